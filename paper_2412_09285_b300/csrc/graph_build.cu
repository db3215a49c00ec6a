// Device construction of a sparse problem's CSR (fem_create_problem for large edge
// lists).  After one copy of the edge list to the device, everything that costs time
// on the host runs here:
//   0. validation (indices in range, no self-loops, finite nonzero weights, positive
//      for bMinCut), the weight flags (all |w| = 1, all integer) and the weight sums,
//      one thread per chunk of kWeightChunk edges (the fp64 chunk sums are added in
//      chunk order on the host, as the host builder adds its own);
//   1. degrees (atomic counts), 2. an exclusive scan to the row pointers,
//   3. a scatter of (column << 32 | edge) keys into the rows,
//   4. a sort of every row by column (one warp per row up to 32 entries, one block
//      per row up to 4096, the host for the rare longer rows),
//   5. one pass per row that rejects a repeated column (a duplicate edge) and writes
//      the packed columns (the +-1 weight in bit 31 when every |w| = 1), the fp32 and
//      fp64 weights and the row normalisations c_i (MaxCut: 1 / sum_j |W_ij|;
//      bMinCut: c^f = q / sum_j W_ij, c^a = q / sqrt(sum_j W_ij)).
// The columns of a row end up in increasing order and every row sum is taken in that
// order in fp64, exactly as in the host builder, so both give the same arrays bit
// for bit.  Long clause lists (Max-k-SAT, p-spin) go through the same machinery
// (device_sat_build at the end of this file): validation, packed literals, counts, the
// scan, a scatter of (clause << 3 | position) keys and the per-variable sorts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fem_internal.h"

namespace fem {
namespace {

constexpr unsigned kMask = 0xffffffffu;
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;
constexpr int kBlockSortMax = 4096;  // longest row sorted by one block in shared memory

// Step 0: chunk c = edges c * kWeightChunk ..; first_bad is the lowest invalid edge
// (all ones when none), flags bit 0 = some |w| != 1, bit 1 = some w not an integer of
// magnitude <= 2^24; csum[c] the chunk's weight sum in edge order; wsum_i the sum of
// the integer weights (meaningful when flags bit 1 is clear).
__global__ void k_check_edges(const int32_t* __restrict__ ei, const int32_t* __restrict__ ej,
                              const double* __restrict__ w, int64_t E, int32_t n, int32_t pos_only,
                              unsigned long long* __restrict__ first_bad, int32_t* __restrict__ flags,
                              double* __restrict__ csum, unsigned long long* __restrict__ wsum_i) {
  const long long nchunks = (E + kWeightChunk - 1) / kWeightChunk;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (long long)gridDim.x * blockDim.x) {
    const long long e0 = c * kWeightChunk, e1 = e0 + kWeightChunk < E ? e0 + kWeightChunk : E;
    double sf = 0.0;
    long long si = 0;
    bool unit = true, integer = true;
    long long bad = -1;
    for (long long e = e0; e < e1; ++e) {
      const int32_t i = ei[e], j = ej[e];
      const double x = w ? w[e] : 1.0;
      const double a = fabs(x);
      if (!((uint32_t)i < (uint32_t)n && (uint32_t)j < (uint32_t)n && i != j && a <= 1.7976931348623157e308 &&
            x != 0.0 && (!pos_only || x > 0.0))) {
        bad = e;
        break;
      }
      unit = unit && a == 1.0;
      const bool small = a <= 16777216.0;
      const long long xi = (long long)(small ? x : 0.0);
      integer = integer && small && (double)xi == x;
      sf = __dadd_rn(sf, x);
      si += xi;
    }
    csum[c] = sf;
    if (bad >= 0) atomicMin(first_bad, (unsigned long long)bad);
    if (!unit || !integer) atomicOr(flags, (unit ? 0 : 1) | (integer ? 0 : 2));
    if (si != 0) atomicAdd(wsum_i, (unsigned long long)si);
  }
}

__global__ void k_degrees(const int32_t* __restrict__ ei, const int32_t* __restrict__ ej, int64_t E,
                          int32_t* __restrict__ deg) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
    atomicAdd(deg + ei[e], 1);
    atomicAdd(deg + ej[e], 1);
  }
}

// Inclusive block scan of one value per thread (256 threads); returns the inclusive
// prefix and writes the block total to *total.
__device__ __forceinline__ int32_t block_scan(int32_t x, int32_t* warp_tot, int32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int32_t y = __shfl_up_sync(kMask, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int32_t y = __shfl_up_sync(kMask, t, off);
      if (lane >= off) t += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  const int32_t res = x + (warp > 0 ? warp_tot[warp - 1] : 0);
  if (threadIdx.x == kScanThreads - 1) *total = res;
  __syncthreads();
  return res;
}

// out[i + 1] = sum of in[tile start .. i] for the tile of i; the tile's total to sums[tile].
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int32_t* __restrict__ in, int32_t n,
                                                            int32_t* __restrict__ out, int32_t* __restrict__ sums) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  __shared__ int32_t total;
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = base + k;
    run += i < n ? in[i] : 0;
    v[k] = run;
  }
  const int32_t incl = block_scan(run, warp_tot, &total);
  const int32_t before = incl - run;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = base + k;
    if (i < n) out[i + 1] = v[k] + before;
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Exclusive scan of the tile totals in place, by one block, 256 at a time with a carry.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int32_t* __restrict__ sums, int32_t nb) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  __shared__ int32_t total;
  int32_t carry = 0;
  for (int c0 = 0; c0 < nb; c0 += kScanThreads) {
    const int i = c0 + threadIdx.x;
    const int32_t x = i < nb ? sums[i] : 0;
    const int32_t incl = block_scan(x, warp_tot, &total);
    if (i < nb) sums[i] = incl - x + carry;
    carry += total;
    __syncthreads();
  }
}

__global__ void k_scan_add(int32_t* __restrict__ out, int32_t n, const int32_t* __restrict__ sums) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i + 1] += sums[i / kScanTile];
}

// Each undirected edge e = (i, j) becomes the key (j << 32 | e) in row i and
// (i << 32 | e) in row j, at a slot taken from the row's cursor.
__global__ void k_scatter(const int32_t* __restrict__ ei, const int32_t* __restrict__ ej, int64_t E,
                          int32_t* __restrict__ cursor, unsigned long long* __restrict__ key) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)ei[e], j = (uint32_t)ej[e];
    key[atomicAdd(cursor + i, 1)] = ((unsigned long long)j << 32) | (uint32_t)e;
    key[atomicAdd(cursor + j, 1)] = ((unsigned long long)i << 32) | (uint32_t)e;
  }
}

// Rows of up to 32 entries: one warp per row, a bitonic sort across the lanes.  Longer
// rows are listed for the block sort.
__global__ void k_sort_rows_warp(const int32_t* __restrict__ row_ptr, int32_t n, unsigned long long* __restrict__ key,
                                 int32_t* __restrict__ big, int32_t* __restrict__ nbig) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += nwarps) {
    const int beg = row_ptr[row], len = row_ptr[row + 1] - beg;
    if (len <= 1) continue;
    if (len > 32) {
      if (lane == 0) big[atomicAdd(nbig, 1)] = (int32_t)row;
      continue;
    }
    unsigned long long x = lane < len ? key[beg + lane] : ~0ull;
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kMask, x, stride);
        const bool keep_min = ((lane & stride) == 0) == ((lane & size) == 0);
        x = keep_min ? (x < y ? x : y) : (x < y ? y : x);
      }
    }
    if (lane < len) key[beg + lane] = x;
  }
}

// Rows of 33 .. kBlockSortMax entries: one block per row, a bitonic sort in shared
// memory over the next power of two.  Longer rows are listed for the host.
__global__ void __launch_bounds__(512) k_sort_rows_block(const int32_t* __restrict__ row_ptr,
                                                         unsigned long long* __restrict__ key,
                                                         const int32_t* __restrict__ big, const int32_t* __restrict__ nbig,
                                                         int32_t* __restrict__ giant, int32_t* __restrict__ ngiant) {
  __shared__ unsigned long long sk[kBlockSortMax];
  const int nb = *nbig;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const int row = big[b];
    const int beg = row_ptr[row], len = row_ptr[row + 1] - beg;
    if (len > kBlockSortMax) {
      if (threadIdx.x == 0) giant[atomicAdd(ngiant, 1)] = row;
      continue;
    }
    int P = 64;
    while (P < len) P <<= 1;
    for (int k = threadIdx.x; k < P; k += blockDim.x) sk[k] = k < len ? key[beg + k] : ~0ull;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int k = threadIdx.x; k < P; k += blockDim.x) {
          const int partner = k ^ stride;
          if (partner > k) {
            const bool asc = (k & size) == 0;
            const unsigned long long a = sk[k], c = sk[partner];
            if ((a > c) == asc) {
              sk[k] = c;
              sk[partner] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int k = threadIdx.x; k < len; k += blockDim.x) key[beg + k] = sk[k];
    __syncthreads();
  }
}

// Clause c of a Max-k-SAT / p-spin list: the first check it fails (0 when it passes):
// 1 pointers (not 0 <= b <= e <= L), 2 more than 8 literals, 3 a literal 0 or out of
// [-n, n], 4 a variable repeated within the clause; *lit is the offending literal.
__host__ __device__ inline int clause_defect(const int64_t* ptr, const int32_t* lits, long long c, long long L, int32_t n,
                                             int32_t* lit) {
  const long long b = ptr[c], e = ptr[c + 1];
  if (b < 0 || e < b || e > L) return 1;
  if (e - b > 8) return 2;
  for (long long k = b; k < e; ++k) {
    const int32_t x = lits[k];
    *lit = x;
    if (x == 0 || x > n || x < -n) return 3;
    const int32_t v = x < 0 ? -x : x;
    for (long long k2 = b; k2 < k; ++k2)
      if ((lits[k2] < 0 ? -lits[k2] : lits[k2]) == v) return 4;
  }
  return 0;
}

// res[0] = lowest failing clause (all ones when none); widths of the others: res[1] max, res[2] min.
__global__ void k_sat_check(const int64_t* __restrict__ ptr, const int32_t* __restrict__ lits, int64_t M, int64_t L,
                            int32_t n, unsigned long long* __restrict__ res) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (long long)gridDim.x * blockDim.x) {
    int32_t lit = 0;
    if (clause_defect(ptr, lits, c, L, n, &lit)) {
      atomicMin(res, (unsigned long long)c);
    } else {
      const unsigned long long w = (unsigned long long)(ptr[c + 1] - ptr[c]);
      atomicMax(res + 1, w);
      atomicMin(res + 2, w);
    }
  }
}

// Packed literals (var << 1 | negated), int32 clause pointers and the occurrence counts.
__global__ void k_sat_count(const int64_t* __restrict__ ptr, const int32_t* __restrict__ lits, int64_t M,
                            int32_t* __restrict__ cl_ptr, int32_t* __restrict__ cl_lit, int32_t* __restrict__ cnt) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (long long)gridDim.x * blockDim.x) {
    const long long b = ptr[c], e = ptr[c + 1];
    cl_ptr[c] = (int32_t)b;
    if (c == M - 1) cl_ptr[M] = (int32_t)e;
    for (long long k = b; k < e; ++k) {
      const int32_t x = lits[k], v = (x < 0 ? -x : x) - 1;
      cl_lit[k] = (v << 1) | (x < 0 ? 1 : 0);
      atomicAdd(cnt + v, 1);
    }
  }
}

// Each literal (clause c, position k) becomes the key (c << 3 | k) in its variable's list.
__global__ void k_sat_scatter(const int32_t* __restrict__ cl_ptr, const int32_t* __restrict__ cl_lit, int64_t M,
                              int32_t* __restrict__ cursor, unsigned long long* __restrict__ key) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (long long)gridDim.x * blockDim.x) {
    const int32_t b = cl_ptr[c], e = cl_ptr[c + 1];
    for (int32_t k = b; k < e; ++k)
      key[atomicAdd(cursor + (cl_lit[k] >> 1), 1)] = ((unsigned long long)c << 3) | (unsigned)(k - b);
  }
}

// p-spin terms: J_v with the literals' negations folded in (fp32, fp64, and int64 when
// an integer of magnitude <= 2^40); res[0] = lowest non-finite term, res[1] bit 0 =
// some J_v not such an integer.
__global__ void k_pspin_terms(const int64_t* __restrict__ ptr, const int32_t* __restrict__ lits,
                              const double* __restrict__ tw, int64_t M, float* __restrict__ pj,
                              double* __restrict__ pj_f, int64_t* __restrict__ pj_i, unsigned long long* __restrict__ res) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (long long)gridDim.x * blockDim.x) {
    double J = tw[c];
    if (!isfinite(J)) {
      atomicMin(res, (unsigned long long)c);
      continue;
    }
    for (long long k = ptr[c]; k < ptr[c + 1]; ++k)
      if (lits[k] < 0) J = -J;
    const bool integer = J == rint(J) && fabs(J) <= 1099511627776.0;
    if (!integer) atomicOr(res + 1, 1ull);
    pj[c] = (float)J;
    pj_f[c] = J;
    pj_i[c] = integer ? (int64_t)J : 0;
  }
}

// Per occurrence: the packed (clause << 3 | position); with every clause of width 3,
// the other two literals (the first with the occurrence's own negation in bit 31) and,
// for p-spin, the term's J.
__global__ void k_sat_occ(const unsigned long long* __restrict__ key, int64_t L, const int32_t* __restrict__ cl_ptr,
                          const int32_t* __restrict__ cl_lit, int32_t* __restrict__ occ, int32_t* __restrict__ oth,
                          const float* __restrict__ pj, float* __restrict__ pjo) {
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < L; o += (long long)gridDim.x * blockDim.x) {
    const int32_t x = (int32_t)key[o], c = x >> 3, pos = x & 7;
    occ[o] = x;
    if (oth) {
      const int32_t b = cl_ptr[c];
      int32_t other[2], k2 = 0;
      for (int32_t k = 0; k < 3; ++k)
        if (k != pos) other[k2++] = cl_lit[b + k];
      const uint32_t own_neg = (uint32_t)(cl_lit[b + pos] & 1);
      oth[2 * o] = (int32_t)((uint32_t)other[0] | (own_neg << 31));
      oth[2 * o + 1] = other[1];
      if (pjo) pjo[o] = pj[c];
    }
  }
}

// One thread per row: duplicate check, packed columns, weights, row normalisations.
// dup[0] is set (and dup[1], dup[2] name the pair) when a row repeats a column.
__global__ void k_finish_rows(const int32_t* __restrict__ row_ptr, const unsigned long long* __restrict__ key,
                              int32_t n, const double* __restrict__ w, int32_t unit, int32_t integer, int32_t kind,
                              int32_t q, uint32_t* __restrict__ col, float* __restrict__ wf, double* __restrict__ w64,
                              float* __restrict__ cnorm, float* __restrict__ cnorm2, int32_t* __restrict__ dup) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double rsum = 0.0, rabs = 0.0;
    uint32_t prev = 0xffffffffu;
    for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const unsigned long long kk = key[k];
      const uint32_t j = (uint32_t)(kk >> 32);
      const double wt = w ? w[(uint32_t)kk] : 1.0;
      if (j == prev && atomicCAS(dup, 0, 1) == 0) {
        dup[1] = (int32_t)i;
        dup[2] = (int32_t)j;
      }
      prev = j;
      col[k] = j | ((unit && wt < 0.0) ? 0x80000000u : 0u);
      if (!unit) wf[k] = (float)wt;
      if (!integer) w64[k] = wt;
      rsum += wt;
      rabs += fabs(wt);
    }
    if (kind == FEM_MAXCUT) {
      if (!unit) cnorm[i] = rabs > 0.0 ? (float)(1.0 / rabs) : 0.f;
    } else {
      cnorm[i] = rsum > 0.0 ? (float)((double)q / rsum) : 0.f;
      cnorm2[i] = rsum > 0.0 ? (float)((double)q / sqrt(rsum)) : 0.f;
    }
  }
}

int grid_for(long long work, int sm_count, int threads = 256) {
  long long b = (work + threads - 1) / threads;
  const long long cap = (long long)sm_count * 8;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// Sorts every segment [ptr[r], ptr[r + 1]) of key, r < nrows, into increasing order:
// one warp per segment of up to 32 keys, one block up to kBlockSortMax, the host for
// the rare longer ones.  big (nrows ints), giant (nrows ints) and counters[0..1] (zero)
// are scratch.  Returns with the stream synchronised.
cudaError_t sort_segments(const int32_t* ptr, int32_t nrows, unsigned long long* key, int32_t* big, int32_t* giant,
                          int32_t* counters, int sm, cudaStream_t s) {
  k_sort_rows_warp<<<grid_for((long long)nrows * 32, sm), 256, 0, s>>>(ptr, nrows, key, big, counters);
  k_sort_rows_block<<<sm * 2, 512, 0, s>>>(ptr, key, big, counters, giant, counters + 1);
  count_launches(2);
  cudaError_t e = cudaGetLastError();
  int32_t ngiant = 0;
  auto sync_copy = [&](void* dst, const void* src, size_t bytes, cudaMemcpyKind kind) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, kind, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  };
  sync_copy(&ngiant, counters + 1, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess || ngiant == 0) return e;
  std::vector<int32_t> rows(ngiant);
  sync_copy(rows.data(), giant, sizeof(int32_t) * (size_t)ngiant, cudaMemcpyDeviceToHost);
  std::vector<unsigned long long> seg;
  for (int32_t r : rows) {
    int32_t be[2] = {0, 0};
    sync_copy(be, ptr + r, sizeof(be), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    seg.resize((size_t)(be[1] - be[0]));
    sync_copy(seg.data(), key + be[0], seg.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    std::sort(seg.begin(), seg.end());
    sync_copy(key + be[0], seg.data(), seg.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  }
  return e;
}

}  // namespace

fem_status device_graph_build(Problem* p, int32_t kind, int32_t q, const fem_problem_desc* d, cudaStream_t s) {
  const int32_t n = d->n;
  const int64_t E = d->n_edges, nnz = 2 * E;
  p->n_edges = E;
  p->nnz = nnz;
  fem_status st;

  // scratch of the build, stream-ordered and released at the end
  const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
  int32_t *ei = nullptr, *ej = nullptr, *deg = nullptr, *sums = nullptr, *cursor = nullptr, *big = nullptr,
          *counters = nullptr;
  double* w = nullptr;
  unsigned long long* key = nullptr;
  std::vector<void*> tmp;
  auto talloc = [&](void** ptr, size_t bytes) -> fem_status {
    const cudaError_t e = cudaMallocAsync(ptr, bytes < 16 ? 16 : bytes, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *ptr = nullptr;
      return fail(FEM_ERR_OOM, "device graph build: %zu bytes of scratch", bytes);
    }
    tmp.push_back(*ptr);
    return FEM_OK;
  };
  auto release = [&]() {
    for (void* x : tmp) cudaFreeAsync(x, s);
    tmp.clear();
  };
  st = FEM_OK;
  if (st == FEM_OK) st = talloc((void**)&ei, sizeof(int32_t) * (size_t)E);
  if (st == FEM_OK) st = talloc((void**)&ej, sizeof(int32_t) * (size_t)E);
  if (st == FEM_OK && d->w) st = talloc((void**)&w, sizeof(double) * (size_t)E);
  if (st == FEM_OK) st = talloc((void**)&deg, sizeof(int32_t) * (size_t)n);
  if (st == FEM_OK) st = talloc((void**)&sums, sizeof(int32_t) * (size_t)ntiles);
  if (st == FEM_OK) st = talloc((void**)&cursor, sizeof(int32_t) * (size_t)n);
  if (st == FEM_OK) st = talloc((void**)&big, sizeof(int32_t) * (size_t)n);
  if (st == FEM_OK) st = talloc((void**)&counters, sizeof(int32_t) * 8);  // nbig, ngiant, dup[3]
  if (st == FEM_OK) st = talloc((void**)&key, sizeof(unsigned long long) * (size_t)nnz);
  const int64_t nchunks = (E + kWeightChunk - 1) / kWeightChunk;
  double* csum = nullptr;
  unsigned long long* check = nullptr;  // first_bad, wsum_i, flags
  if (st == FEM_OK) st = talloc((void**)&csum, sizeof(double) * (size_t)nchunks);
  if (st == FEM_OK) st = talloc((void**)&check, sizeof(unsigned long long) * 3);
  if (st != FEM_OK) {
    release();
    return st;
  }
  // 0. the edge list to the device and its validation; nothing indexes with the
  // endpoints before it has passed
  {
    cudaError_t e0 = cudaMemcpyAsync(ei, d->ei, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s);
    if (e0 == cudaSuccess) e0 = cudaMemcpyAsync(ej, d->ej, sizeof(int32_t) * (size_t)E, cudaMemcpyHostToDevice, s);
    if (e0 == cudaSuccess && d->w)
      e0 = cudaMemcpyAsync(w, d->w, sizeof(double) * (size_t)E, cudaMemcpyHostToDevice, s);
    if (e0 == cudaSuccess) e0 = cudaMemsetAsync(check, 0, sizeof(unsigned long long) * 3, s);
    if (e0 == cudaSuccess) e0 = cudaMemsetAsync(check, 0xff, sizeof(unsigned long long), s);
    if (e0 == cudaSuccess) {
      k_check_edges<<<grid_for(nchunks, p->sm_count), 256, 0, s>>>(ei, ej, w, E, n, kind == FEM_BMINCUT ? 1 : 0,
                                                                    check, reinterpret_cast<int32_t*>(check + 2),
                                                                    csum, check + 1);
      count_launches(1);
      e0 = cudaGetLastError();
    }
    unsigned long long res[3] = {0, 0, 0};
    std::vector<double> hsum((size_t)nchunks);
    if (e0 == cudaSuccess) e0 = cudaMemcpyAsync(res, check, sizeof(res), cudaMemcpyDeviceToHost, s);
    if (e0 == cudaSuccess)
      e0 = cudaMemcpyAsync(hsum.data(), csum, sizeof(double) * (size_t)nchunks, cudaMemcpyDeviceToHost, s);
    if (e0 == cudaSuccess) e0 = cudaStreamSynchronize(s);
    if (e0 != cudaSuccess) {
      release();
      return cuda_fail(e0, "device graph build: edge check");
    }
    if (res[0] != ~0ull) {
      release();
      return edge_error(d, kind, (int64_t)res[0]);
    }
    const int32_t flags = (int32_t)(res[2] & 0xffffffffull);
    p->unit_w = (flags & 1) == 0;
    p->int_w = (flags & 2) == 0;
    p->wtot_i = (int64_t)res[1];
    double tot = 0.0;
    for (double x : hsum) tot += x;
    p->wtot_f = tot;
  }
  const bool unit = p->unit_w, integer = p->int_w;
  if (st == FEM_OK) st = dev_alloc_t(p, &p->row_ptr, (size_t)n + 1);
  if (st == FEM_OK) st = dev_alloc_t(p, &p->col, (size_t)nnz);
  if (st == FEM_OK && !unit) st = dev_alloc_t(p, &p->w, (size_t)nnz);
  if (st == FEM_OK && !integer) st = dev_alloc_t(p, &p->w64, (size_t)nnz);
  const bool need_c = kind != FEM_MAXCUT || !unit;
  if (st == FEM_OK && need_c) st = dev_alloc_t(p, &p->cnorm, (size_t)n);
  if (st == FEM_OK && kind != FEM_MAXCUT) st = dev_alloc_t(p, &p->cnorm2, (size_t)n);
  if (st != FEM_OK) {
    release();
    return st;
  }
  int32_t* giant = cursor;  // the cursors are spent once the keys are placed
  cudaError_t e = cudaSuccess;
  auto step = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  step(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)n, s));
  step(cudaMemsetAsync(counters, 0, sizeof(int32_t) * 8, s));
  step(cudaMemsetAsync(p->row_ptr, 0, sizeof(int32_t), s));
  if (e == cudaSuccess) {
    const int sm = p->sm_count;
    k_degrees<<<grid_for(E, sm), 256, 0, s>>>(ei, ej, E, deg);
    k_scan_tiles<<<ntiles, kScanThreads, 0, s>>>(deg, n, p->row_ptr, sums);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, ntiles);
    k_scan_add<<<grid_for(n, sm), 256, 0, s>>>(p->row_ptr, n, sums);
    step(cudaMemcpyAsync(cursor, p->row_ptr, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    k_scatter<<<grid_for(E, sm), 256, 0, s>>>(ei, ej, E, cursor, key);
    count_launches(5);
    step(cudaGetLastError());
  }
  if (e == cudaSuccess) step(sort_segments(p->row_ptr, n, key, big, giant, counters, p->sm_count, s));
  int32_t dup[3] = {0, 0, 0};
  if (e == cudaSuccess) {
    k_finish_rows<<<grid_for(n, p->sm_count), 256, 0, s>>>(p->row_ptr, key, n, w, unit ? 1 : 0, integer ? 1 : 0, kind, q,
                                                           p->col, p->w, p->w64, p->cnorm, p->cnorm2, counters + 2);
    count_launches(1);
    step(cudaGetLastError());
    if (e == cudaSuccess) step(cudaMemcpyAsync(dup, counters + 2, sizeof(dup), cudaMemcpyDeviceToHost, s));
  }
  release();
  if (e == cudaSuccess) step(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return cuda_fail(e, "device graph build");
  if (dup[0]) return fail(FEM_ERR_INVALID_ARG, "duplicate edge (%d, %d)", dup[1], dup[2]);
  return FEM_OK;
}

}  // namespace fem

namespace fem {

// Max-k-SAT and p-spin clause lists on the device (fem_create_problem for long lists):
// the clause pointers and literals are copied once, validated (k_sat_check: the lowest
// failing clause is reported with the host builder's message), packed, counted per
// variable, scanned into the occurrence pointers, scattered as (clause << 3 | position)
// keys and sorted per variable, so every variable's occurrences are in clause order as
// the host builder lists them; then the per-occurrence tables.  p-spin terms are folded
// with their literals' negations here too.  Sets the clause fields of p (and pj, pj_f,
// pj_i, pjo and *terms_int for p-spin).
fem_status device_sat_build(Problem* p, const fem_problem_desc* d, bool pspin, bool* terms_int, cudaStream_t s) {
  const int32_t n = d->n;
  const int64_t M = d->n_clauses, L = d->clause_ptr[M];
  const int sm = p->sm_count;
  p->n_clauses = M;
  p->n_occ = L;
  const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
  int64_t* dptr = nullptr;
  int32_t *dlits = nullptr, *cnt = nullptr, *sums = nullptr, *cursor = nullptr, *big = nullptr, *counters = nullptr;
  double* tw = nullptr;
  unsigned long long *key = nullptr, *res = nullptr;
  std::vector<void*> tmp;
  auto talloc = [&](void** ptr, size_t bytes) -> fem_status {
    const cudaError_t e = cudaMallocAsync(ptr, bytes < 16 ? 16 : bytes, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *ptr = nullptr;
      return fail(FEM_ERR_OOM, "device clause build: %zu bytes of scratch", bytes);
    }
    tmp.push_back(*ptr);
    return FEM_OK;
  };
  auto release = [&]() {
    for (void* x : tmp) cudaFreeAsync(x, s);
    tmp.clear();
  };
  fem_status st = FEM_OK;
  if (st == FEM_OK) st = talloc((void**)&dptr, sizeof(int64_t) * (size_t)(M + 1));
  if (st == FEM_OK) st = talloc((void**)&dlits, sizeof(int32_t) * (size_t)L);
  if (st == FEM_OK) st = talloc((void**)&res, sizeof(unsigned long long) * 4);
  if (st == FEM_OK && pspin) st = talloc((void**)&tw, sizeof(double) * (size_t)M);
  if (st != FEM_OK) {
    release();
    return st;
  }
  // 0. copy and validate; nothing indexes with a literal before this has passed
  cudaError_t e = cudaMemcpyAsync(dptr, d->clause_ptr, sizeof(int64_t) * (size_t)(M + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dlits, d->lits, sizeof(int32_t) * (size_t)L, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && pspin) e = cudaMemcpyAsync(tw, d->term_weight, sizeof(double) * (size_t)M, cudaMemcpyHostToDevice, s);
  const unsigned long long init[4] = {~0ull, 0ull, ~0ull, 0ull};  // first bad, max width, min width, unused
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_sat_check<<<grid_for(M, sm), 256, 0, s>>>(dptr, dlits, M, L, n, res);
    count_launches(1);
    e = cudaGetLastError();
  }
  unsigned long long chk[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(chk, res, sizeof(chk), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "device clause build: check");
  }
  if (chk[0] != ~0ull) {
    release();
    const long long c = (long long)chk[0];
    int32_t lit = 0;
    const int why = clause_defect(d->clause_ptr, d->lits, c, L, n, &lit);
    if (why == 2) return fail(FEM_ERR_UNSUPPORTED, "clause %lld has more than 8 literals", c);
    if (why == 3) return fail(FEM_ERR_INVALID_ARG, "clause %lld: literal %d out of range", c, lit);
    if (why == 4) return fail(FEM_ERR_INVALID_ARG, "clause %lld repeats variable %d", c, lit < 0 ? -lit : lit);
    return fail(FEM_ERR_INVALID_ARG, "clause_ptr must be non-decreasing and end at the literal count");
  }
  const int32_t max_w = (int32_t)chk[1], min_w = (int32_t)chk[2];
  p->max_width = max_w;
  const bool three = M > 0 && min_w == 3 && max_w == 3;
  // p-spin terms (their validation follows the clauses', as on the host)
  if (pspin) {
    if ((st = dev_alloc_t(p, &p->pj, (size_t)M)) != FEM_OK || (st = dev_alloc_t(p, &p->pj_f, (size_t)M)) != FEM_OK ||
        (st = dev_alloc_t(p, &p->pj_i, (size_t)M)) != FEM_OK) {
      release();
      return st;
    }
    const unsigned long long tinit[2] = {~0ull, 0ull};
    e = cudaMemcpyAsync(res, tinit, sizeof(tinit), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      k_pspin_terms<<<grid_for(M, sm), 256, 0, s>>>(dptr, dlits, tw, M, p->pj, p->pj_f, p->pj_i, res);
      count_launches(1);
      e = cudaGetLastError();
    }
    unsigned long long tr[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(tr, res, sizeof(tr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(e, "device clause build: terms");
    }
    if (tr[0] != ~0ull) {
      release();
      return fail(FEM_ERR_INVALID_ARG, "term_weight[%lld] must be finite", (long long)tr[0]);
    }
    *terms_int = (tr[1] & 1ull) == 0;
  }
  // 1. packed literals, counts, occurrence pointers
  if ((st = dev_alloc_t(p, &p->cl_ptr, (size_t)M + 1)) != FEM_OK || (st = dev_alloc_t(p, &p->cl_lit, (size_t)L)) != FEM_OK ||
      (st = dev_alloc_t(p, &p->occ_ptr, (size_t)n + 1)) != FEM_OK || (st = dev_alloc_t(p, &p->occ, (size_t)L)) != FEM_OK ||
      (three && (st = dev_alloc_t(p, &p->oth, 2 * (size_t)L)) != FEM_OK) ||
      (three && pspin && (st = dev_alloc_t(p, &p->pjo, (size_t)L)) != FEM_OK)) {
    release();
    return st;
  }
  if (st == FEM_OK) st = talloc((void**)&cnt, sizeof(int32_t) * (size_t)n);
  if (st == FEM_OK) st = talloc((void**)&sums, sizeof(int32_t) * (size_t)ntiles);
  if (st == FEM_OK) st = talloc((void**)&cursor, sizeof(int32_t) * (size_t)n);
  if (st == FEM_OK) st = talloc((void**)&big, sizeof(int32_t) * (size_t)n);
  if (st == FEM_OK) st = talloc((void**)&counters, sizeof(int32_t) * 8);
  if (st == FEM_OK) st = talloc((void**)&key, sizeof(unsigned long long) * (size_t)L);
  if (st != FEM_OK) {
    release();
    return st;
  }
  e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, sizeof(int32_t) * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->occ_ptr, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) {
    k_sat_count<<<grid_for(M, sm), 256, 0, s>>>(dptr, dlits, M, p->cl_ptr, p->cl_lit, cnt);
    k_scan_tiles<<<ntiles, kScanThreads, 0, s>>>(cnt, n, p->occ_ptr, sums);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, ntiles);
    k_scan_add<<<grid_for(n, sm), 256, 0, s>>>(p->occ_ptr, n, sums);
    count_launches(4);
    e = cudaGetLastError();
  }
  // 2. keys into the variables' lists, sorted into clause order
  if (e == cudaSuccess) e = cudaMemcpyAsync(cursor, p->occ_ptr, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) {
    k_sat_scatter<<<grid_for(M, sm), 256, 0, s>>>(p->cl_ptr, p->cl_lit, M, cursor, key);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = sort_segments(p->occ_ptr, n, key, big, cursor, counters, sm, s);
  // 3. the per-occurrence tables
  if (e == cudaSuccess && L > 0) {
    k_sat_occ<<<grid_for(L, sm), 256, 0, s>>>(key, L, p->cl_ptr, p->cl_lit, p->occ, three ? p->oth : nullptr,
                                               p->pj, three && pspin ? p->pjo : nullptr);
    count_launches(1);
    e = cudaGetLastError();
  }
  release();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "device clause build");
  return FEM_OK;
}

}  // namespace fem
