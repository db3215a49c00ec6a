// Exact-gradient MaxCut / QUBO step with the neighbour gathers on the tensor memory
// accelerator (SM Eq. grad_m_h, exact mode):
//   g_ir = (gamma/4) [c S_ir + h_ir/beta] (1 - m_ir^2),  S_ir = sum_j W_ij m_jr,
// c = 2 for MaxCut, 1 for QUBO (plus the per-node constant), m = tanh(h/2) of the
// fields the step reads.
//
// The direct-gather kernel (maxcut_sparse.cu) waits on one 128-byte line of m per
// neighbour and warp, most of them L2 misses, with only a few in flight per warp.  Here
// a block works on tiles of 16 consecutive nodes (one block of 32 replicas) and a
// producer warp stages each tile ahead in shared memory:
//   * the tile's CSR entries (coalesced loads), then one TMA gather4 per four entries
//     (cp.async.bulk.tensor tile::gather4 over the [n][R] marginals, a box of one row of
//     32 replicas), so all of the tile's neighbour lines are in flight at once;
//   * the tile's h, m, v rows by bulk copies;
// all completing on the stage's mbarrier.  Four consumer warps then sum each node's
// neighbour rows from shared memory in CSR order and run the same fp32 update as the
// direct kernel, so both give the same bits.  Two stages per block and four blocks per
// SM: each producer fills one stage while its consumers work on the other, its row
// pointers two tiles and its CSR entries one tile ahead in registers.  (Measured at
// n = 2^20, R = 32: 32-node tiles at two blocks per SM 0.373 ms, 8-node tiles at eight
// 0.336 ms, 16-node tiles at four 0.325 ms; the producer loading a tile's row pointers
// and entries only when it fills the stage, 0.612 ms.)  Entries beyond a tile's capacity (hub
// rows) are gathered directly from global memory, in order.  Every wait is bounded; on
// expiry the kernel records FEM's timeout bit and leaves.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "fem_internal.h"
#include "step_common.cuh"

namespace fem {
namespace {

constexpr int kNodes = 16;        // nodes per tile
constexpr int kCap = 128;         // neighbour rows staged per tile (a multiple of 4)
constexpr int kConsumers = 4;     // consumer warps; warp kConsumers is the producer
constexpr int kStages = 2;        // tiles in flight per block
constexpr int kThreads = (kConsumers + 1) * 32;
constexpr unsigned long long kWaitNs = 2000000000ull;

struct GatherArgs {
  const int32_t* row_ptr;
  const uint32_t* col;   // unit weights: the -1 sign in bit 31
  const float* w;        // weights (NULL for unit weights)
  int32_t n, R, wpn;
  const float* h_in;
  float* h_out;
  float* m;
  float* v;
  const float* mag_in;   // m = tanh(h/2) of h_in, [n][R] (also behind the tensor map)
  float* mag_out;
  uint32_t* words_out;
  float ccoef;
  const float* offset;
  int32_t* err;
};

// One stage of shared memory (1 KB aligned, so that both stages' copy targets are).
struct alignas(1024) Stage {
  float rows[kCap * 32];           // gathered neighbour lines, entry k at rows[32 k ..]
  float h[kNodes * 32], m[kNodes * 32], v[kNodes * 32];
  uint32_t col[kCap];
  float w[kCap];
  float off[kNodes];               // QUBO: the nodes' constants of the field
  int32_t rptr[kNodes + 1];        // the tile's row pointers relative to base
  int32_t base;                    // row_ptr of the tile's first node
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the timeout bit set) when the phase has not completed in kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int32_t* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > kWaitNs) {
      atomicOr(err, ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) into shared memory.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Four rows y0..y3 of the 2D map, columns x .. x + 31, to dst (4 x 128 bytes).
__device__ __forceinline__ void gather4(void* dst, const CUtensorMap* tm, int x, int y0, int y1, int y2, int y3,
                                        uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
      ::"r"(smem_u32(dst)), "l"(tm), "r"(x), "r"(y0), "r"(y1), "r"(y2), "r"(y3), "r"(smem_u32(bar))
      : "memory");
}

// R32: the replica count is 32 (one block of replicas per node), a compile-time constant, so
// the state rows' offsets are immediates.  OFF: QUBO's per-node constants of the field are
// staged and added (MaxCut instantiations carry neither the loads nor the registers).
template <int OPT, bool UNIT, bool R32, bool OFF>
__global__ void __launch_bounds__(kThreads, 4) k_exact_gather(const __grid_constant__ CUtensorMap tm_mag, GatherArgs a,
                                                              StepScalars s) {
  const int R = R32 ? 32 : a.R, wpn = R32 ? 1 : a.wpn;
  extern __shared__ uint8_t smem_raw[];
  Stage* st = reinterpret_cast<Stage*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ int32_t abort_flag;
  volatile int32_t* abort_v = &abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long tiles = (long long)((a.n + kNodes - 1) / kNodes) * wpn;
  if (threadIdx.x == 0) {
    for (int b = 0; b < kStages; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], kConsumers);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  long long issued = 0;  // producer: tiles whose copies were issued
  if (warp == kConsumers) {
    // ---- producer.  The row pointers run two tiles ahead and the CSR entries one tile
    // ahead in registers, so a tile's stage is filled without waiting on memory.
    constexpr int kQ = kCap / 32;  // entries per lane and tile
    auto first_node = [&](long long t) { return (int)(wpn == 1 ? t : t / wpn) * kNodes; };
    auto load_rp = [&](long long t, int& rp, int& rl) {
      if (t < tiles) {
        const int i0 = first_node(t);
        rp = __ldg(a.row_ptr + min(i0 + lane, a.n));
        rl = __ldg(a.row_ptr + min(i0 + kNodes, a.n));
      }
    };
    auto load_cols = [&](long long t, int rp, int rl, uint32_t (&c)[kQ], float (&w)[kQ], float& of) {
      if (t >= tiles) return;
      if (OFF) of = __ldg(a.offset + min(first_node(t) + lane, a.n - 1));
      const int base = __shfl_sync(kFullMask, rp, 0), ecap = min(rl - base, kCap);
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        const int k = lane + 32 * q;
        if (k < ecap) {
          c[q] = __ldg(a.col + base + k);
          if (!UNIT) w[q] = __ldg(a.w + base + k);
        }
      }
    };
    uint32_t c1[kQ], c2[kQ];
    float w1[kQ], w2[kQ], of1 = 0.f, of2 = 0.f;
    int rp1 = 0, rl1 = 0, rp2 = 0, rl2 = 0, rp3 = 0, rl3 = 0;
    long long t1 = blockIdx.x, t2 = t1 + gridDim.x, t3 = t2 + gridDim.x;
    load_rp(t1, rp1, rl1);
    load_rp(t2, rp2, rl2);
    load_cols(t1, rp1, rl1, c1, w1, of1);
    for (long long it = 0; t1 < tiles; ++it) {
      load_cols(t2, rp2, rl2, c2, w2, of2);  // in flight while this tile's stage is filled
      load_rp(t3, rp3, rl3);
      const int b = (int)(it % kStages);
      const uint32_t use = (uint32_t)(it / kStages);
      // every lane waits (each then writes the stage), and the warp agrees on the outcome
      const bool ok = __all_sync(kFullMask, mbar_wait(&empty[b], (use & 1) ^ 1, a.err)) && !*abort_v;
      if (!ok) {
        *abort_v = 1;
        break;
      }
      Stage& S = st[b];
      const long long nb = wpn == 1 ? t1 : t1 / wpn;
      const int wb = wpn == 1 ? 0 : (int)(t1 - nb * wpn);
      const int i0 = (int)nb * kNodes, nn = min(kNodes, a.n - i0);
      const int base = __shfl_sync(kFullMask, rp1, 0);
      if (lane < kNodes) {
        S.rptr[lane] = rp1 - base;
        if (OFF) S.off[lane] = of1;
      }
      if (lane == 0) {
        S.rptr[kNodes] = rl1 - base;
        S.base = base;
      }
      const int ecap = min(rl1 - base, kCap);
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        const int k = lane + 32 * q;
        if (k < ecap) {
          S.col[k] = c1[q];
          if (!UNIT) S.w[k] = w1[q];
        }
      }
      __syncwarp();
      const int groups = (ecap + 3) >> 2;
      // bytes this stage expects: four rows per gather, the state rows
      const uint32_t rows_b = (uint32_t)nn * 128u;
      const uint32_t bytes = (uint32_t)groups * 512u + rows_b * (OPT == FEM_OPT_SGD ? 2u : 3u);
      if (lane == 0) mbar_expect_tx(&full[b], bytes);
      for (int g = lane; g < groups; g += 32) {
        const int k = 4 * g;
        const int y0 = (int)(S.col[k] & 0x7fffffffu);
        const int y1 = k + 1 < ecap ? (int)(S.col[k + 1] & 0x7fffffffu) : y0;
        const int y2 = k + 2 < ecap ? (int)(S.col[k + 2] & 0x7fffffffu) : y0;
        const int y3 = k + 3 < ecap ? (int)(S.col[k + 3] & 0x7fffffffu) : y0;
        gather4(S.rows + 32 * k, &tm_mag, wb * 32, y0, y1, y2, y3, &full[b]);
      }
      if (wpn == 1) {
        if (lane == 0) {
          const size_t off = (size_t)i0 * R;
          bulk_load(S.h, a.h_in + off, rows_b, &full[b]);
          bulk_load(S.m, a.m + off, rows_b, &full[b]);
          if (OPT != FEM_OPT_SGD) bulk_load(S.v, a.v + off, rows_b, &full[b]);
        }
      } else if (lane < nn) {
        const size_t off = (size_t)(i0 + lane) * R + (size_t)wb * 32;
        bulk_load(S.h + 32 * lane, a.h_in + off, 128u, &full[b]);
        bulk_load(S.m + 32 * lane, a.m + off, 128u, &full[b]);
        if (OPT != FEM_OPT_SGD) bulk_load(S.v + 32 * lane, a.v + off, 128u, &full[b]);
      }
      issued = it + 1;
      // the next tile's entries become this tile's
      t1 = t2;
      t2 = t3;
      t3 += gridDim.x;
      rp1 = rp2;
      rl1 = rl2;
      rp2 = rp3;
      rl2 = rl3;
      of1 = of2;
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        c1[q] = c2[q];
        w1[q] = w2[q];
      }
    }
    // the stages still owned by the consumers finish before the block leaves (below)
  } else {
    // ---- consumers: warp w takes nodes w, w + 8, w + 16, w + 24 of each tile
    long long it = 0;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
      const int b = (int)(it % kStages);
      const uint32_t use = (uint32_t)(it / kStages);
      const bool ok = __all_sync(kFullMask, mbar_wait(&full[b], use & 1, a.err)) && !*abort_v;
      if (!ok) {
        *abort_v = 1;
        break;
      }
      const Stage& S = st[b];
      const long long nb = wpn == 1 ? t : t / wpn;
      const int wb = wpn == 1 ? 0 : (int)(t - nb * wpn);
      const int i0 = (int)nb * kNodes, nn = min(kNodes, a.n - i0);
      for (int j = warp; j < nn; j += kConsumers) {
        const int i = i0 + j;
        const int beg = S.rptr[j], end = S.rptr[j + 1];
        float facc = 0.f;
        const int e1 = min(end, kCap);
        // unrolled (the sums stay in entry order): less loop overhead per staged row
#pragma unroll 4
        for (int k = beg; k < e1; ++k) {
          const float mj = S.rows[32 * k + lane];
          if (UNIT) facc += (S.col[k] >> 31) ? -mj : mj;
          else facc = fmaf(S.w[k], mj, facc);
        }
        for (int k = max(beg, kCap); k < end; ++k) {  // beyond the staged rows: direct gathers
          const uint32_t c = __ldg(a.col + S.base + k);
          const float mj = a.mag_in[(size_t)(c & 0x7fffffffu) * R + (size_t)wb * 32 + lane];
          if (UNIT) facc += (c >> 31) ? -mj : mj;
          else facc = fmaf(__ldg(a.w + S.base + k), mj, facc);
        }
        float hi = S.h[32 * j + lane], mi = S.m[32 * j + lane];
        float vi = OPT == FEM_OPT_SGD ? 0.f : S.v[32 * j + lane];
        float field = a.ccoef * facc;
        if (OFF) field += S.off[j];
        // field + h/beta as one explicit fma, so that the direct and the tile kernel round it
        // alike however the compiler contracts the code around it
        const float g = s.gq * fmaf(hi, s.inv_beta, field) * one_minus_m2_fast(hi);
        opt_update_fast<OPT>(hi, mi, vi, g, s);
        const size_t idx = (size_t)i * R + (size_t)wb * 32 + lane;
        a.h_out[idx] = hi;
        a.m[idx] = mi;
        if (OPT != FEM_OPT_SGD) a.v[idx] = vi;
        a.mag_out[idx] = tanhf(0.5f * hi);
        const uint32_t ball = __ballot_sync(kFullMask, hi < 0.f);
        if (lane == 0) a.words_out[(size_t)i * wpn + wb] = ball;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[b]);
    }
  }
  __syncthreads();
  if (threadIdx.x == kConsumers * 32) {
    // the last fills of both stages have landed before the block's shared memory is
    // released (after an abort the consumers may not have waited for them)
    for (long long k = issued - kStages < 0 ? 0 : issued - kStages; k < issued; ++k)
      mbar_wait(&full[k % kStages], (uint32_t)((k / kStages) & 1), a.err);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// The [n][R] fp32 marginals as a 2D map whose box is one row of 32 replicas (the
// gather4 form wants boxes one row high).
fem_status mag_map(CUtensorMap* m, const float* base, int32_t n, int32_t R) {
  auto enc = encode_fn();
  if (!enc) return fail(FEM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[2] = {(cuuint64_t)R, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)R * sizeof(float)};
  const cuuint32_t box[2] = {32, 1};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(FEM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return FEM_OK;
}

template <int OPT, bool UNIT, bool R32, bool OFF>
fem_status launch(const CUtensorMap& tm, const GatherArgs& a, const StepScalars& s, int sm_count, cudaStream_t st) {
  constexpr auto k = k_exact_gather<OPT, UNIT, R32, OFF>;
  static int grid_per_sm = 0;
  const size_t smem = kStages * sizeof(Stage) + 1024;
  if (grid_per_sm == 0) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&grid_per_sm, k, kThreads, smem) != cudaSuccess ||
        grid_per_sm < 1) {
      cudaGetLastError();
      grid_per_sm = 0;
      return fail(FEM_ERR_CUDA, "exact-mode gather kernel: no resident block");
    }
  }
  const long long tiles = (long long)((a.n + kNodes - 1) / kNodes) * a.wpn;
  long long grid = (long long)grid_per_sm * sm_count;
  if (grid > tiles) grid = tiles;
  k<<<(int)(grid < 1 ? 1 : grid), kThreads, smem, st>>>(tm, a, s);
  return FEM_OK;
}

template <bool R32, bool OFF>
fem_status dispatch(const Problem* p, const CUtensorMap& tm, const GatherArgs& a, const StepScalars& s,
                    cudaStream_t st) {
  const bool unit = p->unit_w;
  switch (p->optimizer) {
    case FEM_OPT_ADAM: return unit ? launch<FEM_OPT_ADAM, true, R32, OFF>(tm, a, s, p->sm_count, st)
                                   : launch<FEM_OPT_ADAM, false, R32, OFF>(tm, a, s, p->sm_count, st);
    case FEM_OPT_RMSPROP: return unit ? launch<FEM_OPT_RMSPROP, true, R32, OFF>(tm, a, s, p->sm_count, st)
                                      : launch<FEM_OPT_RMSPROP, false, R32, OFF>(tm, a, s, p->sm_count, st);
    default: return unit ? launch<FEM_OPT_SGD, true, R32, OFF>(tm, a, s, p->sm_count, st)
                         : launch<FEM_OPT_SGD, false, R32, OFF>(tm, a, s, p->sm_count, st);
  }
}

}  // namespace

// One exact-mode step of a sparse MaxCut / QUBO problem reading p->h[in] and
// p->mag[in], writing p->h[in ^ 1], p->mag[in ^ 1] and p->words[in ^ 1].
fem_status maxcut_exact_gather_step(Problem* p, int in, const StepScalars& s, cudaStream_t st) {
  if (p->tmap_mag_for[in] != p->mag[in] || p->tmap_mag_R != p->R) {
    for (int b = 0; b < 2; ++b) {
      const fem_status e = mag_map(&p->tmap_mag[b], p->mag[b], p->n, p->R);
      if (e != FEM_OK) return e;
      p->tmap_mag_for[b] = p->mag[b];
    }
    p->tmap_mag_R = p->R;
  }
  GatherArgs a{};
  a.row_ptr = p->row_ptr;
  a.col = p->col;
  a.w = p->unit_w ? nullptr : p->w;
  a.n = p->n;
  a.R = p->R;
  a.wpn = p->words_per_node;
  a.h_in = p->h[in];
  a.h_out = p->h[in ^ 1];
  a.m = p->m;
  a.v = p->v;
  a.mag_in = p->mag[in];
  a.mag_out = p->mag[in ^ 1];
  a.words_out = p->words[in ^ 1];
  a.ccoef = p->qubo ? 1.f : 2.f;
  a.offset = p->qubo ? p->qoff : nullptr;
  a.err = p->err;
  const CUtensorMap& tm = p->tmap_mag[in];
  // R = 32 runs the compile-time replica form, except for QUBO problems (per-node offsets),
  // which measured faster in the run-time form (n = 2^20: 0.3133 ms in the R = 32 form
  // with its offsets at compile time, 0.2983 ms in the run-time form)
  if (p->qubo) return dispatch<false, true>(p, tm, a, s, st);
  return p->R == 32 ? dispatch<true, false>(p, tm, a, s, st) : dispatch<false, false>(p, tm, a, s, st);
}

}  // namespace fem
