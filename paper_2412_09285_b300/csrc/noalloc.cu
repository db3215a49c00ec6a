// Allocation-free cut evaluation: the MaxCut read-out (per-replica cut, energy
// and best replica) for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a memory-pool manager
// that owns all device memory, or a loop that must not allocate because an
// allocation can synchronise the device and stall other streams.  This entry
// point therefore takes every input and output from the caller and keeps its
// only scratch - the per-block partial sums - in a fixed file-scope device array.
// Each GPU that loads the library holds that array (2 MiB) until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "fem_internal.h"
#include "step_common.cuh"

namespace fem {
namespace {

constexpr int kNoallocBlocks = 256;        // partial-sum rows (grid size of the first kernel)
constexpr int kNoallocMaxReplicas = 1024;  // replicas per call
constexpr int kNoallocMaxDevices = 64;

// Partial cuts, [block][replica].  Every call overwrites the rows it reads, so
// nothing has to be cleared between calls; calls that overlap on the GPU race.
__device__ __align__(256) int64_t g_noalloc_partials[kNoallocBlocks * kNoallocMaxReplicas];
// Set by the first kernel when the CSR names a row range or a column outside the
// graph (the access is skipped); read and cleared by the second kernel, so it is
// zero again when the next call starts.
__device__ int32_t g_noalloc_bad;

std::mutex g_noalloc_mutex;
int64_t* g_noalloc_addr[kNoallocMaxDevices] = {};

// Host code cannot use the array's name as a device address: look the address
// up once per device, with that device current.
fem_status noalloc_scratch(int64_t** out) {
  int dev = 0;
  FEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(FEM_ERR_UNSUPPORTED, "device index %d too large", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_addr[dev] = static_cast<int64_t*>(p);
  }
  *out = g_noalloc_addr[dev];
  return FEM_OK;
}

// Same sum as the library's read-out: for every undirected edge (j > i in the
// CSR) with +-1 weight in bit 31 of col, add W_ij when the two sign bits differ.
__global__ void __launch_bounds__(256) k_noalloc_cut_partial(const int32_t* __restrict__ row_ptr,
                                                             const uint32_t* __restrict__ col,
                                                             const uint32_t* __restrict__ words,
                                                             int32_t n, int32_t R, int32_t wpn,
                                                             int64_t* __restrict__ part) {
  __shared__ int64_t s[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wb = blockIdx.y;
  int64_t acc = 0;
  const int nnz = row_ptr[n];
  for (int i = blockIdx.x * 8 + warp; i < n; i += gridDim.x * 8) {
    const uint32_t bi = (words[(size_t)i * wpn + wb] >> lane) & 1u;
    const int beg = row_ptr[i], end = row_ptr[i + 1];
    if (beg < 0 || end < beg || end > nnz) {   // a row outside col[0, row_ptr[n])
      if (lane == 0) g_noalloc_bad = 1;
      continue;
    }
    for (int k0 = beg; k0 < end; k0 += 32) {
      const int k = k0 + lane;
      uint32_t c = 0, wd = 0;
      bool bad = false;
      if (k < end) {
        c = col[k];
        const uint32_t j = c & 0x7fffffffu;
        if (j < (uint32_t)n) wd = words[(size_t)j * wpn + wb];
        else bad = true;
      }
      if (__any_sync(kFullMask, bad)) {       // a column outside the graph: skip the row
        if (lane == 0) g_noalloc_bad = 1;
        break;
      }
      const int cnt = min(32, end - k0);
      for (int e = 0; e < cnt; ++e) {
        const uint32_t ce = __shfl_sync(kFullMask, c, e);
        const uint32_t bj = (__shfl_sync(kFullMask, wd, e) >> lane) & 1u;
        if ((int)(ce & 0x7fffffffu) > i && bj != bi) acc += (ce >> 31) ? -1 : 1;
      }
    }
  }
  s[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    int64_t t = 0;
    for (int k = 0; k < 8; ++k) t += s[k][lane];
    part[(size_t)blockIdx.x * R + (size_t)wb * 32 + lane] = t;
  }
}

// E_r = -cut_r summed over the partial rows in order, then the argmin over
// replicas (lowest index on ties); best = -1 when the CSR was malformed.
__global__ void __launch_bounds__(1024) k_noalloc_finish(const int64_t* __restrict__ part, int32_t nblk,
                                                         int32_t R, int64_t* __restrict__ energy,
                                                         int32_t* __restrict__ best) {
  __shared__ int64_t sv[1024];
  __shared__ int si[1024];
  int64_t bv = 0;
  int bi = 0x7fffffff;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    int64_t t = 0;
    for (int b = 0; b < nblk; ++b) t += part[(size_t)b * R + r];
    energy[r] = -t;
    if (bi == 0x7fffffff || -t < bv) {
      bv = -t;
      bi = r;
    }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      const int oi = si[threadIdx.x + off], mi = si[threadIdx.x];
      const int64_t ov = sv[threadIdx.x + off];
      if (oi != 0x7fffffff && (mi == 0x7fffffff || ov < sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < mi))) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    best[0] = g_noalloc_bad ? -1 : si[0];
    g_noalloc_bad = 0;
  }
}

}  // namespace
}  // namespace fem

using namespace fem;

extern "C" fem_status fem_maxcut_energies_noalloc(const int32_t* row_ptr, const uint32_t* col, int32_t n,
                                                  const uint32_t* words, int32_t replicas,
                                                  int64_t* energy, int32_t* best_replica, void* stream) {
  if (!row_ptr || !col || !words || !energy || !best_replica || n < 1)
    return fail(FEM_ERR_INVALID_ARG, "all pointers must be non-NULL and n >= 1");
  if (replicas < 32 || replicas % 32 != 0)
    return fail(FEM_ERR_UNSUPPORTED, "replicas must be a positive multiple of 32");
  if (replicas > kNoallocMaxReplicas)
    return fail(FEM_ERR_UNSUPPORTED, "replicas (%d) exceeds the static scratch limit of %d", replicas,
                kNoallocMaxReplicas);
  int64_t* part = nullptr;
  fem_status st = noalloc_scratch(&part);
  if (st != FEM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int blocks = (n + 7) / 8;
  if (blocks > kNoallocBlocks) blocks = kNoallocBlocks;
  const int wpn = replicas / 32;
  k_noalloc_cut_partial<<<dim3(blocks, wpn), 256, 0, s>>>(row_ptr, col, words, n, replicas, wpn, part);
  k_noalloc_finish<<<1, 1024, 0, s>>>(part, blocks, replicas, energy, best_replica);
  count_launches(2);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}
