// Read-out reductions shared by the problem kinds: per-replica sums of per-block
// partials in a fixed order, and the argmin over replicas.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fem {

constexpr int kRedThreads = 256;  // block size of the per-replica reductions

// Sum of part[b * stride + col] over b in [0, nblk), by one block: thread t adds
// b = t, t + 256, ... in order, then a fixed tree over the threads.  Every run adds
// in the same order, so floating-point sums are reproducible.
template <typename T>
__device__ __forceinline__ T column_sum(const T* __restrict__ part, int nblk, size_t stride, size_t col,
                                        T* sh /* [kRedThreads] */) {
  T acc = T(0);
  for (int b = threadIdx.x; b < nblk; b += kRedThreads) acc += part[(size_t)b * stride + col];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int off = kRedThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  const T res = sh[0];
  __syncthreads();
  return res;
}

// best[0] = argmin_r e_f[r] over r in [0, R), the lowest index on ties (one block of
// 1024 threads).
__global__ void __launch_bounds__(1024) k_argmin_replica(const double* __restrict__ e_f, int32_t R,
                                                         int32_t* __restrict__ best);

}  // namespace fem
