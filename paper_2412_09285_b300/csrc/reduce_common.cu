// The argmin over replicas shared by the read-outs.
#include "reduce_common.cuh"

namespace fem {

__global__ void __launch_bounds__(1024) k_argmin_replica(const double* __restrict__ e_f, int32_t R,
                                                         int32_t* __restrict__ best) {
  __shared__ double sval[1024];
  __shared__ int sidx[1024];
  double bv = 0.0;
  int bi = 0x7fffffff;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double v = e_f[r];
    if (bi == 0x7fffffff || v < bv) {
      bv = v;
      bi = r;
    }
  }
  sval[threadIdx.x] = bv;
  sidx[threadIdx.x] = bi;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      const double ov = sval[threadIdx.x + off];
      const int oi = sidx[threadIdx.x + off], mi = sidx[threadIdx.x];
      if (oi != 0x7fffffff && (mi == 0x7fffffff || ov < sval[threadIdx.x] || (ov == sval[threadIdx.x] && oi < mi))) {
        sval[threadIdx.x] = ov;
        sidx[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) best[0] = sidx[0];
}

}  // namespace fem
