// Dense couplings from the caller to the device: one copy of the n x n fp32 matrix,
// then, on the device,
//   1. its validation: every entry an integer with |J_ij| <= 127 (exact in bf16 and
//      int8), a zero diagonal, symmetry; the lowest offending (i, j) in row-major
//      order is reported with the message of the first check it fails;
//   2. the operands the kernels read: the n_pad x n_pad fp32, bf16, e4m3 and int8
//      copies (zero padding), the row normalisations c_i = 1 / sum_j |J_ij| (SM, after
//      Eq. maxcut_modified_gradient), the sum of the couplings above the diagonal, and
//      whether every |J_ij| <= 16 (then e4m3 holds them exactly).
// The sums are of integers, so they are exact in any order.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <cmath>

#include "fem_internal.h"

namespace fem {
namespace {

// The first check entry (i, j) fails: 1 not an integer with |x| <= 127, 2 nonzero
// diagonal, 3 differs from its transpose (checked for j > i); 0 when it passes.
__device__ __host__ inline int dense_defect(float x, float xt, int i, int j) {
  if (!(fabsf(x) <= 127.f) || x != rintf(x)) return 1;
  if (i == j && x != 0.f) return 2;
  if (j > i && x != xt) return 3;
  return 0;
}

__global__ void k_dense_check(const float* __restrict__ J, int32_t n, unsigned long long* __restrict__ first_bad) {
  const long long total = (long long)n * n;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (long long)i * n);
    const float x = J[e];
    const float xt = j > i ? J[(long long)j * n + i] : x;
    if (dense_defect(x, xt, i, j)) atomicMin(first_bad, (unsigned long long)e);
  }
}

__global__ void k_dense_convert(const float* __restrict__ J, int32_t n, int32_t np, float* __restrict__ J32,
                                uint16_t* __restrict__ J16, uint8_t* __restrict__ J8, int8_t* __restrict__ Ji8) {
  const long long total = (long long)np * np;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / np), j = (int)(e - (long long)i * np);
    const float x = i < n && j < n ? J[(long long)i * n + j] : 0.f;
    J32[e] = x;
    J16[e] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
    J8[e] = (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
    Ji8[e] = (int8_t)x;
  }
}

// One warp per row: c_i, the couplings above the diagonal, and |J_ij| > 16 anywhere.
__global__ void k_dense_rows(const float* __restrict__ J, int32_t n, float* __restrict__ cn,
                             unsigned long long* __restrict__ wtot, int32_t* __restrict__ over16) {
  const int lane = threadIdx.x & 31;
  for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((long long)gridDim.x * blockDim.x) >> 5) {
    long long ra = 0, up = 0;
    bool big = false;
    for (int j = lane; j < n; j += 32) {
      const float x = J[i * n + j];
      const long long xi = (long long)x;  // an integer with |x| <= 127 (validated)
      ra += xi < 0 ? -xi : xi;
      if (j > i) up += xi;
      big = big || fabsf(x) > 16.f;
    }
    for (int off = 16; off > 0; off >>= 1) {
      ra += __shfl_xor_sync(0xffffffffu, ra, off);
      up += __shfl_xor_sync(0xffffffffu, up, off);
    }
    big = __any_sync(0xffffffffu, big);
    if (lane == 0) {
      cn[i] = ra > 0 ? (float)(1.0 / (double)ra) : 0.f;
      if (up != 0) atomicAdd(wtot, (unsigned long long)up);
      if (big) atomicOr(over16, 1);
    }
  }
}

int grid_of(long long work, int sm_count) {
  long long b = (work + 255) / 256;
  const long long cap = (long long)sm_count * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

fem_status dense_build(Problem* p, const float* J, cudaStream_t s) {
  const int n = p->n, np = p->n_pad;
  const size_t nn = (size_t)n * n, pp = (size_t)np * np;
  float* Jd = nullptr;
  unsigned long long* res = nullptr;  // first bad entry, sum above the diagonal, |J| > 16 flag
  cudaError_t e = cudaMallocAsync((void**)&Jd, nn * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&res, 3 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (Jd) cudaFreeAsync(Jd, s);
    return fail(FEM_ERR_OOM, "dense couplings: %zu bytes of staging", nn * sizeof(float));
  }
  auto release = [&]() {
    cudaFreeAsync(Jd, s);
    cudaFreeAsync(res, s);
  };
  unsigned long long h[3] = {0, 0, 0};
  e = cudaMemcpyAsync(Jd, J, nn * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(res, 0, 3 * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(res, 0xff, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    k_dense_check<<<grid_of((long long)nn, p->sm_count), 256, 0, s>>>(Jd, n, res);
    count_launches(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "dense couplings: validation");
  }
  if (h[0] != ~0ull) {
    release();
    const int i = (int)(h[0] / (unsigned long long)n), j = (int)(h[0] % (unsigned long long)n);
    const float x = J[(size_t)i * n + j];
    const int why = dense_defect(x, j > i ? J[(size_t)j * n + i] : x, i, j);
    if (why == 1) return fail(FEM_ERR_INVALID_ARG, "dense_J[%d][%d] must be an integer with |J| <= 127", i, j);
    if (why == 2) return fail(FEM_ERR_INVALID_ARG, "dense_J must have a zero diagonal");
    return fail(FEM_ERR_INVALID_ARG, "dense_J must be symmetric");
  }
  fem_status st;
  if ((st = dev_alloc_t(p, &p->J32, pp)) != FEM_OK || (st = dev_alloc(p, &p->J16, pp * 2)) != FEM_OK ||
      (st = dev_alloc(p, &p->J8, pp)) != FEM_OK || (st = dev_alloc(p, (void**)&p->Ji8, pp)) != FEM_OK ||
      (st = dev_alloc_t(p, &p->rowabs, (size_t)np)) != FEM_OK) {
    release();
    return st;
  }
  e = cudaMemsetAsync(p->rowabs, 0, (size_t)np * sizeof(float), s);
  if (e == cudaSuccess) {
    k_dense_convert<<<grid_of((long long)pp, p->sm_count), 256, 0, s>>>(
        Jd, n, np, p->J32, reinterpret_cast<uint16_t*>(p->J16), reinterpret_cast<uint8_t*>(p->J8), p->Ji8);
    k_dense_rows<<<grid_of((long long)n * 32, p->sm_count), 256, 0, s>>>(Jd, n, p->rowabs, res + 1,
                                                                       reinterpret_cast<int32_t*>(res + 2));
    count_launches(2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s);
  release();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "dense couplings: conversion");
  p->dense_wtot = (int64_t)h[1];
  p->dense_fp8_ok = (h[2] & 0xffffffffull) == 0;
  return FEM_OK;
}

}  // namespace fem
