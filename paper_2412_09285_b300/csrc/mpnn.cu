// Warm-start network for MaxCut FEM: forward, backward, Adam training step and
// inference, all on the GPU.  (Not from the paper: a learned initialisation of the
// local fields, judged against the plain random-initialised FEM.)
//
//   P = D^-1 W;  s_i = [1, deg_i/mean deg, sum_j W_ij / deg_i, 1/sqrt(deg_i + 1)]
//   x^0 = s;  a^l = P x^(l-1);  x^l = tanh(x^(l-1) A_l + a^l B_l + b_l),  l = 1..3, width 64
//   theta = x^3 C + c (4 taps);  u_0 = z, u_k = P u_(k-1);  y_ir = sum_k theta_ik u_k,ir
//   loss = mean_ir (tanh(y_ir/2) - tanh(h_ir/2))^2,  h = FEM's fields at the target step
//
// Weights: fp32 master copy (Adam state beside it) and a bf16 copy read by the
// forward kernels, which accumulate in fp32.  Activations are fp32.  Weight
// gradients are reduced over nodes per block and then summed over blocks in a fixed
// order (deterministic).  Buffers of one call are stream-ordered allocations.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fem_internal.h"
#include "reduce_common.cuh"
#include "step_common.cuh"

namespace fem {
namespace {

constexpr int kH = 64, kF0 = 4, kTaps = 4;
// parameter blocks (row-major), in the library's order
constexpr int kOffA1 = 0, kOffB1 = kOffA1 + kF0 * kH, kOffb1 = kOffB1 + kF0 * kH;
constexpr int kOffA2 = kOffb1 + kH, kOffB2 = kOffA2 + kH * kH, kOffb2 = kOffB2 + kH * kH;
constexpr int kOffA3 = kOffb2 + kH, kOffB3 = kOffA3 + kH * kH, kOffb3 = kOffB3 + kH * kH;
constexpr int kOffC = kOffb3 + kH, kOffc = kOffC + kH * kTaps, kNParams = kOffc + kTaps;
static_assert(kNParams == 17348, "parameter count");

__host__ __device__ constexpr int off_A(int l) { return l == 1 ? kOffA1 : (l == 2 ? kOffA2 : kOffA3); }
__host__ __device__ constexpr int off_B(int l) { return l == 1 ? kOffB1 : (l == 2 ? kOffB2 : kOffB3); }
__host__ __device__ constexpr int off_b(int l) { return l == 1 ? kOffb1 : (l == 2 ? kOffb2 : kOffb3); }

struct Graph {
  const int32_t* row_ptr;
  const uint32_t* col;
  const float* w;  // NULL: +-1 in bit 31 of col
  int32_t n;
};

__device__ __forceinline__ float edge_w(const Graph& g, int k, uint32_t c) {
  return g.w ? g.w[k] : ((c >> 31) ? -1.f : 1.f);
}

// Structural features s_i.
__global__ void k_feats(Graph g, float mean_deg, float* __restrict__ x0) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
    const int b = g.row_ptr[i], e = g.row_ptr[i + 1];
    float rs = 0.f;
    for (int k = b; k < e; ++k) rs += edge_w(g, k, g.col[k]);
    const float d = (float)(e - b);
    x0[i * kF0 + 0] = 1.f;
    x0[i * kF0 + 1] = d / mean_deg;
    x0[i * kF0 + 2] = d > 0.f ? rs / d : 0.f;
    x0[i * kF0 + 3] = rsqrtf(d + 1.f);
  }
}

// out = P X (transpose = 0) or P^T X = W D^-1 X (transpose = 1); X is [n][F].
// One warp per node; a lane holds two features (f and f + 32) of a 64-feature chunk.
// The node's column indices are loaded 32 at a time (one coalesced load) and eight
// neighbours' rows are gathered before any is added, so a warp waits for one memory
// round trip per eight neighbours; the sums keep the neighbour order.
constexpr int kSpmmGather = 8;

template <bool TRANSPOSE>
__global__ void __launch_bounds__(256) k_spmm(Graph g, const float* __restrict__ X, int F,
                                              float* __restrict__ out) {
  constexpr bool transpose = TRANSPOSE;
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < g.n; i += (gridDim.x * blockDim.x) >> 5) {
    const int b = g.row_ptr[i], e = g.row_ptr[i + 1];
    for (int f0 = 0; f0 < F; f0 += 64) {
      const int fa = f0 + lane, fb = f0 + 32 + lane;
      float acc_a = 0.f, acc_b = 0.f;
      for (int k0 = b; k0 < e; k0 += 32) {
        const int kk = k0 + lane;
        uint32_t c = 0;
        float wk = 0.f, dk = 1.f;
        if (kk < e) {
          c = g.col[kk];
          wk = edge_w(g, kk, c);
          if (transpose) {
            const int j = (int)(c & 0x7fffffffu);
            dk = (float)(g.row_ptr[j + 1] - g.row_ptr[j]);
          }
        }
        const int cnt = min(32, e - k0);
        for (int u0 = 0; u0 < cnt; u0 += kSpmmGather) {
          float xa[kSpmmGather], xb[kSpmmGather];
#pragma unroll
          for (int u = 0; u < kSpmmGather; ++u) {
            const int j = (int)(__shfl_sync(kFullMask, c, u0 + u) & 0x7fffffffu);
            const bool ok = u0 + u < cnt;
            xa[u] = ok && fa < F ? X[(size_t)j * F + fa] : 0.f;
            xb[u] = ok && fb < F ? X[(size_t)j * F + fb] : 0.f;
          }
#pragma unroll
          for (int u = 0; u < kSpmmGather; ++u) {
            if (u0 + u < cnt) {
              const float w = __shfl_sync(kFullMask, wk, u0 + u);
              float x1 = xa[u], x2 = xb[u];
              if (transpose) {
                const float dj = __shfl_sync(kFullMask, dk, u0 + u);
                x1 = dj > 0.f ? x1 / dj : 0.f;
                x2 = dj > 0.f ? x2 / dj : 0.f;
              }
              acc_a = fmaf(w, x1, acc_a);
              acc_b = fmaf(w, x2, acc_b);
            }
          }
        }
      }
      if (!transpose) {
        acc_a = (e > b) ? acc_a / (float)(e - b) : 0.f;
        acc_b = (e > b) ? acc_b / (float)(e - b) : 0.f;
      }
      if (fa < F) out[(size_t)i * F + fa] = acc_a;
      if (fb < F) out[(size_t)i * F + fb] = acc_b;
    }
  }
}

// x_out = tanh(x_in A + a B + b): 32 nodes per block; thread = (4 consecutive outputs,
// 2 nodes 16 apart), so every shared-memory load of the weights (float4) and of the
// inputs (broadcast) feeds 4 or 8 multiply-adds.
__global__ void __launch_bounds__(256) k_layer_fwd(const float* __restrict__ x_in, const float* __restrict__ a,
                                                   int n, int din, const __nv_bfloat16* __restrict__ wts, int l,
                                                   float* __restrict__ x_out) {
  __shared__ __align__(16) float sA[kH * kH], sB[kH * kH];
  __shared__ float sx[32][kH], sa[32][kH];
  for (int t = threadIdx.x; t < din * kH; t += blockDim.x) {
    sA[t] = __bfloat162float(wts[off_A(l) + t]);
    sB[t] = __bfloat162float(wts[off_B(l) + t]);
  }
  const int o4 = (threadIdx.x & 15) * 4, ng = threadIdx.x >> 4;
  float bo[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) bo[c] = __bfloat162float(wts[off_b(l) + o4 + c]);
  for (int i0 = blockIdx.x * 32; i0 < n; i0 += gridDim.x * 32) {
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * din; t += blockDim.x) {
      const int r = t / din, p = t % din, i = i0 + r;
      sx[r][p] = i < n ? x_in[(size_t)i * din + p] : 0.f;
      sa[r][p] = i < n ? a[(size_t)i * din + p] : 0.f;
    }
    __syncthreads();
    float acc[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[h][c] = bo[c];
    for (int p = 0; p < din; ++p) {
      const float4 wa = *reinterpret_cast<const float4*>(&sA[p * kH + o4]);
      const float4 wb = *reinterpret_cast<const float4*>(&sB[p * kH + o4]);
      const float wav[4] = {wa.x, wa.y, wa.z, wa.w}, wbv[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float xv = sx[ng + 16 * h][p], av = sa[ng + 16 * h][p];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[h][c] = fmaf(xv, wav[c], fmaf(av, wbv[c], acc[h][c]));
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + ng + 16 * h;
      if (i < n) {
        float4 y;
        y.x = tanhf(acc[h][0]);
        y.y = tanhf(acc[h][1]);
        y.z = tanhf(acc[h][2]);
        y.w = tanhf(acc[h][3]);
        *reinterpret_cast<float4*>(&x_out[(size_t)i * kH + o4]) = y;
      }
    }
  }
}

// theta = x3 C + c (4 taps per node).
__global__ void k_head(const float* __restrict__ x3, int n, const __nv_bfloat16* __restrict__ wts,
                       float* __restrict__ theta) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * kTaps; e += gridDim.x * blockDim.x) {
    const int i = e / kTaps, k = e % kTaps;
    float acc = __bfloat162float(wts[kOffc + k]);
    for (int p = 0; p < kH; ++p) acc = fmaf(x3[(size_t)i * kH + p], __bfloat162float(wts[kOffC + p * kTaps + k]), acc);
    theta[e] = acc;
  }
}

// y_ir = sum_k theta_ik u_k,ir; optionally the loss terms, dL/dy and dtheta_ik =
// sum_r dy_ir u_k,ir.  Warp per node, lanes over replicas.  u is [kTaps][n][R].
__global__ void k_predict(const float* __restrict__ theta, const float* __restrict__ u, int n, int R,
                          const float* __restrict__ m_t, float inv_count, float* __restrict__ y,
                          float* __restrict__ dtheta, float* __restrict__ loss_node) {
  const int lane = threadIdx.x & 31;
  const size_t nR = (size_t)n * R;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
    float th[kTaps], dth[kTaps] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < kTaps; ++k) th[k] = theta[i * kTaps + k];
    float ls = 0.f;
    for (int r0 = 0; r0 < R; r0 += 32) {
      const int r = r0 + lane;
      if (r >= R) continue;
      const size_t e = (size_t)i * R + r;
      float uk[kTaps], yy = 0.f;
#pragma unroll
      for (int k = 0; k < kTaps; ++k) {
        uk[k] = u[k * nR + e];
        yy = fmaf(th[k], uk[k], yy);
      }
      if (y) y[e] = yy;
      if (m_t) {
        const float t = tanhf(0.5f * yy), d = t - tanhf(0.5f * m_t[e]);  // m_t holds target fields
        ls = fmaf(d, d, ls);
        const float dy = d * (1.f - t * t) * inv_count;  // 2 (t - m) * (1 - t^2)/2 / count
#pragma unroll
        for (int k = 0; k < kTaps; ++k) dth[k] = fmaf(dy, uk[k], dth[k]);
      }
    }
    if (m_t) {
#pragma unroll
      for (int k = 0; k < kTaps; ++k)
        for (int off = 16; off > 0; off >>= 1) dth[k] += __shfl_xor_sync(kFullMask, dth[k], off);
      for (int off = 16; off > 0; off >>= 1) ls += __shfl_xor_sync(kFullMask, ls, off);
      if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kTaps; ++k) dtheta[i * kTaps + k] = dth[k];
        loss_node[i] = ls;
      }
    }
  }
}

// dx3 = dtheta C^T (per node, 64 outputs).
__global__ void k_head_bwd_dx(const float* __restrict__ dtheta, int n, const __nv_bfloat16* __restrict__ wts,
                              float* __restrict__ dx) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)n * kH; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / kH;
    const int p = (int)(e % kH);
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < kTaps; ++k) acc = fmaf(dtheta[i * kTaps + k], __bfloat162float(wts[kOffC + p * kTaps + k]), acc);
    dx[e] = acc;
  }
}

// dpre = dx * (1 - x_out^2), in place in dx.
__global__ void k_tanh_bwd(float* __restrict__ dx, const float* __restrict__ x_out, size_t total) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    dx[e] *= 1.f - x_out[e] * x_out[e];
}

// Per-block partial of G[p][o] = sum_i U[i][p] V[i][o] (U: [n][P], V: [n][O]),
// written to part[block][P*O].  Thread t owns entries t, t + 256, ...
__global__ void __launch_bounds__(256) k_outer_partial(const float* __restrict__ U, int Pd,
                                                       const float* __restrict__ V, int Od, int n, int chunk,
                                                       float* __restrict__ part) {
  __shared__ float su[16][kH], sv[16][kH];
  float acc[16];
  const int PO = Pd * Od;
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.f;
  const int i_begin = blockIdx.x * chunk, i_end = min(n, i_begin + chunk);
  for (int i0 = i_begin; i0 < i_end; i0 += 16) {
    __syncthreads();
    for (int t = threadIdx.x; t < 16 * kH; t += blockDim.x) {
      const int r = t / kH, c = t % kH, i = i0 + r;
      su[r][c] = (i < i_end && c < Pd) ? U[(size_t)i * Pd + c] : 0.f;
      sv[r][c] = (i < i_end && c < Od) ? V[(size_t)i * Od + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int idx = threadIdx.x + q * 256;
      if (idx < PO) {
        const int p = idx / Od, o = idx % Od;
        float s = acc[q];
        for (int r = 0; r < 16; ++r) s = fmaf(su[r][p], sv[r][o], s);
        acc[q] = s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int idx = threadIdx.x + q * 256;
    if (idx < PO) part[(size_t)blockIdx.x * PO + idx] = acc[q];
  }
}

// Column sums (bias gradients) per block: part[block][O] = sum_i V[i][o].
__global__ void k_colsum_partial(const float* __restrict__ V, int Od, int n, int chunk, float* __restrict__ part) {
  const int o = threadIdx.x;
  if (o >= Od) return;
  const int i_begin = blockIdx.x * chunk, i_end = min(n, i_begin + chunk);
  float s = 0.f;
  for (int i = i_begin; i < i_end; ++i) s += V[(size_t)i * Od + o];
  part[(size_t)blockIdx.x * Od + o] = s;
}

// grad[off + e] = sum over blocks (in order) of part[block][e].
__global__ void k_reduce_blocks(const float* __restrict__ part, int nblk, int size, float* __restrict__ grad, int off) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < size; e += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * size + e];
    grad[off + e] = s;
  }
}

// dx_in = dpre A^T (+ accumulate == 0) and da = dpre B^T, per node.
__global__ void __launch_bounds__(256) k_layer_bwd_dx(const float* __restrict__ dpre, int n, int din,
                                                      const __nv_bfloat16* __restrict__ wts, int l,
                                                      float* __restrict__ dx_in, float* __restrict__ da) {
  __shared__ float sA[kH * kH], sB[kH * kH];
  __shared__ float sd[32][kH];
  for (int t = threadIdx.x; t < din * kH; t += blockDim.x) {
    sA[t] = __bfloat162float(wts[off_A(l) + t]);
    sB[t] = __bfloat162float(wts[off_B(l) + t]);
  }
  const int p = threadIdx.x & (kH - 1), ng = threadIdx.x >> 6;
  for (int i0 = blockIdx.x * 32; i0 < n; i0 += gridDim.x * 32) {
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * kH; t += blockDim.x) {
      const int r = t / kH, o = t % kH, i = i0 + r;
      sd[r][o] = i < n ? dpre[(size_t)i * kH + o] : 0.f;
    }
    __syncthreads();
    if (p < din) {
      for (int r = ng; r < 32; r += 4) {
        float ax = 0.f, aa = 0.f;
        for (int o = 0; o < kH; ++o) {
          ax = fmaf(sd[r][o], sA[p * kH + o], ax);
          aa = fmaf(sd[r][o], sB[p * kH + o], aa);
        }
        if (i0 + r < n) {
          dx_in[(size_t)(i0 + r) * din + p] = ax;
          da[(size_t)(i0 + r) * din + p] = aa;
        }
      }
    }
  }
}

__global__ void k_add(float* __restrict__ x, const float* __restrict__ y, size_t total) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    x[e] += y[e];
}

// Adam on the fp32 master weights, then the bf16 copy.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, int size, float lr_t,
                       float b1, float b2, float inv_sqrt_bc2, float eps) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < size; e += gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = fmaf(b1, m[e], (1.f - b1) * gg);
    const float vv = fmaf(b2, v[e], (1.f - b2) * gg * gg);
    m[e] = mm;
    v[e] = vv;
    const float ww = w[e] - lr_t * mm / (sqrtf(vv) * inv_sqrt_bc2 + eps);
    w[e] = ww;
    wb[e] = __float2bfloat16_rn(ww);
  }
}

__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int size) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < size; e += gridDim.x * blockDim.x)
    wb[e] = __float2bfloat16_rn(w[e]);
}

// Per-replica sums of squares of y ([n][R]) over row chunks: part[b][r] (fp64).
constexpr int kRmsRows = 512;
__global__ void k_col_sumsq_partial(const float* __restrict__ y, int n, int R, double* __restrict__ part) {
  const int i0 = blockIdx.x * kRmsRows, i1 = min(n, i0 + kRmsRows);
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double acc = 0.0;
    for (int i = i0; i < i1; ++i) {
      const double v = y[(size_t)i * R + r];
      acc += v * v;
    }
    part[(size_t)blockIdx.x * R + r] = acc;
  }
}

// scale[r] = rms / sqrt(mean_i y_ir^2) (0 for an all-zero column); one block per replica.
__global__ void __launch_bounds__(kRedThreads) k_col_scale(const double* __restrict__ part, int nblk, int n, int R,
                                                           float rms, float* __restrict__ scale) {
  __shared__ double sh[kRedThreads];
  const int r = blockIdx.x;
  const double ss = column_sum<double>(part, nblk, R, r, sh);
  if (threadIdx.x == 0) scale[r] = ss > 0.0 ? (float)(rms / sqrt(ss / n)) : 0.f;
}

__global__ void k_scale_cols(float* __restrict__ y, size_t total, int R, const float* __restrict__ scale) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x)
    y[e] *= scale[e % R];
}

}  // namespace

struct Mpnn {
  float* w = nullptr;  // fp32 master
  float* m = nullptr;
  float* v = nullptr;
  float* g = nullptr;
  __nv_bfloat16* wb = nullptr;
  int64_t steps = 0;
  int sm_count = 148;
  // workspace of a call's activations, grown to the largest call so far (a call that
  // needs more takes stream-ordered allocations for the rest, and the next call finds
  // the workspace grown); calls on one network must not overlap on the GPU
  uint8_t* arena = nullptr;
  size_t arena_cap = 0;
};

namespace {

int blocks_for(size_t work, int sm_count, int per = 8) {
  size_t b = (work + 255) / 256;
  const size_t cap = (size_t)sm_count * per;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

struct Pass {
  // forward activations
  float *x[4] = {nullptr, nullptr, nullptr, nullptr}, *a[4] = {nullptr, nullptr, nullptr, nullptr};
  float *theta = nullptr, *u = nullptr, *dtheta = nullptr, *loss_node = nullptr;
  // backward scratch
  float *dx = nullptr, *dx_in = nullptr, *da = nullptr, *tmp = nullptr, *part = nullptr;
  Mpnn* net = nullptr;
  size_t used = 0;  // bytes of the network's workspace handed out in this call
  std::vector<void*> mine;
};

fem_status pass_alloc(Pass& ps, void** p, size_t bytes, cudaStream_t s) {
  const size_t need = (bytes + 255) & ~(size_t)255;
  if (ps.net && ps.used + need <= ps.net->arena_cap) {
    *p = ps.net->arena + ps.used;
  } else {
    FEM_CUDA(cudaMallocAsync(p, bytes, s));
    ps.mine.push_back(*p);
  }
  ps.used += need;
  return FEM_OK;
}

void pass_free(Pass& ps, cudaStream_t s) {
  for (void* p : ps.mine) cudaFreeAsync(p, s);
  ps.mine.clear();
  // grow the workspace to this call's size for the next call (cudaFree waits for the
  // device, so no queued kernel still reads the old one)
  if (ps.net && ps.used > ps.net->arena_cap) {
    if (ps.net->arena) cudaFree(ps.net->arena);
    ps.net->arena = nullptr;
    ps.net->arena_cap = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, ps.used) == cudaSuccess) {
      ps.net->arena = (uint8_t*)p;
      ps.net->arena_cap = ps.used;
    } else {
      cudaGetLastError();  // without a workspace the next call allocates again
    }
  }
}

// Forward pass; with m_t also the loss terms and dL/dtheta.
fem_status forward(const Mpnn* net, const Problem* pr, const float* z, int R, const float* m_t, float* y_out,
                   Pass& ps, cudaStream_t s) {
  const Graph g{pr->row_ptr, pr->col, pr->unit_w ? nullptr : pr->w, pr->n};
  const int n = pr->n;
  const int sm = net->sm_count;
  fem_status st;
  if ((st = pass_alloc(ps, (void**)&ps.x[0], (size_t)n * kF0 * 4, s)) != FEM_OK) return st;
  for (int l = 1; l <= 3; ++l) {
    if ((st = pass_alloc(ps, (void**)&ps.a[l], (size_t)n * (l == 1 ? kF0 : kH) * 4, s)) != FEM_OK) return st;
    if ((st = pass_alloc(ps, (void**)&ps.x[l], (size_t)n * kH * 4, s)) != FEM_OK) return st;
  }
  if ((st = pass_alloc(ps, (void**)&ps.theta, (size_t)n * kTaps * 4, s)) != FEM_OK) return st;
  if ((st = pass_alloc(ps, (void**)&ps.u, (size_t)kTaps * n * R * 4, s)) != FEM_OK) return st;
  const float mean_deg = n > 0 ? (float)((double)pr->nnz / n) : 1.f;
  const int wb_nodes = blocks_for((size_t)n * 32, sm);
  k_feats<<<blocks_for(n, sm), 256, 0, s>>>(g, mean_deg > 0.f ? mean_deg : 1.f, ps.x[0]);
  for (int l = 1; l <= 3; ++l) {
    const int din = l == 1 ? kF0 : kH;
    k_spmm<false><<<wb_nodes, 256, 0, s>>>(g, ps.x[l - 1], din, ps.a[l]);
    k_layer_fwd<<<blocks_for((size_t)n * 8, sm), 256, 0, s>>>(ps.x[l - 1], ps.a[l], n, din, net->wb, l, ps.x[l]);
  }
  k_head<<<blocks_for((size_t)n * kTaps, sm), 256, 0, s>>>(ps.x[3], n, net->wb, ps.theta);
  FEM_CUDA(cudaMemcpyAsync(ps.u, z, (size_t)n * R * 4, cudaMemcpyDeviceToDevice, s));
  for (int k = 1; k < kTaps; ++k)
    k_spmm<false><<<wb_nodes, 256, 0, s>>>(g, ps.u + (size_t)(k - 1) * n * R, R, ps.u + (size_t)k * n * R);
  if (m_t) {
    if ((st = pass_alloc(ps, (void**)&ps.dtheta, (size_t)n * kTaps * 4, s)) != FEM_OK) return st;
    if ((st = pass_alloc(ps, (void**)&ps.loss_node, (size_t)n * 4, s)) != FEM_OK) return st;
  }
  k_predict<<<wb_nodes, 256, 0, s>>>(ps.theta, ps.u, n, R, m_t, 1.f / ((float)n * (float)R), y_out, ps.dtheta,
                                     ps.loss_node);
  count_launches(2 + 6 + (kTaps - 1) + 1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

// Backward pass into net->g (all parameters).  Requires forward(..., m_t).
fem_status backward(Mpnn* net, const Problem* pr, Pass& ps, cudaStream_t s) {
  const Graph g{pr->row_ptr, pr->col, pr->unit_w ? nullptr : pr->w, pr->n};
  const int n = pr->n, sm = net->sm_count;
  const int chunk = 256;
  const int nblk = (n + chunk - 1) / chunk;
  fem_status st;
  if ((st = pass_alloc(ps, (void**)&ps.dx, (size_t)n * kH * 4, s)) != FEM_OK) return st;
  if ((st = pass_alloc(ps, (void**)&ps.dx_in, (size_t)n * kH * 4, s)) != FEM_OK) return st;
  if ((st = pass_alloc(ps, (void**)&ps.da, (size_t)n * kH * 4, s)) != FEM_OK) return st;
  if ((st = pass_alloc(ps, (void**)&ps.tmp, (size_t)n * kH * 4, s)) != FEM_OK) return st;
  if ((st = pass_alloc(ps, (void**)&ps.part, (size_t)nblk * kH * kH * 4, s)) != FEM_OK) return st;
  int launches = 0;
  // head: dC = x3^T dtheta, dc = colsum dtheta, dx3 = dtheta C^T
  k_outer_partial<<<nblk, 256, 0, s>>>(ps.x[3], kH, ps.dtheta, kTaps, n, chunk, ps.part);
  k_reduce_blocks<<<blocks_for(kH * kTaps, sm), 256, 0, s>>>(ps.part, nblk, kH * kTaps, net->g, kOffC);
  k_colsum_partial<<<nblk, 64, 0, s>>>(ps.dtheta, kTaps, n, chunk, ps.part);
  k_reduce_blocks<<<1, 256, 0, s>>>(ps.part, nblk, kTaps, net->g, kOffc);
  k_head_bwd_dx<<<blocks_for((size_t)n * kH, sm), 256, 0, s>>>(ps.dtheta, n, net->wb, ps.dx);
  launches += 5;
  for (int l = 3; l >= 1; --l) {
    const int din = l == 1 ? kF0 : kH;
    k_tanh_bwd<<<blocks_for((size_t)n * kH, sm), 256, 0, s>>>(ps.dx, ps.x[l], (size_t)n * kH);
    k_outer_partial<<<nblk, 256, 0, s>>>(ps.x[l - 1], din, ps.dx, kH, n, chunk, ps.part);
    k_reduce_blocks<<<blocks_for(din * kH, sm), 256, 0, s>>>(ps.part, nblk, din * kH, net->g, off_A(l));
    k_outer_partial<<<nblk, 256, 0, s>>>(ps.a[l], din, ps.dx, kH, n, chunk, ps.part);
    k_reduce_blocks<<<blocks_for(din * kH, sm), 256, 0, s>>>(ps.part, nblk, din * kH, net->g, off_B(l));
    k_colsum_partial<<<nblk, 64, 0, s>>>(ps.dx, kH, n, chunk, ps.part);
    k_reduce_blocks<<<1, 256, 0, s>>>(ps.part, nblk, kH, net->g, off_b(l));
    launches += 7;
    if (l > 1) {
      k_layer_bwd_dx<<<blocks_for((size_t)n * 8, sm), 256, 0, s>>>(ps.dx, n, din, net->wb, l, ps.dx_in, ps.da);
      k_spmm<true><<<blocks_for((size_t)n * 32, sm), 256, 0, s>>>(g, ps.da, din, ps.tmp);
      k_add<<<blocks_for((size_t)n * din, sm), 256, 0, s>>>(ps.dx_in, ps.tmp, (size_t)n * din);
      std::swap(ps.dx, ps.dx_in);
      launches += 3;
    }
  }
  count_launches(launches);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

fem_status read_loss(const Pass& ps, int n, int R, double* loss, cudaStream_t s) {
  if (!loss) return FEM_OK;
  std::vector<float> ln(n);
  FEM_CUDA(cudaMemcpyAsync(ln.data(), ps.loss_node, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  double t = 0.0;
  for (float x : ln) t += x;
  *loss = t / ((double)n * R);
  return FEM_OK;
}

}  // namespace
}  // namespace fem

struct fem_mpnn : public fem::Mpnn {};

using namespace fem;

extern "C" {

int32_t fem_mpnn_num_params(void) { return kNParams; }

fem_status fem_mpnn_create(const float* params, fem_mpnn_t* out) {
  if (!params || !out) return fail(FEM_ERR_INVALID_ARG, "params and out must be non-NULL");
  *out = nullptr;
  fem_mpnn* net = new fem_mpnn();
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&net->sm_count, cudaDevAttrMultiProcessorCount, dev);
  const size_t b = kNParams * sizeof(float);
  cudaError_t e = cudaMalloc((void**)&net->w, b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&net->m, b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&net->v, b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&net->g, b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&net->wb, kNParams * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemcpy(net->w, params, b, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(net->m, 0, b);
  if (e == cudaSuccess) e = cudaMemset(net->v, 0, b);
  if (e == cudaSuccess) {
    k_to_bf16<<<(kNParams + 255) / 256, 256>>>(net->w, net->wb, kNParams);
    count_launches(1);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    fem_mpnn_destroy(net);
    return cuda_fail(e, "fem_mpnn_create");
  }
  *out = net;
  return FEM_OK;
}

void fem_mpnn_destroy(fem_mpnn_t net) {
  if (!net) return;
  cudaFree(net->w);
  cudaFree(net->m);
  cudaFree(net->v);
  cudaFree(net->g);
  cudaFree(net->wb);
  cudaFree(net->arena);
  delete net;
}

fem_status fem_mpnn_get_params(fem_mpnn_t net, float* params) {
  if (!net || !params) return fail(FEM_ERR_INVALID_ARG, "net and params must be non-NULL");
  FEM_CUDA(cudaMemcpy(params, net->w, kNParams * sizeof(float), cudaMemcpyDeviceToHost));
  return FEM_OK;
}

static fem_status mpnn_check(fem_mpnn_t net, fem_problem_t g, const float* z, int32_t R) {
  if (!net || !g || !z) return fail(FEM_ERR_INVALID_ARG, "net, graph and z must be non-NULL");
  if (g->kind != FEM_MAXCUT || g->dense) return fail(FEM_ERR_UNSUPPORTED, "the network runs on sparse MaxCut graphs");
  if (R < 1) return fail(FEM_ERR_INVALID_ARG, "replicas must be >= 1");
  return FEM_OK;
}

fem_status fem_mpnn_predict(fem_mpnn_t net, fem_problem_t g, const float* z, int32_t R, float rms, float* y,
                            void* stream) {
  fem_status st = mpnn_check(net, g, z, R);
  if (st != FEM_OK) return st;
  if (!y) return fail(FEM_ERR_INVALID_ARG, "y must be non-NULL");
  if (!(rms >= 0.f)) return fail(FEM_ERR_INVALID_ARG, "rms must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  Pass ps;
  ps.net = net;
  st = forward(net, g, z, R, nullptr, y, ps, s);
  if (st == FEM_OK && rms > 0.f) {
    const int n = g->n, nblk = (n + kRmsRows - 1) / kRmsRows;
    double* part = nullptr;
    float* scale = nullptr;
    if ((st = pass_alloc(ps, (void**)&part, (size_t)nblk * R * sizeof(double), s)) == FEM_OK &&
        (st = pass_alloc(ps, (void**)&scale, (size_t)R * sizeof(float), s)) == FEM_OK) {
      k_col_sumsq_partial<<<nblk, 256, 0, s>>>(y, n, R, part);
      k_col_scale<<<R, kRedThreads, 0, s>>>(part, nblk, n, R, rms, scale);
      k_scale_cols<<<blocks_for((size_t)n * R, net->sm_count), 256, 0, s>>>(y, (size_t)n * R, R, scale);
      count_launches(3);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_fail(e, "fem_mpnn_predict normalisation");
    }
  }
  pass_free(ps, s);
  return st;
}

fem_status fem_mpnn_grad(fem_mpnn_t net, fem_problem_t g, const float* z, const float* m_t, int32_t R,
                         float* grad, double* loss, void* stream) {
  fem_status st = mpnn_check(net, g, z, R);
  if (st != FEM_OK) return st;
  if (!m_t) return fail(FEM_ERR_INVALID_ARG, "h_target must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  Pass ps;
  ps.net = net;
  st = forward(net, g, z, R, m_t, nullptr, ps, s);
  if (st == FEM_OK) st = backward(net, g, ps, s);
  if (st == FEM_OK) st = read_loss(ps, g->n, R, loss, s);
  if (st == FEM_OK && grad) {
    const cudaError_t e = cudaMemcpyAsync(grad, net->g, kNParams * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_fail(e, "fem_mpnn_grad copy");
  }
  pass_free(ps, s);
  if (st == FEM_OK) FEM_CUDA(cudaStreamSynchronize(s));
  return st;
}

fem_status fem_mpnn_train_step(fem_mpnn_t net, fem_problem_t g, const float* z, const float* m_t, int32_t R,
                               double lr, double* loss, void* stream) {
  fem_status st = fem_mpnn_grad(net, g, z, m_t, R, nullptr, loss, stream);
  if (st != FEM_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  net->steps += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float lr_t = (float)(lr / (1.0 - std::pow(b1, (double)net->steps)));
  const float isb = (float)(1.0 / std::sqrt(1.0 - std::pow(b2, (double)net->steps)));
  k_adam<<<(kNParams + 255) / 256, 256, 0, s>>>(net->w, net->m, net->v, net->g, net->wb, kNParams, lr_t, (float)b1,
                                               (float)b2, isb, 1e-8f);
  count_launches(1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

}  // extern "C"
