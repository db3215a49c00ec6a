// Device helpers shared by the step kernels: the optimizer updates and the
// single-field marginal algebra.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "fem_internal.h"

namespace fem {

constexpr unsigned kFullMask = 0xffffffffu;

// One optimizer update of one field with PyTorch's semantics (Methods,
// "Hyperparameter tunning": the paper uses torch.optim's Adam, RMSprop and SGD).
//   Adam:    m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
//            h -= lr/(1-b1^t) * m / (sqrt(v)/sqrt(1-b2^t) + eps)
//   RMSprop: v = a v + (1-a) g^2;  avg = sqrt(v) + eps;
//            momentum mu > 0: buf = mu buf + g/avg, h -= lr buf;  else h -= lr g/avg
//   SGD:     momentum mu != 0: buf = g (first step) or mu buf + (1-d) g;  h -= lr buf
// The L2 weight decay adds wd*h to g first.  `m` doubles as the momentum buffer
// of RMSprop and SGD.  Every multiply-add is an explicit fmaf, so the rounding does
// not depend on how the compiler contracts the surrounding kernel's code (kernels
// that must agree bit for bit share these sequences).
template <int OPT>
__device__ __forceinline__ void opt_update(float& h, float& m, float& v, float g,
                                           const StepScalars& s) {
  if (s.wd != 0.f) g = fmaf(s.wd, h, g);
  if (OPT == FEM_OPT_ADAM) {
    m = fmaf(s.b1, m, s.omb1 * g);
    v = fmaf(s.b2, v, s.omb2 * g * g);
    const float denom = fmaf(sqrtf(v), s.inv_sqrt_bc2, s.eps);
    h = fmaf(-s.lr, m / denom, h);
  } else if (OPT == FEM_OPT_RMSPROP) {
    v = fmaf(s.b1, v, s.omb1 * g * g);
    const float avg = sqrtf(v) + s.eps;
    if (s.momentum > 0.f) {
      m = fmaf(s.momentum, m, g / avg);
      h = fmaf(-s.lr, m, h);
    } else {
      h = fmaf(-s.lr, g / avg, h);
    }
  } else {
    if (s.b1 != 0.f) {
      m = s.first ? g : fmaf(s.b1, m, s.omb1 * g);
      g = m;
    }
    h = fmaf(-s.lr, g, h);
  }
}

// The approximate operations of the step kernels.  Each takes one hardware instruction
// in its .ftz form (denormal input and result flushed to zero; the plain forms wrap the
// instruction in denormal handling, which costs kernels bound by instruction issue), and
// never on a value whose denormals matter: a quotient multiplies its numerator, which
// keeps IEEE denormals, by the reciprocal of a normal divisor, so a denormal gradient
// still moves a denormal field, and its sign, as in exact arithmetic.  The products are
// __fmul_rn, which the compiler never contracts into a neighbouring add, so kernels
// that share these sequences round alike.
// Square root (PTX sqrt.approx, a few ulp); a denormal argument gives 0 (callers add
// eps to it).
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// 1 / b (PTX rcp.approx, 1 ulp) for |b| in [2^-126, 2^126]; 0 above that range.
__device__ __forceinline__ float rcp_approx(float b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
  return r;
}
// a / b as a times rcp_approx(b) (2 ulp); above the range it gives 0, where |a / b| is below
// 2^-126 for every caller here anyway.
__device__ __forceinline__ float div_approx(float a, float b) { return __fmul_rn(a, rcp_approx(b)); }
// e^x by the identity e^x = 2^(x log2 e) on the approximate base-2 exponential (PTX
// ex2.approx): relative error about 2^-22 + |x| 2^-24, the second term from rounding
// the product; 0 for x below about -87.3 (results under 2^-126).
__device__ __forceinline__ float exp_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__fmul_rn(x, 1.4426950408889634f)));
  return y;
}
// ln x = log2(x) ln 2 on the approximate base-2 logarithm (PTX lg2.approx), x normal.
__device__ __forceinline__ float log_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return __fmul_rn(y, 0.6931471805599453f);
}

// The same updates with approximate divisions and square roots (div_approx,
// sqrt_approx); the divisors here are >= eps and far below 2^126.
// opt_update_fast_core is the update of a gradient that already includes wd*h
// (callers that must not branch per element add it with an fmaf, which leaves g
// unchanged when wd == 0).
template <int OPT>
__device__ __forceinline__ void opt_update_fast_core(float& h, float& m, float& v, float g,
                                                     const StepScalars& s) {
  if (OPT == FEM_OPT_ADAM) {
    m = fmaf(s.b1, m, s.omb1 * g);
    v = fmaf(s.b2, v, s.omb2 * g * g);
    h = fmaf(-s.lr, div_approx(m, fmaf(sqrt_approx(v), s.inv_sqrt_bc2, s.eps)), h);
  } else if (OPT == FEM_OPT_RMSPROP) {
    v = fmaf(s.b1, v, s.omb1 * g * g);
    const float q = div_approx(g, sqrt_approx(v) + s.eps);
    if (s.momentum > 0.f) {
      m = fmaf(s.momentum, m, q);
      h = fmaf(-s.lr, m, h);
    } else {
      h = fmaf(-s.lr, q, h);
    }
  } else {
    if (s.b1 != 0.f) {
      m = s.first ? g : fmaf(s.b1, m, s.omb1 * g);
      g = m;
    }
    h = fmaf(-s.lr, g, h);
  }
}

template <int OPT>
__device__ __forceinline__ void opt_update_fast(float& h, float& m, float& v, float g,
                                                const StepScalars& s) {
  if (s.wd != 0.f) g = fmaf(s.wd, h, g);
  opt_update_fast_core<OPT>(h, m, v, g, s);
}

// Calls f(OPT) with the run-time optimizer as a compile-time constant: one
// warp-uniform branch around a whole block of updates, so their arithmetic can
// interleave instead of being split by a branch per update.
template <class F>
__device__ __forceinline__ void with_opt(int opt, F&& f) {
  if (opt == FEM_OPT_ADAM) f(std::integral_constant<int, FEM_OPT_ADAM>{});
  else if (opt == FEM_OPT_RMSPROP) f(std::integral_constant<int, FEM_OPT_RMSPROP>{});
  else f(std::integral_constant<int, FEM_OPT_SGD>{});
}

// Transpose of a 32 x 32 bit matrix held one row per lane (lane e holds row e):
// afterwards lane r holds column r, i.e. bit e of the result is bit r of row e.
// Five butterfly stages exchange blocks of 16, 8, 4, 2 and 1 bits.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int j = 16 >> s;
    const uint32_t m = masks[s];
    const uint32_t y = __shfl_xor_sync(kFullMask, x, j);
    x = (lane & j) ? (((y >> j) & m) | (x & ~m)) : ((x & m) | ((y << j) & ~m));
  }
  return x;
}

// Element index e = i*R + r -> (i, r); 32-bit division whenever e < 2^32.
__device__ __forceinline__ void split_element(long long e, int R, int& i, int& r) {
  if ((unsigned long long)e < 4294967296ull) {
    const uint32_t el = (uint32_t)e, ii = el / (uint32_t)R;
    i = (int)ii;
    r = (int)(el - ii * (uint32_t)R);
  } else {
    i = (int)(e / R);
    r = (int)(e - (long long)i * R);
  }
}

// 1 - tanh(h/2)^2 with the fast exponential (relative error ~1e-6).
__device__ __forceinline__ float one_minus_m2_fast(float h) {
  const float e = exp_approx(-fabsf(h));
  const float d = 1.f + e;
  return div_approx(4.f * e, d * d);
}

// The same update with the optimizer chosen at run time (a warp-uniform branch).
__device__ __forceinline__ void opt_update_rt(int opt, float& h, float& m, float& v, float g,
                                              const StepScalars& s) {
  if (opt == FEM_OPT_ADAM) opt_update<FEM_OPT_ADAM>(h, m, v, g, s);
  else if (opt == FEM_OPT_RMSPROP) opt_update<FEM_OPT_RMSPROP>(h, m, v, g, s);
  else opt_update<FEM_OPT_SGD>(h, m, v, g, s);
}

// opt_update_fast with the optimizer chosen at run time (a warp-uniform branch).
__device__ __forceinline__ void opt_update_fast_rt(int opt, float& h, float& m, float& v, float g,
                                                   const StepScalars& s) {
  if (opt == FEM_OPT_ADAM) opt_update_fast<FEM_OPT_ADAM>(h, m, v, g, s);
  else if (opt == FEM_OPT_RMSPROP) opt_update_fast<FEM_OPT_RMSPROP>(h, m, v, g, s);
  else opt_update_fast<FEM_OPT_SGD>(h, m, v, g, s);
}

// 1 - m^2 for m = tanh(h/2) = 2 sigmoid(h) - 1, evaluated as 4e/(1+e)^2 with
// e = exp(-|h|) so that it keeps full relative accuracy when |m| -> 1.
__device__ __forceinline__ float one_minus_m2(float h) {
  const float e = expf(-fabsf(h));
  const float d = 1.f + e;
  return 4.f * e / (d * d);
}

}  // namespace fem
