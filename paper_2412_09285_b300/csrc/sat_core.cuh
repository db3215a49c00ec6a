// Per-element Max-k-SAT step (shared by the single-problem and batched kernels).
// See sat.cu for the method and the data layout.
#pragma once

#include "fem_internal.h"
#include "step_common.cuh"

namespace fem {

struct SatArgs {
  const int32_t* cl_ptr;   // [M+1]
  const int32_t* cl_lit;   // [n_occ]: (var << 1) | negated
  const int32_t* occ_ptr;  // [n+1]
  const int32_t* occ;      // [n_occ]: (clause << 3) | position
  const int2* oth;         // [n_occ] or NULL: 3-SAT, the other two literals (own negation in bit 31)
  const float* jw;         // p-spin: term coefficients J_v (NULL: Max-k-SAT)
  const float* lin;        // p-spin: fields b_i
  int32_t n, R, opt;
  float* h;
  float* m;
  float* v;
  const float* P_in;
  float* P_out;
};

// sigmoid with the fast exponential and reciprocal (relative error ~1e-6)
__device__ __forceinline__ float sigmoidf_fast(float x) { return __fdividef(1.f, 1.f + __expf(-x)); }

// The update of element e = i*R + r (variable i, replica r) of one step.
// p-spin (a.jw != NULL, SM multi-variable interactions): the marginal buffers hold
// m = tanh(h/2), a term's factor for spin k is m_k, and
//   g_i = gamma (1 - m_i^2)/4 [2 (sum_{v ni i} J_v prod_{k in v, k != i} m_k + b_i) + h_i/beta].
__device__ __forceinline__ void sat_element(const SatArgs& a, const StepScalars& s, long long e) {
  {
    int i, r;
    split_element(e, a.R, i, r);
    float hi = a.h[e], mi = a.m[e];
    float vi = a.opt == FEM_OPT_SGD ? 0.f : a.v[e];
    const bool pspin = a.jw != nullptr;
    float G = 0.f;
    const int ob = a.occ_ptr[i], oe = a.occ_ptr[i + 1];
    for (int o = ob; o < oe; ++o) {
      const int x = a.occ[o];
      const int c = x >> 3, pos = x & 7;
      const int cb = a.cl_ptr[c], ce = a.cl_ptr[c + 1];
      float prod = 1.f;
      float sgn = 1.f;
      for (int b = cb; b < ce; ++b) {
        const int lit = a.cl_lit[b];
        if (b - cb == pos) {
          sgn = (lit & 1) ? -1.f : 1.f;
          continue;
        }
        const float pk = a.P_in[(size_t)(lit >> 1) * a.R + r];
        prod *= pspin ? pk : ((lit & 1) ? pk : 1.f - pk);
      }
      G = fmaf(pspin ? a.jw[c] : sgn, prod, G);
    }
    const float g = pspin ? s.gq * fmaf(2.f, G + a.lin[i], hi * s.inv_beta) * one_minus_m2_fast(hi)
                          : s.gq * (hi * s.inv_beta - G) * one_minus_m2_fast(hi);
    opt_update_fast_rt(a.opt, hi, mi, vi, g, s);
    a.h[e] = hi;
    a.m[e] = mi;
    if (a.opt != FEM_OPT_SGD) a.v[e] = vi;
    a.P_out[e] = pspin ? tanhf(0.5f * hi) : sigmoidf_fast(hi);
  }
}

// The same update for 3-SAT, a warp at a time (all 32 lanes call it together; lanes
// with act == false contribute nothing).  The G = min(R, 32) lanes of a variable
// (R == 16 or R % 32 == 0) load G occurrences' other-literal pairs at once, then
// issue the marginal gathers of 8 occurrences before using any of them, so a
// variable waits for a few memory round trips instead of four per occurrence.  The
// products and the sum over occurrences run in the order of sat_element, so both
// give the same bits.
__device__ __forceinline__ bool sat_k3_shape(const SatArgs& a) {
  return a.oth && !a.jw && (a.R == 16 || a.R % 32 == 0);
}

__device__ __forceinline__ void sat_element_k3(const SatArgs& a, const StepScalars& s, long long e, bool act,
                                               int lane) {
  const int G = a.R >= 32 ? 32 : 16;
  const bool sgd = a.opt == FEM_OPT_SGD;
  int i = 0, r = 0, ob = 0, nocc = 0;
  float hi = 0.f, mi = 0.f, vi = 0.f;
  if (act) {
    split_element(e, a.R, i, r);
    hi = a.h[e];
    mi = a.m[e];
    vi = sgd ? 0.f : a.v[e];
    ob = a.occ_ptr[i];
    nocc = a.occ_ptr[i + 1] - ob;
  }
  int maxocc = nocc;
  if (G == 16) maxocc = max(maxocc, __shfl_xor_sync(kFullMask, maxocc, 16));
  const int sub = lane & (G - 1), gbase = lane & ~(G - 1);
  float Gs = 0.f;
  for (int j0 = 0; j0 < maxocc; j0 += G) {
    int2 ot = make_int2(0, 0);
    if (j0 + sub < nocc) ot = a.oth[ob + j0 + sub];
    const int cnt = min(max(nocc - j0, 0), G), lim = min(maxocc - j0, G);
    for (int jb = 0; jb < lim; jb += 8) {
      int la[8], lb[8];
      float pa[8], pb[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int src = gbase + ((jb + u) & (G - 1));
        la[u] = __shfl_sync(kFullMask, ot.x, src);
        lb[u] = __shfl_sync(kFullMask, ot.y, src);
        const bool v = jb + u < cnt;
        pa[u] = v ? a.P_in[(size_t)(((uint32_t)la[u] & 0x7fffffffu) >> 1) * a.R + r] : 0.f;
        pb[u] = v ? a.P_in[(size_t)((uint32_t)lb[u] >> 1) * a.R + r] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (jb + u < cnt) {
          const float ua = (la[u] & 1) ? pa[u] : 1.f - pa[u];
          const float ub = (lb[u] & 1) ? pb[u] : 1.f - pb[u];
          Gs = fmaf(la[u] < 0 ? -1.f : 1.f, ua * ub, Gs);
        }
      }
    }
  }
  if (act) {
    const float g = s.gq * (hi * s.inv_beta - Gs) * one_minus_m2_fast(hi);
    opt_update_fast_rt(a.opt, hi, mi, vi, g, s);
    a.h[e] = hi;
    a.m[e] = mi;
    if (!sgd) a.v[e] = vi;
    a.P_out[e] = sigmoidf_fast(hi);
  }
}

}  // namespace fem
