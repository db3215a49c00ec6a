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
  const float* jwo;        // p-spin with 3-spin terms: J_v of each occurrence's term (with oth)
  const float* lin;        // p-spin: fields b_i
  int32_t n, R, opt;
  float* h;
  float* m;
  float* v;
  const float* P_in;
  float* P_out;
};

// sigmoid with the fast exponential and reciprocal (relative error ~1e-6)
__device__ __forceinline__ float sigmoidf_fast(float x) { return div_approx(1.f, 1.f + exp_approx(-x)); }

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

// The same update for 3-literal clauses or 3-spin terms with four replicas per thread
// (R % 4 == 0): the thread of element e (a multiple of 4) updates replicas r..r+3 of
// variable i with float4 loads of the state and of both other literals' marginals, so
// the occurrence table, the address arithmetic and the literal decoding are paid once
// per four replicas.  Max-3-SAT: a factor P or 1 - P is fma(+-1, P, 0 or 1), which
// rounds exactly as either; p-spin (PSPIN): the factors are the mean spins m and each
// occurrence carries its term's J.  The products and the sum over occurrences run in
// the order of sat_element, so both give the same bits.  Occurrences are taken U at a
// time: their other-literal pairs, then all 2U marginal gathers, then the arithmetic
// (U = 2 where registers are scarce).
__device__ __forceinline__ bool sat_k3_shape(const SatArgs& a) {
  return a.oth && a.R % 4 == 0 && (!a.jw || a.jwo);
}

__device__ __forceinline__ float4 ld_f4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st_f4(float* p, const float4& x) { *reinterpret_cast<float4*>(p) = x; }

// The streaming state (h, m, v: read once and written once per step) with the
// evict-first cache hint when STREAM, so that it displaces less of the gathered mean
// spins in L2; measured faster for the 3-spin step and slower for Max-3-SAT, which
// keeps plain accesses.
template <bool STREAM>
__device__ __forceinline__ float4 ld_state(const float* p) {
  if constexpr (STREAM) return __ldcs(reinterpret_cast<const float4*>(p));
  else return ld_f4(p);
}
template <bool STREAM>
__device__ __forceinline__ void st_state(float* p, const float4& x) {
  if constexpr (STREAM) __stcs(reinterpret_cast<float4*>(p), x);
  else st_f4(p, x);
}

template <bool PSPIN>
__device__ __forceinline__ float sat_factor(int lit, float p) {
  if (PSPIN) return p;
  return fmaf((lit & 1) ? 1.f : -1.f, p, (lit & 1) ? 0.f : 1.f);  // negated literal: P, else 1 - P
}

// RC: the replica count as a compile-time constant (0: a.R at run time).
template <int U, bool PSPIN, int RC = 0>
__device__ __forceinline__ void sat_element_k3(const SatArgs& a, const StepScalars& s, long long e) {
  const int R = RC ? RC : a.R;
  int i, r;
  split_element(e, R, i, r);
  const bool sgd = a.opt == FEM_OPT_SGD;
  float4 h = ld_state<PSPIN>(a.h + e), m = ld_state<PSPIN>(a.m + e);
  float4 v = sgd ? make_float4(0.f, 0.f, 0.f, 0.f) : ld_state<PSPIN>(a.v + e);
  const int ob = a.occ_ptr[i], oe = a.occ_ptr[i + 1];
  const float* P = a.P_in + r;
  float G0 = 0.f, G1 = 0.f, G2 = 0.f, G3 = 0.f;
  for (int o = ob; o < oe; o += U) {
    int2 ot[U];
    float sg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      ot[u] = o + u < oe ? a.oth[o + u] : make_int2(0, 0);
      if (PSPIN) sg[u] = o + u < oe ? a.jwo[o + u] : 0.f;
    }
    float4 pa[U], pb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (o + u < oe) {
        pa[u] = ld_f4(P + (size_t)(((uint32_t)ot[u].x & 0x7fffffffu) >> 1) * R);
        pb[u] = ld_f4(P + (size_t)((uint32_t)ot[u].y >> 1) * R);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (o + u < oe) {
        if (!PSPIN) sg[u] = ot[u].x < 0 ? -1.f : 1.f;  // the own literal's negation
        G0 = fmaf(sg[u], sat_factor<PSPIN>(ot[u].x, pa[u].x) * sat_factor<PSPIN>(ot[u].y, pb[u].x), G0);
        G1 = fmaf(sg[u], sat_factor<PSPIN>(ot[u].x, pa[u].y) * sat_factor<PSPIN>(ot[u].y, pb[u].y), G1);
        G2 = fmaf(sg[u], sat_factor<PSPIN>(ot[u].x, pa[u].z) * sat_factor<PSPIN>(ot[u].y, pb[u].z), G2);
        G3 = fmaf(sg[u], sat_factor<PSPIN>(ot[u].x, pa[u].w) * sat_factor<PSPIN>(ot[u].y, pb[u].w), G3);
      }
    }
  }
  float* hv = &h.x;
  float* mv = &m.x;
  float* vv = &v.x;
  const float Gs[4] = {G0, G1, G2, G3};
  const float lin = PSPIN ? a.lin[i] : 0.f;
  float4 pout;
  float* pv = &pout.x;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float hi = hv[c], mi = mv[c], vi = vv[c];
    const float g = PSPIN ? s.gq * fmaf(2.f, Gs[c] + lin, hi * s.inv_beta) * one_minus_m2_fast(hi)
                          : s.gq * (hi * s.inv_beta - Gs[c]) * one_minus_m2_fast(hi);
    opt_update_fast_rt(a.opt, hi, mi, vi, g, s);
    hv[c] = hi;
    mv[c] = mi;
    vv[c] = vi;
    pv[c] = PSPIN ? tanhf(0.5f * hi) : sigmoidf_fast(hi);
  }
  st_state<PSPIN>(a.h + e, h);
  st_state<PSPIN>(a.m + e, m);
  if (!sgd) st_state<PSPIN>(a.v + e, v);
  st_f4(a.P_out + e, pout);
}

}  // namespace fem
