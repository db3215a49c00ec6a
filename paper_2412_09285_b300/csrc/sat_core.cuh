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
  int32_t n, R, opt;
  float* h;
  float* m;
  float* v;
  const float* P_in;
  float* P_out;
};

__device__ __forceinline__ float sigmoidf_acc(float x) { return 1.f / (1.f + expf(-x)); }

// The update of element e = i*R + r (variable i, replica r) of one step.
__device__ __forceinline__ void sat_element(const SatArgs& a, const StepScalars& s, long long e) {
  {
    const int i = (int)(e / a.R);
    const int r = (int)(e - (long long)i * a.R);
    float hi = a.h[e], mi = a.m[e];
    float vi = a.opt == FEM_OPT_SGD ? 0.f : a.v[e];
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
        prod *= (lit & 1) ? pk : 1.f - pk;
      }
      G = fmaf(sgn, prod, G);
    }
    const float g = s.gq * (hi * s.inv_beta - G) * one_minus_m2(hi);
    opt_update_rt(a.opt, hi, mi, vi, g, s);
    a.h[e] = hi;
    a.m[e] = mi;
    if (a.opt != FEM_OPT_SGD) a.v[e] = vi;
    a.P_out[e] = sigmoidf_acc(hi);
  }
}

}  // namespace fem
