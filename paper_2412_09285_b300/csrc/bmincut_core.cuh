// Per-element bMinCut step (shared by the single-problem and batched kernels).
// See bmincut_sparse.cu for the method and the data layout.
#pragma once

#include "fem_internal.h"
#include "step_common.cuh"

namespace fem {

template <int Q>
struct QBits {
  static constexpr int B = Q <= 2 ? 1 : (Q <= 4 ? 2 : 4);
  static constexpr int RPW = 32 / B;  // replicas per word
  static constexpr uint32_t MASK = (1u << B) - 1u;
};

constexpr float kPsumScale = 4294967296.0f;         // 2^32
constexpr float kPsumInv = 2.3283064365386963e-10f;  // 2^-32

struct BmcArgs {
  const int32_t* row_ptr;
  const uint32_t* col;
  const float* w;  // NULL for unit weights
  const float* cf;
  const float* ca;
  const int32_t* nodew;  // node weights V_i, NULL: all 1
  float cw;              // coupling coefficient: bMinCut -2 (exact) / -1 (paper, times c^f); colouring +1
  float lam_scale;       // 1 for bMinCut, 0 for colouring (no balance term)
  int32_t n, R, wpn, opt;
  const float* h_in;
  float* h_out;
  float* m;
  float* v;
  const float* d_in;  // exact mode: q (P_j(s) - 1/q) of the fields h_in, [n][R][q]
  float* d_out;       // exact mode: the same of the updated fields, gathered by the next step
  const uint32_t* words_in;
  uint32_t* words_out;
  const int32_t* cnt_in;
  int32_t* cnt_out;
  int32_t* cnt_zero;
  const unsigned long long* ps_in;
  unsigned long long* ps_out;
  unsigned long long* ps_zero;
};

// Softmax with the fast exponential and reciprocal (relative error ~1e-6; Z >= 1).
template <int Q>
__device__ __forceinline__ void softmax_q(const float (&h)[Q], float (&P)[Q], float (&lnP)[Q]) {
  float mx = h[0];
#pragma unroll
  for (int s = 1; s < Q; ++s) mx = fmaxf(mx, h[s]);
  float ex[Q], Z = 0.f;
#pragma unroll
  for (int s = 0; s < Q; ++s) {
    ex[s] = exp_approx(h[s] - mx);
    Z += ex[s];
  }
  const float invZ = div_approx(1.f, Z), lz = log_approx(Z);
#pragma unroll
  for (int s = 0; s < Q; ++s) {
    P[s] = ex[s] * invZ;
    lnP[s] = h[s] - mx - lz;
  }
}

// q (P(s) - 1/q) of the softmax of h.  With u(s) = expm1(h(s) - max h) and
// Z = sum_s exp(h(s) - max h) = q + sum_s u(s), it equals (q u(s) - sum_s' u(s')) / Z.
// u is accurate relative to |h(s) - max h|, so near a uniform P, where those gaps are
// as small as the differences h(s) - h(s'), the result keeps full relative accuracy
// (P - 1/q formed in fp32 would not); q expm1 per element instead of q^2.
template <int Q>
__device__ __forceinline__ void centred_q(const float (&h)[Q], float (&d)[Q]) {
  float mx = h[0];
#pragma unroll
  for (int q = 1; q < Q; ++q) mx = fmaxf(mx, h[q]);
  float u[Q], su = 0.f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    u[q] = expm1f(h[q] - mx);
    su += u[q];
  }
  const float invZ = div_approx(1.f, (float)Q + su);  // Z in [1, q]
#pragma unroll
  for (int q = 0; q < Q; ++q) d[q] = fmaf((float)Q, u[q], -su) * invZ;
}

template <int Q>
__device__ __forceinline__ int argmax_q(const float (&h)[Q]) {
  int best = 0;
  float bv = h[0];
#pragma unroll
  for (int s = 1; s < Q; ++s)
    if (h[s] > bv) {
      bv = h[s];
      best = s;
    }
  return best;
}

// A node-replica's q fields are contiguous ([n][R][q]), so q = 8 and q = 4 start on
// 16-byte boundaries and q = 6 and q = 2 on 8-byte ones.
template <int Q>
__device__ __forceinline__ void load_q(const float* p, float (&x)[Q]) {
  if constexpr (Q % 4 == 0) {
#pragma unroll
    for (int s = 0; s < Q; s += 4) {
      const float4 t = *reinterpret_cast<const float4*>(p + s);
      x[s] = t.x; x[s + 1] = t.y; x[s + 2] = t.z; x[s + 3] = t.w;
    }
  } else if constexpr (Q % 2 == 0) {
#pragma unroll
    for (int s = 0; s < Q; s += 2) {
      const float2 t = *reinterpret_cast<const float2*>(p + s);
      x[s] = t.x; x[s + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int s = 0; s < Q; ++s) x[s] = p[s];
  }
}

template <int Q>
__device__ __forceinline__ void store_q(float* p, const float (&x)[Q]) {
  if constexpr (Q % 4 == 0) {
#pragma unroll
    for (int s = 0; s < Q; s += 4)
      *reinterpret_cast<float4*>(p + s) = make_float4(x[s], x[s + 1], x[s + 2], x[s + 3]);
  } else if constexpr (Q % 2 == 0) {
#pragma unroll
    for (int s = 0; s < Q; s += 2) *reinterpret_cast<float2*>(p + s) = make_float2(x[s], x[s + 1]);
  } else {
#pragma unroll
    for (int s = 0; s < Q; ++s) p[s] = x[s];
  }
}

// The update of element e = i*R + r (node i, replica r) of one step: marginals,
// neighbour contraction, centred gradient, optimizer, argmax word and the block's
// shared-memory counts (scnt / sps, [R][Q]).  All 32 lanes of the warp must call it
// together (word packing shuffles); lanes with act == false contribute nothing.
// RC: the replica count as a compile-time constant (0: a.R at run time), for
// immediate offsets and shifts instead of run-time multiplies and divisions.
template <int Q, int MODE, int RC = 0>
__device__ __forceinline__ void bmincut_element(const BmcArgs& a, const StepScalars& s, long long e,
                                                bool act, int lane, int32_t* scnt,
                                                unsigned long long* sps) {
  constexpr int B = QBits<Q>::B, RPW = QBits<Q>::RPW;
  const int R = RC ? RC : a.R, wpn = RC ? RC * B / 32 : a.wpn;
  constexpr uint32_t SM = QBits<Q>::MASK;
  {
    int i = 0, r = 0;
    if (act) split_element(e, R, i, r);
    const int wsel = r / RPW, sh = (r % RPW) * B;
    float h[Q], mm[Q], vv[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) h[q] = mm[q] = vv[q] = 0.f;
    const size_t idx = ((size_t)i * R + r) * Q;
    float acc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) acc[q] = 0.f;
    int own = 0, Vi = 1;
    float cf = 0.f, ca = 0.f;
    int beg = 0, end = 0;
    // Paper mode, unit weights, one packed word per node (R * B == 32: q = 2 with
    // R = 32, q = 3, 4 with R = 16): the lanes of a node load up to R neighbours'
    // words at once, a warp bit-transpose turns them into bit planes, and popcounts
    // give the per-state counts (warp-uniform condition; every lane takes part).
    const bool planes = MODE == FEM_GRAD_PAPER && B <= 2 && !a.w && R * B == 32;
    // q = 5..8 (4 bits per replica) with R = 16: two packed words per node, one bit-plane
    // pass per word
    const bool planes4 = MODE == FEM_GRAD_PAPER && B == 4 && !a.w && R == 16;
    if (act) {
      load_q<Q>(a.h_in + idx, h);
      load_q<Q>(a.m + idx, mm);
      if (a.opt != FEM_OPT_SGD) load_q<Q>(a.v + idx, vv);
      beg = a.row_ptr[i];
      end = a.row_ptr[i + 1];
      if (a.nodew) Vi = a.nodew[i];
      if (MODE == FEM_GRAD_PAPER) {
        own = (int)((a.words_in[(size_t)i * wpn + wsel] >> sh) & SM);
        cf = a.cf[i];
        ca = a.ca[i];
      }
    }
    if (MODE == FEM_GRAD_PAPER && planes) {
      const int G = R;  // lanes per node: 16 or 32
      const int deg = end - beg, sub = lane & (G - 1);
      int maxdeg = deg;
      if (G == 16) maxdeg = max(maxdeg, __shfl_xor_sync(kFullMask, maxdeg, 16));
      uint32_t c[4] = {0u, 0u, 0u, 0u};
      for (int k0 = 0; k0 < maxdeg; k0 += G) {
        const int kk = k0 + sub;
        uint32_t w = 0u;
        if (kk < deg) w = a.words_in[a.col[beg + kk] & 0x7fffffffu];
        const uint32_t t = warp_transpose32(w, lane);  // lane b: bit e = bit b of lane e's word
        const int nv = min(max(deg - k0, 0), G);
        const uint32_t vm = (nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u)) << (lane & ~(G - 1));
        if (B == 1) {
          c[1] += __popc(t & vm);
          c[0] += __popc(~t & vm);
        } else {
          const uint32_t lo = __shfl_sync(kFullMask, t, 2 * sub), hi = __shfl_sync(kFullMask, t, 2 * sub + 1);
          c[0] += __popc(~lo & ~hi & vm);
          c[1] += __popc(lo & ~hi & vm);
          c[2] += __popc(~lo & hi & vm);
          c[3] += __popc(lo & hi & vm);
        }
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[q] = (float)c[q < 4 ? q : 0];
    } else if (MODE == FEM_GRAD_PAPER && B == 4 && planes4) {
      // Lanes 0-15 and 16-31 are two nodes; lane sub holds replica sub, whose state sits
      // in bits 4(sub % 8) .. of word sub / 8.  Each pass loads one word of up to 16
      // neighbours per node, transposes, and the lanes whose replicas live in that word
      // count their neighbours per state from three bit planes (states < 8).
      const int deg = end - beg, sub = lane & 15;
      const int maxdeg = max(deg, __shfl_xor_sync(kFullMask, deg, 16));
      const int myw = sub >> 3, base = (sub & 7) * 4;
      uint32_t c8[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) c8[q] = 0u;
      for (int k0 = 0; k0 < maxdeg; k0 += 16) {
        const int kk = k0 + sub;
        const bool have = kk < deg;
        const uint32_t j = have ? (a.col[beg + kk] & 0x7fffffffu) : 0u;
        const int nv = min(max(deg - k0, 0), 16);
        const uint32_t vm = (nv >= 16 ? 0xffffu : ((1u << nv) - 1u)) << (lane & 16);
#pragma unroll
        for (int w = 0; w < 2; ++w) {
          const uint32_t word = have ? a.words_in[(size_t)j * 2 + w] : 0u;
          const uint32_t t = warp_transpose32(word, lane);  // lane b: bit e = bit b of lane e's word
          const uint32_t p0 = __shfl_sync(kFullMask, t, base);
          const uint32_t p1 = __shfl_sync(kFullMask, t, base + 1);
          const uint32_t p2 = __shfl_sync(kFullMask, t, base + 2);
          if (myw == w) {
#pragma unroll
            for (int q = 0; q < Q; ++q)
              c8[q] += __popc(((q & 1) ? p0 : ~p0) & ((q & 2) ? p1 : ~p1) & ((q & 4) ? p2 : ~p2) & vm);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) acc[q] = (float)c8[q];
    } else if (MODE == FEM_GRAD_EXACT || act) {
      // in exact mode every lane takes this branch (its sums shuffle within the warp); an
      // inactive lane has beg == end, so its loops add nothing
      if (MODE == FEM_GRAD_PAPER) {
        if (!a.w && end - beg < (Q <= 4 ? 65536 : 256)) {
          // unit weights: integer counts packed 16 (q <= 4) or 8 bits wide in one word,
          // the same exact sums as the float path below
          constexpr int F = Q <= 4 ? 16 : 8;
          unsigned long long pk = 0ull;
          for (int k = beg; k < end; ++k) {
            const uint32_t j = a.col[k] & 0x7fffffffu;
            const uint32_t sj = (a.words_in[(size_t)j * wpn + wsel] >> sh) & SM;
            pk += 1ull << (F * sj);
          }
#pragma unroll
          for (int q = 0; q < Q; ++q) acc[q] = (float)(uint32_t)((pk >> (F * q)) & ((1ull << F) - 1ull));
        } else {
          for (int k = beg; k < end; ++k) {
            const uint32_t j = a.col[k] & 0x7fffffffu;
            const float wk = a.w ? a.w[k] : 1.f;
            const int sj = (int)((a.words_in[(size_t)j * wpn + wsel] >> sh) & SM);
#pragma unroll
            for (int q = 0; q < Q; ++q) acc[q] += (sj == q) ? wk : 0.f;
          }
        }
      } else {
        // accumulate sum_j W_ij (P_j(s) - 1/q): the constant drops out of every
        // difference below.  Each neighbour's q (P_j(s) - 1/q) (centred_q) was written
        // by the step that produced h_j, once per node rather than once per edge.
        // G neighbours at a time: their gathers, then the sums in neighbour order (the
        // same arithmetic as one at a time).  When a node's replicas fill aligned groups
        // of lanes (R = 16: half a warp; R a multiple of 32: whole warps), its lanes load
        // the node's column indices (and weights) with one coalesced load per group of
        // entries and pass them on by shuffles, so a thread waits for one memory round
        // trip per G neighbours; otherwise each thread loads them itself (two).
        constexpr int G = Q <= 4 ? 4 : 2;
        if (R == 16 || R % 32 == 0) {
          const int L = R == 16 ? 16 : 32;  // lanes per node
          const int sub = lane & (L - 1), gbase = lane & ~(L - 1);
          const int deg = end - beg;
          // the loops run to the larger degree of the warp's nodes, so that every lane
          // takes part in the shuffles (the lanes of one node share deg)
          const int maxdeg = L == 16 ? max(deg, __shfl_xor_sync(kFullMask, deg, 16)) : deg;
          for (int c0 = 0; c0 < maxdeg; c0 += L) {
            const int kk = c0 + sub;
            const bool have = kk < deg;
            const uint32_t myc = have ? (a.col[beg + kk] & 0x7fffffffu) : 0u;
            const float myw = have && a.w ? a.w[beg + kk] : 1.f;
            const int cnt = min(maxdeg - c0, L);
            for (int k0 = 0; k0 < cnt; k0 += G) {
              uint32_t jj[G];
              float wkk[G];
              bool okk[G];
#pragma unroll
              for (int u = 0; u < G; ++u) {
                const int e = k0 + u;
                okk[u] = e < L && c0 + e < deg;
                const int src = gbase + (e < L ? e : L - 1);
                jj[u] = __shfl_sync(kFullMask, myc, src);
                wkk[u] = __shfl_sync(kFullMask, myw, src);
              }
              float dj[G][Q];
#pragma unroll
              for (int u = 0; u < G; ++u) {
                if (okk[u]) {
                  load_q<Q>(a.d_in + ((size_t)jj[u] * R + r) * Q, dj[u]);
                } else {
#pragma unroll
                  for (int q = 0; q < Q; ++q) dj[u][q] = 0.f;
                }
              }
#pragma unroll
              for (int u = 0; u < G; ++u) {
                if (okk[u]) {
#pragma unroll
                  for (int q = 0; q < Q; ++q) acc[q] = fmaf(wkk[u], dj[u][q] * (1.f / Q), acc[q]);
                }
              }
            }
          }
        } else {
          for (int k0 = beg; k0 < end; k0 += G) {
            uint32_t jj[G];
            float wkk[G];
#pragma unroll
            for (int u = 0; u < G; ++u) {
              const bool ok = k0 + u < end;
              jj[u] = ok ? (a.col[k0 + u] & 0x7fffffffu) : 0u;
              wkk[u] = ok && a.w ? a.w[k0 + u] : 1.f;
            }
            float dj[G][Q];
#pragma unroll
            for (int u = 0; u < G; ++u) {
              if (k0 + u < end) {
                load_q<Q>(a.d_in + ((size_t)jj[u] * R + r) * Q, dj[u]);
              } else {
#pragma unroll
                for (int q = 0; q < Q; ++q) dj[u][q] = 0.f;
              }
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
              if (k0 + u < end) {
#pragma unroll
                for (int q = 0; q < Q; ++q) acc[q] = fmaf(wkk[u], dj[u][q] * (1.f / Q), acc[q]);
              }
            }
          }
        }
      }
    }
    // Centred gradient ghat(s) - sum_s' P(s') ghat(s') = sum_s' P(s') [ghat(s) - ghat(s')],
    // with every difference formed before it is scaled: integer count differences
    // (paper), exact fixed-point column-sum differences (exact), ln P(s) - ln P(s') =
    // h(s) - h(s').  Algebraically the formula above; in fp32 it avoids cancelling the
    // large s-independent parts (deg/q, lambda N/q) of ghat.
    float P[Q], lnP[Q];
    softmax_q<Q>(h, P, lnP);
    const float lam = s.lambda * a.lam_scale;
    int32_t nc[Q];
    unsigned long long ps[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      if (MODE == FEM_GRAD_PAPER) nc[q] = act ? a.cnt_in[r * Q + q] - (own == q ? Vi : 0) : 0;
      else ps[q] = act ? a.ps_in[r * Q + q] : 0ull;
    }
    // d(s, s') is antisymmetric bit for bit (each step is an exact difference, a product
    // or an fma, all odd under negation in round-to-nearest), and d(s, s) = +0 leaves
    // the sum unchanged (it starts at +0 and never becomes -0), so only the pairs s < s'
    // are formed; the sums still run over s' in order.
    float dm[Q][Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
#pragma unroll
      for (int q2 = q + 1; q2 < Q; ++q2) {
        float d;
        // node weights (SM, node-weighted balance term): lambda c^a_i V_i [n(s) - V_i e_i(s)]
        // (paper) and 2 lambda V_i [sum_j V_j P_j(s) - V_i P_i(s)] (exact); V_i = 1 gives
        // the unweighted forms with the same roundings
        // the coupling term enters with a.cw: -c^f / -2 (bMinCut: cut edges are cheap to
        // keep together) or +c^f / +1 (colouring: same colours across an edge cost)
        if (MODE == FEM_GRAD_PAPER) {
          d = (a.cw * cf) * (acc[q] - acc[q2]) + lam * (ca * (float)Vi) * (float)(nc[q] - nc[q2]);
        } else {
          const float dcol = (float)(long long)(ps[q] - ps[q2]) * kPsumInv;
          d = a.cw * (acc[q] - acc[q2]) + 2.f * lam * (float)Vi * (dcol - (float)Vi * (P[q] - P[q2]));
        }
        dm[q][q2] = fmaf(h[q] - h[q2], s.inv_beta, d);
      }
    }
    float cen[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      float c = 0.f;
#pragma unroll
      for (int q2 = 0; q2 < Q; ++q2)
        if (q2 != q) c = fmaf(P[q2], q < q2 ? dm[q][q2] : -dm[q2][q], c);
      cen[q] = c;
    }
    with_opt(a.opt, [&](auto O) {
#pragma unroll
      for (int q = 0; q < Q; ++q) opt_update_fast<decltype(O)::value>(h[q], mm[q], vv[q], s.gq * cen[q] * P[q], s);
    });
    const int sn = argmax_q<Q>(h);
    if (act) {
      store_q<Q>(a.h_out + idx, h);
      store_q<Q>(a.m + idx, mm);
      if (a.opt != FEM_OPT_SGD) store_q<Q>(a.v + idx, vv);
      atomicAdd(&scnt[r * Q + sn], Vi);
      if (MODE == FEM_GRAD_EXACT) {
        float Pn[Q], ln[Q], dn[Q];
        softmax_q<Q>(h, Pn, ln);
#pragma unroll
        for (int q = 0; q < Q; ++q)
          atomicAdd(&sps[r * Q + q], __float2ull_rn(Pn[q] * kPsumScale) * (unsigned long long)Vi);
        centred_q<Q>(h, dn);
        store_q<Q>(a.d_out + idx, dn);
      }
    }
    uint32_t word = act ? ((uint32_t)sn << sh) : 0u;
#pragma unroll
    for (int off = 1; off < RPW; off <<= 1) word |= __shfl_xor_sync(kFullMask, word, off);
    if (act && (r % RPW) == 0) a.words_out[(size_t)i * wpn + wsel] = word;
  }
}

}  // namespace fem
