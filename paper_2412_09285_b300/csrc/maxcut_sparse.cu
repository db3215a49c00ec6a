// MaxCut on sparse graphs: the fused per-step kernel (neighbour contraction +
// single-field gradient + optimizer) and the read-out of cuts.
//
// Single-field form (SM "Simplification of FEM for solving the MaxCut problem",
// Eq. grad_m_h): P_i = sigmoid(h_i), m_i = tanh(h_i/2),
//   paper mode: g_i = (gamma/4) [c_i sum_j W_ij sgn(m_j) + h_i/beta] (1 - m_i^2)
//   exact mode: g_i = (gamma/4) [2 sum_j W_ij m_j      + h_i/beta] (1 - m_i^2)
// with c_i = 1/sum_j |W_ij| (SM, after Eq. maxcut_modified_gradient; 0 when isolated).
//
// Layout: h, m, v are [n][R] fp32 with the R replicas of a node contiguous, so a
// warp (lane = replica) reads and writes 128 B per array per node.  The
// discretised state sgn(m_j) of 32 replicas is one uint32 per node ("sign word";
// bit r set <=> h_jr < 0 <=> state -1), ping-ponged between steps, so a
// neighbour gather moves 4 bytes per edge instead of 128.
#include "fem_internal.h"
#include "reduce_common.cuh"
#include "step_common.cuh"

namespace fem {
namespace {

struct MaxcutArgs {
  const int32_t* row_ptr;
  const uint32_t* col;
  const float* w;
  const float* cnorm;
  int32_t n, R, wpn;
  const float* h_in;
  float* h_out;
  float* m;
  float* v;
  const uint32_t* words_in;
  uint32_t* words_out;
  const float* mag_in;  // exact mode: m_j = tanh(h_j / 2) of the fields this step reads
  float* mag_out;       // exact mode: m of the updated fields, for the next step
  float ccoef;          // exact mode: coefficient of sum_j W_ij m_j (2 for MaxCut, 1 for QUBO)
  const float* offset;  // exact mode: per-node constant of the field (QUBO), NULL for MaxCut
};

// Exact-mode step, direct gathers: one warp per (node, block of 32 replicas); lane =
// replica.  Neighbour column indices are loaded 32 at a time (one coalesced load) and
// broadcast by shuffles; each lane gathers its replica's m_j of every neighbour (a
// 128-byte line per neighbour and warp).  Bound by those gathers, most of which miss
// L2 at n = 2^20 (m is 128 MiB).  The default exact-mode kernel is the TMA-gather
// tile kernel (maxcut_gather.cu), which computes the same sums in the same order with
// the same update; this one stays as its reference (fem_set_tma_gather(0)).
template <int OPT, bool UNIT>
__global__ void __launch_bounds__(256) k_maxcut_step(MaxcutArgs a, StepScalars s) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long items = (long long)a.n * a.wpn;
  for (long long it = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items;
       it += nwarps) {
    const int i = (int)(it / a.wpn);
    const int wb = (int)(it - (long long)i * a.wpn);
    const size_t idx = (size_t)i * a.R + (size_t)wb * 32 + lane;
    float hi = a.h_in[idx];
    float mi = a.m[idx];
    float vi = (OPT == FEM_OPT_SGD) ? 0.f : a.v[idx];
    const int beg = a.row_ptr[i], end = a.row_ptr[i + 1];
    float facc = 0.f;
    for (int k0 = beg; k0 < end; k0 += 32) {
      const int k = k0 + lane;
      uint32_t c = 0;
      float wk = 0.f;
      if (k < end) {
        c = a.col[k];
        if (!UNIT) wk = a.w[k];
      }
      const int cnt = min(32, end - k0);
      for (int e = 0; e < cnt; ++e) {
        const uint32_t ce = __shfl_sync(kFullMask, c, e);
        const float mj = a.mag_in[(size_t)(ce & 0x7fffffffu) * a.R + (size_t)wb * 32 + lane];
        if (UNIT) {
          facc += (ce >> 31) ? -mj : mj;
        } else {
          facc = fmaf(__shfl_sync(kFullMask, wk, e), mj, facc);
        }
      }
    }
    // MaxCut: 2 sum_j W_ij m_j.  QUBO: with p = (1 + m)/2, 2 sum_j Q_ij p_j + d_i =
    // sum_j Q_ij m_j + (sum_j Q_ij + d_i)
    float field = a.ccoef * facc;
    if (a.offset) field += a.offset[i];
    // field + h/beta as one explicit fma, so that the direct and the tile kernel round it
    // alike however the compiler contracts the code around it
    const float g = s.gq * fmaf(hi, s.inv_beta, field) * one_minus_m2_fast(hi);
    opt_update_fast<OPT>(hi, mi, vi, g, s);
    a.h_out[idx] = hi;
    a.m[idx] = mi;
    if (OPT != FEM_OPT_SGD) a.v[idx] = vi;
    a.mag_out[idx] = tanhf(0.5f * hi);  // gathered by the next step
    const uint32_t ball = __ballot_sync(kFullMask, hi < 0.f);
    if (lane == 0) a.words_out[(size_t)i * a.wpn + wb] = ball;
  }
}

// Paper-mode step, tuned for HBM streaming.  A warp owns NPW consecutive nodes
// (one block of 32 replicas) per iteration and issues every load of the group
// before it computes: the 3*NPW state lines (h, m, v), then one coalesced load
// of up to 32 CSR entries covering the whole group, then 32 parallel gathers of
// the neighbours' sign words.  The row pointers of the next group are fetched a
// group ahead.  Each gathered word is pre-XORed with the weight sign (unit
// weights), so one shuffle and one bit test per edge give the neighbour term:
//   sum_j W_ij sgn(m_j) = deg_i - 2 * #{j : W_ij sgn(m_j) = -1}.
// R32: the replica count is 32 (one sign word per node), a compile-time constant.
template <int OPT, bool UNIT, int NPW, bool R32 = false>
__global__ void __launch_bounds__(256, 5) k_maxcut_step_paper(MaxcutArgs a, StepScalars s) {
  const int R = R32 ? 32 : a.R, wpn = R32 ? 1 : a.wpn;
  const int lane = threadIdx.x & 31;
  const int ngroups = (a.n + NPW - 1) / NPW;
  const long long total = (long long)ngroups * wpn;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  auto row_ptrs = [&](long long gg) -> int {
    if (gg >= total) return 0;
    const int ng = wpn == 1 ? (int)gg : (int)(gg / wpn);
    return lane <= NPW ? __ldg(a.row_ptr + min(ng * NPW + lane, a.n)) : 0;
  };
  int rp = row_ptrs(g);
  for (; g < total; g += nwarps) {
    const int ng = wpn == 1 ? (int)g : (int)(g / wpn);
    const int wb = wpn == 1 ? 0 : (int)(g - (long long)ng * wpn);
    const int i0 = ng * NPW;
    float h[NPW], m[NPW], v[NPW];
#pragma unroll
    for (int k = 0; k < NPW; ++k) {
      h[k] = 0.f; m[k] = 0.f; v[k] = 0.f;
      if (i0 + k < a.n) {
        const size_t idx = (size_t)(i0 + k) * R + (size_t)wb * 32 + lane;
        h[k] = a.h_in[idx];
        m[k] = a.m[idx];
        if (OPT != FEM_OPT_SGD) v[k] = a.v[idx];
      }
    }
    int rb[NPW + 1];
#pragma unroll
    for (int k = 0; k <= NPW; ++k) rb[k] = __shfl_sync(kFullMask, rp, k);
    rp = row_ptrs(g + nwarps);  // prefetch the next group's row pointers
    const int bN = rb[NPW];
    int cb = rb[0];
    uint32_t adj = 0;
    float wv = 0.f;
    auto load_chunk = [&](int base) {
      const int e = base + lane;
      adj = 0;
      wv = 0.f;
      if (e < bN) {
        const uint32_t c = __ldg(a.col + e);
        const uint32_t wd = __ldg(a.words_in + (size_t)(c & 0x7fffffffu) * wpn + wb);
        if (UNIT) {
          adj = wd ^ (0u - (c >> 31));
        } else {
          adj = wd;
          wv = __ldg(a.w + e);
        }
      }
    };
    load_chunk(cb);
    // Unit weights: the group's CSR entries in chunks of 32 (one chunk in the common
    // case).  A 32 x 32 bit transpose across the warp turns "lane e holds the word of
    // entry e" into "lane r holds, for every entry e, bit r of its word"; a node's count
    // in a chunk is then one popcount under the node's entry mask.  The next chunk's
    // column and word loads are issued before the current chunk is counted.
    int nneg_u[NPW];
#pragma unroll
    for (int k = 0; k < NPW; ++k) nneg_u[k] = 0;
    if (UNIT && bN - rb[0] <= 32) {
      const uint32_t tr = warp_transpose32(adj, lane);
#pragma unroll
      for (int k = 0; k < NPW; ++k) {
        const int len = rb[k + 1] - rb[k];
        nneg_u[k] = __popc(tr & (len == 0 ? 0u : (len >= 32 ? 0xffffffffu : ((1u << len) - 1u)) << (rb[k] - rb[0])));
      }
    } else if (UNIT) {
      for (int c0 = rb[0]; c0 < bN; c0 += 32) {
        const uint32_t cur = adj;
        if (c0 + 32 < bN) load_chunk(c0 + 32);
        const uint32_t tr = warp_transpose32(cur, lane);
#pragma unroll
        for (int k = 0; k < NPW; ++k) {
          const int lo = max(rb[k], c0) - c0, hi = min(rb[k + 1], c0 + 32) - c0;
          if (hi > lo) {
            const int len = hi - lo;
            nneg_u[k] += __popc(tr & ((len >= 32 ? 0xffffffffu : ((1u << len) - 1u)) << lo));
          }
        }
      }
    }
    uint32_t ball[NPW];
#pragma unroll
    for (int k = 0; k < NPW; ++k) {
      int nneg = nneg_u[k];
      float facc = 0.f;
      if (!UNIT) {
        for (int e = rb[k]; e < rb[k + 1]; ++e) {
          if (e >= cb + 32) {
            cb += 32;
            load_chunk(cb);
          }
          const uint32_t bit = (__shfl_sync(kFullMask, adj, e - cb) >> lane) & 1u;
          const float w = __shfl_sync(kFullMask, wv, e - cb);
          facc += bit ? -w : w;
        }
      }
      const int deg = rb[k + 1] - rb[k];
      const float field = UNIT ? (deg > 0 ? div_approx((float)(deg - 2 * nneg), (float)deg) : 0.f)
                               : (a.cnorm[min(i0 + k, a.n - 1)] * facc);
      float hk = h[k], mk = m[k], vk = v[k];
      const float gk = s.gq * (field + hk * s.inv_beta) * one_minus_m2_fast(hk);
      opt_update_fast<OPT>(hk, mk, vk, gk, s);
      ball[k] = __ballot_sync(kFullMask, hk < 0.f);
      if (i0 + k < a.n) {
        const size_t idx = (size_t)(i0 + k) * R + (size_t)wb * 32 + lane;
        a.h_out[idx] = hk;
        a.m[idx] = mk;
        if (OPT != FEM_OPT_SGD) a.v[idx] = vk;
      }
    }
    uint32_t mine = ball[0];
#pragma unroll
    for (int k = 1; k < NPW; ++k) mine = lane == k ? ball[k] : mine;
    if (lane < NPW && i0 + lane < a.n) a.words_out[(size_t)(i0 + lane) * wpn + wb] = mine;
  }
}

// Sign words of the fields: bit r of word (i, b) is set when h[i][32b + r] < 0 (and,
// when mag is non-NULL, m = tanh(h/2) for the exact-mode gathers).  With copy
// non-NULL the fields are also written there: a fresh start reads the caller's
// initial fields once, instead of a device copy followed by this pass.
__global__ void k_pack_sign_words(const float* __restrict__ h, int32_t n, int32_t R,
                                  int32_t wpn, uint32_t* __restrict__ words, float* __restrict__ mag,
                                  float* __restrict__ copy) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long it = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       it < (long long)n * wpn; it += nwarps) {
    const float x = h[it * 32 + lane];  // [n][R] with R = 32 wpn: item it covers elements it*32..
    const uint32_t b = __ballot_sync(kFullMask, x < 0.f);
    if (lane == 0) words[it] = b;
    if (mag) mag[it * 32 + lane] = tanhf(0.5f * x);
    if (copy) copy[it * 32 + lane] = x;
  }
}

// Per-block partial cuts: cut_r = sum over undirected edges (j > i in the CSR)
// of W_ij [bit_ir != bit_jr].  blockIdx.y selects the block of 32 replicas;
// the lane is the replica.  Integer weights accumulate in int64, others in fp64
// in CSR order, then the 8 warps of the block are added in warp order.
template <bool UNIT, bool INTW>
__global__ void __launch_bounds__(256) k_maxcut_cut_partial(
    const int32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const float* __restrict__ w, const double* __restrict__ w64,
    const uint32_t* __restrict__ words, int32_t n, int32_t R, int32_t wpn,
    int64_t* __restrict__ part_i, double* __restrict__ part_f) {
  __shared__ int64_t si[8][32];
  __shared__ double sf[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wb = blockIdx.y;
  int64_t acc_i = 0;
  double acc_f = 0.0;
  for (int i = blockIdx.x * 8 + warp; i < n; i += gridDim.x * 8) {
    const uint32_t bi = (words[(size_t)i * wpn + wb] >> lane) & 1u;
    const int beg = row_ptr[i], end = row_ptr[i + 1];
    for (int k0 = beg; k0 < end; k0 += 32) {
      const int k = k0 + lane;
      uint32_t c = 0, word = 0;
      if (k < end) {
        c = col[k];
        word = words[(size_t)(c & 0x7fffffffu) * wpn + wb];
      }
      const int cnt = min(32, end - k0);
      for (int e = 0; e < cnt; ++e) {
        const uint32_t ce = __shfl_sync(kFullMask, c, e);
        const uint32_t bj = (__shfl_sync(kFullMask, word, e) >> lane) & 1u;
        const uint32_t j = ce & 0x7fffffffu;
        if ((int)j <= i || bj == bi) continue;
        if (INTW) {
          acc_i += UNIT ? ((ce >> 31) ? -1 : 1) : (int64_t)w[k0 + e];
        } else {
          acc_f += w64[k0 + e];
        }
      }
    }
  }
  si[warp][lane] = acc_i;
  sf[warp][lane] = acc_f;
  __syncthreads();
  if (warp == 0) {
    int64_t ti = 0;
    double tf = 0.0;
    for (int k = 0; k < 8; ++k) {
      ti += si[k][lane];
      tf += sf[k][lane];
    }
    const size_t o = (size_t)blockIdx.x * R + (size_t)wb * 32 + lane;
    if (INTW) part_i[o] = ti;
    else part_f[o] = tf;
  }
}

// Unit-weight partial objectives, NPW consecutive nodes per warp.  The group's CSR
// entries are read 32 at a time (one coalesced load); lane e forms the 32-replica word
// of entry e's edge term from the two endpoints' sign words - MaxCut: the states
// differ (XOR); QUBO: both variables are 1 (neither bit set) - and a 32 x 32 warp bit
// transpose gives lane r, for every entry, replica r's bit.  One popcount under the
// mask of entries with W = +1 minus one under W = -1 then adds a chunk's edges to
// replica r's count (each undirected edge once: the entry with j > i).  The sums are
// integers, so the grouping does not change the result.  The row pointers of the next
// group are fetched while the current one is counted.
template <bool QUBO, int NPW>
__global__ void __launch_bounds__(256) k_maxcut_cut_grouped(
    const int32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col, const int64_t* __restrict__ lin_i,
    const uint32_t* __restrict__ words, int32_t n, int32_t R, int32_t wpn, int64_t* __restrict__ part_i) {
  __shared__ int64_t si[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wb = blockIdx.y;
  const int ngroups = (n + NPW - 1) / NPW;
  const int stride = gridDim.x * 8;
  int64_t acc = 0;
  int g = blockIdx.x * 8 + warp;
  int rp = (g < ngroups && lane <= NPW) ? __ldg(row_ptr + min(g * NPW + lane, n)) : 0;
  for (; g < ngroups; g += stride) {
    const int i0 = g * NPW;
    const uint32_t own = (lane < NPW && i0 + lane < n) ? __ldg(words + (size_t)(i0 + lane) * wpn + wb) : 0u;
    int rb[NPW + 1];
#pragma unroll
    for (int k = 0; k <= NPW; ++k) rb[k] = __shfl_sync(kFullMask, rp, k);
    const int gn = g + stride;
    rp = (gn < ngroups && lane <= NPW) ? __ldg(row_ptr + min(gn * NPW + lane, n)) : 0;
    for (int c0 = rb[0]; c0 < rb[NPW]; c0 += 32) {
      const int e = c0 + lane;
      const bool valid = e < rb[NPW];
      int k = 0;
#pragma unroll
      for (int kk = 1; kk < NPW; ++kk) k += (e >= rb[kk]) ? 1 : 0;
      const uint32_t wi = __shfl_sync(kFullMask, own, k);
      uint32_t c = 0, wj = 0;
      if (valid) {
        c = __ldg(col + e);
        wj = __ldg(words + (size_t)(c & 0x7fffffffu) * wpn + wb);
      }
      const bool take = valid && (int)(c & 0x7fffffffu) > i0 + k;
      const uint32_t pm = __ballot_sync(kFullMask, take && !(c >> 31));
      const uint32_t nm = __ballot_sync(kFullMask, take && (c >> 31));
      const uint32_t x = QUBO ? ~(wi | wj) : (wi ^ wj);
      const uint32_t tr = warp_transpose32(x, lane);
      const int d = __popc(tr & pm) - __popc(tr & nm);
      acc += QUBO ? 2 * d : d;
    }
    if (QUBO) {   // the linear terms of the group's variables that are 1
#pragma unroll
      for (int k = 0; k < NPW; ++k) {
        const uint32_t wk = __shfl_sync(kFullMask, own, k);
        if (i0 + k < n && !((wk >> lane) & 1u)) acc += __ldg(lin_i + i0 + k);
      }
    }
  }
  si[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    int64_t t = 0;
    for (int k = 0; k < 8; ++k) t += si[k][lane];
    part_i[(size_t)blockIdx.x * R + (size_t)wb * 32 + lane] = t;
  }
}

// Sum the partials of every replica in block order, set E_r = -cut_r, then the
// argmin over replicas with the lowest index winning ties.  One block.
// QUBO energy partials: E_r = sum_{i<j} 2 Q_ij s_i s_j + sum_i d_i s_i with s = 1 where
// h >= 0 (sign bit clear); same blocking and fixed summation order as the cut partials.
template <bool UNIT, bool INTW>
__global__ void __launch_bounds__(256) k_qubo_partial(
    const int32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const float* __restrict__ w, const double* __restrict__ w64, const int64_t* __restrict__ lin_i,
    const double* __restrict__ lin_f, const uint32_t* __restrict__ words, int32_t n, int32_t R, int32_t wpn,
    int64_t* __restrict__ part_i, double* __restrict__ part_f) {
  __shared__ int64_t si[8][32];
  __shared__ double sf[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wb = blockIdx.y;
  int64_t acc_i = 0;
  double acc_f = 0.0;
  for (int i = blockIdx.x * 8 + warp; i < n; i += gridDim.x * 8) {
    const uint32_t bi = (words[(size_t)i * wpn + wb] >> lane) & 1u;
    if (!bi) {
      if (INTW) acc_i += lin_i[i];
      else acc_f += lin_f[i];
    }
    const int beg = row_ptr[i], end = row_ptr[i + 1];
    for (int k0 = beg; k0 < end; k0 += 32) {
      const int k = k0 + lane;
      uint32_t c = 0, word = 0;
      if (k < end) {
        c = col[k];
        word = words[(size_t)(c & 0x7fffffffu) * wpn + wb];
      }
      const int cnt = min(32, end - k0);
      for (int e = 0; e < cnt; ++e) {
        const uint32_t ce = __shfl_sync(kFullMask, c, e);
        const uint32_t bj = (__shfl_sync(kFullMask, word, e) >> lane) & 1u;
        const uint32_t j = ce & 0x7fffffffu;
        if ((int)j <= i || bi || bj) continue;
        if (INTW) acc_i += 2 * (UNIT ? ((ce >> 31) ? -1 : 1) : (int64_t)w[k0 + e]);
        else acc_f += 2.0 * w64[k0 + e];
      }
    }
  }
  si[warp][lane] = acc_i;
  sf[warp][lane] = acc_f;
  __syncthreads();
  if (warp == 0) {
    int64_t ti = 0;
    double tf = 0.0;
    for (int k = 0; k < 8; ++k) {
      ti += si[k][lane];
      tf += sf[k][lane];
    }
    const size_t o = (size_t)blockIdx.x * R + (size_t)wb * 32 + lane;
    if (INTW) part_i[o] = ti;
    else part_f[o] = tf;
  }
}

// E_r = -cut_r (MaxCut, negate) or the QUBO energy for replica r = blockIdx.x (the
// argmin follows in k_argmin_replica).
template <bool INTW>
__global__ void __launch_bounds__(kRedThreads) k_maxcut_finish(const int64_t* __restrict__ part_i,
                                                               const double* __restrict__ part_f,
                                                               int32_t nblk, int32_t R, int32_t negate,
                                                               int64_t* __restrict__ e_i,
                                                               double* __restrict__ e_f) {
  __shared__ int64_t shi[kRedThreads];
  __shared__ double shf[kRedThreads];
  const int r = blockIdx.x;
  if (INTW) {
    const int64_t t = column_sum<int64_t>(part_i, nblk, R, r, shi);
    if (threadIdx.x == 0) {
      e_i[r] = negate ? -t : t;
      e_f[r] = (double)(negate ? -t : t);
    }
  } else {
    const double t = column_sum<double>(part_f, nblk, R, r, shf);
    if (threadIdx.x == 0) {
      e_i[r] = 0;
      e_f[r] = negate ? -t : t;
    }
  }
}

// states[i] = +1 / -1 of replica r (from the sign words).
// States from sign words: a set bit (h < 0) is `lo` (MaxCut -1, QUBO 0), a clear bit 1.
__global__ void k_maxcut_states_one(const uint32_t* __restrict__ words, int32_t n, int32_t wpn,
                                    const int32_t* __restrict__ best, int32_t* __restrict__ out, int32_t lo) {
  const int r = best[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    out[i] = ((words[(size_t)i * wpn + (r >> 5)] >> (r & 31)) & 1u) ? lo : 1;
  }
}

__global__ void k_maxcut_states_all(const uint32_t* __restrict__ words, int32_t n, int32_t R,
                                    int32_t wpn, int32_t* __restrict__ out, int32_t lo) {
  const size_t total = (size_t)n * R;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = e / R;
    const int r = (int)(e - i * R);
    out[e] = ((words[i * wpn + (r >> 5)] >> (r & 31)) & 1u) ? lo : 1;
  }
}

constexpr int kNodesPerWarp = 4;

// Persistent grid: exactly the resident blocks (occupancy x SMs), never more
// than the work needs, so the grid-stride loop runs in a single wave.  The
// occupancy is queried once per kernel (K is the kernel itself, not its type).
template <auto K>
int resident_grid(int sm_count, long long warps_needed) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, K, 256, 0) != cudaSuccess || b < 1) b = 1;
    per_sm = b;
  }
  long long blocks = (warps_needed + 7) / 8;
  const long long cap = (long long)per_sm * sm_count;
  if (blocks > cap) blocks = cap;
  return (int)(blocks < 1 ? 1 : blocks);
}

// Graphs with fewer groups of kNodesPerWarp nodes than this many warps run one node
// per warp instead (more warps in flight when a step is latency-bound).
constexpr long long kSmallGraphWarps = 4096;

template <int MODE, int OPT, bool UNIT>
void launch_step(const MaxcutArgs& a, const StepScalars& s, int sm_count, long long warps,
                 cudaStream_t st) {
  const long long per_node = (long long)a.n * a.wpn;
  if (MODE == FEM_GRAD_PAPER) {
    if (warps < kSmallGraphWarps && a.R == 32) {
      constexpr auto k = k_maxcut_step_paper<OPT, UNIT, 1, true>;
      k<<<resident_grid<k>(sm_count, per_node), 256, 0, st>>>(a, s);
    } else if (warps < kSmallGraphWarps) {
      constexpr auto k = k_maxcut_step_paper<OPT, UNIT, 1>;
      k<<<resident_grid<k>(sm_count, per_node), 256, 0, st>>>(a, s);
    } else if (a.R == 32) {
      constexpr auto k = k_maxcut_step_paper<OPT, UNIT, kNodesPerWarp, true>;
      k<<<resident_grid<k>(sm_count, warps), 256, 0, st>>>(a, s);
    } else {
      constexpr auto k = k_maxcut_step_paper<OPT, UNIT, kNodesPerWarp>;
      k<<<resident_grid<k>(sm_count, warps), 256, 0, st>>>(a, s);
    }
  } else {
    constexpr auto k = k_maxcut_step<OPT, UNIT>;
    k<<<resident_grid<k>(sm_count, per_node), 256, 0, st>>>(a, s);
  }
}

using StepFn = void (*)(const MaxcutArgs&, const StepScalars&, int, long long, cudaStream_t);

template <int MODE, bool UNIT>
StepFn pick_opt(int opt) {
  switch (opt) {
    case FEM_OPT_ADAM: return launch_step<MODE, FEM_OPT_ADAM, UNIT>;
    case FEM_OPT_RMSPROP: return launch_step<MODE, FEM_OPT_RMSPROP, UNIT>;
    default: return launch_step<MODE, FEM_OPT_SGD, UNIT>;
  }
}

StepFn pick_step(int mode, int opt, bool unit) {
  if (mode == FEM_GRAD_PAPER) return unit ? pick_opt<FEM_GRAD_PAPER, true>(opt) : pick_opt<FEM_GRAD_PAPER, false>(opt);
  return unit ? pick_opt<FEM_GRAD_EXACT, true>(opt) : pick_opt<FEM_GRAD_EXACT, false>(opt);
}

int grid_for_warps(const Problem* p, long long warps) {
  long long blocks = (warps + 7) / 8;
  const long long cap = (long long)p->sm_count * 8;
  if (blocks > cap) blocks = cap;
  return (int)(blocks < 1 ? 1 : blocks);
}

}  // namespace

fem_status maxcut_pack_words(Problem* p, int hbuf, int wbuf, cudaStream_t s, const float* src) {
  const long long items = (long long)p->n * p->words_per_node;
  k_pack_sign_words<<<grid_for_warps(p, items), 256, 0, s>>>(
      src ? src : p->h[hbuf], p->n, p->R, p->words_per_node, p->words[wbuf],
      p->grad_mode == FEM_GRAD_EXACT ? p->mag[wbuf] : nullptr, src ? p->h[hbuf] : nullptr);
  count_launches(1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

fem_status maxcut_sparse_steps(Problem* p, const fem_anneal_params& a,
                               const std::vector<StepScalars>& sc, cudaStream_t s) {
  const StepFn fn = pick_step(p->grad_mode, p->optimizer, p->unit_w);
  const long long groups = (long long)((p->n + kNodesPerWarp - 1) / kNodesPerWarp) * p->words_per_node;
  MaxcutArgs args{};
  args.row_ptr = p->row_ptr;
  args.col = p->col;
  args.w = p->w;
  args.cnorm = p->cnorm;
  args.n = p->n;
  args.R = p->R;
  args.wpn = p->words_per_node;
  args.m = p->m;
  args.v = p->v;
  args.ccoef = p->qubo ? 1.f : 2.f;
  args.offset = p->qubo ? p->qoff : nullptr;
  if (p->grad_mode == FEM_GRAD_PAPER && tma_gather_enabled() && groups >= kSmallGraphWarps) {
    // the staged tile kernel (maxcut_paper_tile.cu): the same arithmetic and bits
    for (size_t k = 0; k < sc.size(); ++k) {
      const fem_status st = maxcut_paper_tile_step(p, p->cur, sc[k], s);
      if (st != FEM_OK) return st;
      p->cur ^= 1;
    }
    count_launches((int64_t)sc.size());
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
  }
  if (p->grad_mode == FEM_GRAD_EXACT && tma_gather_enabled()) {
    // the TMA-gather kernel (maxcut_gather.cu): the same arithmetic and bits
    for (size_t k = 0; k < sc.size(); ++k) {
      const fem_status st = maxcut_exact_gather_step(p, p->cur, sc[k], s);
      if (st != FEM_OK) return st;
      p->cur ^= 1;
    }
    count_launches((int64_t)sc.size());
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
  }
  for (size_t k = 0; k < sc.size(); ++k) {
    if (p->grad_mode == FEM_GRAD_PAPER) {
      args.h_in = p->h[0];
      args.h_out = p->h[0];
    } else {
      args.h_in = p->h[p->cur];
      args.h_out = p->h[p->cur ^ 1];
    }
    args.words_in = p->words[p->cur];
    args.words_out = p->words[p->cur ^ 1];
    args.mag_in = p->mag[p->cur];
    args.mag_out = p->mag[p->cur ^ 1];
    fn(args, sc[k], p->sm_count, groups, s);
    p->cur ^= 1;
  }
  count_launches((int64_t)sc.size());
  FEM_CUDA(cudaGetLastError());
  (void)a;
  return FEM_OK;
}

const float* maxcut_current_fields(const Problem* p) {
  return p->grad_mode == FEM_GRAD_PAPER ? p->h[0] : p->h[p->cur];
}

fem_status maxcut_readout(Problem* p, cudaStream_t s) {
  const int wpn = p->words_per_node;
  const dim3 grid(p->part_blocks, wpn);
  const uint32_t* words = p->words[p->cur];
  const bool intw = p->int_w && (!p->qubo || p->qlin_int);
  if (intw && p->unit_w) {   // the common case: grouped nodes and bit-sliced counts
    if (p->qubo)
      k_maxcut_cut_grouped<true, kNodesPerWarp><<<grid, 256, 0, s>>>(p->row_ptr, p->col, p->qlin_i, words, p->n,
                                                                     p->R, wpn, p->part_i);
    else
      k_maxcut_cut_grouped<false, kNodesPerWarp><<<grid, 256, 0, s>>>(p->row_ptr, p->col, p->qlin_i, words, p->n,
                                                                      p->R, wpn, p->part_i);
  } else if (p->qubo) {
    if (intw)
      k_qubo_partial<false, true><<<grid, 256, 0, s>>>(p->row_ptr, p->col, p->w, p->w64, p->qlin_i, p->qlin_f,
                                                       words, p->n, p->R, wpn, p->part_i, p->part_f);
    else
      k_qubo_partial<false, false><<<grid, 256, 0, s>>>(p->row_ptr, p->col, p->w, p->w64, p->qlin_i, p->qlin_f,
                                                        words, p->n, p->R, wpn, p->part_i, p->part_f);
  } else if (intw) {
    k_maxcut_cut_partial<false, true><<<grid, 256, 0, s>>>(p->row_ptr, p->col, p->w, p->w64, words,
                                                           p->n, p->R, wpn, p->part_i, p->part_f);
  } else {
    k_maxcut_cut_partial<false, false><<<grid, 256, 0, s>>>(p->row_ptr, p->col, p->w, p->w64, words,
                                                            p->n, p->R, wpn, p->part_i, p->part_f);
  }
  const int negate = p->qubo ? 0 : 1;
  if (intw)
    k_maxcut_finish<true><<<p->R, kRedThreads, 0, s>>>(p->part_i, p->part_f, p->part_blocks, p->R, negate,
                                                        p->energy_i, p->energy_f);
  else
    k_maxcut_finish<false><<<p->R, kRedThreads, 0, s>>>(p->part_i, p->part_f, p->part_blocks, p->R, negate,
                                                         p->energy_i, p->energy_f);
  k_argmin_replica<<<1, 1024, 0, s>>>(p->energy_f, p->R, p->best);
  k_maxcut_states_one<<<(p->n + 255) / 256 < 1024 ? (p->n + 255) / 256 : 1024, 256, 0, s>>>(
      words, p->n, wpn, p->best, p->states_dev, p->qubo ? 0 : -1);
  count_launches(4);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

fem_status maxcut_states_all(Problem* p, int32_t* out_dev, cudaStream_t s) {
  const size_t total = (size_t)p->n * p->R;
  size_t blocks = (total + 255) / 256;
  if (blocks > (size_t)p->sm_count * 16) blocks = (size_t)p->sm_count * 16;
  k_maxcut_states_all<<<(int)blocks, 256, 0, s>>>(p->words[p->cur], p->n, p->R, p->words_per_node,
                                                  out_dev, p->qubo ? 0 : -1);
  count_launches(1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

}  // namespace fem
