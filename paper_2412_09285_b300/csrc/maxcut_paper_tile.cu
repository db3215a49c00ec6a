// Paper-mode sparse MaxCut step (SM Eq. maxcut_modified_gradient) with its operands
// staged ahead in shared memory:
//   g_ir = (gamma/4) [c_i sum_j W_ij sgn(m_jr) + h_ir/beta] (1 - m_ir^2),
// c_i = 1/deg_i for unit weights (the sum counted from sign words), 1/sum_j |W_ij| else.
//
// The direct kernel (k_maxcut_step_paper in maxcut_sparse.cu) has each warp load its
// group's state, CSR entries and neighbours' sign words itself, so its issue slots wait
// on two dependent memory round trips per group.  Here a block works on tiles of 16
// nodes (four groups of four, one block of 32 replicas) and a producer warp prepares
// each tile in shared memory: the tile's h, m, v rows by bulk copies completing on the
// stage's mbarrier, and the neighbours' sign words (XOR-ed with the weight signs)
// gathered by the producer's lanes from registers, with the row pointers three tiles,
// the CSR entries two tiles and the words one tile ahead.  Four consumer warps, one
// group each, then run the direct kernel's arithmetic on the staged operands (the
// warp bit transpose, the popcounts, the update), in its order, so both give the same
// bits.  Entries beyond a tile's capacity (hub rows) are read directly.  Every wait is
// bounded.
#include <cuda_runtime.h>

#include "fem_internal.h"
#include "step_common.cuh"

namespace fem {
namespace {

constexpr int kNpw = 4;                      // nodes per consumer warp (a group)
constexpr int kConsumers = 4;                // consumer warps; warp kConsumers is the producer
constexpr int kNodes = kNpw * kConsumers;    // nodes per tile
constexpr int kCap = 192;                    // CSR entries staged per tile (a multiple of 32)
constexpr int kQ = kCap / 32;                // entries per producer lane
constexpr int kStages = 2;
constexpr int kThreads = (kConsumers + 1) * 32;
constexpr unsigned long long kWaitNs = 2000000000ull;
// the producer holds a tile's kNodes + 1 row pointers one per lane
static_assert(kNodes < 32, "a tile's row pointers must fit the producer warp's lanes");

struct PArgs {
  const int32_t* row_ptr;
  const uint32_t* col;   // unit weights: the -1 sign in bit 31
  const float* w;        // weights (NULL for unit weights)
  const float* cnorm;    // c_i (weighted graphs)
  int32_t n, R, wpn;
  float* h;              // read and written in place (paper mode)
  float* m;
  float* v;
  const uint32_t* words_in;
  uint32_t* words_out;
  int32_t* err;
};

struct alignas(128) Stage {
  float h[kNodes * 32], m[kNodes * 32], v[kNodes * 32];
  uint32_t adj[kCap];              // entry k's neighbour sign word (XOR the weight sign for unit weights)
  float w[kCap];
  float cn[kNodes];                // weights: c_i; unit weights: 1/deg_i (0 for deg_i = 0)
  uint32_t mask[kNodes];           // unit weights: node's entries within its group's first 32
  int32_t rptr[kNodes + 1];        // the tile's row pointers relative to base
  int32_t base;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int32_t* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > kWaitNs) {
      atomicOr(err, ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Resident blocks per SM the registers are budgeted for: seven with unit weights (measured
// faster than six and eight), six for SGD in the run-time replica form (seven spill there),
// five with weights.
template <int OPT, bool UNIT, bool R32>
constexpr int tile_blocks() { return !UNIT ? 5 : (OPT == FEM_OPT_SGD && !R32 ? 6 : 7); }

// R32: the replica count is 32 (one sign word per node), a compile-time constant, so the
// state rows' offsets are immediates.
template <int OPT, bool UNIT, bool R32>
__global__ void __launch_bounds__(kThreads, tile_blocks<OPT, UNIT, R32>()) k_paper_tile(PArgs a, StepScalars s) {
  const int R = R32 ? 32 : a.R, wpn = R32 ? 1 : a.wpn;
  __shared__ __align__(128) Stage st[kStages];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages];
  __shared__ int32_t abort_flag;
  volatile int32_t* abort_v = &abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long tiles = (long long)((a.n + kNodes - 1) / kNodes) * wpn;
  if (threadIdx.x == 0) {
    for (int b = 0; b < kStages; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], kConsumers);
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto tile_pos = [&](long long t, int& i0, int& wb) {
    const long long nb = wpn == 1 ? t : t / wpn;
    wb = wpn == 1 ? 0 : (int)(t - nb * wpn);
    i0 = (int)nb * kNodes;
  };

  long long issued = 0;
  if (warp == kConsumers) {
    // ---- producer: row pointers three tiles, entries two tiles, words one tile ahead
    const long long G = gridDim.x;
    auto load_rp = [&](long long t) -> int {
      if (t >= tiles) return 0;
      int i0, wb;
      tile_pos(t, i0, wb);
      return lane <= kNodes ? __ldg(a.row_ptr + min(i0 + lane, a.n)) : 0;
    };
    auto load_cols = [&](long long t, int rp, uint32_t (&c)[kQ]) {
      if (t >= tiles) return;
      const int base = __shfl_sync(kFullMask, rp, 0), ecap = min(__shfl_sync(kFullMask, rp, kNodes) - base, kCap);
#pragma unroll
      for (int q = 0; q < kQ; ++q)
        if (lane + 32 * q < ecap) c[q] = __ldg(a.col + base + lane + 32 * q);
    };
    auto load_adj = [&](long long t, int rp, const uint32_t (&c)[kQ], uint32_t (&adj)[kQ], float (&w)[kQ],
                        float& cn) {
      if (t >= tiles) return;
      int i0, wb;
      tile_pos(t, i0, wb);
      const int base = __shfl_sync(kFullMask, rp, 0), ecap = min(__shfl_sync(kFullMask, rp, kNodes) - base, kCap);
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        const int k = lane + 32 * q;
        if (k < ecap) {
          const uint32_t wd = __ldg(a.words_in + (size_t)(c[q] & 0x7fffffffu) * wpn + wb);
          adj[q] = UNIT ? wd ^ (0u - (c[q] >> 31)) : wd;
          if (!UNIT) w[q] = __ldg(a.w + base + k);
        }
      }
      if (!UNIT) cn = __ldg(a.cnorm + min(i0 + lane, a.n - 1));
    };
    uint32_t c1[kQ], c2[kQ], a0[kQ], a1[kQ];
    float w0[kQ], w1[kQ], cn0 = 0.f, cn1 = 0.f;
    const long long t0 = blockIdx.x;
    int r0 = load_rp(t0), r1 = load_rp(t0 + G), r2 = load_rp(t0 + 2 * G), r3 = 0;
    {
      uint32_t c0[kQ];
      load_cols(t0, r0, c0);
      load_cols(t0 + G, r1, c1);
      load_adj(t0, r0, c0, a0, w0, cn0);
    }
    long long t = t0;
    for (long long it = 0; t < tiles; ++it) {
      r3 = load_rp(t + 3 * G);
      load_cols(t + 2 * G, r2, c2);
      load_adj(t + G, r1, c1, a1, w1, cn1);
      const int b = (int)(it % kStages);
      const uint32_t use = (uint32_t)(it / kStages);
      const bool ok = __all_sync(kFullMask, mbar_wait(&empty[b], (use & 1) ^ 1, a.err)) && !*abort_v;
      if (!ok) {
        *abort_v = 1;
        break;
      }
      Stage& S = st[b];
      int i0, wb;
      tile_pos(t, i0, wb);
      const int nn = min(kNodes, a.n - i0);
      const int base = __shfl_sync(kFullMask, r0, 0);
      const int ecap = min(__shfl_sync(kFullMask, r0, kNodes) - base, kCap);
      if (lane <= kNodes) S.rptr[lane] = r0 - base;
      if (lane == 0) S.base = base;
      if (!UNIT && lane < kNodes) S.cn[lane] = cn0;
      if (UNIT) {
        // per node of the tile (lane = node): 1/deg with the reciprocal of the direct
        // kernel's quotient, and the node's entry mask within its group's first 32 entries
        const int rnext = __shfl_down_sync(kFullMask, r0, 1);
        const int gfirst = __shfl_sync(kFullMask, r0, lane & ~(kNpw - 1) & 31);
        const int glast = __shfl_sync(kFullMask, r0, ((lane & ~(kNpw - 1)) + kNpw) & 31);
        if (lane < kNodes) {
          const int len = rnext - r0, off = r0 - gfirst;
          S.cn[lane] = len > 0 ? rcp_approx((float)len) : 0.f;
          S.mask[lane] = (glast - gfirst > 32 || len == 0) ? 0u
                         : (len >= 32 ? 0xffffffffu : ((1u << len) - 1u) << off);
        }
      }
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        const int k = lane + 32 * q;
        if (k < ecap) {
          S.adj[k] = a0[q];
          if (!UNIT) S.w[k] = w0[q];
        }
      }
      __syncwarp();
      const uint32_t rows_b = (uint32_t)nn * 128u;
      if (lane == 0) mbar_expect_tx(&full[b], rows_b * (OPT == FEM_OPT_SGD ? 2u : 3u));
      if (wpn == 1) {
        if (lane == 0) {
          const size_t off = (size_t)i0 * R;
          bulk_load(S.h, a.h + off, rows_b, &full[b]);
          bulk_load(S.m, a.m + off, rows_b, &full[b]);
          if (OPT != FEM_OPT_SGD) bulk_load(S.v, a.v + off, rows_b, &full[b]);
        }
      } else if (lane < nn) {
        const size_t off = (size_t)(i0 + lane) * R + (size_t)wb * 32;
        bulk_load(S.h + 32 * lane, a.h + off, 128u, &full[b]);
        bulk_load(S.m + 32 * lane, a.m + off, 128u, &full[b]);
        if (OPT != FEM_OPT_SGD) bulk_load(S.v + 32 * lane, a.v + off, 128u, &full[b]);
      }
      issued = it + 1;
      t += G;
      r0 = r1;
      r1 = r2;
      r2 = r3;
      cn0 = cn1;
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        c1[q] = c2[q];
        a0[q] = a1[q];
        w0[q] = w1[q];
      }
    }
  } else {
    // ---- consumers: warp w takes group w (nodes 4w .. 4w + 3) of each tile
    long long it = 0;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
      const int b = (int)(it % kStages);
      const uint32_t use = (uint32_t)(it / kStages);
      const bool ok = __all_sync(kFullMask, mbar_wait(&full[b], use & 1, a.err)) && !*abort_v;
      if (!ok) {
        *abort_v = 1;
        break;
      }
      const Stage& S = st[b];
      int i0t, wb;
      tile_pos(t, i0t, wb);
      const int i0 = i0t + kNpw * warp;
      if (i0 < a.n) {
        const int gbase = S.base;
        // entry e of the tile (relative to its base): the staged word, or beyond the
        // staged ones the direct load the direct kernel makes
        auto adj_at = [&](int e) -> uint32_t {
          if (e < kCap) return S.adj[e];
          const uint32_t c = __ldg(a.col + gbase + e);
          const uint32_t wd = __ldg(a.words_in + (size_t)(c & 0x7fffffffu) * wpn + wb);
          return UNIT ? wd ^ (0u - (c >> 31)) : wd;
        };
        auto w_at = [&](int e) -> float { return e < kCap ? S.w[e] : __ldg(a.w + gbase + e); };
        int rb[kNpw + 1];
#pragma unroll
        for (int k = 0; k <= kNpw; ++k) rb[k] = S.rptr[kNpw * warp + k];
        const int bN = rb[kNpw];
        float h[kNpw], m[kNpw], v[kNpw];
#pragma unroll
        for (int k = 0; k < kNpw; ++k) {
          const int j = kNpw * warp + k;
          const bool in = i0 + k < a.n;
          h[k] = in ? S.h[32 * j + lane] : 0.f;
          m[k] = in ? S.m[32 * j + lane] : 0.f;
          v[k] = (in && OPT != FEM_OPT_SGD) ? S.v[32 * j + lane] : 0.f;
        }
        int nneg_u[kNpw];
#pragma unroll
        for (int k = 0; k < kNpw; ++k) nneg_u[k] = 0;
        if (UNIT && bN - rb[0] <= 32) {
          const uint32_t adj = rb[0] + lane < bN ? adj_at(rb[0] + lane) : 0u;
          const uint32_t tr = warp_transpose32(adj, lane);
#pragma unroll
          for (int k = 0; k < kNpw; ++k) nneg_u[k] = __popc(tr & S.mask[kNpw * warp + k]);
        } else if (UNIT) {
          for (int c0 = rb[0]; c0 < bN; c0 += 32) {
            const uint32_t cur = c0 + lane < bN ? adj_at(c0 + lane) : 0u;
            const uint32_t tr = warp_transpose32(cur, lane);
#pragma unroll
            for (int k = 0; k < kNpw; ++k) {
              const int lo = max(rb[k], c0) - c0, hi = min(rb[k + 1], c0 + 32) - c0;
              if (hi > lo) {
                const int len = hi - lo;
                nneg_u[k] += __popc(tr & ((len >= 32 ? 0xffffffffu : ((1u << len) - 1u)) << lo));
              }
            }
          }
        }
        uint32_t ball[kNpw];
#pragma unroll
        for (int k = 0; k < kNpw; ++k) {
          float facc = 0.f;
          if (!UNIT) {
            for (int e = rb[k]; e < rb[k + 1]; ++e) {
              const uint32_t bit = (adj_at(e) >> lane) & 1u;
              const float w = w_at(e);
              facc += bit ? -w : w;
            }
          }
          const int deg = rb[k + 1] - rb[k];
          // unit weights: div_approx((float)(deg - 2 nneg), (float)deg) of the direct kernel,
          // with the producer's reciprocal (0 for deg = 0, where the numerator is 0 too)
          const float field = UNIT ? __fmul_rn((float)(deg - 2 * nneg_u[k]), S.cn[kNpw * warp + k])
                                   : (S.cn[kNpw * warp + k] * facc);
          float hk = h[k], mk = m[k], vk = v[k];
          const float gk = s.gq * (field + hk * s.inv_beta) * one_minus_m2_fast(hk);
          opt_update_fast<OPT>(hk, mk, vk, gk, s);
          ball[k] = __ballot_sync(kFullMask, hk < 0.f);
          if (i0 + k < a.n) {
            const size_t idx = (size_t)(i0 + k) * R + (size_t)wb * 32 + lane;
            a.h[idx] = hk;
            a.m[idx] = mk;
            if (OPT != FEM_OPT_SGD) a.v[idx] = vk;
          }
        }
        uint32_t mine = ball[0];
#pragma unroll
        for (int k = 1; k < kNpw; ++k) mine = lane == k ? ball[k] : mine;
        if (lane < kNpw && i0 + lane < a.n) a.words_out[(size_t)(i0 + lane) * wpn + wb] = mine;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[b]);
    }
  }
  __syncthreads();
  if (threadIdx.x == kConsumers * 32) {
    // the last fills of the stages have landed before the block's shared memory is released
    for (long long k = issued - kStages < 0 ? 0 : issued - kStages; k < issued; ++k)
      mbar_wait(&full[k % kStages], (uint32_t)((k / kStages) & 1), a.err);
  }
}

template <int OPT, bool UNIT, bool R32>
fem_status launch(const PArgs& a, const StepScalars& s, int sm_count, cudaStream_t st) {
  constexpr auto k = k_paper_tile<OPT, UNIT, R32>;
  static int per_sm = 0;
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0) != cudaSuccess || per_sm < 1) {
      cudaGetLastError();
      per_sm = 0;
      return fail(FEM_ERR_CUDA, "paper-mode tile kernel: no resident block");
    }
  }
  const long long tiles = (long long)((a.n + kNodes - 1) / kNodes) * a.wpn;
  long long grid = (long long)per_sm * sm_count;
  if (grid > tiles) grid = tiles;
  k<<<(int)(grid < 1 ? 1 : grid), kThreads, 0, st>>>(a, s);
  return FEM_OK;
}

}  // namespace

// One paper-mode step of a sparse MaxCut problem (h, m, v in place), reading words[in]
// and writing words[in ^ 1].
fem_status maxcut_paper_tile_step(Problem* p, int in, const StepScalars& s, cudaStream_t st) {
  PArgs a{};
  a.row_ptr = p->row_ptr;
  a.col = p->col;
  a.w = p->unit_w ? nullptr : p->w;
  a.cnorm = p->cnorm;
  a.n = p->n;
  a.R = p->R;
  a.wpn = p->words_per_node;
  a.h = p->h[0];
  a.m = p->m;
  a.v = p->v;
  a.words_in = p->words[in];
  a.words_out = p->words[in ^ 1];
  a.err = p->err;
  const bool unit = p->unit_w;
  if (p->R == 32) {
    switch (p->optimizer) {
      case FEM_OPT_ADAM: return unit ? launch<FEM_OPT_ADAM, true, true>(a, s, p->sm_count, st)
                                     : launch<FEM_OPT_ADAM, false, true>(a, s, p->sm_count, st);
      case FEM_OPT_RMSPROP: return unit ? launch<FEM_OPT_RMSPROP, true, true>(a, s, p->sm_count, st)
                                        : launch<FEM_OPT_RMSPROP, false, true>(a, s, p->sm_count, st);
      default: return unit ? launch<FEM_OPT_SGD, true, true>(a, s, p->sm_count, st)
                           : launch<FEM_OPT_SGD, false, true>(a, s, p->sm_count, st);
    }
  }
  switch (p->optimizer) {
    case FEM_OPT_ADAM: return unit ? launch<FEM_OPT_ADAM, true, false>(a, s, p->sm_count, st)
                                   : launch<FEM_OPT_ADAM, false, false>(a, s, p->sm_count, st);
    case FEM_OPT_RMSPROP: return unit ? launch<FEM_OPT_RMSPROP, true, false>(a, s, p->sm_count, st)
                                      : launch<FEM_OPT_RMSPROP, false, false>(a, s, p->sm_count, st);
    default: return unit ? launch<FEM_OPT_SGD, true, false>(a, s, p->sm_count, st)
                         : launch<FEM_OPT_SGD, false, false>(a, s, p->sm_count, st);
  }
}

}  // namespace fem
