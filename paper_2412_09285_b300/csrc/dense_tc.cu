// MaxCut on dense couplings (complete graphs, e.g. Sherrington-Kirkpatrick J = +-1):
// the per-step contraction S = J M on the tcgen05 tensor cores with the single-field
// gradient and the optimizer fused into the epilogue, a CUDA-core fp32 variant of the
// same step, and an exact integer read-out.
//
// Step t, replica r, row i (SM Eq. grad_m_h):
//   paper: S_ir = sum_j J_ij sgn(m_jr),  g = (gamma/4)[c_i S_ir + h_ir/beta](1 - m_ir^2)
//   exact: S_ir = sum_j J_ij m_jr,       g = (gamma/4)[2 S_ir + h_ir/beta](1 - m_ir^2)
// c_i = 1/sum_j |J_ij|.  sgn(m) = +-1 and integer J are exact in bf16 and (|J| <= 16)
// in e4m3, and the fp32 accumulation of at most 2^24 unit terms is exact, so the
// paper-mode contraction is bit-exact on the tensor cores.  In exact mode m is split
// into m_hi = bf16(m) and m_lo = bf16(m - m_hi) and both products accumulate into the
// same TMEM tile (about 16 bits of m).
//
// Layout (dense problems only): h, m, v are [R][n_pad] fp32 (rows of one replica
// contiguous), so the epilogue thread that owns row i of a tile reads and writes
// consecutive addresses across a warp for every replica column.  The next step's
// operand M^T is written as [R][n_pad] bf16 / e4m3, K-major for the tensor cores.
//
// Tensor-core kernel: CTA = 512 threads, tile = 128 rows (i) x 128 replicas (r),
// K loop over j in 128-byte chunks fed by TMA (128B swizzle) through a 6-stage
// (hi+lo: 4-stage) mbarrier pipeline; thread 0 issues the copies, thread 32 issues
// tcgen05.mma into a 128-column fp32 TMEM accumulator; then all 16 warps read TMEM
// (tcgen05.ld 32x32b: warp w owns lane quadrant w%4 and 32 replica columns) and run
// the fused epilogue.  Every wait is bounded in time; on expiry the kernel records
// FEM's timeout bit and leaves, freeing its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "fem_internal.h"
#include "step_common.cuh"

namespace fem {
namespace {

constexpr int kTile = 128;        // rows (i) and replica columns (r) per CTA
constexpr int kMaxStages = 6;
constexpr int kThreads = 512;  // 16 warps: all run the epilogue (lane quadrant = warp % 4)
__host__ __device__ constexpr int stages_for(int prec) { return prec == FEM_PREC_BF16X2 ? 4 : 6; }
constexpr int kChunkBytes = 128;  // K bytes per pipeline stage (one swizzle row)
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on any wait

struct DenseArgs {
  int32_t n, n_pad, R, opt, mode, prec;
  float* h;
  float* m;
  float* v;
  const float* cnorm;
  void* mt_out;     // next step's operand (bf16 or e4m3), [R][n_pad]
  void* mt_lo_out;  // exact mode low part (bf16) or NULL
  int32_t* err;
  int64_t* part;  // read-out: per (row tile, replica) partial sums
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
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
// Bounded wait: false (and the timeout bit set) if the phase has not completed in kWaitNs.
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
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// CTA pair: a copy into this CTA's shared memory whose completion is counted on an
// mbarrier of the pair's even CTA (`bar` is its shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// CTA-pair forms: one warp of each CTA of the pair executes them; the allocation has
// the same address in both CTAs.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Every thread of both CTAs of the pair; also orders their memory accesses.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared variable in the CTA of the given rank of this cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// CTA pair (M = 256): A rows 0..127 come from this CTA's shared memory and rows
// 128..255 from the same offsets in the other CTA's; B's N columns are split the same
// way, and each CTA's tensor memory receives its own 128 rows of D.
__device__ __forceinline__ void umma_f16_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_f8_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// Arrives on the barrier at this offset in both CTAs of the pair once the MMAs issued
// so far have completed.
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar) {
  const uint16_t both = 0x3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(both)
      : "memory");
}
// TMEM <-> registers, 32 lanes x 8 columns.  A load is issued without waiting; its
// outputs are tied to tmem_wait_ld, which every reader calls first (it waits for all
// earlier loads of the thread), so no use can be scheduled before the data arrives.
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05) for a K-major tile whose rows are 128
// bytes with the 128-byte swizzle: start address >> 4, leading offset unused (1),
// stride between 8-row groups 1024 B, descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: fp32 accumulator, A and B of format `fmt` (kind::f16:
// 1 = bf16; kind::f8f6f4: 0 = e4m3), both K-major, N = 128, M = 128 (one CTA) or
// 256 (a CTA pair).
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t m = kTile) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTile >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// One element of the fused epilogue: the gradient from the accumulated field S_ir
// and the optimizer update of (h, m, v).  Returns the next step's operand entry (bf16
// or e4m3 bits; with the bf16 hi+lo split the low part goes to *lo); the caller
// stores it.  Branch-free for Adam at fixed (PREC, OPT, PAPER), so the elements of
// a chunk interleave.
template <int PREC, int OPT, bool PAPER>
__device__ __forceinline__ uint32_t epi_element(const StepScalars& s, float cn, uint32_t acc_bits, float& h,
                                                float& m, float& v, uint32_t* lo) {
  // explicit roundings: the per-step and the persistent kernels agree bit for bit
  const float field = __fmul_rn(cn, __uint_as_float(acc_bits));
  float g = __fmul_rn(__fmul_rn(s.gq, fmaf(h, s.inv_beta, field)), one_minus_m2_fast(h));
  g = fmaf(s.wd, h, g);  // L2 weight decay; exactly g when wd == 0
  opt_update_fast_core<OPT>(h, m, v, g, s);
  if (PAPER) {
    *lo = 0u;
    if (PREC == FEM_PREC_FP8) return h < 0.f ? 0xB8u : 0x38u;  // e4m3 -1 / +1
    return h < 0.f ? 0xBF80u : 0x3F80u;                        // bf16 -1 / +1
  }
  const float mm = tanhf(0.5f * h);
  const uint16_t hi = bf16_bits(mm);
  *lo = PREC == FEM_PREC_BF16X2 ? bf16_bits(mm - __bfloat162float(__ushort_as_bfloat16(hi))) : 0u;
  return hi;
}

// Calls f(OPT, PAPER) with the run-time optimizer and gradient mode as compile-time
// constants (one warp-uniform branch per call instead of several per element).
template <class F>
__device__ __forceinline__ void with_opt_mode(int opt, int mode, F&& f) {
  using A = std::integral_constant<int, FEM_OPT_ADAM>;
  using Rm = std::integral_constant<int, FEM_OPT_RMSPROP>;
  using Sg = std::integral_constant<int, FEM_OPT_SGD>;
  if (mode == FEM_GRAD_PAPER) {
    if (opt == FEM_OPT_ADAM) f(A{}, std::true_type{});
    else if (opt == FEM_OPT_RMSPROP) f(Rm{}, std::true_type{});
    else f(Sg{}, std::true_type{});
  } else {
    if (opt == FEM_OPT_ADAM) f(A{}, std::false_type{});
    else if (opt == FEM_OPT_RMSPROP) f(Rm{}, std::false_type{});
    else f(Sg{}, std::false_type{});
  }
}

template <int PREC>
__device__ __forceinline__ void store_operand(void* base, size_t idx, uint32_t bits) {
  if (PREC == FEM_PREC_FP8) reinterpret_cast<uint8_t*>(base)[idx] = (uint8_t)bits;
  else reinterpret_cast<uint16_t*>(base)[idx] = (uint16_t)bits;
}

// ------------------------------------------------------------ the fused step
// READ: the exact read-out instead of a step.  With B = sgn(h) (+-1) the accumulator
// holds S_ir = sum_j J_ij s_jr exactly, and the epilogue writes the partial
// Q_r = sum_{i in tile} s_ir S_ir to a.part[blockIdx.x][r] (no state is changed).
template <int PREC, bool READ = false>  // FEM_PREC_BF16, FEM_PREC_BF16X2 or FEM_PREC_FP8
__global__ void __launch_bounds__(kThreads, 1) k_dense_step_tc(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB,
                                                         const __grid_constant__ CUtensorMap tmBlo,
                                                         DenseArgs a, StepScalars s) {
  constexpr bool X2 = PREC == FEM_PREC_BF16X2;
  constexpr int kElem = PREC == FEM_PREC_FP8 ? 1 : 2;
  constexpr int kChunkK = kChunkBytes / kElem;     // K elements per stage
  constexpr int kMmaK = PREC == FEM_PREC_FP8 ? 32 : 16;
  constexpr uint32_t kTileBytes = kTile * kChunkBytes;  // 16 KB
  constexpr uint32_t kStageBytes = kTileBytes * (X2 ? 3 : 2);
  constexpr uint32_t kIdesc = make_idesc(PREC == FEM_PREC_FP8 ? 0u : 1u);

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int kStages = stages_for(PREC);
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t empty[kMaxStages];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base_slot;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i0 = blockIdx.x * kTile, r0 = blockIdx.y * kTile;
  const int nchunks = a.n_pad / kChunkK;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_base_slot, kTile);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;

  if (threadIdx.x == 0) {
    // producer: TMA copies of J rows i0.. and M^T rows r0.. for every K chunk
    for (int k = 0; k < nchunks; ++k) {
      const int st = k % kStages;
      if (!mbar_wait(&empty[st], ((k / kStages) & 1) ^ 1, a.err)) break;
      uint8_t* sa = smem + st * kStageBytes;
      mbar_expect_tx(&full[st], kStageBytes);
      tma_load_2d(sa, &tmA, k * kChunkK, i0, &full[st]);
      tma_load_2d(sa + kTileBytes, &tmB, k * kChunkK, r0, &full[st]);
      if (X2) tma_load_2d(sa + 2 * kTileBytes, &tmBlo, k * kChunkK, r0, &full[st]);
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer: 128 / (mma K bytes) instructions per stage into the TMEM tile
    for (int k = 0; k < nchunks; ++k) {
      const int st = k % kStages;
      if (!mbar_wait(&full[st], (k / kStages) & 1, a.err)) break;
      tc_fence_after();
      const uint32_t sa = smem_u32(smem + st * kStageBytes);
      const uint64_t da = desc_sw128(sa), db = desc_sw128(sa + kTileBytes);
      const uint64_t dblo = desc_sw128(sa + 2 * kTileBytes);
#pragma unroll
      for (int kk = 0; kk < kChunkK / kMmaK; ++kk) {
        const uint64_t adv = (uint64_t)((kk * kMmaK * kElem) >> 4);
        const uint32_t acc = (k > 0 || kk > 0) ? 1u : 0u;
        if (PREC == FEM_PREC_FP8) umma_f8(tmem, da + adv, db + adv, kIdesc, acc);
        else umma_f16(tmem, da + adv, db + adv, kIdesc, acc);
        if (X2) umma_f16(tmem, da + adv, dblo + adv, kIdesc, 1u);
      }
      umma_commit(&empty[st]);  // frees the stage once these MMAs have read it
    }
    umma_commit(&done);
  }
  __syncwarp();

  if constexpr (READ) {
    __shared__ int32_t red[4][kTile];
    const int quad = warp & 3, c0 = (warp >> 2) * 32;
    const int i = i0 + quad * 32 + lane;
    const bool row = i < a.n;
    const bool ok = mbar_wait(&done, 0, a.err);
    tc_fence_after();
    if (__all_sync(kFullMask, ok)) {
#pragma unroll 1
      for (int cb = 0; cb < 32; cb += 8) {
        float hv[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) hv[c] = row ? a.h[(size_t)(r0 + c0 + cb + c) * a.n_pad + i] : 0.f;
        uint32_t acc[8];
        tmem_ld8_issue(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c0 + cb), acc);
        tmem_wait_ld(acc);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int S = (int)__uint_as_float(acc[c]);
          const int v = row ? (hv[c] >= 0.f ? S : -S) : 0;
          const int tot = __reduce_add_sync(kFullMask, v);
          if (lane == 0) red[quad][c0 + cb + c] = tot;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < kTile)
      a.part[(size_t)blockIdx.x * a.R + r0 + threadIdx.x] =
          (int64_t)red[0][threadIdx.x] + red[1][threadIdx.x] + red[2][threadIdx.x] + red[3][threadIdx.x];
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
      tc_fence_after();
      tmem_dealloc(tmem, kTile);
    }
    return;
  }

  // epilogue: thread = TMEM lane = row i of the tile.  Warp w reads TMEM lanes
  // 32*(w%4).. (its quadrant) and the 32 replica columns 32*(w/4)..; the state of 8
  // columns is loaded in one batch (the first batch before the MMAs complete), so a
  // thread waits for four memory round trips instead of one per column.
  constexpr int kB = 8;
  const int quad = warp & 3, c0 = (warp >> 2) * 32;
  const int i = i0 + quad * 32 + lane;
  const bool row = i < a.n;
  const bool sgd = a.opt == FEM_OPT_SGD;
  float* __restrict__ h_io = a.h;
  float* __restrict__ m_io = a.m;
  float* __restrict__ v_io = a.v;
  float hv[kB], mv[kB], vv[kB];
  auto load_batch = [&](int cb) {
#pragma unroll
    for (int c = 0; c < kB; ++c) {
      const size_t idx = (size_t)(r0 + c0 + cb + c) * a.n_pad + i;
      hv[c] = h_io[idx];
      mv[c] = m_io[idx];
      vv[c] = sgd ? 0.f : v_io[idx];
    }
  };
  if (row) load_batch(0);
  const bool ok = mbar_wait(&done, 0, a.err);
  tc_fence_after();
  if (__all_sync(kFullMask, ok)) {
    const float cn = row ? (a.mode == FEM_GRAD_PAPER ? a.cnorm[i] : 2.f) : 0.f;
#pragma unroll 1
    for (int cb = 0; cb < 32; cb += kB) {  // R % 128 == 0: every column is a replica
      uint32_t acc[kB];
      tmem_ld8_issue(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(c0 + cb), acc);
      tmem_wait_ld(acc);
      if (!row) continue;
      if (cb > 0) load_batch(cb);
      with_opt_mode(a.opt, a.mode, [&](auto O, auto P) {
        constexpr int OPT = decltype(O)::value;
        constexpr bool PAPER = decltype(P)::value;
#pragma unroll
        for (int c = 0; c < kB; ++c) {
          const size_t idx = (size_t)(r0 + c0 + cb + c) * a.n_pad + i;
          float h = hv[c], m = mv[c], v = vv[c];
          uint32_t lo;
          store_operand<PREC>(a.mt_out, idx, epi_element<PREC, OPT, PAPER>(s, cn, acc[c], h, m, v, &lo));
          if (X2 && !PAPER) reinterpret_cast<uint16_t*>(a.mt_lo_out)[idx] = (uint16_t)lo;
          h_io[idx] = h;
          m_io[idx] = m;
          if (OPT != FEM_OPT_SGD) v_io[idx] = v;
        }
      });
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTile);
  }
}

// --------------------------------------------- persistent anneal (one launch)
// The step above, run for a whole window of steps by one launch.  Each CTA keeps its
// 128 x 128 tile of h, m and v in tensor memory for the whole window (TMEM columns
// 128.., 256.., 384..; the accumulator uses 0..127), so the optimizer state is read
// from global memory once at the start and written once at the end.
//
// Per step the only data a CTA needs from other CTAs is the next operand M^T of its
// replica block, written by the n_pad/128 CTAs that share blockIdx.y; those CTAs meet
// at a counter barrier in global memory after each step (release/acquire at GPU
// scope, plus a proxy fence because the operand is written with ordinary stores and
// read by TMA).
//
// PAIR: two CTAs (a cluster of 2, row tiles 2p and 2p + 1) issue M = 256 MMAs
// together.  Each loads its own 128 rows of J and half of the 128 replica columns of
// M^T, so a CTA copies 1.5 instead of 2 bytes into shared memory per byte of J it
// uses.  Both CTAs' copies of a stage complete on the even CTA's barrier, which
// expects the bytes of both; the even CTA issues the MMAs, and its commits arrive on
// the barriers of both CTAs.
//
// All waits are bounded; a CTA that gives up records the timeout bit, lets its copies
// and MMAs in flight land, frees its TMEM and leaves, and the CTAs waiting for it give
// up in turn.
constexpr int kTmemCols = 4 * kTile;  // accumulator, h, m, v

struct DenseAnnealArgs {
  DenseArgs a;               // h, m, v ([R][n_pad], read at the start, written at the end), cnorm, err
  void* mt[2];               // operand ping-pong: step t reads mt[t & 1] and writes mt[(t + 1) & 1]
  void* mt_lo[2];            // exact mode low parts (bf16 hi + lo), else NULL
  const StepScalars* sc;     // [n_steps], the scalars of steps t_begin ..
  int32_t t_begin, n_steps;
  int32_t* bar;              // one arrival counter per replica block (stride 32 ints), zero at launch
  unsigned long long bar_wait_ns;  // limit on the step barrier (the copy and MMA waits keep kWaitNs)
  int32_t stall_tile;        // tests: the CTAs of this row tile never arrive at the barrier (-1: none)
};

__device__ __forceinline__ bool wait_counter(const int32_t* ctr, int32_t target, int32_t* err,
                                             unsigned long long limit_ns) {
  const unsigned long long t0 = global_ns();
  while (true) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= target) return true;
    if (global_ns() - t0 >= limit_ns) {
      atomicOr(err, ERR_TIMEOUT);
      return false;
    }
  }
}

__host__ __device__ constexpr int anneal_stages(int prec, bool pair) {
  return pair ? (prec == FEM_PREC_BF16X2 ? 6 : 8) : stages_for(prec);
}
__host__ __device__ constexpr uint32_t anneal_stage_bytes(int prec, bool pair) {
  return (uint32_t)(kTile * kChunkBytes + (pair ? kTile / 2 : kTile) * kChunkBytes * (prec == FEM_PREC_BF16X2 ? 2 : 1));
}
constexpr int kMaxAnnealStages = 8;

template <int PREC, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1) k_dense_anneal_tc(const __grid_constant__ CUtensorMap tmA,
                                                           const __grid_constant__ CUtensorMap tmB0,
                                                           const __grid_constant__ CUtensorMap tmB1,
                                                           const __grid_constant__ CUtensorMap tmBlo0,
                                                           const __grid_constant__ CUtensorMap tmBlo1,
                                                           const DenseAnnealArgs x) {
  constexpr bool X2 = PREC == FEM_PREC_BF16X2;
  constexpr int kElem = PREC == FEM_PREC_FP8 ? 1 : 2;
  constexpr int kChunkK = kChunkBytes / kElem;
  constexpr int kMmaK = PREC == FEM_PREC_FP8 ? 32 : 16;
  constexpr int kBRows = PAIR ? kTile / 2 : kTile;  // replica rows of M^T this CTA copies
  constexpr uint32_t kATileBytes = kTile * kChunkBytes;
  constexpr uint32_t kBTileBytes = kBRows * kChunkBytes;
  constexpr uint32_t kStageBytes = anneal_stage_bytes(PREC, PAIR);
  constexpr uint32_t kIdesc = make_idesc(PREC == FEM_PREC_FP8 ? 0u : 1u, PAIR ? 2 * kTile : kTile);
  constexpr int kStages = anneal_stages(PREC, PAIR);
  static_assert(kStageBytes % 1024 == 0 && kBTileBytes % 1024 == 0, "128B-swizzled tiles need 1 KB alignment");
  constexpr int kCols = 8;  // replica columns per TMEM load / store in the epilogue

  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kMaxAnnealStages];
  __shared__ __align__(8) uint64_t empty[kMaxAnnealStages];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tmem_base_slot;
  __shared__ int32_t abort_flag;
  __shared__ StepScalars s_sc[2];  // step k's scalars in s_sc[k & 1] (thread 0 loads the next during step k)
  volatile int32_t* abort_v = &abort_flag;

  const DenseArgs& a = x.a;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool issuer = rank == 0;  // issues the MMAs (always, without PAIR)
  const int i0 = blockIdx.x * kTile, r0 = blockIdx.y * kTile;
  const int nchunks = a.n_pad / kChunkK;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    if (x.n_steps > 0) s_sc[0] = x.sc[0];
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (PAIR) cluster_sync_all();  // the other CTA's barriers exist before anything arrives on them
  if (warp == 0) {
    if (PAIR) tmem_alloc_pair(&tmem_base_slot, kTmemCols);
    else tmem_alloc(&tmem_base_slot, kTmemCols);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_slot;

  // epilogue geometry: thread = TMEM lane = row i; warp w owns lane quadrant w % 4
  // and the 32 replica columns 32 * (w / 4) ..
  const int quad = warp & 3, c0 = (warp >> 2) * 32;
  const int i = i0 + quad * 32 + lane;
  const bool row = i < a.n;
  const bool sgd = a.opt == FEM_OPT_SGD;
  const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;  // + region * kTile + column
  const float cn = row ? (a.mode == FEM_GRAD_PAPER ? a.cnorm[i] : 2.f) : 0.f;

  // state: global [R][n_pad] -> TMEM (padding rows hold zeros and are never updated)
#pragma unroll
  for (int cb = 0; cb < 32; cb += kCols) {
    uint32_t hr[kCols], mr[kCols], vr[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) {
      const size_t idx = (size_t)(r0 + c0 + cb + c) * a.n_pad + i;
      hr[c] = row ? __float_as_uint(a.h[idx]) : 0u;
      mr[c] = row ? __float_as_uint(a.m[idx]) : 0u;
      vr[c] = (row && !sgd) ? __float_as_uint(a.v[idx]) : 0u;
    }
    tmem_st8(tl + 1 * kTile + cb, hr);
    tmem_st8(tl + 2 * kTile + cb, mr);
    tmem_st8(tl + 3 * kTile + cb, vr);
  }
  tmem_wait_st();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  int issued = 0;  // producer: TMA stage loads issued so far (thread 0 only)
  for (int k = 0; k < x.n_steps; ++k) {
    const int t = x.t_begin + k, in = t & 1;
    if (threadIdx.x == 0) {
      const CUtensorMap* mb = in ? &tmB1 : &tmB0;
      const CUtensorMap* mlo = in ? &tmBlo1 : &tmBlo0;
      for (int kc = 0; kc < nchunks; ++kc) {
        const int g = k * nchunks + kc, st = g % kStages;
        if (!mbar_wait(&empty[st], ((g / kStages) & 1) ^ 1, a.err)) {
          *abort_v = 1;
          break;
        }
        uint8_t* sa = smem + st * kStageBytes;
        const int x0 = kc * kChunkK, rb = r0 + (int)rank * kBRows;
        if (issuer) {
          mbar_expect_tx(&full[st], PAIR ? 2 * kStageBytes : kStageBytes);  // a pair: both CTAs' copies
          tma_load_2d(sa, &tmA, x0, i0, &full[st]);
          tma_load_2d(sa + kATileBytes, mb, x0, rb, &full[st]);
          if (X2) tma_load_2d(sa + kATileBytes + kBTileBytes, mlo, x0, rb, &full[st]);
        } else {
          const uint32_t bar = cluster_addr(&full[st], 0);
          tma_load_2d_pair(sa, &tmA, x0, i0, bar);
          tma_load_2d_pair(sa + kATileBytes, mb, x0, rb, bar);
          if (X2) tma_load_2d_pair(sa + kATileBytes + kBTileBytes, mlo, x0, rb, bar);
        }
        issued = g + 1;
      }
      if (k + 1 < x.n_steps) s_sc[(k + 1) & 1] = x.sc[k + 1];  // read by step k + 1's epilogue
    } else if (threadIdx.x == 32 && issuer) {
      for (int kc = 0; kc < nchunks; ++kc) {
        const int g = k * nchunks + kc, st = g % kStages;
        if (!mbar_wait(&full[st], (g / kStages) & 1, a.err)) {
          *abort_v = 1;
          break;
        }
        tc_fence_after();
        const uint32_t sa = smem_u32(smem + st * kStageBytes);
        const uint64_t da = desc_sw128(sa), db = desc_sw128(sa + kATileBytes);
        const uint64_t dblo = desc_sw128(sa + kATileBytes + kBTileBytes);
#pragma unroll
        for (int kk = 0; kk < kChunkK / kMmaK; ++kk) {
          const uint64_t adv = (uint64_t)((kk * kMmaK * kElem) >> 4);
          const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
          if (PAIR) {
            if (PREC == FEM_PREC_FP8) umma_f8_pair(tmem, da + adv, db + adv, kIdesc, acc);
            else umma_f16_pair(tmem, da + adv, db + adv, kIdesc, acc);
            if (X2) umma_f16_pair(tmem, da + adv, dblo + adv, kIdesc, 1u);
          } else {
            if (PREC == FEM_PREC_FP8) umma_f8(tmem, da + adv, db + adv, kIdesc, acc);
            else umma_f16(tmem, da + adv, db + adv, kIdesc, acc);
            if (X2) umma_f16(tmem, da + adv, dblo + adv, kIdesc, 1u);
          }
        }
        if (PAIR) umma_commit_pair(&empty[st]);
        else umma_commit(&empty[st]);
      }
      // also after a failed wait: done then tracks the MMAs issued
      if (PAIR) umma_commit_pair(&done);
      else umma_commit(&done);
    }
    __syncwarp();

    const bool ok = mbar_wait(&done, k & 1, a.err);
    tc_fence_after();
    if (!ok) *abort_v = 1;
    if (__all_sync(kFullMask, ok) && !*abort_v) {
      const StepScalars s = s_sc[k & 1];  // registers: the operand stores below are generic and could alias it
      void* mt_out = x.mt[(t + 1) & 1];
      void* mt_lo_out = x.mt_lo[(t + 1) & 1];
#pragma unroll
      for (int cb = 0; cb < 32; cb += kCols) {
        uint32_t acc[kCols], hr[kCols], mr[kCols], vr[kCols];
        tmem_ld8_issue(tl + cb, acc);
        tmem_ld8_issue(tl + 1 * kTile + cb, hr);
        tmem_ld8_issue(tl + 2 * kTile + cb, mr);
        tmem_ld8_issue(tl + 3 * kTile + cb, vr);
        tmem_wait_ld(acc);
        tmem_wait_ld(hr);
        tmem_wait_ld(mr);
        tmem_wait_ld(vr);
        if (row) {
          // all arithmetic of the chunk first, then its operand stores
          with_opt_mode(a.opt, a.mode, [&](auto O, auto P) {
            constexpr int OPT = decltype(O)::value;
            constexpr bool PAPER = decltype(P)::value;
            uint32_t lo[kCols];
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
              float h = __uint_as_float(hr[c]), m = __uint_as_float(mr[c]);
              float v = OPT == FEM_OPT_SGD ? 0.f : __uint_as_float(vr[c]);
              acc[c] = epi_element<PREC, OPT, PAPER>(s, cn, acc[c], h, m, v, &lo[c]);
              hr[c] = __float_as_uint(h);
              mr[c] = __float_as_uint(m);
              vr[c] = __float_as_uint(v);
            }
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
              const size_t idx = (size_t)(r0 + c0 + cb + c) * a.n_pad + i;
              store_operand<PREC>(mt_out, idx, acc[c]);
              if (X2 && !PAPER) reinterpret_cast<uint16_t*>(mt_lo_out)[idx] = (uint16_t)lo[c];
            }
          });
        }
        tmem_st8(tl + 1 * kTile + cb, hr);
        tmem_st8(tl + 2 * kTile + cb, mr);
        tmem_st8(tl + 3 * kTile + cb, vr);
      }
      tmem_wait_st();
    }

    // the operand of step t + 1 is complete once every CTA of this replica block is here
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && k + 1 < x.n_steps && !*abort_v) {
      int32_t* ctr = x.bar + blockIdx.y * 32;
      asm volatile("fence.proxy.async.global;" ::: "memory");
      if ((int)blockIdx.x != x.stall_tile)
        asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(ctr) : "memory");  // cumulative over bar.sync
      if (!wait_counter(ctr, (k + 1) * (int32_t)gridDim.x, a.err, x.bar_wait_ns)) *abort_v = 1;
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    if (*abort_v) break;
  }

  if (*abort_v) {
    // let the stage loads still in flight land before the CTA's shared memory is released
    // (a pair's odd CTA counts its copies on the even CTA's barriers, which wait for both)
    if (threadIdx.x == 0 && issuer)
      for (int g = issued - kStages < 0 ? 0 : issued - kStages; g < issued; ++g)
        mbar_wait(&full[g % kStages], (g / kStages) & 1, a.err);
  } else {
    // state: TMEM -> global
#pragma unroll
    for (int cb = 0; cb < 32; cb += kCols) {
      uint32_t hr[kCols], mr[kCols], vr[kCols];
      tmem_ld8_issue(tl + 1 * kTile + cb, hr);
      tmem_ld8_issue(tl + 2 * kTile + cb, mr);
      tmem_ld8_issue(tl + 3 * kTile + cb, vr);
      tmem_wait_ld(hr);
      tmem_wait_ld(mr);
      tmem_wait_ld(vr);
      if (row) {
#pragma unroll
        for (int c = 0; c < kCols; ++c) {
          const size_t idx = (size_t)(r0 + c0 + cb + c) * a.n_pad + i;
          a.h[idx] = __uint_as_float(hr[c]);
          a.m[idx] = __uint_as_float(mr[c]);
          if (!sgd) a.v[idx] = __uint_as_float(vr[c]);
        }
      }
    }
  }
  tc_fence_before();
  // neither CTA of a pair leaves while the other may still use its shared or tensor memory
  if (PAIR) cluster_sync_all();
  else __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    if (PAIR) tmem_dealloc_pair(tmem, kTmemCols);
    else tmem_dealloc(tmem, kTmemCols);
  }
}

// ------------------------------------------- CUDA-core fp32 step (the plain FEM)
// S = J M^T on the CUDA cores: a 128 x 128 output tile (rows i x replicas r) per
// 256-thread block, 8 x 8 per thread as two 4 x 4 quadrants 64 apart (so the
// epilogue's float4 accesses of h, m, v along i coalesce across the 16 threads of a
// row), K in tiles of 8 staged k-major in shared memory and double-buffered: the next
// tile's global loads are in flight while the current one is multiplied.  The same
// epilogue as the tensor-core kernels, in fp32 with IEEE operations.
constexpr int kF32Tile = 128, kF32K = 8;

__global__ void __launch_bounds__(256) k_dense_step_fp32(const float* __restrict__ J, const float* __restrict__ M,
                                                         DenseArgs a, StepScalars s) {
  __shared__ __align__(16) float sJ[2][kF32K][kF32Tile];
  __shared__ __align__(16) float sM[2][kF32K][kF32Tile];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * kF32Tile, r0 = blockIdx.y * kF32Tile;
  // global -> shared: thread t moves 4 consecutive k of row t / 2 of each operand tile
  const int lrow = tid >> 1, lk = (tid & 1) * 4;
  const float* gJ = J + (size_t)(i0 + lrow) * a.n_pad + lk;
  const bool mrow = r0 + lrow < a.R;
  const float* gM = M + (size_t)(mrow ? r0 + lrow : 0) * a.n_pad + lk;
  float4 nj = *reinterpret_cast<const float4*>(gJ);
  float4 nm = mrow ? *reinterpret_cast<const float4*>(gM) : make_float4(0.f, 0.f, 0.f, 0.f);
  auto stash = [&](int b) {
    sJ[b][lk + 0][lrow] = nj.x; sJ[b][lk + 1][lrow] = nj.y; sJ[b][lk + 2][lrow] = nj.z; sJ[b][lk + 3][lrow] = nj.w;
    sM[b][lk + 0][lrow] = nm.x; sM[b][lk + 1][lrow] = nm.y; sM[b][lk + 2][lrow] = nm.z; sM[b][lk + 3][lrow] = nm.w;
  };
  stash(0);
  __syncthreads();
  float acc[8][8];
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[p][q] = 0.f;
  const int ntiles = a.n_pad / kF32K;
  for (int kt = 0; kt < ntiles; ++kt) {
    const int b = kt & 1;
    if (kt + 1 < ntiles) {
      nj = *reinterpret_cast<const float4*>(gJ + (kt + 1) * kF32K);
      nm = mrow ? *reinterpret_cast<const float4*>(gM + (kt + 1) * kF32K) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int kk = 0; kk < kF32K; ++kk) {
      const float4 x0 = *reinterpret_cast<const float4*>(&sJ[b][kk][tx * 4]);
      const float4 x1 = *reinterpret_cast<const float4*>(&sJ[b][kk][64 + tx * 4]);
      const float4 y0 = *reinterpret_cast<const float4*>(&sM[b][kk][ty * 4]);
      const float4 y1 = *reinterpret_cast<const float4*>(&sM[b][kk][64 + ty * 4]);
      const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const float y[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
      for (int p = 0; p < 8; ++p)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(x[p], y[q], acc[p][q]);
    }
    if (kt + 1 < ntiles) stash(b ^ 1);
    __syncthreads();
  }
  float* mt = reinterpret_cast<float*>(a.mt_out);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int r = r0 + (q < 4 ? ty * 4 + q : 64 + ty * 4 + q - 4);
    if (r >= a.R) continue;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int ib = i0 + half * 64 + tx * 4;   // 4 consecutive rows
      if (ib >= a.n) continue;
      const size_t idx = (size_t)r * a.n_pad + ib;
      float4 hv = *reinterpret_cast<const float4*>(a.h + idx);
      float4 mv = *reinterpret_cast<const float4*>(a.m + idx);
      float4 vv = a.opt == FEM_OPT_SGD ? make_float4(0.f, 0.f, 0.f, 0.f) : *reinterpret_cast<const float4*>(a.v + idx);
      float4 ov;
      float* hp = &hv.x;
      float* mp = &mv.x;
      float* vp = &vv.x;
      float* op = &ov.x;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = ib + e;
        if (i >= a.n) {   // padding rows keep their (zero) state and operand
          op[e] = 0.f;
          continue;
        }
        const float cn = a.mode == FEM_GRAD_PAPER ? a.cnorm[i] : 2.f;
        const float g = s.gq * (cn * acc[half * 4 + e][q] + hp[e] * s.inv_beta) * one_minus_m2(hp[e]);
        opt_update_rt(a.opt, hp[e], mp[e], vp[e], g, s);
        op[e] = a.mode == FEM_GRAD_PAPER ? (hp[e] < 0.f ? -1.f : 1.f) : tanhf(0.5f * hp[e]);
      }
      *reinterpret_cast<float4*>(a.h + idx) = hv;
      *reinterpret_cast<float4*>(a.m + idx) = mv;
      if (a.opt != FEM_OPT_SGD) *reinterpret_cast<float4*>(a.v + idx) = vv;
      *reinterpret_cast<float4*>(mt + idx) = ov;
    }
  }
}

// The operand of the first step from the fields: sign(h) or m = tanh(h/2).
__global__ void k_dense_operand(const float* __restrict__ h, int32_t n, int32_t n_pad, int32_t R, int32_t mode,
                                int32_t prec, void* __restrict__ out, void* __restrict__ out_lo) {
  const size_t total = (size_t)R * n_pad;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n_pad);
    const float hv = h[e];
    const bool live = i < n;
    if (prec == FEM_PREC_FP32) {
      reinterpret_cast<float*>(out)[e] = !live ? 0.f : (mode == FEM_GRAD_PAPER ? (hv < 0.f ? -1.f : 1.f) : tanhf(0.5f * hv));
    } else if (prec == FEM_PREC_FP8) {
      reinterpret_cast<uint8_t*>(out)[e] = !live ? 0u : (hv < 0.f ? 0xB8u : 0x38u);
    } else if (mode == FEM_GRAD_PAPER) {
      reinterpret_cast<uint16_t*>(out)[e] = !live ? 0u : (hv < 0.f ? 0xBF80u : 0x3F80u);
      if (out_lo) reinterpret_cast<uint16_t*>(out_lo)[e] = 0u;
    } else {
      const float mm = live ? tanhf(0.5f * hv) : 0.f;
      const uint16_t hi = bf16_bits(mm);
      reinterpret_cast<uint16_t*>(out)[e] = hi;
      if (out_lo) reinterpret_cast<uint16_t*>(out_lo)[e] = bf16_bits(mm - __bfloat162float(__ushort_as_bfloat16(hi)));
    }
  }
}

// [n][R] <-> [R][n_pad] transposes of fp32 fields (32 x 32 tiles through shared memory).
__global__ void k_transpose_nr_to_rn(const float* __restrict__ src, int32_t n, int32_t R, int32_t n_pad,
                                     float* __restrict__ dst) {
  __shared__ float t[32][33];
  const int bi = blockIdx.x * 32, br = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int i = bi + y, r = br + threadIdx.x;
    t[y][threadIdx.x] = (i < n && r < R) ? src[(size_t)i * R + r] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = br + y, i = bi + threadIdx.x;
    if (r < R && i < n_pad) dst[(size_t)r * n_pad + i] = t[threadIdx.x][y];
  }
}
__global__ void k_transpose_rn_to_nr(const float* __restrict__ src, int32_t n, int32_t R, int32_t n_pad,
                                     float* __restrict__ dst) {
  __shared__ float t[32][33];
  const int bi = blockIdx.x * 32, br = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = br + y, i = bi + threadIdx.x;
    t[y][threadIdx.x] = (r < R && i < n) ? src[(size_t)r * n_pad + i] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int i = bi + y, r = br + threadIdx.x;
    if (i < n && r < R) dst[(size_t)i * R + r] = t[threadIdx.x][y];
  }
}

// Read-out: Q_r = sum_ij J_ij s_ir s_jr in exact integer arithmetic, s = +1 where
// h >= 0 else -1; a 32 x 32 (rows x replicas) tile per block with int8 couplings.
__global__ void __launch_bounds__(1024) k_dense_quad(const int8_t* __restrict__ J8, const float* __restrict__ h,
                                                     int32_t n, int32_t n_pad, int32_t R,
                                                     int64_t* __restrict__ part) {
  __shared__ int8_t sJ[32][33];
  __shared__ int8_t sS[32][33];
  __shared__ int64_t red[32][33];
  const int tr = threadIdx.x & 31, ti = threadIdx.x >> 5;  // replica, row
  const int i0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  int32_t acc = 0;
  for (int j0 = 0; j0 < n_pad; j0 += 32) {
    sJ[ti][tr] = J8[(size_t)(i0 + ti) * n_pad + j0 + tr];
    const int rr = r0 + ti, jj = j0 + tr;
    sS[ti][tr] = (rr < R && jj < n) ? (h[(size_t)rr * n_pad + jj] >= 0.f ? 1 : -1) : 0;
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) acc += (int32_t)sJ[ti][k] * (int32_t)sS[tr][k];
    __syncthreads();
  }
  const int i = i0 + ti, r = r0 + tr;
  const int si = (i < n && r < R) ? (h[(size_t)r * n_pad + i] >= 0.f ? 1 : -1) : 0;
  red[ti][tr] = (int64_t)acc * si;
  __syncthreads();
  if (ti == 0 && r < R) {
    int64_t t = 0;
    for (int k = 0; k < 32; ++k) t += red[k][tr];
    part[(size_t)blockIdx.x * R + r] = t;
  }
}

// E_r = -cut_r with cut_r = (W_tot - Q_r / 2) / 2, argmin over replicas, and the
// winning replica's +-1 states.
__global__ void __launch_bounds__(1024) k_dense_finish(const int64_t* __restrict__ part, int32_t nblk, int32_t R,
                                                       int64_t wtot, int64_t* __restrict__ e_i,
                                                       double* __restrict__ e_f, int32_t* __restrict__ best) {
  __shared__ int64_t sv[1024];
  __shared__ int si[1024];
  int64_t bv = 0;
  int bi = 0x7fffffff;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    int64_t q = 0;
    for (int b = 0; b < nblk; ++b) q += part[(size_t)b * R + r];
    const int64_t cut = (wtot - q / 2) / 2;
    e_i[r] = -cut;
    e_f[r] = (double)(-cut);
    if (bi == 0x7fffffff || -cut < bv) {
      bv = -cut;
      bi = r;
    }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      const int oi = si[threadIdx.x + off], mi = si[threadIdx.x];
      const int64_t ov = sv[threadIdx.x + off];
      if (oi != 0x7fffffff && (mi == 0x7fffffff || ov < sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < mi))) {
        sv[threadIdx.x] = ov;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) best[0] = si[0];
}

__global__ void k_dense_states(const float* __restrict__ h, int32_t n, int32_t n_pad, int32_t R,
                               const int32_t* __restrict__ best, int32_t* __restrict__ out, int32_t all) {
  const size_t total = all ? (size_t)n * R : (size_t)n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = all ? e / R : e;
    const int r = all ? (int)(e - i * R) : best[0];
    out[e] = h[(size_t)r * n_pad + i] >= 0.f ? 1 : -1;
  }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2D K-major map: rows x n_pad elements, box = box_rows rows x 128 bytes, 128B swizzle.
fem_status make_map(CUtensorMap* m, const void* base, int rows, int n_pad, int elem_bytes, int box_rows = kTile) {
  auto enc = get_encode();
  if (!enc) return fail(FEM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n_pad * elem_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)(kChunkBytes / elem_bytes), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                         const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(FEM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return FEM_OK;
}

size_t tc_smem_bytes(int prec) {
  return (size_t)stages_for(prec) * kTile * kChunkBytes * (prec == FEM_PREC_BF16X2 ? 3 : 2) + 1024;
}

template <int PREC>
fem_status launch_tc(Problem* p, const DenseArgs& a, const StepScalars& s, int in, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    FEM_CUDA(cudaFuncSetAttribute(k_dense_step_tc<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem_bytes(PREC)));
    attr = true;
  }
  const CUtensorMap* mb = &p->tmap_b[in];
  const CUtensorMap* mlo = PREC == FEM_PREC_BF16X2 ? &p->tmap_blo[in] : mb;
  const dim3 grid(p->n_pad / kTile, (p->R + kTile - 1) / kTile);
  k_dense_step_tc<PREC><<<grid, kThreads, tc_smem_bytes(PREC), st>>>(
      PREC == FEM_PREC_FP8 ? p->tmap_a8 : p->tmap_a16, *mb, *mlo, a, s);
  return FEM_OK;
}

size_t anneal_smem_bytes(int prec, bool pair) {
  return (size_t)anneal_stages(prec, pair) * anneal_stage_bytes(prec, pair) + 1024;
}

cudaLaunchConfig_t anneal_config(Problem* p, int prec, bool pair, cudaLaunchAttribute* attr, bool cooperative,
                                 cudaStream_t st) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(p->n_pad / kTile, p->R / kTile);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = anneal_smem_bytes(prec, pair);
  cfg.stream = st;
  int na = 0;
  if (pair) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = 2;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  if (cooperative) {
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cfg;
}

// Whether a persistent kernel can run this problem: tensor-core precision, whole
// replica tiles, an even number of row tiles for CTA pairs, and every CTA co-resident
// (one per SM; for pairs, as many co-resident clusters as the grid has).
template <int PREC, bool PAIR>
bool anneal_fits(Problem* p) {
  if (p->R % kTile != 0 || p->R == 0) return false;
  const int tiles = p->n_pad / kTile;
  if (PAIR && tiles % 2 != 0) return false;
  const long grid = (long)tiles * (p->R / kTile);
  static int per_sm = -1;
  if (per_sm < 0) {
    if (cudaFuncSetAttribute(k_dense_anneal_tc<PREC, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)anneal_smem_bytes(PREC, PAIR)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_anneal_tc<PREC, PAIR>, kThreads,
                                                      anneal_smem_bytes(PREC, PAIR)) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 0;
    }
  }
  if (per_sm <= 0 || grid > (long)per_sm * p->sm_count) return false;
  if (!PAIR) return true;
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = anneal_config(p, PREC, true, attr, false, nullptr);
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_dense_anneal_tc<PREC, PAIR>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (long)clusters * 2 >= grid;
}

// The persistent kernel a window runs on: 2 = CTA pairs, 1 = one CTA per tile, 0 = none.
int anneal_kind(Problem* p) {
  const bool single_only = p->dense_launch == FEM_DENSE_PERSISTENT_SINGLE;
  switch (p->precision) {
    case FEM_PREC_BF16:
      return !single_only && anneal_fits<FEM_PREC_BF16, true>(p) ? 2 : anneal_fits<FEM_PREC_BF16, false>(p) ? 1 : 0;
    case FEM_PREC_BF16X2:
      return !single_only && anneal_fits<FEM_PREC_BF16X2, true>(p) ? 2
             : anneal_fits<FEM_PREC_BF16X2, false>(p)              ? 1
                                                                   : 0;
    case FEM_PREC_FP8:
      return !single_only && anneal_fits<FEM_PREC_FP8, true>(p) ? 2 : anneal_fits<FEM_PREC_FP8, false>(p) ? 1 : 0;
    default: return 0;
  }
}

template <int PREC, bool PAIR>
fem_status launch_anneal_tc(Problem* p, const DenseArgs& a, int t_begin, int n_steps, cudaStream_t st) {
  DenseAnnealArgs x{};
  x.a = a;
  for (int b = 0; b < 2; ++b) {
    x.mt[b] = p->mt[b];
    x.mt_lo[b] = p->mt_lo[b];
  }
  x.sc = p->dense_sc;
  x.t_begin = t_begin;
  x.n_steps = n_steps;
  x.bar = p->dense_bar;
  x.bar_wait_ns = (unsigned long long)p->barrier_wait_ns;
  x.stall_tile = p->stall_tile;
  FEM_CUDA(cudaMemsetAsync(p->dense_bar, 0, (size_t)(p->R / kTile) * 32 * sizeof(int32_t), st));
  const bool x2 = PREC == FEM_PREC_BF16X2;
  const CUtensorMap* b = PAIR ? p->tmap_bh : p->tmap_b;
  const CUtensorMap* blo = PAIR ? p->tmap_blo_h : p->tmap_blo;
  const CUtensorMap& ta = PREC == FEM_PREC_FP8 ? p->tmap_a8 : p->tmap_a16;
  // One CTA per tile: a cooperative launch guarantees that all CTAs are co-resident.
  // CTA pairs: a cluster launch, with co-residency from the cluster occupancy check in
  // anneal_fits (a CTA that was never scheduled alongside the others would only make
  // them time out at the step barrier).
  cudaLaunchAttribute attr[2];
  cudaLaunchConfig_t cfg = anneal_config(p, PREC, PAIR, attr, !PAIR, st);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_dense_anneal_tc<PREC, PAIR>, ta, b[0], b[1], x2 ? blo[0] : b[0],
                                           x2 ? blo[1] : b[1], x);
  if (e != cudaSuccess) return cuda_fail(e, "persistent dense launch");
  return FEM_OK;
}

// The step-scalar table of a window on the device (grown as needed; the old table is
// released after the stream has drained, since a running anneal may still read it).
fem_status upload_scalars(Problem* p, const std::vector<StepScalars>& sc, cudaStream_t s) {
  if ((int64_t)sc.size() > p->dense_sc_cap) {
    if (p->dense_sc) {
      FEM_CUDA(cudaStreamSynchronize(s));
      cudaFree(p->dense_sc);
      p->allocs.erase(std::remove(p->allocs.begin(), p->allocs.end(), (void*)p->dense_sc), p->allocs.end());
      p->dense_sc = nullptr;
      p->dense_sc_cap = 0;
    }
    const int64_t cap = std::max<int64_t>((int64_t)sc.size(), 1024);
    fem_status st = dev_alloc_t(p, &p->dense_sc, (size_t)cap);
    if (st != FEM_OK) return st;
    p->dense_sc_cap = cap;
  }
  FEM_CUDA(cudaMemcpyAsync(p->dense_sc, sc.data(), sc.size() * sizeof(StepScalars), cudaMemcpyHostToDevice, s));
  return FEM_OK;
}

}  // namespace

int dense_pad(int n) { return ((n + kTile - 1) / kTile) * kTile; }

// Host-side construction of the dense couplings (validated by the caller):
// fp32, bf16, e4m3 and int8 copies padded to n_pad with zeros, row sums |J|, W_tot.
fem_status dense_upload(Problem* p, const float* J, cudaStream_t s) {
  p->dense = true;
  p->n_pad = dense_pad(p->n);
  const fem_status st = dense_build(p, J, s);  // validation and operands, on the device
  if (st != FEM_OK) return st;
  fem_status e = make_map(&p->tmap_a16, p->J16, p->n_pad, p->n_pad, 2);
  if (e != FEM_OK) return e;
  return make_map(&p->tmap_a8, p->J8, p->n_pad, p->n_pad, 1);
}

// State for R replicas: h, m, v [R][n_pad] and two operand buffers per part.
fem_status dense_state(Problem* p, int R, int prec, cudaStream_t s) {
  const size_t per = (size_t)R * p->n_pad;
  // the buffers of the previous replica count or precision are released first
  // (cudaFree waits for the device, so no queued work still uses them)
  auto release = [p](auto*& ptr) {
    if (!ptr) return;
    cudaFree(ptr);
    p->allocs.erase(std::remove(p->allocs.begin(), p->allocs.end(), (void*)ptr), p->allocs.end());
    ptr = nullptr;
  };
  for (int b = 0; b < 2; ++b) {
    release(p->h[b]);
    release(p->mt[b]);
    release(p->mt_lo[b]);
  }
  release(p->m);
  release(p->v);
  release(p->part_i);
  release(p->part_f);
  release(p->energy_i);
  release(p->energy_f);
  release(p->best);
  release(p->states_dev);
  p->dense_R_alloc = 0;  // no state until every buffer below is in place
  p->R = 0;
  fem_status st;
  for (int b = 0; b < 2; ++b)
    if ((st = dev_alloc_t(p, &p->h[b], per)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->m, per)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->v, per)) != FEM_OK) return st;
  const int eb = prec == FEM_PREC_FP32 ? 4 : (prec == FEM_PREC_FP8 ? 1 : 2);
  for (int b = 0; b < 2; ++b) {
    p->mt_lo[b] = nullptr;
    if ((st = dev_alloc(p, &p->mt[b], per * eb)) != FEM_OK) return st;
    // the K padding (columns n..n_pad-1) is never written by a step: it must hold zeros,
    // not arbitrary bits (0 x NaN would reach the accumulator); cleared on the anneal's
    // stream, so the first contraction is ordered after it
    FEM_CUDA(cudaMemsetAsync(p->mt[b], 0, per * eb, s));
    if (prec == FEM_PREC_BF16X2) {
      if ((st = dev_alloc(p, &p->mt_lo[b], per * 2)) != FEM_OK) return st;
      FEM_CUDA(cudaMemsetAsync(p->mt_lo[b], 0, per * 2, s));
    }
    if (prec != FEM_PREC_FP32 && (st = make_map(&p->tmap_b[b], p->mt[b], R, p->n_pad, eb)) != FEM_OK) return st;
    if (prec != FEM_PREC_FP32 && (st = make_map(&p->tmap_bh[b], p->mt[b], R, p->n_pad, eb, kTile / 2)) != FEM_OK)
      return st;
    if (prec == FEM_PREC_BF16X2 && (st = make_map(&p->tmap_blo[b], p->mt_lo[b], R, p->n_pad, 2)) != FEM_OK)
      return st;
    if (prec == FEM_PREC_BF16X2 && (st = make_map(&p->tmap_blo_h[b], p->mt_lo[b], R, p->n_pad, 2, kTile / 2)) != FEM_OK)
      return st;
  }
  p->part_blocks = p->n_pad / 32;
  if ((st = dev_alloc_t(p, &p->part_i, (size_t)p->part_blocks * R)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->part_f, (size_t)R)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->energy_i, (size_t)R)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->energy_f, (size_t)R)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->best, 1)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->states_dev, (size_t)p->n)) != FEM_OK) return st;
  p->dense_R_alloc = R;
  p->dense_prec_alloc = prec;
  p->R = R;
  return FEM_OK;
}

// Fields [n][R] (host or device) -> h[0] as [R][n_pad], and the first operand.
fem_status dense_set_fields(Problem* p, const float* h_nr, bool on_device, cudaStream_t s) {
  const size_t bytes = (size_t)p->n * p->R * 4;
  float* tmp = nullptr;
  FEM_CUDA(cudaMallocAsync((void**)&tmp, bytes, s));
  cudaError_t e = cudaMemcpyAsync(tmp, h_nr, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    const dim3 grid((p->n_pad + 31) / 32, (p->R + 31) / 32);
    k_transpose_nr_to_rn<<<grid, dim3(32, 8), 0, s>>>(tmp, p->n, p->R, p->n_pad, p->h[0]);
    count_launches(1);
    e = cudaGetLastError();
  }
  cudaFreeAsync(tmp, s);
  if (e != cudaSuccess) return cuda_fail(e, "dense fields upload");
  return FEM_OK;
}

fem_status dense_get(Problem* p, const float* src_rn, float* dst_nr_host, cudaStream_t s) {
  const size_t bytes = (size_t)p->n * p->R * 4;
  float* tmp = nullptr;
  FEM_CUDA(cudaMallocAsync((void**)&tmp, bytes, s));
  const dim3 grid((p->n + 31) / 32, (p->R + 31) / 32);
  k_transpose_rn_to_nr<<<grid, dim3(32, 8), 0, s>>>(src_rn, p->n, p->R, p->n_pad, tmp);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst_nr_host, tmp, bytes, cudaMemcpyDefault, s);
  cudaFreeAsync(tmp, s);
  if (e != cudaSuccess) return cuda_fail(e, "dense fields download");
  return FEM_OK;
}

fem_status dense_put(Problem* p, float* dst_rn, const float* src_nr_host, cudaStream_t s) {
  const size_t bytes = (size_t)p->n * p->R * 4;
  float* tmp = nullptr;
  FEM_CUDA(cudaMallocAsync((void**)&tmp, bytes, s));
  cudaError_t e = cudaMemcpyAsync(tmp, src_nr_host, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    const dim3 grid((p->n_pad + 31) / 32, (p->R + 31) / 32);
    k_transpose_nr_to_rn<<<grid, dim3(32, 8), 0, s>>>(tmp, p->n, p->R, p->n_pad, dst_rn);
    count_launches(1);
    e = cudaGetLastError();
  }
  cudaFreeAsync(tmp, s);
  if (e != cudaSuccess) return cuda_fail(e, "dense state upload");
  return FEM_OK;
}

// Operand for step t from the current fields.
fem_status dense_operand(Problem* p, int t, cudaStream_t s) {
  const size_t total = (size_t)p->R * p->n_pad;
  int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)p->sm_count * 16);
  k_dense_operand<<<blocks, 256, 0, s>>>(p->h[0], p->n, p->n_pad, p->R, p->grad_mode, p->precision,
                                         p->mt[t & 1], p->mt_lo[t & 1]);
  count_launches(1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

bool dense_persistent_ok(Problem* p) { return anneal_kind(p) > 0; }

fem_status dense_steps(Problem* p, const std::vector<StepScalars>& sc, int t_begin, cudaStream_t s) {
  DenseArgs a{};
  a.n = p->n;
  a.n_pad = p->n_pad;
  a.R = p->R;
  a.opt = p->optimizer;
  a.mode = p->grad_mode;
  a.prec = p->precision;
  a.h = p->h[0];
  a.m = p->m;
  a.v = p->v;
  a.cnorm = p->rowabs;
  a.err = p->err;
  // AUTO takes the persistent kernel for windows of two or more steps
  const bool forced = p->dense_launch == FEM_DENSE_PERSISTENT || p->dense_launch == FEM_DENSE_PERSISTENT_SINGLE;
  const int kind = sc.empty() || p->dense_launch == FEM_DENSE_PER_STEP || !(forced || sc.size() > 1)
                       ? 0
                       : anneal_kind(p);
  if (forced && kind == 0 && !sc.empty())
    return fail(FEM_ERR_UNSUPPORTED, "persistent dense anneal needs a tensor-core precision, R %% 128 == 0 and "
                "(n_pad/128)*(R/128) co-resident CTAs");
  if (kind > 0) {
    fem_status st = upload_scalars(p, sc, s);
    if (st == FEM_OK) {
      const int64_t flags = (int64_t)(p->R / kTile) * 32;  // one counter per replica block, 128 bytes apart
      if (p->dense_bar_cap < flags) {  // first use, or more replica blocks than before
        if (p->dense_bar) {
          FEM_CUDA(cudaStreamSynchronize(s));
          cudaFree(p->dense_bar);
          p->allocs.erase(std::remove(p->allocs.begin(), p->allocs.end(), (void*)p->dense_bar), p->allocs.end());
          p->dense_bar = nullptr;
          p->dense_bar_cap = 0;
        }
        if ((st = dev_alloc_t(p, &p->dense_bar, (size_t)flags)) != FEM_OK) return st;
        p->dense_bar_cap = flags;
      }
    }
    if (st == FEM_OK) {
      const int n = (int)sc.size();
      switch (p->precision * 2 + (kind == 2 ? 1 : 0)) {
        case FEM_PREC_BF16 * 2: st = launch_anneal_tc<FEM_PREC_BF16, false>(p, a, t_begin, n, s); break;
        case FEM_PREC_BF16 * 2 + 1: st = launch_anneal_tc<FEM_PREC_BF16, true>(p, a, t_begin, n, s); break;
        case FEM_PREC_BF16X2 * 2: st = launch_anneal_tc<FEM_PREC_BF16X2, false>(p, a, t_begin, n, s); break;
        case FEM_PREC_BF16X2 * 2 + 1: st = launch_anneal_tc<FEM_PREC_BF16X2, true>(p, a, t_begin, n, s); break;
        case FEM_PREC_FP8 * 2: st = launch_anneal_tc<FEM_PREC_FP8, false>(p, a, t_begin, n, s); break;
        default: st = launch_anneal_tc<FEM_PREC_FP8, true>(p, a, t_begin, n, s); break;
      }
    }
    if (st != FEM_OK) return st;
    p->dense_last_launch = kind == 2 ? FEM_DENSE_PERSISTENT : FEM_DENSE_PERSISTENT_SINGLE;
    count_launches(1);
    FEM_CUDA(cudaGetLastError());
    return FEM_OK;
  }
  if (!sc.empty()) p->dense_last_launch = FEM_DENSE_PER_STEP;
  for (size_t k = 0; k < sc.size(); ++k) {
    const int t = t_begin + (int)k, in = t & 1, out = (t + 1) & 1;
    a.mt_out = p->mt[out];
    a.mt_lo_out = p->mt_lo[out];
    fem_status st = FEM_OK;
    switch (p->precision) {
      case FEM_PREC_FP32: {
        const dim3 grid(p->n_pad / kF32Tile, (p->R + kF32Tile - 1) / kF32Tile);
        k_dense_step_fp32<<<grid, 256, 0, s>>>(p->J32, reinterpret_cast<const float*>(p->mt[in]), a, sc[k]);
        break;
      }
      case FEM_PREC_BF16: st = launch_tc<FEM_PREC_BF16>(p, a, sc[k], in, s); break;
      case FEM_PREC_BF16X2: st = launch_tc<FEM_PREC_BF16X2>(p, a, sc[k], in, s); break;
      default: st = launch_tc<FEM_PREC_FP8>(p, a, sc[k], in, s); break;
    }
    if (st != FEM_OK) return st;
  }
  count_launches((int64_t)sc.size());
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

// Read-out on the tensor cores: S = J sgn(h) with +-1 operands (exact), reduced to
// Q_r per 128-row tile in the epilogue.  Paper mode at BF16 / FP8 reuses the current
// operand (it is sgn(h)); otherwise sgn(h) is written as bf16 into the ping-pong
// buffer the next step overwrites anyway.
template <int PREC>
fem_status launch_read(Problem* p, int b, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    FEM_CUDA(cudaFuncSetAttribute(k_dense_step_tc<PREC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem_bytes(PREC)));
    attr = true;
  }
  DenseArgs a{};
  a.n = p->n;
  a.n_pad = p->n_pad;
  a.R = p->R;
  a.h = p->h[0];
  a.err = p->err;
  a.part = p->part_i;
  const dim3 grid(p->n_pad / kTile, p->R / kTile);
  k_dense_step_tc<PREC, true><<<grid, kThreads, tc_smem_bytes(PREC), st>>>(
      PREC == FEM_PREC_FP8 ? p->tmap_a8 : p->tmap_a16, p->tmap_b[b], p->tmap_b[b], a, StepScalars{});
  return FEM_OK;
}

fem_status dense_readout(Problem* p, cudaStream_t s) {
  int nblk = p->n_pad / 32;
  if (p->precision == FEM_PREC_FP32 || p->R % kTile != 0) {
    const dim3 grid(p->n_pad / 32, (p->R + 31) / 32);
    k_dense_quad<<<grid, 1024, 0, s>>>(p->Ji8, p->h[0], p->n, p->n_pad, p->R, p->part_i);
  } else {
    const int t = p->steps_done;
    fem_status st;
    if (p->grad_mode == FEM_GRAD_PAPER && p->precision != FEM_PREC_BF16X2) {
      st = p->precision == FEM_PREC_FP8 ? launch_read<FEM_PREC_FP8>(p, t & 1, s)
                                         : launch_read<FEM_PREC_BF16>(p, t & 1, s);
    } else {
      const int b = (t + 1) & 1;
      const size_t total = (size_t)p->R * p->n_pad;
      const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)p->sm_count * 16);
      k_dense_operand<<<blocks, 256, 0, s>>>(p->h[0], p->n, p->n_pad, p->R, FEM_GRAD_PAPER, FEM_PREC_BF16,
                                             p->mt[b], nullptr);
      count_launches(1);
      st = launch_read<FEM_PREC_BF16>(p, b, s);
    }
    if (st != FEM_OK) return st;
    nblk = p->n_pad / kTile;
  }
  k_dense_finish<<<1, 1024, 0, s>>>(p->part_i, nblk, p->R, p->dense_wtot, p->energy_i, p->energy_f, p->best);
  k_dense_states<<<(p->n + 255) / 256, 256, 0, s>>>(p->h[0], p->n, p->n_pad, p->R, p->best, p->states_dev, 0);
  count_launches(3);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

fem_status dense_states_all(Problem* p, int32_t* out, cudaStream_t s) {
  const size_t total = (size_t)p->n * p->R;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)p->sm_count * 16);
  k_dense_states<<<blocks, 256, 0, s>>>(p->h[0], p->n, p->n_pad, p->R, p->best, out, 1);
  count_launches(1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

}  // namespace fem
