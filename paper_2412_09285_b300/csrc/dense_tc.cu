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

#include <cmath>
#include <cstring>

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
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

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
// 1 = bf16; kind::f8f6f4: 0 = e4m3), both K-major, N = 128, M = 128.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTile >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// ------------------------------------------------------------ the fused step
template <int PREC>  // FEM_PREC_BF16, FEM_PREC_BF16X2 or FEM_PREC_FP8
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

  // epilogue: thread = TMEM lane = row i of the tile
  const bool ok = mbar_wait(&done, 0, a.err);
  tc_fence_after();
  if (ok) {
    // warp w reads TMEM lanes 32*(w%4).. (its quadrant) and replica columns 32*(w/4)..
    const int quad = warp & 3;
    const int i = i0 + quad * 32 + lane;
    const bool row = i < a.n;
    const float cn = row ? (a.mode == FEM_GRAD_PAPER ? a.cnorm[i] : 2.f) : 0.f;
    for (int c0 = (warp >> 2) * 32; c0 < kTile; c0 += 32 * (kThreads / 128)) {
      uint32_t acc[32];
      tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, acc);
      if (!row) continue;
#pragma unroll
      for (int c = 0; c < 32; ++c) {  // R % 128 == 0: every column is a replica
        const int r = r0 + c0 + c;
        const size_t idx = (size_t)r * a.n_pad + i;
        float hv = a.h[idx], mv = a.m[idx], vv = a.opt == FEM_OPT_SGD ? 0.f : a.v[idx];
        const float field = cn * __uint_as_float(acc[c]);
        const float g = s.gq * (field + hv * s.inv_beta) * one_minus_m2_fast(hv);
        opt_update_rt(a.opt, hv, mv, vv, g, s);
        a.h[idx] = hv;
        a.m[idx] = mv;
        if (a.opt != FEM_OPT_SGD) a.v[idx] = vv;
        if (a.mode == FEM_GRAD_PAPER) {
          if (PREC == FEM_PREC_FP8)
            reinterpret_cast<uint8_t*>(a.mt_out)[idx] = hv < 0.f ? 0xB8u : 0x38u;  // e4m3 -1 / +1
          else
            reinterpret_cast<uint16_t*>(a.mt_out)[idx] = hv < 0.f ? 0xBF80u : 0x3F80u;  // bf16 -1 / +1
        } else {
          const float mm = tanhf(0.5f * hv);
          const uint16_t hi = bf16_bits(mm);
          reinterpret_cast<uint16_t*>(a.mt_out)[idx] = hi;
          if (X2) {
            const float res = mm - __bfloat162float(__ushort_as_bfloat16(hi));
            reinterpret_cast<uint16_t*>(a.mt_lo_out)[idx] = bf16_bits(res);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTile);
  }
}

// ------------------------------------------- CUDA-core fp32 step (the plain FEM)
// 64 x 64 output tile per 256-thread block, 4 x 4 per thread, K tiles of 16 in
// shared memory; the same epilogue as the tensor-core kernel.
__global__ void __launch_bounds__(256) k_dense_step_fp32(const float* __restrict__ J, const float* __restrict__ M,
                                                         DenseArgs a, StepScalars s) {
  __shared__ float sJ[16][64 + 4];
  __shared__ float sM[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < a.n_pad; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e & 15, rr = e >> 4;
      sJ[kk][rr] = J[(size_t)(i0 + rr) * a.n_pad + k0 + kk];
      sM[kk][rr] = (r0 + rr < a.R) ? M[(size_t)(r0 + rr) * a.n_pad + k0 + kk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float x[4], y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        x[q] = sJ[kk][tx + 16 * q];
        y[q] = sM[kk][ty + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(x[p], y[q], acc[p][q]);
    }
    __syncthreads();
  }
  float* mt = reinterpret_cast<float*>(a.mt_out);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int i = i0 + tx + 16 * p;
    if (i >= a.n) continue;
    const float cn = a.mode == FEM_GRAD_PAPER ? a.cnorm[i] : 2.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + ty + 16 * q;
      if (r >= a.R) continue;
      const size_t idx = (size_t)r * a.n_pad + i;
      float hv = a.h[idx], mv = a.m[idx], vv = a.opt == FEM_OPT_SGD ? 0.f : a.v[idx];
      const float g = s.gq * (cn * acc[p][q] + hv * s.inv_beta) * one_minus_m2(hv);
      opt_update_rt(a.opt, hv, mv, vv, g, s);
      a.h[idx] = hv;
      a.m[idx] = mv;
      if (a.opt != FEM_OPT_SGD) a.v[idx] = vv;
      mt[idx] = a.mode == FEM_GRAD_PAPER ? (hv < 0.f ? -1.f : 1.f) : tanhf(0.5f * hv);
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

// 2D K-major map: rows x n_pad elements, box = 128 rows x 128 bytes, 128B swizzle.
fem_status make_map(CUtensorMap* m, const void* base, int rows, int n_pad, int elem_bytes) {
  auto enc = get_encode();
  if (!enc) return fail(FEM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[2] = {(cuuint64_t)n_pad, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n_pad * elem_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)(kChunkBytes / elem_bytes), (cuuint32_t)kTile};
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

}  // namespace

int dense_pad(int n) { return ((n + kTile - 1) / kTile) * kTile; }

// Host-side construction of the dense couplings (validated by the caller):
// fp32, bf16, e4m3 and int8 copies padded to n_pad with zeros, row sums |J|, W_tot.
fem_status dense_upload(Problem* p, const float* J, cudaStream_t s) {
  const int n = p->n, np = dense_pad(n);
  p->dense = true;
  p->n_pad = np;
  std::vector<float> j32((size_t)np * np, 0.f);
  std::vector<uint16_t> j16((size_t)np * np, 0);
  std::vector<uint8_t> j8((size_t)np * np, 0);
  std::vector<int8_t> ji((size_t)np * np, 0);
  std::vector<float> cn(np, 0.f);
  int64_t wtot = 0;
  bool fp8_ok = true;
  for (int i = 0; i < n; ++i) {
    double ra = 0;
    for (int j = 0; j < n; ++j) {
      const float x = J[(size_t)i * n + j];
      const size_t o = (size_t)i * np + j;
      j32[o] = x;
      uint16_t b;
      const __nv_bfloat16 bb = __float2bfloat16_rn(x);
      std::memcpy(&b, &bb, 2);
      j16[o] = b;
      const __nv_fp8_e4m3 f8(x);
      std::memcpy(&j8[o], &f8, 1);
      if (std::fabs(x) > 16.f) fp8_ok = false;
      ji[o] = (int8_t)x;
      ra += std::fabs(x);
      if (j > i) wtot += (int64_t)x;
    }
    cn[i] = ra > 0 ? (float)(1.0 / ra) : 0.f;
  }
  p->dense_wtot = wtot;
  p->dense_fp8_ok = fp8_ok;
  fem_status st;
  if ((st = dev_alloc_t(p, &p->J32, j32.size())) != FEM_OK) return st;
  if ((st = dev_alloc(p, &p->J16, j16.size() * 2)) != FEM_OK) return st;
  if ((st = dev_alloc(p, &p->J8, j8.size())) != FEM_OK) return st;
  if ((st = dev_alloc(p, (void**)&p->Ji8, ji.size())) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->rowabs, cn.size())) != FEM_OK) return st;
  FEM_CUDA(cudaMemcpyAsync(p->J32, j32.data(), j32.size() * 4, cudaMemcpyHostToDevice, s));
  FEM_CUDA(cudaMemcpyAsync(p->J16, j16.data(), j16.size() * 2, cudaMemcpyHostToDevice, s));
  FEM_CUDA(cudaMemcpyAsync(p->J8, j8.data(), j8.size(), cudaMemcpyHostToDevice, s));
  FEM_CUDA(cudaMemcpyAsync(p->Ji8, ji.data(), ji.size(), cudaMemcpyHostToDevice, s));
  FEM_CUDA(cudaMemcpyAsync(p->rowabs, cn.data(), cn.size() * 4, cudaMemcpyHostToDevice, s));
  FEM_CUDA(cudaStreamSynchronize(s));  // the host staging vectors die at return
  fem_status e = make_map(&p->tmap_a16, p->J16, np, np, 2);
  if (e != FEM_OK) return e;
  return make_map(&p->tmap_a8, p->J8, np, np, 1);
}

// State for R replicas: h, m, v [R][n_pad] and two operand buffers per part.
fem_status dense_state(Problem* p, int R, int prec) {
  const size_t per = (size_t)R * p->n_pad;
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
    // not arbitrary bits (0 x NaN would reach the accumulator)
    FEM_CUDA(cudaMemset(p->mt[b], 0, per * eb));
    if (prec == FEM_PREC_BF16X2) {
      if ((st = dev_alloc(p, &p->mt_lo[b], per * 2)) != FEM_OK) return st;
      FEM_CUDA(cudaMemset(p->mt_lo[b], 0, per * 2));
    }
    if (prec != FEM_PREC_FP32 && (st = make_map(&p->tmap_b[b], p->mt[b], R, p->n_pad, eb)) != FEM_OK) return st;
    if (prec == FEM_PREC_BF16X2 && (st = make_map(&p->tmap_blo[b], p->mt_lo[b], R, p->n_pad, 2)) != FEM_OK)
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
  for (size_t k = 0; k < sc.size(); ++k) {
    const int t = t_begin + (int)k, in = t & 1, out = (t + 1) & 1;
    a.mt_out = p->mt[out];
    a.mt_lo_out = p->mt_lo[out];
    fem_status st = FEM_OK;
    switch (p->precision) {
      case FEM_PREC_FP32: {
        const dim3 grid(p->n_pad / 64, (p->R + 63) / 64);
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

fem_status dense_readout(Problem* p, cudaStream_t s) {
  const dim3 grid(p->n_pad / 32, (p->R + 31) / 32);
  k_dense_quad<<<grid, 1024, 0, s>>>(p->Ji8, p->h[0], p->n, p->n_pad, p->R, p->part_i);
  k_dense_finish<<<1, 1024, 0, s>>>(p->part_i, p->n_pad / 32, p->R, p->dense_wtot, p->energy_i, p->energy_f, p->best);
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
