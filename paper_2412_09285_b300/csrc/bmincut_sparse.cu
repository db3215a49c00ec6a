// Balanced q-way MinCut on sparse graphs: the fused per-step kernel (softmax
// marginals, neighbour contraction, balance term, chain rule, optimizer) and the
// read-out of cut, group sizes and energy.
//
// Gradient (SM "The bMinCut problem" and Eq. gradients_wrt_h):
//   g_i(s) = gamma [ghat_i(s) - sum_s' P_i(s') ghat_i(s')] P_i(s),  P_i = softmax(h_i)
//   paper: ghat = -c^f_i sum_j W_ij e_j(s) + lambda c^a_i [n(s) - e_i(s)] + ln P_i(s)/beta
//   exact: ghat = -2 sum_j W_ij P_j(s) + 2 lambda [sum_j P_j(s) - P_i(s)] + ln P_i(s)/beta
// c^f = q/sum_j W_ij, c^a = q/sqrt(sum_j W_ij) (0 for isolated nodes).  The "+1" of
// (ln P + 1)/beta and every other s-independent term cancel in the centred form
// and are not evaluated.
//
// Layout: h, m, v are [n][R][q] fp32 (the q fields of one replica contiguous).
// The argmax state of each (node, replica) is packed B bits wide (B = 1, 2, 4 for
// q = 2, <= 4, <= 8) into uint32 words, R*B/32 words per node, ping-ponged between
// steps.  The per-replica group counts n(s) = sum_j e_j(s) (paper mode) and the
// fixed-point column sums sum_j P_j(s) * 2^32 (exact mode, integer atomics, so the
// result does not depend on the order of the additions) are produced by step t for
// step t+1 in a rotation of three buffers: step t reads buffer t%3, writes
// (t+1)%3 and zeroes (t+2)%3 for the step after.
#include <cmath>

#include "bmincut_core.cuh"
#include "reduce_common.cuh"

namespace fem {
namespace {

// Resident blocks per SM the registers are budgeted for: paper mode with q <= 4 six in the
// R = 16 form and five otherwise (each measured faster than one block fewer), three for
// q >= 7, else four (more would spill).
template <int Q, int MODE, int RC>
constexpr int bmincut_blocks() { return Q >= 7 ? 3 : ((Q <= 4 && MODE == FEM_GRAD_PAPER) ? (RC == 16 ? 6 : 5) : 4); }

// One thread per (node, replica); a warp covers 32 consecutive (node, replica)
// pairs, so R % RPW == 0 keeps every packed word inside one group of lanes.
// RC: the replica count as a compile-time constant (0: run time).  OPTC: the optimizer as a
// compile-time constant (-1: run time); the element code then holds one update, not three.
template <int Q, int MODE, int RC = 0, int OPTC = -1>
__global__ void __launch_bounds__(256, bmincut_blocks<Q, MODE, RC>()) k_bmincut_step(BmcArgs args, StepScalars s) {
  BmcArgs a = args;
  if (OPTC >= 0) a.opt = OPTC;
  extern __shared__ unsigned long long smem_u64[];
  const int R = RC ? RC : a.R;
  const int RQ = R * Q;
  unsigned long long* sps = smem_u64;                                // [R*Q] exact mode
  int32_t* scnt = reinterpret_cast<int32_t*>(smem_u64 + (MODE == FEM_GRAD_EXACT ? RQ : 0));
  for (int x = threadIdx.x; x < RQ; x += blockDim.x) {
    scnt[x] = 0;
    if (MODE == FEM_GRAD_EXACT) sps[x] = 0ull;
  }
  if (blockIdx.x == 0) {
    for (int x = threadIdx.x; x < RQ; x += blockDim.x) {
      a.cnt_zero[x] = 0;
      if (MODE == FEM_GRAD_EXACT) a.ps_zero[x] = 0ull;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long total = (long long)a.n * R;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
       base += stride) {
    const long long e = base + lane;
    bmincut_element<Q, MODE, RC>(a, s, e, e < total, lane, scnt, sps);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < RQ; x += blockDim.x) {
    if (scnt[x]) atomicAdd(&a.cnt_out[x], scnt[x]);
    if (MODE == FEM_GRAD_EXACT && sps[x]) atomicAdd(&a.ps_out[x], sps[x]);
  }
}

// From fields h: packed argmax words, group counts and fixed-point column sums.
// Counts and sums gather in shared memory ([R][q] per block) and reach the global
// buffers with one integer atomic per entry and block (exact, so order-free).
template <int Q>
__global__ void __launch_bounds__(256) k_bmincut_derive(const float* __restrict__ h, int32_t n, int32_t R,
                                                        int32_t wpn, const int32_t* __restrict__ nodew,
                                                        uint32_t* __restrict__ words,
                                                        int32_t* __restrict__ cnt,
                                                        unsigned long long* __restrict__ ps,
                                                        float* __restrict__ d) {
  constexpr int B = QBits<Q>::B, RPW = QBits<Q>::RPW;
  extern __shared__ unsigned long long smem_d[];
  const int RQ = R * Q;
  unsigned long long* sps = smem_d;
  int32_t* scnt = reinterpret_cast<int32_t*>(smem_d + RQ);
  for (int x = threadIdx.x; x < RQ; x += blockDim.x) {
    sps[x] = 0ull;
    scnt[x] = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long total = (long long)n * R;
  for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total;
       base += (long long)gridDim.x * blockDim.x) {
    const long long e = base + lane;
    const bool act = e < total;
    int i = 0, r = 0;
    if (act) split_element(e, R, i, r);
    float x[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) x[q] = 0.f;
    if (act) load_q<Q>(h + ((size_t)i * R + r) * Q, x);
    const int sn = argmax_q<Q>(x);
    if (act) {
      const int Vi = nodew ? nodew[i] : 1;
      atomicAdd(&scnt[r * Q + sn], Vi);
      float P[Q], ln[Q];
      softmax_q<Q>(x, P, ln);
#pragma unroll
      for (int q = 0; q < Q; ++q)
        atomicAdd(&sps[r * Q + q], __float2ull_rn(P[q] * kPsumScale) * (unsigned long long)Vi);
      if (d) {  // exact mode: what the neighbours' terms gather at this step
        float c[Q];
        centred_q<Q>(x, c);
        store_q<Q>(d + ((size_t)i * R + r) * Q, c);
      }
    }
    uint32_t word = act ? ((uint32_t)sn << ((r % RPW) * B)) : 0u;
#pragma unroll
    for (int off = 1; off < RPW; off <<= 1) word |= __shfl_xor_sync(kFullMask, word, off);
    if (act && (r % RPW) == 0) words[(size_t)i * wpn + r / RPW] = word;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < RQ; x += blockDim.x) {
    if (scnt[x]) atomicAdd(&cnt[x], scnt[x]);
    if (sps[x]) atomicAdd(&ps[x], sps[x]);
  }
}

// Per-block partial cut (undirected edges, j > i) and group sizes per replica.
// Block = 16 nodes x 16 replicas; blockIdx.y selects the block of 16 replicas.
// Each thread keeps its own (fixed) replica, so every sum runs in a fixed order.
template <int Q, bool INTW>
__global__ void __launch_bounds__(256) k_bmincut_cut_partial(
    const int32_t* __restrict__ row_ptr, const uint32_t* __restrict__ col,
    const float* __restrict__ w, const double* __restrict__ w64, const uint32_t* __restrict__ words,
    const int32_t* __restrict__ nodew, int32_t n, int32_t R, int32_t wpn, int64_t* __restrict__ part_i,
    double* __restrict__ part_f, int64_t* __restrict__ part_cnt) {
  constexpr int B = QBits<Q>::B, RPW = QBits<Q>::RPW;
  constexpr uint32_t SM = QBits<Q>::MASK;
  __shared__ int64_t si[256];
  __shared__ double sf[256];
  __shared__ int32_t sc[256 * Q];
  const int nl = threadIdx.x >> 4, rl = threadIdx.x & 15;
  const int r = blockIdx.y * 16 + rl;
  const int wsel = r / RPW, sh = (r % RPW) * B;
  int64_t acc_i = 0;
  double acc_f = 0.0;
  int32_t cnt[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) cnt[q] = 0;
  for (int i = blockIdx.x * 16 + nl; i < n; i += gridDim.x * 16) {
    const int si_ = (int)((words[(size_t)i * wpn + wsel] >> sh) & SM);
#pragma unroll
    for (int q = 0; q < Q; ++q) cnt[q] += (si_ == q) ? (nodew ? nodew[i] : 1) : 0;
    const int beg = row_ptr[i], end = row_ptr[i + 1];
    for (int k = beg; k < end; ++k) {
      const int j = (int)(col[k] & 0x7fffffffu);
      if (j <= i) continue;
      const int sj = (int)((words[(size_t)j * wpn + wsel] >> sh) & SM);
      if (sj == si_) continue;
      if (INTW) acc_i += w ? (int64_t)w[k] : 1;
      else acc_f += w64[k];
    }
  }
  si[threadIdx.x] = acc_i;
  sf[threadIdx.x] = acc_f;
#pragma unroll
  for (int q = 0; q < Q; ++q) sc[threadIdx.x * Q + q] = cnt[q];
  __syncthreads();
  if (nl == 0) {
    int64_t ti = 0;
    double tf = 0.0;
    int64_t tc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) tc[q] = 0;
    for (int k = 0; k < 16; ++k) {
      ti += si[k * 16 + rl];
      tf += sf[k * 16 + rl];
#pragma unroll
      for (int q = 0; q < Q; ++q) tc[q] += sc[(k * 16 + rl) * Q + q];
    }
    const size_t o = (size_t)blockIdx.x * R + r;
    part_i[o] = ti;
    part_f[o] = tf;
#pragma unroll
    for (int q = 0; q < Q; ++q) part_cnt[o * Q + q] = tc[q];
  }
}

// E_r = cut_r + lambda_max * sum_s n_s (n_s - 1) for replica r = blockIdx.x (the
// argmin follows in k_argmin_replica).
template <int Q>
__global__ void __launch_bounds__(kRedThreads) k_bmincut_finish(
    const int64_t* __restrict__ part_i, const double* __restrict__ part_f,
    const int64_t* __restrict__ part_cnt, int32_t nblk, int32_t R, int32_t intw, int32_t lam_is_int,
    double lam, int64_t sum_v2, int32_t coloring, int64_t wtot_i, double wtot_f, int64_t* __restrict__ e_i,
    double* __restrict__ e_f) {
  __shared__ int64_t shi[kRedThreads];
  __shared__ double shf[kRedThreads];
  const int r = blockIdx.x;
  const int64_t ci = intw ? column_sum<int64_t>(part_i, nblk, R, r, shi) : 0;
  const double cfv = intw ? 0.0 : column_sum<double>(part_f, nblk, R, r, shf);
  // sum_s [n_s^2 - sum_{i in s} V_i^2] = sum_s n_s^2 - sum_i V_i^2 (n_s(n_s - 1) unweighted)
  int64_t bal = -sum_v2;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int64_t sz = column_sum<int64_t>(part_cnt, nblk, (size_t)R * Q, (size_t)r * Q + q, shi);
    bal += sz * sz;
  }
  if (threadIdx.x == 0 && coloring) {  // violated edges = all edges - cut edges
    e_i[r] = intw ? wtot_i - ci : 0;
    e_f[r] = intw ? (double)(wtot_i - ci) : wtot_f - cfv;
  } else if (threadIdx.x == 0) {
    double ef;
    if (intw && lam_is_int) {
      const int64_t ei = ci + (int64_t)lam * bal;
      e_i[r] = ei;
      ef = (double)ei;
    } else {
      e_i[r] = 0;
      ef = (intw ? (double)ci : cfv) + lam * (double)bal;
    }
    e_f[r] = ef;
  }
}

template <int Q>
__global__ void k_bmincut_states(const uint32_t* __restrict__ words, int32_t n, int32_t R,
                                 int32_t wpn, const int32_t* __restrict__ best, int32_t* __restrict__ out,
                                 int32_t all) {
  constexpr int B = QBits<Q>::B, RPW = QBits<Q>::RPW;
  constexpr uint32_t SM = QBits<Q>::MASK;
  const size_t total = all ? (size_t)n * R : (size_t)n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t i = all ? e / R : e;
    const int r = all ? (int)(e - i * R) : best[0];
    out[e] = (int32_t)((words[i * wpn + r / RPW] >> ((r % RPW) * B)) & SM);
  }
}

template <typename K>
int resident_grid(K kernel, int sm_count, long long threads, size_t smem) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  long long blocks = (threads + 255) / 256;
  const long long cap = (long long)per_sm * sm_count;
  if (blocks > cap) blocks = cap;
  return (int)(blocks < 1 ? 1 : blocks);
}

template <int Q>
fem_status steps_q(Problem* p, const std::vector<StepScalars>& sc, int t_begin, cudaStream_t st) {
  BmcArgs a{};
  a.row_ptr = p->row_ptr;
  a.col = p->col;
  a.w = p->unit_w ? nullptr : p->w;
  a.cf = p->cnorm;
  a.ca = p->cnorm2;
  a.nodew = p->nodew;
  a.cw = p->coloring ? 1.f : (p->grad_mode == FEM_GRAD_EXACT ? -2.f : -1.f);
  a.lam_scale = p->coloring ? 0.f : 1.f;
  a.n = p->n;
  a.R = p->R;
  a.wpn = p->words_per_node;
  a.opt = p->optimizer;
  a.m = p->m;
  a.v = p->v;
  const bool exact = p->grad_mode == FEM_GRAD_EXACT;
  if (exact && (!p->mag[0] || !p->mag[1])) return fail(FEM_ERR_STATE, "exact-mode buffers are not allocated");
  const size_t smem = (size_t)p->R * Q * (exact ? 12 : 4);
  // R = 16 (with its one or two packed words per node) runs an instantiation with the
  // replica count fixed at compile time
  const bool r16 = p->R == 16 && p->words_per_node == 16 * QBits<Q>::B / 32;
  // ... and, with Adam (the default), the optimizer too
  const bool adam = p->optimizer == FEM_OPT_ADAM;
  auto kern = exact ? (r16 ? (adam ? k_bmincut_step<Q, FEM_GRAD_EXACT, 16, FEM_OPT_ADAM> : k_bmincut_step<Q, FEM_GRAD_EXACT, 16>)
                           : k_bmincut_step<Q, FEM_GRAD_EXACT>)
                    : (r16 ? (adam ? k_bmincut_step<Q, FEM_GRAD_PAPER, 16, FEM_OPT_ADAM> : k_bmincut_step<Q, FEM_GRAD_PAPER, 16>)
                           : k_bmincut_step<Q, FEM_GRAD_PAPER>);
  if (smem > 48 * 1024) FEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = resident_grid(kern, p->sm_count, (long long)p->n * p->R, smem);
  for (size_t k = 0; k < sc.size(); ++k) {
    const int t = t_begin + (int)k;
    a.h_in = exact ? p->h[t & 1] : p->h[0];
    a.h_out = exact ? p->h[(t + 1) & 1] : p->h[0];
    a.words_in = p->words[t & 1];
    a.words_out = p->words[(t + 1) & 1];
    a.cnt_in = p->cnt[t % 3];
    a.cnt_out = p->cnt[(t + 1) % 3];
    a.cnt_zero = p->cnt[(t + 2) % 3];
    a.ps_in = p->psum[t % 3];
    a.ps_out = p->psum[(t + 1) % 3];
    a.ps_zero = p->psum[(t + 2) % 3];
    a.d_in = exact ? p->mag[t & 1] : nullptr;
    a.d_out = exact ? p->mag[(t + 1) & 1] : nullptr;
    kern<<<grid, 256, smem, st>>>(a, sc[k]);
  }
  count_launches((int64_t)sc.size());
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

// Derived data for step t from the fields step t reads: words[t%2], counts and
// column sums in buffer t%3; buffer (t+1)%3, which step t accumulates into, is zeroed.
template <int Q>
fem_status derive_q(Problem* p, int t, cudaStream_t st) {
  if (p->grad_mode == FEM_GRAD_EXACT && !p->mag[t & 1])
    return fail(FEM_ERR_STATE, "exact-mode buffers are not allocated");
  const size_t rq = (size_t)p->R * Q;
  const float* h = p->grad_mode == FEM_GRAD_PAPER ? p->h[0] : p->h[t & 1];
  for (int b : {t % 3, (t + 1) % 3}) {
    FEM_CUDA(cudaMemsetAsync(p->cnt[b], 0, rq * sizeof(int32_t), st));
    FEM_CUDA(cudaMemsetAsync(p->psum[b], 0, rq * sizeof(unsigned long long), st));
  }
  const size_t smem = rq * (sizeof(unsigned long long) + sizeof(int32_t));
  if (smem > 48 * 1024)
    FEM_CUDA(cudaFuncSetAttribute(k_bmincut_derive<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = resident_grid(k_bmincut_derive<Q>, p->sm_count, (long long)p->n * p->R, smem);
  k_bmincut_derive<Q><<<grid, 256, smem, st>>>(h, p->n, p->R, p->words_per_node, p->nodew, p->words[t & 1],
                                              p->cnt[t % 3], p->psum[t % 3],
                                              p->grad_mode == FEM_GRAD_EXACT ? p->mag[t & 1] : nullptr);
  count_launches(1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

template <int Q>
fem_status readout_q(Problem* p, cudaStream_t st) {
  const dim3 grid(p->part_blocks, p->R / 16);
  const uint32_t* words = p->words[p->steps_done & 1];
  if (p->int_w)
    k_bmincut_cut_partial<Q, true><<<grid, 256, 0, st>>>(p->row_ptr, p->col, p->unit_w ? nullptr : p->w,
                                                         p->w64, words, p->nodew, p->n, p->R, p->words_per_node,
                                                         p->part_i, p->part_f, p->part_cnt);
  else
    k_bmincut_cut_partial<Q, false><<<grid, 256, 0, st>>>(p->row_ptr, p->col, p->unit_w ? nullptr : p->w,
                                                          p->w64, words, p->nodew, p->n, p->R, p->words_per_node,
                                                          p->part_i, p->part_f, p->part_cnt);
  const double lam = p->lambda_max;
  k_bmincut_finish<Q><<<p->R, kRedThreads, 0, st>>>(p->part_i, p->part_f, p->part_cnt, p->part_blocks, p->R,
                                                     p->int_w ? 1 : 0, lam == std::floor(lam) ? 1 : 0, lam,
                                                     p->nodew_sq, p->coloring ? 1 : 0, p->wtot_i, p->wtot_f,
                                                     p->energy_i, p->energy_f);
  k_argmin_replica<<<1, 1024, 0, st>>>(p->energy_f, p->R, p->best);
  k_bmincut_states<Q><<<(p->n + 255) / 256 < 1024 ? (p->n + 255) / 256 : 1024, 256, 0, st>>>(
      words, p->n, p->R, p->words_per_node, p->best, p->states_dev, 0);
  count_launches(4);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

template <int Q>
fem_status states_q(Problem* p, int32_t* out, cudaStream_t st) {
  const size_t total = (size_t)p->n * p->R;
  size_t blocks = (total + 255) / 256;
  if (blocks > (size_t)p->sm_count * 16) blocks = (size_t)p->sm_count * 16;
  k_bmincut_states<Q><<<(int)blocks, 256, 0, st>>>(p->words[p->steps_done & 1], p->n, p->R,
                                                   p->words_per_node, p->best, out, 1);
  count_launches(1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

}  // namespace

int bmincut_bits(int q) { return q <= 2 ? 1 : (q <= 4 ? 2 : 4); }

fem_status bmincut_sparse_steps(Problem* p, const std::vector<StepScalars>& sc, int t_begin,
                                cudaStream_t s) {
  switch (p->q) {
    case 2: return steps_q<2>(p, sc, t_begin, s);
    case 3: return steps_q<3>(p, sc, t_begin, s);
    case 4: return steps_q<4>(p, sc, t_begin, s);
    case 5: return steps_q<5>(p, sc, t_begin, s);
    case 6: return steps_q<6>(p, sc, t_begin, s);
    case 7: return steps_q<7>(p, sc, t_begin, s);
    default: return steps_q<8>(p, sc, t_begin, s);
  }
}

fem_status bmincut_derive(Problem* p, int t, cudaStream_t s) {
  switch (p->q) {
    case 2: return derive_q<2>(p, t, s);
    case 3: return derive_q<3>(p, t, s);
    case 4: return derive_q<4>(p, t, s);
    case 5: return derive_q<5>(p, t, s);
    case 6: return derive_q<6>(p, t, s);
    case 7: return derive_q<7>(p, t, s);
    default: return derive_q<8>(p, t, s);
  }
}

fem_status bmincut_readout(Problem* p, cudaStream_t s) {
  switch (p->q) {
    case 2: return readout_q<2>(p, s);
    case 3: return readout_q<3>(p, s);
    case 4: return readout_q<4>(p, s);
    case 5: return readout_q<5>(p, s);
    case 6: return readout_q<6>(p, s);
    case 7: return readout_q<7>(p, s);
    default: return readout_q<8>(p, s);
  }
}

fem_status bmincut_states_all(Problem* p, int32_t* out, cudaStream_t s) {
  switch (p->q) {
    case 2: return states_q<2>(p, out, s);
    case 3: return states_q<3>(p, out, s);
    case 4: return states_q<4>(p, out, s);
    case 5: return states_q<5>(p, out, s);
    case 6: return states_q<6>(p, out, s);
    case 7: return states_q<7>(p, out, s);
    default: return states_q<8>(p, out, s);
  }
}

}  // namespace fem
