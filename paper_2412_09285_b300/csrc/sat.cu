// Max-k-SAT: the fused per-step kernel (clause products through the variable ->
// occurrence transpose, single-field gradient, optimizer) and the read-out of
// unsatisfied clauses.
//
// Single field P_i = P(sigma_i = 1) = sigmoid(h_i).  With u_mk = 1 - P_k(W_mk)
// (a positive literal gives 1 - P_k, a negated one P_k) and s_mi = +1 / -1 for a
// positive / negated literal of variable i in clause m, the gradient of
// F = sum_m prod_{k in m} u_mk - S/beta (Methods Eq. maxksat_F; SM "The MaxSAT
// problem", taken through Eq. gradients_wrt_h for the two states) is
//   g_i = gamma P_i (1 - P_i) [ -sum_{m ni i} s_mi prod_{k in m, k != i} u_mk + h_i/beta ].
// P_i(1 - P_i) = (1 - m_i^2)/4, so the kernel uses the single-field scale gamma/4.
//
// Layout: h, m, v and the marginals P are [n][R] fp32.  P is ping-ponged between
// steps (step t reads P[t%2], writes P[(t+1)%2]); the neighbour gathers read P,
// so no exponential is evaluated per gathered literal.  h is updated in place.
#include <algorithm>

#include "reduce_common.cuh"
#include "sat_core.cuh"

namespace fem {
namespace {

// PATH: 0 the per-element update (any clause widths, any R); 1 Max-3-SAT and 2 3-spin
// terms with four replicas per thread (R % 4 == 0).  One kernel per path, so each is
// compiled with only the registers it needs.  The four-replica paths wait on their
// marginal gathers, so they are built for more resident blocks (5 and 4 per SM; 5 for
// 3-spin terms in the R = 16 form, whose registers allow it), taking one and two
// occurrences at a time, which fits their registers without spills.
// RC: the replica count as a compile-time constant for the four-replica paths (0: run time).
template <int PATH, int RC = 0>
__global__ void __launch_bounds__(256, PATH == 1 ? 5 : (PATH == 2 ? (RC ? 5 : 4) : 1)) k_sat_step(SatArgs a, StepScalars s) {
  const long long total = (long long)a.n * (RC ? RC : a.R);
  if (PATH > 0) {
    for (long long e = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4; e < total;
         e += (long long)gridDim.x * blockDim.x * 4)
      sat_element_k3<PATH == 1 ? 1 : 2, PATH == 2, RC>(a, s, e);
    return;
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    sat_element(a, s, e);
}

using SatStep = void (*)(SatArgs, StepScalars);

// The gathered marginals of the fields: P = sigmoid(h) (Max-k-SAT) or m = tanh(h/2) (p-spin).
__global__ void k_sat_marginals(const float* __restrict__ h, long long total, float* __restrict__ P, int32_t pspin) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x)
    P[e] = pspin ? tanhf(0.5f * h[e]) : sigmoidf_fast(h[e]);
}

// p-spin energy partials: per replica, sum over terms of J_v prod_{i in v} sigma_i plus
// sum_i b_i sigma_i, sigma = +1 where h >= 0 else -1; block = 16 rows (terms, then
// spins) x 16 replicas, each thread summing its rows in a fixed order.
template <bool INTW>
__global__ void __launch_bounds__(256) k_pspin_partial(const int32_t* __restrict__ cl_ptr,
                                                       const int32_t* __restrict__ cl_lit, int64_t M,
                                                       const int64_t* __restrict__ J_i, const double* __restrict__ J_f,
                                                       const int64_t* __restrict__ b_i, const double* __restrict__ b_f,
                                                       int32_t n, const float* __restrict__ h, int32_t R,
                                                       int64_t* __restrict__ part_i, double* __restrict__ part_f) {
  __shared__ int64_t si[256];
  __shared__ double sf[256];
  const int rw = threadIdx.x >> 4, rl = threadIdx.x & 15;
  const int r = blockIdx.y * 16 + rl;
  int64_t acc_i = 0;
  double acc_f = 0.0;
  if (r < R) {
    for (long long c = (long long)blockIdx.x * 16 + rw; c < M; c += (long long)gridDim.x * 16) {
      int sgn = 1;
      for (int b = cl_ptr[c]; b < cl_ptr[c + 1]; ++b)
        if (h[(size_t)(cl_lit[b] >> 1) * R + r] < 0.f) sgn = -sgn;
      if (INTW) acc_i += sgn * J_i[c];
      else acc_f += sgn * J_f[c];
    }
    for (long long i = (long long)blockIdx.x * 16 + rw; i < n; i += (long long)gridDim.x * 16) {
      const int sgn = h[(size_t)i * R + r] >= 0.f ? 1 : -1;
      if (INTW) acc_i += sgn * b_i[i];
      else acc_f += sgn * b_f[i];
    }
  }
  si[threadIdx.x] = acc_i;
  sf[threadIdx.x] = acc_f;
  __syncthreads();
  if (rw == 0 && r < R) {
    int64_t ti = 0;
    double tf = 0.0;
    for (int k = 0; k < 16; ++k) {
      ti += si[k * 16 + rl];
      tf += sf[k * 16 + rl];
    }
    if (INTW) part_i[(size_t)blockIdx.x * R + r] = ti;
    else part_f[(size_t)blockIdx.x * R + r] = tf;
  }
}

// p-spin energy of replica r = blockIdx.x from the partials (integer or fp64).
__global__ void __launch_bounds__(kRedThreads) k_pspin_finish(const int64_t* __restrict__ part_i,
                                                              const double* __restrict__ part_f, int32_t nblk,
                                                              int32_t R, int32_t intw, int64_t* __restrict__ e_i,
                                                              double* __restrict__ e_f) {
  __shared__ int64_t shi[kRedThreads];
  __shared__ double shf[kRedThreads];
  const int r = blockIdx.x;
  if (intw) {
    const int64_t t = column_sum<int64_t>(part_i, nblk, R, r, shi);
    if (threadIdx.x == 0) {
      e_i[r] = t;
      e_f[r] = (double)t;
    }
  } else {
    const double t = column_sum<double>(part_f, nblk, R, r, shf);
    if (threadIdx.x == 0) {
      e_i[r] = 0;
      e_f[r] = t;
    }
  }
}

// Per-block partial counts of unsatisfied clauses; a thread keeps one replica.
// Block = 16 clauses x 16 replicas; blockIdx.y selects the block of 16 replicas.
// A variable takes the value 1 when h >= 0.
__global__ void __launch_bounds__(256) k_sat_unsat_partial(const int32_t* __restrict__ cl_ptr,
                                                           const int32_t* __restrict__ cl_lit,
                                                           int64_t M, const float* __restrict__ h,
                                                           int32_t R, int64_t* __restrict__ part) {
  __shared__ int64_t sc[256];
  const int cl = threadIdx.x >> 4, rl = threadIdx.x & 15;
  const int r = blockIdx.y * 16 + rl;
  int64_t cnt = 0;
  if (r < R) {
    for (long long c = (long long)blockIdx.x * 16 + cl; c < M; c += (long long)gridDim.x * 16) {
      bool sat = false;
      for (int b = cl_ptr[c]; b < cl_ptr[c + 1]; ++b) {
        const int lit = cl_lit[b];
        const bool one = h[(size_t)(lit >> 1) * R + r] >= 0.f;
        sat |= (lit & 1) ? !one : one;
      }
      cnt += sat ? 0 : 1;
    }
  }
  sc[threadIdx.x] = cnt;
  __syncthreads();
  if (cl == 0 && r < R) {
    int64_t t = 0;
    for (int k = 0; k < 16; ++k) t += sc[k * 16 + rl];
    part[(size_t)blockIdx.x * R + r] = t;
  }
}

// Unsatisfied clauses of replica r = blockIdx.x (the argmin follows in k_argmin_replica).
__global__ void __launch_bounds__(kRedThreads) k_sat_finish(const int64_t* __restrict__ part, int32_t nblk,
                                                            int32_t R, int64_t* __restrict__ e_i,
                                                            double* __restrict__ e_f) {
  __shared__ int64_t sh[kRedThreads];
  const int r = blockIdx.x;
  const int64_t t = column_sum<int64_t>(part, nblk, R, r, sh);
  if (threadIdx.x == 0) {
    e_i[r] = t;
    e_f[r] = (double)t;
  }
}

// States: 1 where h >= 0, else `lo` (Max-k-SAT 0, p-spin -1).
__global__ void k_sat_states(const float* __restrict__ h, int32_t n, int32_t R,
                             const int32_t* __restrict__ best, int32_t* __restrict__ out, int32_t all, int32_t lo) {
  const size_t total = all ? (size_t)n * R : (size_t)n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t idx = all ? e : e * R + best[0];
    out[e] = h[idx] >= 0.f ? 1 : lo;
  }
}

int grid_for(const Problem* p, long long threads, int per_sm) {
  long long blocks = (threads + 255) / 256;
  const long long cap = (long long)per_sm * p->sm_count;
  if (blocks > cap) blocks = cap;
  return (int)(blocks < 1 ? 1 : blocks);
}

}  // namespace

// Marginals read by step t (buffer t%2) from the current fields.
fem_status sat_marginals(Problem* p, int t, cudaStream_t st) {
  const long long total = (long long)p->n * p->R;
  k_sat_marginals<<<grid_for(p, total, 8), 256, 0, st>>>(p->h[0], total, p->satP[t & 1], p->pspin ? 1 : 0);
  count_launches(1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

fem_status sat_steps(Problem* p, const std::vector<StepScalars>& sc, int t_begin, cudaStream_t st) {
  // path 3: path 2 (3-spin terms) with R = 16 fixed at compile time.  The same form of
  // path 1 (Max-3-SAT) spilled at its five resident blocks per SM and was slower.
  static const SatStep kernels[4] = {k_sat_step<0>, k_sat_step<1>, k_sat_step<2>, k_sat_step<2, 16>};
  static int per_sm[4] = {0, 0, 0, 0};
  int path = (p->oth && p->R % 4 == 0) ? (!p->pspin ? 1 : (p->pjo ? 2 : 0)) : 0;
  if (path == 2 && p->R == 16) path = 3;
  if (per_sm[path] == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernels[path], 256, 0) != cudaSuccess || b < 1) b = 1;
    per_sm[path] = b;
  }
  SatArgs a{};
  a.cl_ptr = p->cl_ptr;
  a.cl_lit = p->cl_lit;
  a.occ_ptr = p->occ_ptr;
  a.occ = p->occ;
  a.oth = reinterpret_cast<const int2*>(p->oth);
  a.jw = p->pspin ? p->pj : nullptr;
  a.jwo = p->pspin ? p->pjo : nullptr;
  a.lin = p->pspin ? p->qoff : nullptr;
  a.n = p->n;
  a.R = p->R;
  a.opt = p->optimizer;
  a.h = p->h[0];
  a.m = p->m;
  a.v = p->v;
  const int grid = grid_for(p, (long long)p->n * p->R, per_sm[path]);
  for (size_t k = 0; k < sc.size(); ++k) {
    const int t = t_begin + (int)k;
    a.P_in = p->satP[t & 1];
    a.P_out = p->satP[(t + 1) & 1];
    kernels[path]<<<grid, 256, 0, st>>>(a, sc[k]);
  }
  count_launches((int64_t)sc.size());
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

fem_status sat_readout(Problem* p, cudaStream_t st) {
  const int nb = (int)std::min<long long>(std::max<long long>(1, (p->n_clauses + 15) / 16),
                                          (long long)p->part_blocks);
  const dim3 grid(nb, (p->R + 15) / 16);
  if (p->pspin) {
    if (p->pspin_int)
      k_pspin_partial<true><<<grid, 256, 0, st>>>(p->cl_ptr, p->cl_lit, p->n_clauses, p->pj_i, p->pj_f, p->qlin_i,
                                                  p->qlin_f, p->n, p->h[0], p->R, p->part_i, p->part_f);
    else
      k_pspin_partial<false><<<grid, 256, 0, st>>>(p->cl_ptr, p->cl_lit, p->n_clauses, p->pj_i, p->pj_f, p->qlin_i,
                                                   p->qlin_f, p->n, p->h[0], p->R, p->part_i, p->part_f);
    k_pspin_finish<<<p->R, kRedThreads, 0, st>>>(p->part_i, p->part_f, nb, p->R, p->pspin_int ? 1 : 0,
                                                  p->energy_i, p->energy_f);
  } else {
    k_sat_unsat_partial<<<grid, 256, 0, st>>>(p->cl_ptr, p->cl_lit, p->n_clauses, p->h[0], p->R, p->part_i);
    k_sat_finish<<<p->R, kRedThreads, 0, st>>>(p->part_i, nb, p->R, p->energy_i, p->energy_f);
  }
  k_argmin_replica<<<1, 1024, 0, st>>>(p->energy_f, p->R, p->best);
  k_sat_states<<<(p->n + 255) / 256 < 1024 ? (p->n + 255) / 256 : 1024, 256, 0, st>>>(
      p->h[0], p->n, p->R, p->best, p->states_dev, 0, p->pspin ? -1 : 0);
  count_launches(4);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

fem_status sat_states_all(Problem* p, int32_t* out, cudaStream_t st) {
  const size_t total = (size_t)p->n * p->R;
  size_t blocks = (total + 255) / 256;
  if (blocks > (size_t)p->sm_count * 16) blocks = (size_t)p->sm_count * 16;
  k_sat_states<<<(int)blocks, 256, 0, st>>>(p->h[0], p->n, p->R, p->best, out, 1, p->pspin ? -1 : 0);
  count_launches(1);
  FEM_CUDA(cudaGetLastError());
  return FEM_OK;
}

}  // namespace fem
