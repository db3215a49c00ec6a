// Internal declarations of libfem (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fem.h"
#include "step_scalars.h"

namespace fem {

// The device-side definitions (error bits, step scalars) are in step_scalars.h.


struct Problem {
  int32_t kind = 0, n = 0, q = 2;
  int device = 0, sm_count = 148;

  // ---- graph, CSR over directed entries (each undirected edge twice)
  int64_t n_edges = 0, nnz = 0;
  bool unit_w = true;        // every |w| == 1: the sign lives in bit 31 of col
  bool int_w = true;         // every w integer with |w| <= 2^24: exact int64 objectives
  int32_t* row_ptr = nullptr;  // [n+1]
  uint32_t* col = nullptr;     // [nnz], bit 31 = weight sign when unit_w
  float* w = nullptr;          // [nnz] when !unit_w
  double* w64 = nullptr;       // [nnz] fp64 weights when !int_w (objectives)
  float* cnorm = nullptr;      // MaxCut c_i = 1/sum|W_ij| (when !unit_w); bMinCut c^f
  float* cnorm2 = nullptr;     // bMinCut c^a
  int32_t* nodew = nullptr;    // bMinCut node weights V_i (NULL: all 1)
  bool coloring = false;       // FEM_COLORING on the bMinCut data path (kind == FEM_BMINCUT)
  bool qubo = false;           // FEM_QUBO on the MaxCut data path (kind == FEM_MAXCUT)
  float* qoff = nullptr;       // per-node constant of the gradient: QUBO sum_j Q_ij + d_i, p-spin b_i
  int64_t* qlin_i = nullptr;   // QUBO d_i / p-spin b_i, integer (read-out)
  double* qlin_f = nullptr;    // the same, fp64
  bool qlin_int = true;
  bool pspin = false;          // FEM_PSPIN on the Max-k-SAT data path (kind == FEM_MAXKSAT)
  float* pj = nullptr;         // p-spin term coefficients J_v (negations folded in), fp32 for the steps
  float* pjo = nullptr;        // 3-spin terms only: J_v of each occurrence's term, in occurrence order
  int64_t* pj_i = nullptr;     // the same, integer (read-out)
  double* pj_f = nullptr;      // the same, fp64 (read-out)
  bool pspin_int = true;       // every J_v and b_i is an integer
  int64_t wtot_i = 0;          // sum of the edge weights (integer weights)
  double wtot_f = 0.0;         // the same in fp64
  int64_t nodew_sq = 0;        // sum_i V_i^2 (n when unweighted)

  // ---- clauses (Max-k-SAT)
  int64_t n_clauses = 0, n_occ = 0;
  int32_t* cl_ptr = nullptr;   // [M+1]
  int32_t* cl_lit = nullptr;   // [n_occ]: (var << 1) | negated
  int32_t* occ_ptr = nullptr;  // [n+1]: variable -> occurrences
  int32_t* occ = nullptr;      // [n_occ]: (clause << 3) | position
  int32_t* oth = nullptr;      // [2 n_occ]: 3-SAT only, the other two literals per occurrence
  int32_t max_width = 0;

  // ---- dense couplings (MaxCut, dense_J)
  bool dense = false;
  int32_t n_pad = 0;           // n rounded up to the tensor tile
  float* J32 = nullptr;        // fp32 [n_pad][n_pad]
  void* J16 = nullptr;         // bf16 [n_pad][n_pad]
  void* J8 = nullptr;          // e4m3 [n_pad][n_pad]
  int8_t* Ji8 = nullptr;       // int8 [n_pad][n_pad] (exact read-out)
  float* rowabs = nullptr;     // c_i = 1 / sum_j |J_ij|
  int64_t dense_wtot = 0;      // sum_{i<j} J_ij
  bool dense_fp8_ok = false;   // every |J_ij| <= 16 (exact in e4m3)
  int32_t dense_R_alloc = 0, dense_prec_alloc = -1;
  void* mt_lo[2] = {nullptr, nullptr};  // exact mode, bf16 low parts
  CUtensorMap tmap_a16, tmap_a8, tmap_b[2], tmap_blo[2];
  CUtensorMap tmap_bh[2], tmap_blo_h[2];  // the same operands in boxes of 64 replica rows (CTA pairs)
  int32_t dense_launch = 0;               // fem_dense_launch
  int32_t dense_last_launch = 0;          // the fem_dense_launch kind the last window ran on
  int64_t barrier_wait_ns = 2000000000;   // persistent kernel: limit on its step barrier
  int32_t stall_tile = -1;                // tests: row tile whose CTAs never arrive at the step barrier
  StepScalars* dense_sc = nullptr;        // persistent anneal: the window's step scalars
  int64_t dense_sc_cap = 0;
  int32_t* dense_bar = nullptr;           // persistent anneal: per replica block arrival counters (stride 32)
  int64_t dense_bar_cap = 0;              // ints allocated

  // ---- replica state
  int32_t R = 0, steps_done = 0, n_steps = 0;
  bool initialised = false;
  int32_t grad_mode = 1, optimizer = 0, precision = 0;
  int32_t cur = 0;             // which h / words buffer is current
  // CUDA graphs of short-step windows (small sparse problems), see fem_anneal
  struct StepGraph {
    int32_t t_begin, cur_before, cur_after, R, opt, mode;
    std::vector<StepScalars> sc;
    int64_t launches;
    cudaGraphExec_t exec;
  };
  std::vector<StepGraph> step_graphs;
  cudaStream_t capture_stream = nullptr;
  bool stepped_uncaptured = false;  // one window ran directly (one-time setup is done)
  float* h[2] = {nullptr, nullptr};
  float* m = nullptr;
  float* v = nullptr;
  uint32_t* words[2] = {nullptr, nullptr};
  // exact mode, what a neighbour term gathers, ping-pong: sparse MaxCut / QUBO m = tanh(h/2)
  // ([n][R]); bMinCut and colouring q (P(s) - 1/q) ([n][R][q], allocated on first use)
  float* mag[2] = {nullptr, nullptr};
  CUtensorMap tmap_mag[2];                       // exact-mode MaxCut: mag[b] for the gather kernel
  const float* tmap_mag_for[2] = {nullptr, nullptr};
  int32_t tmap_mag_R = 0;
  int32_t words_per_node = 0;
  void* mt[2] = {nullptr, nullptr};    // dense: discretised marginals for the tensor cores
  int32_t* cnt[3] = {nullptr, nullptr, nullptr};  // bMinCut group counts n_r(s), [R][q], rotating
  unsigned long long* psum[3] = {nullptr, nullptr, nullptr};  // bMinCut 2^32 * sum_j P_j(s)
  double lambda_max = 0.0;
  float* satP[2] = {nullptr, nullptr};  // Max-k-SAT marginals P = sigmoid(h), ping-ponged

  // ---- readout scratch
  int32_t part_blocks = 0;
  int64_t* part_i = nullptr;   // [part_blocks][R]
  double* part_f = nullptr;
  int64_t* part_cnt = nullptr; // [part_blocks][R][q] (bMinCut group sizes)
  int64_t* energy_i = nullptr; // [R]
  double* energy_f = nullptr;  // [R]
  int32_t* best = nullptr;     // [1]
  int32_t* states_dev = nullptr;  // [n]
  StepScalars* d_steps = nullptr;  // per-step scalars table
  int32_t d_steps_cap = 0;

  int32_t* err = nullptr;      // sticky device error word
  std::vector<void*> allocs;   // every cudaMalloc, freed by fem_destroy
  uint64_t alloc_gen = 0;      // bumped by every allocation: holders of device pointers
                               // (batch descriptors) rebuild when it changes
};

// ---- error reporting (thread-local last error)
fem_status fail(fem_status s, const char* fmt, ...);

// Edge lists are validated in chunks of kWeightChunk consecutive edges (on the host for
// small lists, on the device for large ones); the fp64 weight sum is the sum, in chunk
// order, of the chunks' sums taken in edge order, so both give the same total.
constexpr int64_t kWeightChunk = 256;
// The error for invalid edge e (the first check it fails, in the order the builders check).
fem_status edge_error(const fem_problem_desc* d, int32_t kind, int64_t e);
fem_status cuda_fail(cudaError_t e, const char* what);
#define FEM_CUDA(call)                                       \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::fem::cuda_fail(e_, #call); \
  } while (0)

fem_status dev_alloc(Problem* p, void** ptr, size_t bytes);
template <typename T>
fem_status dev_alloc_t(Problem* p, T** ptr, size_t count) {
  return dev_alloc(p, reinterpret_cast<void**>(ptr), count * sizeof(T));
}

// ---- kernel launch accounting (fem_kernel_launches)
void count_launches(int64_t k);

// ---- step scalars
std::vector<StepScalars> make_step_scalars(const fem_anneal_params& a, int32_t q_single_field_scale);

// ---- MaxCut sparse (maxcut_sparse.cu)
fem_status maxcut_sparse_steps(Problem* p, const fem_anneal_params& a,
                               const std::vector<StepScalars>& sc, cudaStream_t s);
fem_status maxcut_readout(Problem* p, cudaStream_t s);

// ---- bMinCut sparse (bmincut_sparse.cu)
int bmincut_bits(int q);
fem_status bmincut_sparse_steps(Problem* p, const std::vector<StepScalars>& sc, int t_begin,
                                cudaStream_t s);
fem_status bmincut_derive(Problem* p, int t, cudaStream_t s);
fem_status bmincut_readout(Problem* p, cudaStream_t s);
fem_status bmincut_states_all(Problem* p, int32_t* out, cudaStream_t s);

// ---- dense MaxCut on the tensor cores (dense_tc.cu)
int dense_pad(int n);
fem_status dense_upload(Problem* p, const float* J, cudaStream_t s);
// dense_build.cu: validates the caller's n x n couplings on the device and writes the
// operand copies, c_i, the sum above the diagonal and the e4m3 flag into p.
fem_status dense_build(Problem* p, const float* J, cudaStream_t s);
// maxcut_gather.cu: one exact-mode sparse MaxCut / QUBO step with TMA gathers, reading
// h[in], mag[in] and writing h[in ^ 1], mag[in ^ 1], words[in ^ 1].
fem_status maxcut_exact_gather_step(Problem* p, int in, const StepScalars& s, cudaStream_t st);
// maxcut_paper_tile.cu: one paper-mode sparse MaxCut step with staged operands, reading
// words[in] and writing words[in ^ 1] (h, m, v in place).
fem_status maxcut_paper_tile_step(Problem* p, int in, const StepScalars& s, cudaStream_t st);
// Whether the sparse MaxCut / QUBO steps take the staged tile kernels (fem_set_tma_gather).
bool tma_gather_enabled();
fem_status dense_state(Problem* p, int R, int prec, cudaStream_t s);
fem_status dense_set_fields(Problem* p, const float* h_nr, bool on_device, cudaStream_t s);
fem_status dense_get(Problem* p, const float* src_rn, float* dst_nr_host, cudaStream_t s);
fem_status dense_put(Problem* p, float* dst_rn, const float* src_nr_host, cudaStream_t s);
fem_status dense_operand(Problem* p, int t, cudaStream_t s);
fem_status dense_steps(Problem* p, const std::vector<StepScalars>& sc, int t_begin, cudaStream_t s);
bool dense_persistent_ok(Problem* p);
fem_status dense_readout(Problem* p, cudaStream_t s);
fem_status dense_states_all(Problem* p, int32_t* out, cudaStream_t s);

// ---- Max-k-SAT (sat.cu)
fem_status sat_marginals(Problem* p, int t, cudaStream_t s);
fem_status sat_steps(Problem* p, const std::vector<StepScalars>& sc, int t_begin, cudaStream_t s);
fem_status sat_readout(Problem* p, cudaStream_t s);
fem_status sat_states_all(Problem* p, int32_t* out, cudaStream_t s);

}  // namespace fem

// The opaque handle of the C ABI is the internal problem record.
struct fem_problem : public fem::Problem {};
