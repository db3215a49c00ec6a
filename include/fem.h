/*
 * fem.h - C ABI of the B300 Free-Energy Machine library (libfem.so).
 *
 * The Free-Energy Machine (FEM) minimises R replicas of the variational
 * mean-field free energy F = U - S/beta over marginals P_i(s) = softmax(h_i)(s)
 * while beta is annealed upwards, then reads every replica out by argmax and
 * keeps the replica of lowest energy (Results, "Free-Energy Machine", and its
 * argmax / argmin equations).  This library runs that per-step replica update on
 * one GPU: the coupling contraction, the hand-written gradient of F, the
 * optimizer step and the schedule, then the argmax and an exact objective.
 *
 * Problems (Results, Eqs. maxcut1, bmincut, maxksat_E):
 *   FEM_MAXCUT   E = -sum_{(i,j) in E} W_ij [s_i != s_j]                 (q = 2)
 *   FEM_BMINCUT  E =  sum_{(i,j) in E} W_ij [s_i != s_j]
 *                    + lambda_max * sum_s n_s (n_s - 1)                    (q >= 2)
 *   FEM_MAXKSAT  E = number of unsatisfied clauses                         (q = 2)
 *
 * Conventions shared by every call:
 *   - Every call returns a fem_status; nothing aborts, traps or prints.
 *     fem_last_error() gives a one-line reason for the last failure on the
 *     calling thread.
 *   - Host input buffers are copied before the call returns; the caller keeps
 *     ownership of everything it passes in.  Outputs go to caller buffers.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream) on the
 *     device that was current when the problem was created.  fem_anneal is
 *     asynchronous on that stream; fem_read_* synchronise it.
 *   - Device kernels never trap.  A device-side check (index bounds, a bounded
 *     wait that ran out) sets a sticky error flag in the problem; the next
 *     fem_read_* or fem_sync call reports it as FEM_ERR_DEVICE / FEM_ERR_TIMEOUT.
 *   - A handle is not thread-safe; concurrent calls on one handle are undefined.
 *
 * Layouts of per-replica state (fp32, replica-contiguous per variable):
 *   single-field problems (MaxCut, Max-k-SAT): h[n][R]      (element i*R + r)
 *   q-state problems (bMinCut):                h[n][R][q]   (element (i*R + r)*q + s)
 */
#ifndef FEM_H
#define FEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FEM_OK = 0,
  FEM_ERR_INVALID_ARG = 1, /* a pointer, size, index, weight or flag is out of range   */
  FEM_ERR_UNSUPPORTED = 2, /* valid input this build does not handle (e.g. R % 32 != 0) */
  FEM_ERR_OOM = 3,         /* a device allocation failed                               */
  FEM_ERR_CUDA = 4,        /* a CUDA runtime call failed                               */
  FEM_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                       */
  FEM_ERR_STATE = 6,       /* call out of order (e.g. resume before initialisation)    */
  FEM_ERR_DEVICE = 7       /* a device-side bounds check failed                        */
} fem_status;

/* FEM_COLORING: graph colouring, the q-state Potts energy of violated edges
 * E = sum_{(i,j) in E} W_ij delta(sigma_i, sigma_j) (SM, problems of multi-valued
 * variables), on the bMinCut data path with the coupling's sign reversed and no
 * balance term (lambda_max is ignored); the read-out energy is E itself. */
/* FEM_QUBO: binary sigma_i in {0, 1} with E = sum_{i != j} Q_ij sigma_i sigma_j +
 * sum_i d_i sigma_i (SM, COPs that translate into QUBO formulations; the diagonal of
 * Q is the linear term d because sigma_i^2 = sigma_i).  The graph lists each
 * off-diagonal pair once with w = Q_ij; d comes from fem_problem_desc.linear.  One
 * sigmoid field per variable, FEM_GRAD_EXACT only; the read-out energy is E and a
 * variable's state is 1 where h >= 0. */
/* FEM_PSPIN: spins sigma_i in {-1, +1} with multi-spin terms (p-spin glasses, the
 * quantum error-correction Hamiltonian; SM, problems with multi-variable
 * interactions): E = sum_v J_v prod_{i in v} sigma_i + sum_i b_i sigma_i.  Terms come
 * in clause_ptr / lits (1 to 8 distinct variables each; a negated literal multiplies
 * its term by -1), J_v in term_weight, b_i in linear (NULL: 0).  One sigmoid field per
 * spin (m = tanh(h/2)), the exact gradient in both modes; the read-out energy is E and
 * a spin's state is +1 where h >= 0, else -1. */
typedef enum {
  FEM_MAXCUT = 0, FEM_BMINCUT = 1, FEM_MAXKSAT = 2, FEM_COLORING = 3, FEM_QUBO = 4, FEM_PSPIN = 5
} fem_kind;

/* Methods, "Different annealing schedules for the inverse temperature":
 *   exponential          beta(t) = exp(ln b_min + t (ln b_max - ln b_min)/(N_step - 1))
 *   inverse-proportional 1/beta(t) = 1/b_min + t (1/b_max - 1/b_min)/(N_step - 1)
 * t = 0 .. N_step-1; N_step = 1 gives beta(0) = b_min. */
typedef enum { FEM_SCHED_EXPONENTIAL = 0, FEM_SCHED_INVERSE_PROPORTIONAL = 1 } fem_schedule;

/* Methods, "Hyperparameter tunning": the PyTorch Adam, RMSprop and SGD updates. */
typedef enum { FEM_OPT_ADAM = 0, FEM_OPT_RMSPROP = 1, FEM_OPT_SGD = 2 } fem_optimizer;

/* FEM_GRAD_EXACT: the true gradient dF/dh (SM Eqs. S-maxcut_gradient, the bMinCut
 *   gradient, the MaxSAT gradient, through the chain rule Eq. gradients_wrt_h).
 * FEM_GRAD_PAPER: the manipulated gradients the paper benchmarks - one-hot
 *   discretisation e_j of the neighbours and per-node normalisers c_i
 *   (SM Eq. maxcut_modified_gradient and the bMinCut manipulated gradient).
 *   Max-k-SAT is never manipulated, so both modes are the same there. */
typedef enum { FEM_GRAD_EXACT = 0, FEM_GRAD_PAPER = 1 } fem_grad_mode;

/* Arithmetic of the dense J.M contraction (dense_J problems only):
 *   FP32     CUDA-core fp32 products and sums (the plain FP32 FEM).
 *   BF16     tensor cores, bf16 operands, fp32 accumulation.
 *   BF16X2   tensor cores, M split as m_hi + m_lo in bf16 (two products), fp32 accumulation.
 *   FP8      tensor cores, e4m3 operands, fp32 accumulation (FEM_GRAD_PAPER only:
 *            the discretised +-1 marginals and integer couplings |J| <= 16 are exact). */
typedef enum { FEM_PREC_FP32 = 0, FEM_PREC_BF16 = 1, FEM_PREC_BF16X2 = 2, FEM_PREC_FP8 = 3 } fem_precision;

/* How a dense tensor-core anneal is launched (fem_set_dense_launch).  All give
 * bit-identical fields; they differ only in where the optimizer state lives and how
 * the CTAs share the contraction.
 *   AUTO        PERSISTENT when the problem fits it, else PER_STEP (the default).
 *   PER_STEP    one kernel per step; h, m, v stay in global memory.
 *   PERSISTENT  one kernel per fem_anneal window: every CTA keeps its 128 x 128
 *               (rows x replicas) tile of h, m, v in tensor memory for the whole
 *               window and meets the other CTAs of its replica block at a barrier
 *               after each step.  With an even number of row tiles, CTAs run in
 *               pairs (clusters of 2) that issue 256-row MMAs together, each copying
 *               half of the operand; otherwise one CTA per tile.  Needs precision BF16, BF16X2 or FP8, R % 128 == 0 and
 *               (n_pad/128) * (R/128) co-resident CTAs (one per SM), where n_pad = n
 *               rounded up to 128; fem_anneal returns FEM_ERR_UNSUPPORTED otherwise.
 *   PERSISTENT_SINGLE  PERSISTENT without CTA pairs (one CTA per row tile). */
typedef enum {
  FEM_DENSE_AUTO = 0,
  FEM_DENSE_PER_STEP = 1,
  FEM_DENSE_PERSISTENT = 2,
  FEM_DENSE_PERSISTENT_SINGLE = 3
} fem_dense_launch;

typedef struct fem_problem* fem_problem_t; /* opaque; owned by the library until fem_destroy */

/* Problem description.  All pointers are HOST pointers; they are read during
 * fem_create_problem only.
 *   kind       fem_kind.
 *   n          number of variables, 1 <= n < 2^31.
 *   q          states per variable: 2 for MaxCut and Max-k-SAT, 2..8 for bMinCut.
 *   Graph (MaxCut, bMinCut), undirected, each edge listed once:
 *     n_edges, ei[n_edges], ej[n_edges], w[n_edges]
 *       0 <= ei, ej < n, ei != ej, no pair repeated; w finite and nonzero
 *       (bMinCut: w > 0, SM "The bMinCut problem" uses W_ij > 0).  w may be NULL
 *       for unit weights.  Integer weights with |w| <= 2^24 give exact int64
 *       objectives; other weights give fp64 objectives summed in a fixed order.
 *     dense_J    optional n*n row-major couplings (MaxCut only).  When non-NULL the
 *       dense tensor-core path is used and ei/ej/w are ignored.  Must be symmetric
 *       with a zero diagonal and integer entries, |J_ij| <= 127 (exact in bf16 and
 *       int8; FEM_PREC_FP8 further needs |J_ij| <= 16).
 *   Clauses (Max-k-SAT), DIMACS style:
 *     n_clauses, clause_ptr[n_clauses + 1] (clause_ptr[0] = 0, non-decreasing),
 *     lits[clause_ptr[n_clauses]]: signed 1-based variable indices, +v for the
 *     literal v and -v for its negation; a clause must not repeat a variable.
 *   node_weight  optional (bMinCut only), n node weights V_i: positive integers
 *                <= 2^20 with sum < 2^31 (FEM_ERR_INVALID_ARG otherwise).  The balance
 *                term becomes lambda sum_s [(sum_i V_i P_i(s))^2 - sum_i V_i^2 P_i(s)^2]
 *                with the matching gradients (SM, the FPGA task's community graphs,
 *                where a coarsened node weighs the number of nodes it groups), and
 *                the read-out energy cut + lambda_max sum_s [n_s^2 - sum_{i in s} V_i^2]
 *                with n_s = sum_{i in s} V_i.  NULL: every V_i = 1.
 *   linear       optional (QUBO and p-spin), n coefficients of the linear term (d_i,
 *                b_i); NULL: 0.
 *   term_weight  p-spin only (required there): n_clauses coefficients J_v of the terms.
 */
typedef struct {
  int32_t kind;
  int32_t n;
  int32_t q;
  int64_t n_edges;
  const int32_t* ei;
  const int32_t* ej;
  const double* w;
  const float* dense_J;
  int64_t n_clauses;
  const int64_t* clause_ptr;
  const int32_t* lits;
  const double* node_weight;
  const double* linear;
  const double* term_weight;
} fem_problem_desc;

/* Anneal parameters.
 *   replicas     R >= 1; MaxCut sparse: R % 32 == 0; bMinCut: R % 16 == 0 and R*bits(q) % 32 == 0;
 *                Max-k-SAT: R % 16 == 0; dense: R % 128 == 0.  Fixed by the call with t_begin == 0.
 *   n_steps      N_step of the schedules (>= 1).
 *   t_begin, t_end  run steps t_begin .. t_end-1 (0 <= t_begin <= t_end <= n_steps).
 *                t_begin == 0 (re)initialises the fields from h_init and zeroes the
 *                optimizer state; t_begin > 0 resumes and must equal the number of
 *                steps already run (else FEM_ERR_STATE).  Splitting [0, T) into
 *                [0, a) + [a, T) gives bit-identical fields.
 *   schedule, beta_min, beta_max   see fem_schedule (0 < beta_min, 0 < beta_max).
 *   optimizer, lr, beta1, beta2, eps, weight_decay, momentum, alpha, dampening
 *                PyTorch semantics; unused fields are ignored.
 *   gamma_grad   the gradient scale gamma_grad of Eq. gradients_wrt_h.
 *   lambda_max   bMinCut: lambda(t) = lambda_max * t/(N_step - 1) (SM, bMinCut demonstration),
 *                and the weight of the balance term in the read-out energy.
 *   grad_mode    fem_grad_mode.
 *   precision    fem_precision (dense_J problems only).
 *   h_init       required when t_begin == 0: initial fields in the layout of the
 *                file header, fp32, host pointer (or device pointer when
 *                h_init_is_device != 0). */
typedef struct {
  int32_t replicas;
  int32_t n_steps;
  int32_t t_begin;
  int32_t t_end;
  int32_t schedule;
  double beta_min;
  double beta_max;
  int32_t optimizer;
  double lr;
  double beta1;
  double beta2;
  double eps;
  double weight_decay;
  double momentum;
  double alpha;
  double dampening;
  double gamma_grad;
  double lambda_max;
  int32_t grad_mode;
  int32_t precision;
  const float* h_init;
  int32_t h_init_is_device;
} fem_anneal_params;

/* Validate `desc`, build the device-side problem (CSR with the +-1 weight packed
 * into the column index when |w| == 1, normalisers c_i, c^f_i, c^a_i; the clause
 * list and its variable-occurrence transpose; or the dense couplings) and copy it
 * to the current device on `stream`.  Returns FEM_ERR_INVALID_ARG on malformed
 * input (self-loop, duplicate edge, index out of range, repeated variable in a
 * clause, non-symmetric dense_J ...).  On success *out owns device memory until
 * fem_destroy. */
fem_status fem_create_problem(const fem_problem_desc* desc, void* stream, fem_problem_t* out);

/* Run anneal steps [t_begin, t_end) of FEM (Results "Free-Energy Machine"): per step,
 * beta(t) (and lambda(t)), the coupling contraction, the gradient of F with respect
 * to the fields, and one optimizer step on all R replicas.  Asynchronous.  A fresh
 * start (t_begin == 0) allocates the replica state on first use and whenever R
 * changes (the buffers of the previous R are freed first, which waits for the
 * device): fields, optimizer moments and derived buffers, about 16-24 bytes per
 * field and replica (q fields per node for bMinCut; an exact-mode bMinCut anneal
 * adds two more fp32 copies of the field array).  Returns FEM_ERR_OOM if an
 * allocation fails, FEM_ERR_STATE for a resume whose t_begin, R, n_steps, gradient
 * mode or optimizer differ from the run being resumed. */
fem_status fem_anneal(fem_problem_t p, const fem_anneal_params* prm, void* stream);

/* Read out (Results, argmax and argmin equations): each replica's state is the
 * argmax of its marginals (single field: h >= 0 selects the state of P = sigmoid(h);
 * q states: the lowest index among maximal fields), its energy E is computed
 * exactly (int64 for integer weights, fp64 in a fixed order otherwise), and the
 * replica of minimum E wins (lowest index on ties).  Synchronises `stream`.
 *   best_replica  out, may be NULL.
 *   states        out, may be NULL: the winning replica's states, n int32
 *                 (MaxCut +1/-1; bMinCut 0..q-1; Max-k-SAT 0/1).
 *   energy_i64    out, may be NULL: R energies (integer-weighted problems).
 *   energy_f64    out, may be NULL: R energies as fp64 (all problems).
 * MaxCut energies are minus the cut.  Returns FEM_ERR_STATE before any anneal. */
fem_status fem_read_best(fem_problem_t p, int32_t* best_replica, int32_t* states,
                         int64_t* energy_i64, double* energy_f64, void* stream);

/* Batches: many sparse bMinCut and Max-k-SAT problems advanced together (the
 * batched, heterogeneous form of the per-step update).  Two kernel launches per step
 * (one for the q-state members, one for the clause-shaped members) walk a work list of
 * (member, node range) items across all members, the step loop
 * is captured in a CUDA graph and replayed, and the work-item size is chosen by
 * timing candidates on the first steps of the first call (cached per problem shape;
 * every candidate gives bit-identical results).  Each member keeps its own state:
 * after a batched anneal, fem_read_best / fem_read_fields on a member behave as if
 * that member had been annealed alone with the same parameters (bit-identical).
 *   fem_batch_create  members must be sparse bMinCut or Max-k-SAT problems on one
 *                     device; bMinCut members must share q.  The members must outlive
 *                     the batch.  The batch owns only its work list and graph.
 *   fem_batch_anneal  fem_anneal semantics for every member with the same parameters
 *                     (replicas % 16 == 0); h_init[k] is member k's initial fields
 *                     (host, required when t_begin == 0, else ignored). */
typedef struct fem_batch* fem_batch_t;
fem_status fem_batch_create(fem_problem_t const* probs, int32_t count, fem_batch_t* out);
fem_status fem_batch_anneal(fem_batch_t b, const fem_anneal_params* prm, const float* const* h_init,
                            void* stream);

/* One-shot form of the three batch calls: fem_batch_create, fem_batch_anneal and
 * fem_batch_destroy for `count` problems.  The work list and the step-loop graph are
 * built for this call and released at its end, so it synchronises `stream`; the
 * work-item size chosen by timing stays cached per problem shape across calls.
 * Results equal those of the batch object (and of annealing each member alone). */
fem_status fem_anneal_batch(fem_problem_t const* probs, int32_t count, const fem_anneal_params* prm,
                            const float* const* h_init, void* stream);
void fem_batch_destroy(fem_batch_t b);

/* Warm-start network (not from the paper: a learned initialisation of the local
 * fields for sparse MaxCut, judged against plain random-initialised FEM).
 *   P = D^-1 W;  s_i = [1, deg_i / mean deg, sum_j W_ij / deg_i, 1/sqrt(deg_i + 1)]
 *   x^0 = s;  x^l = tanh(x^(l-1) A_l + (P x^(l-1)) B_l + b_l),  l = 1..3, width 64
 *   theta = x^3 C + c (4 taps);  u_0 = z, u_k = P u_(k-1);  y_ir = sum_k theta_ik u_k,ir
 *   loss = mean_ir (tanh(y_ir / 2) - tanh(h_ir / 2))^2,  h = target fields (FEM's own
 *          converged fields)
 * z is a replica's initial fields in units of 0.001 (the paper's 0.001*randn scale),
 * y the predicted fields; y is odd in z (MaxCut's spin-flip symmetry).  Parameters:
 * fem_mpnn_num_params() fp32 values in the order A1[4][64], B1[4][64], b1[64],
 * A2[64][64], B2[64][64], b2[64], A3, B3, b3, C[64][4], c[4] (row-major).  The
 * forward pass reads the weights rounded to bf16 and accumulates in fp32; the
 * gradient is with respect to those rounded weights; the optimizer (Adam,
 * beta 0.9/0.999, eps 1e-8) updates the fp32 master copy.
 *   graph: a sparse MaxCut problem (its CSR is used).  z, h_target, y: DEVICE
 *   pointers, [n][R] fp32.  grad: HOST, num_params floats (may be NULL).
 *   rms (fem_mpnn_predict): 0 returns y as is; rms > 0 rescales every replica's
 *   column to root-mean-square rms, y_ir * rms / sqrt(mean_i y_ir^2) (the network
 *   fixes the direction of the warm start, the caller its magnitude; an all-zero
 *   column stays zero).  FEM_ERR_INVALID_ARG for rms < 0 or NaN.
 * A network keeps a device workspace for its activations, grown to the largest call
 * so far (a call that needs more allocates the rest stream-ordered and the workspace
 * is grown when it ends, a step that waits for the device); calls on one network must
 * not overlap on the GPU. */
typedef struct fem_mpnn* fem_mpnn_t;
int32_t fem_mpnn_num_params(void);
fem_status fem_mpnn_create(const float* params_host, fem_mpnn_t* out);
fem_status fem_mpnn_get_params(fem_mpnn_t net, float* params_host);
fem_status fem_mpnn_predict(fem_mpnn_t net, fem_problem_t graph, const float* z, int32_t replicas, float rms,
                            float* y, void* stream);
fem_status fem_mpnn_grad(fem_mpnn_t net, fem_problem_t graph, const float* z, const float* h_target,
                         int32_t replicas, float* grad_host, double* loss, void* stream);
fem_status fem_mpnn_train_step(fem_mpnn_t net, fem_problem_t graph, const float* z, const float* h_target,
                               int32_t replicas, double lr, double* loss, void* stream);
void fem_mpnn_destroy(fem_mpnn_t net);

/* Copy the current fields to `h_host` (layout of the file header; n*R (single
 * field) or n*R*q floats).  The destination may be host memory or a device buffer
 * of the problem's device (the warm-start trainer reads fields straight into a
 * device tensor).  Synchronises `stream`. */
fem_status fem_read_fields(fem_problem_t p, float* h_host, void* stream);

/* Copy every replica's argmax states to `states_host`, n*R int32, layout [n][R]. */
fem_status fem_read_states(fem_problem_t p, int32_t* states_host, void* stream);

/* Checkpoint: copy the fields h and the optimizer state to host buffers in the
 * layout of the fields (any pointer may be NULL).  m holds Adam's first moment or
 * the momentum buffer of RMSprop/SGD; v holds Adam's second moment or RMSprop's
 * running square average.  Together with fem_problem_info's steps_done this is
 * the complete state of an anneal.  Synchronises `stream`. */
fem_status fem_read_state(fem_problem_t p, float* h, float* m, float* v, void* stream);

/* Restore a checkpoint: overwrite h, m and v from host buffers (m or v NULL =
 * zeros) and set the number of steps already run to `steps_done`
 * (0 <= steps_done <= n_steps), so that the next fem_anneal resumes with
 * t_begin = steps_done.  The problem must already be initialised by a
 * fem_anneal call with t_begin == 0, which fixes R, N_step, the gradient mode and
 * the optimizer (FEM_ERR_STATE otherwise).  Derived per-step data (discretised
 * states, group counts) are recomputed from h.  Synchronises `stream`. */
fem_status fem_write_state(fem_problem_t p, const float* h, const float* m, const float* v,
                           int32_t steps_done, void* stream);

/* Number of steps run so far, and the problem's sizes (any pointer may be NULL):
 * n, q, R (0 before the first anneal), and the number of units one step processes
 * per replica (|E| undirected edges for graphs, n(n-1)/2 for dense_J, the
 * literal-occurrence count for clause lists). */
fem_status fem_problem_info(fem_problem_t p, int32_t* steps_done, int32_t* n, int32_t* q,
                            int32_t* replicas, int64_t* units_per_replica);

/* Synchronise `stream` and report any sticky device-side error. */
fem_status fem_sync(fem_problem_t p, void* stream);

/* Select how later fem_anneal calls on a dense problem are launched (fem_dense_launch);
 * FEM_ERR_INVALID_ARG for other values or a problem without dense couplings. */
fem_status fem_set_dense_launch(fem_problem_t p, int32_t mode);

/* The kernel the last fem_anneal window of a dense problem ran on: FEM_DENSE_PER_STEP,
 * FEM_DENSE_PERSISTENT (CTA pairs) or FEM_DENSE_PERSISTENT_SINGLE; 0 before the
 * first window, and for problems without dense couplings. */
fem_status fem_dense_last_launch(fem_problem_t p, int32_t* mode);

/* Failure detection (no counterpart in the paper).
 *   fem_set_step_barrier_timeout: the limit, in ns, on the persistent dense kernel's
 *     per-step barrier between CTAs (default 2 s).  A CTA that waits longer records
 *     FEM_ERR_TIMEOUT in the problem's sticky error word, lets its own copies and MMAs
 *     land, frees its tensor memory and returns; the others give up in turn.  The error
 *     surfaces on the next fem_read_* / fem_sync call; an fem_anneal with t_begin == 0
 *     clears it.
 *   fem_inject_step_stall: the persistent dense kernel's CTAs of row tile `row_tile`
 *     (rows 128 * row_tile ..) stop arriving at the step barrier, so the waits of the
 *     other CTAs of their replica blocks run out (tests of the timeout path without a
 *     GPU fault); -1 switches it off.  FEM_ERR_INVALID_ARG for row_tile < -1.
 *   fem_inject_allocation_failure: after `after` >= 0 further successful device
 *     allocations of problems, the next one fails with FEM_ERR_OOM (then the injection
 *     switches itself off); -1 disables it.  Process-wide, for tests. */
fem_status fem_set_step_barrier_timeout(fem_problem_t p, int64_t ns);
fem_status fem_inject_step_stall(fem_problem_t p, int32_t row_tile);
void fem_inject_allocation_failure(int64_t after);

/* Release every resource owned by p (NULL is ignored). */
void fem_destroy(fem_problem_t p);

/* Static English name of a status code. */
const char* fem_status_string(fem_status s);

/* One-line description of the last failure on the calling thread ("" if none). */
const char* fem_last_error(void);

/* The schedule values step t of the anneal described by `a` uses: beta_t (the
 * exponential or inverse-proportional schedule from beta_min to beta_max over
 * a->n_steps steps; Methods, "Different annealing schedules") and the balance
 * weight lambda_t = lambda_max * t / (n_steps - 1) (SM, bMinCut demonstration).
 * Only a->schedule, beta_min, beta_max, lambda_max and n_steps are read.  A caller
 * that starts an anneal part-way along a schedule (a warm start) takes its beta from
 * here.  Host-only and synchronous.  FEM_ERR_INVALID_ARG unless 0 <= t < n_steps,
 * both betas are finite and > 0 and the schedule is known.  Either output may be
 * NULL. */
fem_status fem_schedule_value(const fem_anneal_params* a, int32_t t, double* beta, double* lambda);

/* Number of CUDA kernels this library has launched in the process so far (all
 * handles, all threads).  Lets a caller count the device work behind a call. */
int64_t fem_kernel_launches(void);

/* Where fem_create_problem builds a sparse graph's CSR: graphs with at least
 * min_edges undirected edges on the device of the call (degrees, a prefix sum, a
 * scatter of (column, edge) keys and a per-row sort), smaller ones on the host; a
 * negative value keeps every build on the host.  Both give the same arrays bit for
 * bit.  The device builder validates the copied edge list on the device (indices,
 * self-loops, weights; chunk sums of the weights added in the same order as on the
 * host) before anything indexes with it, the host builder on the host threads; either
 * reports the lowest invalid edge, or a duplicate edge, as FEM_ERR_INVALID_ARG with the
 * same message.  Process-wide; the default is 65536.  Clause lists (Max-k-SAT and
 * p-spin) follow the same threshold on their literal count: long lists are copied once
 * and validated, transposed (occurrences in clause order) and, for p-spin, folded with
 * the literals' negations on the device, with the host builder's tables and messages.
 * Dense couplings are always copied once and validated and converted on the device. */
void fem_set_device_graph_build(int64_t min_edges);

/* Which kernels run the sparse MaxCut and QUBO steps: on (the default) the tile kernels
 * that stage their operands in shared memory ahead of use - exact mode with TMA gather4
 * copies of the neighbours' lines, paper mode (unit or +-1 weights, graphs of at least
 * 4096 groups of four nodes) with bulk copies of the state and sign words gathered by a
 * producer warp - off the kernels that load everything directly.  Both compute the same
 * sums in the same order and give the same bits.  Process-wide. */
void fem_set_tma_gather(int32_t on);

/* MaxCut energies of caller-provided sign words, without allocating.
 * The paper has no counterpart: this is a library service for callers that cannot
 * call cudaMalloc - for example code whose device memory is owned by a pool manager,
 * or a loop that must not allocate because an allocation can synchronise the device.
 * The caller passes every input and output (all DEVICE pointers on the current
 * device); the only scratch is a fixed 2 MiB array in the library's device image,
 * which each GPU that loads the library holds until the process exits.
 *   row_ptr[n+1], col[row_ptr[n]]  the graph in the library's CSR form: every
 *        undirected edge in both rows, column index in bits 0-30 and the edge weight
 *        (+1 or -1 only) in bit 31 (set = -1).
 *   words[n][replicas/32]  bit r of word (i, r/32) set <=> replica r puts node i in
 *        state -1.
 *   energy[replicas]  out: E_r = -cut_r (int64); best_replica[1] out: argmin E,
 *        lowest index on ties.
 * replicas must be a multiple of 32 and at most 1024 (FEM_ERR_UNSUPPORTED beyond).
 * Asynchronous on `stream`, so the CSR cannot be validated on the host: the kernel
 * checks that every row lies in [0, row_ptr[n]) and every column is below n, skips
 * anything outside (no access beyond those bounds) and then writes best_replica = -1;
 * the energies of such a call are meaningless.  col must hold row_ptr[n] entries.
 * The first call on a device looks up the scratch address (a CUDA runtime query),
 * so make that first call before any stream capture; the address is cached for the
 * life of the process and is invalid after cudaDeviceReset.  Calls share the scratch
 * array: calls that overlap on the GPU (different streams, no ordering between them)
 * race and give wrong results. */
fem_status fem_maxcut_energies_noalloc(const int32_t* row_ptr, const uint32_t* col, int32_t n,
                                       const uint32_t* words, int32_t replicas, int64_t* energy,
                                       int32_t* best_replica, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FEM_H */
