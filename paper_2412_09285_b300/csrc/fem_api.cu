// The C ABI of libfem: argument validation, host-side problem builders, state
// management and dispatch to the kernels.  Nothing here prints or aborts.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "fem_internal.h"

namespace fem {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};
constexpr long long kGraphMaxElems = 1ll << 21;  // node x replica (x q) elements of a "small" problem
constexpr int64_t kGraphMinSteps = 16;

void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

fem_status fail(fem_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

fem_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error so the context stays usable
  if (e == cudaErrorMemoryAllocation) return fail(FEM_ERR_OOM, "%s: out of device memory", what);
  return fail(FEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Failure injection for tests: >= 0 makes the allocation after that many successful
// ones fail as if the device were out of memory (then it switches itself off).
static std::atomic<int64_t> g_fail_alloc_after{-1};

fem_status dev_alloc(Problem* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  int64_t left = g_fail_alloc_after.load();
  while (left >= 0 && !g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
  }
  if (left == 0) return fail(FEM_ERR_OOM, "allocation of %zu bytes failed (injected)", bytes);
  const cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(FEM_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  p->allocs.push_back(*ptr);
  ++p->alloc_gen;
  return FEM_OK;
}

template <typename T>
static fem_status upload(Problem* p, T** dst, const std::vector<T>& src, cudaStream_t s) {
  fem_status st = dev_alloc_t(p, dst, src.size());
  if (st != FEM_OK) return st;
  if (!src.empty()) FEM_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T),
                                             cudaMemcpyHostToDevice, s));
  return FEM_OK;
}

// ---------------------------------------------------------------------------
// Per-step scalars: the beta schedule (Methods, "Different annealing schedules"),
// the lambda ramp (SM bMinCut demonstration) and the optimizer constants.
// ---------------------------------------------------------------------------
static double beta_at(const fem_anneal_params& a, int t) {
  if (a.n_steps == 1) return a.beta_min;
  if (a.schedule == FEM_SCHED_EXPONENTIAL)
    return std::exp((std::log(a.beta_max) - std::log(a.beta_min)) / (a.n_steps - 1) * t +
                    std::log(a.beta_min));
  return 1.0 / ((1.0 / a.beta_max - 1.0 / a.beta_min) / (a.n_steps - 1) * t + 1.0 / a.beta_min);
}

static double lambda_at(const fem_anneal_params& a, int t) {
  return a.n_steps == 1 ? 0.0 : a.lambda_max * (double)t / (double)(a.n_steps - 1);
}

std::vector<StepScalars> make_step_scalars(const fem_anneal_params& a, int32_t single_field) {
  std::vector<StepScalars> out;
  out.reserve(a.t_end - a.t_begin);
  for (int t = a.t_begin; t < a.t_end; ++t) {
    StepScalars s;
    std::memset(&s, 0, sizeof(s));
    const double beta = beta_at(a, t);
    const double lam = lambda_at(a, t);
    s.inv_beta = (float)(1.0 / beta);
    s.lambda = (float)lam;
    s.gq = (float)(single_field ? a.gamma_grad / 4.0 : a.gamma_grad);
    const int tt = t + 1;
    switch (a.optimizer) {
      case FEM_OPT_ADAM:
        s.lr = (float)(a.lr / (1.0 - std::pow(a.beta1, tt)));
        s.b1 = (float)a.beta1;
        s.omb1 = (float)(1.0 - a.beta1);
        s.b2 = (float)a.beta2;
        s.omb2 = (float)(1.0 - a.beta2);
        s.inv_sqrt_bc2 = (float)(1.0 / std::sqrt(1.0 - std::pow(a.beta2, tt)));
        s.eps = (float)a.eps;
        break;
      case FEM_OPT_RMSPROP:
        s.lr = (float)a.lr;
        s.b1 = (float)a.alpha;
        s.omb1 = (float)(1.0 - a.alpha);
        s.eps = (float)a.eps;
        s.momentum = (float)a.momentum;
        break;
      default:
        s.lr = (float)a.lr;
        s.b1 = (float)a.momentum;
        s.omb1 = (float)(1.0 - a.dampening);
        s.first = tt == 1;
        break;
    }
    s.wd = (float)a.weight_decay;
    out.push_back(s);
  }
  return out;
}

// Declared in the kernel files.
// Validates the edge list on the device (setting unit_w, int_w and the weight sums of
// p) and builds the CSR there.
fem_status device_graph_build(Problem* p, int32_t kind, int32_t q, const fem_problem_desc* d, cudaStream_t s);
// Validates a clause list on the device and builds its tables there (p-spin: also the
// folded term coefficients; *terms_int tells whether they are all integers).
fem_status device_sat_build(Problem* p, const fem_problem_desc* d, bool pspin, bool* terms_int, cudaStream_t s);
fem_status maxcut_pack_words(Problem* p, int hbuf, int wbuf, cudaStream_t s, const float* src = nullptr);
const float* maxcut_current_fields(const Problem* p);
fem_status maxcut_states_all(Problem* p, int32_t* out_dev, cudaStream_t s);

// The field buffer step `steps_done` reads.  Paper-mode graph problems and
// Max-k-SAT update h in place; exact-mode graph problems ping-pong it.
static float* fields_for_step(Problem* p, int t) {
  if (p->kind == FEM_MAXKSAT || p->grad_mode == FEM_GRAD_PAPER) return p->h[0];
  return p->h[t & 1];
}
static const float* current_fields(Problem* p) { return fields_for_step(p, p->steps_done); }

// ---------------------------------------------------------------------------
// Graph builder: validated undirected edge list -> CSR of directed entries.
// Host-only (no CUDA call), so malformed input is rejected before any device work.
// ---------------------------------------------------------------------------
struct HostGraph {
  int64_t n_edges = 0;
  bool unit = true, integer = true;
  int64_t wsum_i = 0;   // sum of the edge weights (exact when they are integers)
  double wsum_f = 0.0;
  std::vector<int32_t> row_ptr;
  std::vector<uint32_t> col;
  std::vector<float> wf, cnorm, cnorm2;
  std::vector<double> w64;
};

// Graphs with at least this many edges build their CSR on the device
// (fem_set_device_graph_build); below it the host builder is quicker than the launches.
static std::atomic<int64_t> g_device_build_min_edges{1 << 16};

// One unit of the host edge scan: the first invalid edge, the weight flags and the
// integer sum; the fp64 sums of its chunks go to csum.
struct EdgeScan {
  int64_t bad = -1;  // lowest invalid edge of the unit, or -1
  bool unit = true, integer = true;
  int64_t wsum_i = 0;
};

constexpr int64_t kScanUnit = 256 * kWeightChunk;  // edges per unit of work of a host thread

// Edges e0 .. e1-1 (e0 a multiple of kWeightChunk).  The flags and sums stay in
// registers until the end (the records of neighbouring threads share cache lines).
static void scan_edges(int32_t kind, const fem_problem_desc* d, int64_t e0, int64_t e1, EdgeScan& out,
                       double* csum) {
  const uint32_t n = (uint32_t)d->n;
  const bool pos_only = kind == FEM_BMINCUT;
  int64_t si = 0;
  bool unit = true, integer = true;
  int64_t bad = -1;
  for (int64_t c0 = e0; c0 < e1 && bad < 0; c0 += kWeightChunk) {
    const int64_t c1 = std::min(e1, c0 + kWeightChunk);
    double sf = 0.0;
    for (int64_t e = c0; e < c1; ++e) {
      const int32_t i = d->ei[e], j = d->ej[e];
      const double w = d->w ? d->w[e] : 1.0;
      const double a = std::fabs(w);
      // in range, no self-loop, finite (NaN fails the comparison) and nonzero
      if (!((uint32_t)i < n && (uint32_t)j < n && i != j && a <= 1.7976931348623157e308 && w != 0.0 &&
            (!pos_only || w > 0.0))) {
        bad = e;
        break;
      }
      unit = unit && a == 1.0;
      const bool small = a <= 16777216.0;
      const int64_t wi = (int64_t)(small ? w : 0.0);
      integer = integer && small && (double)wi == w;
      sf += w;
      si += wi;
    }
    csum[c0 / kWeightChunk] = sf;
  }
  EdgeScan r;
  r.bad = bad;
  r.unit = unit;
  r.integer = integer;
  r.wsum_i = si;
  out = r;
}

fem_status edge_error(const fem_problem_desc* d, int32_t kind, int64_t e) {
  const int32_t i = d->ei[e], j = d->ej[e], n = d->n;
  const double w = d->w ? d->w[e] : 1.0;
  if (i < 0 || i >= n || j < 0 || j >= n)
    return fail(FEM_ERR_INVALID_ARG, "edge %lld: endpoint out of range [0, %d)", (long long)e, n);
  if (i == j) return fail(FEM_ERR_INVALID_ARG, "edge %lld: self-loop at %d", (long long)e, i);
  if (!std::isfinite(w) || w == 0.0)
    return fail(FEM_ERR_INVALID_ARG, "edge %lld: weight must be finite and nonzero", (long long)e);
  (void)kind;  // the remaining check: bMinCut weights are positive
  return fail(FEM_ERR_INVALID_ARG, "edge %lld: bMinCut weights must be positive", (long long)e);
}

// The checks every edge list gets before it is read.
static fem_status edge_list_basics(const fem_problem_desc* d) {
  if (d->n_edges < 0) return fail(FEM_ERR_INVALID_ARG, "n_edges < 0");
  if (d->n_edges > 0 && (!d->ei || !d->ej)) return fail(FEM_ERR_INVALID_ARG, "ei/ej must be non-NULL");
  if (2 * d->n_edges >= (int64_t)INT32_MAX) return fail(FEM_ERR_UNSUPPORTED, "2|E| must be < 2^31");
  return FEM_OK;
}

// Validation, weight flags and sums on the host, before any device work, over
// several host threads for long lists; with build, the CSR too (the device builder
// takes large lists and validates them itself).  The error names the lowest invalid edge.
static fem_status host_graph(int32_t kind, int32_t q, const fem_problem_desc* d, HostGraph& g, bool build = true) {
  const int32_t n = d->n;
  const int64_t E = d->n_edges;
  fem_status st0 = edge_list_basics(d);
  if (st0 != FEM_OK) return st0;
  const int64_t nunits = (E + kScanUnit - 1) / kScanUnit;
  std::vector<EdgeScan> part((size_t)nunits);
  std::vector<double> csum((size_t)((E + kWeightChunk - 1) / kWeightChunk), 0.0);
  auto run = [&](int64_t u) {
    scan_edges(kind, d, u * kScanUnit, std::min(E, (u + 1) * kScanUnit), part[u], csum.data());
  };
  const int64_t hw = std::max<int64_t>(1, (int64_t)std::thread::hardware_concurrency());
  const int nth = (int)std::min<int64_t>({nunits, hw, 16});
  if (nth > 1) {
    std::atomic<int64_t> next{0};
    auto worker = [&]() {
      for (int64_t u; (u = next.fetch_add(1)) < nunits;) run(u);
    };
    std::vector<std::thread> pool;
    try {
      for (int t = 1; t < nth; ++t) pool.emplace_back(worker);
    } catch (...) {  // fewer threads: the calling thread scans what is left
    }
    worker();
    for (auto& t : pool) t.join();
  } else {
    for (int64_t u = 0; u < nunits; ++u) run(u);
  }
  bool unit = true, integer = true;
  for (const EdgeScan& r : part) {
    if (r.bad >= 0) return edge_error(d, kind, r.bad);
    unit = unit && r.unit;
    integer = integer && r.integer;
    g.wsum_i += r.wsum_i;
  }
  for (double x : csum) g.wsum_f += x;
  g.n_edges = E;
  g.unit = unit;
  g.integer = integer;
  if (!build) return FEM_OK;
  std::vector<int32_t> deg((size_t)n + 1, 0);
  for (int64_t e = 0; e < E; ++e) {
    deg[d->ei[e]]++;
    deg[d->ej[e]]++;
  }
  std::vector<int32_t>& row_ptr = g.row_ptr;
  row_ptr.assign(n + 1, 0);
  for (int32_t i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + deg[i];
  const int64_t nnz = row_ptr[n];
  std::vector<std::pair<int32_t, double>> ent(nnz);
  std::vector<int32_t> fillp(row_ptr.begin(), row_ptr.end() - 1);
  for (int64_t e = 0; e < E; ++e) {
    const int32_t i = d->ei[e], j = d->ej[e];
    const double w = d->w ? d->w[e] : 1.0;
    ent[fillp[i]++] = {j, w};
    ent[fillp[j]++] = {i, w};
  }
  g.col.assign(nnz, 0);
  g.wf.assign(unit ? 0 : nnz, 0.f);
  g.w64.assign(integer ? 0 : nnz, 0.0);
  std::vector<double> rsum(n, 0.0), rabs(n, 0.0);
  for (int32_t i = 0; i < n; ++i) {
    auto b = ent.begin() + row_ptr[i], en = ent.begin() + row_ptr[i + 1];
    std::sort(b, en, [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
      return x.first < y.first;
    });
    for (auto it = b; it != en; ++it) {
      if (it != b && (it - 1)->first == it->first)
        return fail(FEM_ERR_INVALID_ARG, "duplicate edge (%d, %d)", i, it->first);
      const int64_t k = it - ent.begin();
      g.col[k] = (uint32_t)it->first | ((unit && it->second < 0) ? 0x80000000u : 0u);
      if (!unit) g.wf[k] = (float)it->second;
      if (!integer) g.w64[k] = it->second;
      rsum[i] += it->second;
      rabs[i] += std::fabs(it->second);
    }
  }
  g.n_edges = E;
  g.unit = unit;
  g.integer = integer;
  if (kind == FEM_MAXCUT) {
    // c_i = 1 / sum_j |W_ij| (SM, after Eq. maxcut_modified_gradient); unit weights
    // derive it from the degree inside the kernel.
    if (!unit) {
      g.cnorm.resize(n);
      for (int32_t i = 0; i < n; ++i) g.cnorm[i] = rabs[i] > 0 ? (float)(1.0 / rabs[i]) : 0.f;
    }
  } else {
    // c^f_i = q / sum_j W_ij, c^a_i = q / sqrt(sum_j W_ij) (SM "The bMinCut problem").
    g.cnorm.resize(n);
    g.cnorm2.resize(n);
    for (int32_t i = 0; i < n; ++i) {
      g.cnorm[i] = rsum[i] > 0 ? (float)(q / rsum[i]) : 0.f;
      g.cnorm2[i] = rsum[i] > 0 ? (float)(q / std::sqrt(rsum[i])) : 0.f;
    }
  }
  return FEM_OK;
}

static fem_status upload_graph(Problem* p, const HostGraph& g, cudaStream_t s) {
  p->n_edges = g.n_edges;
  p->nnz = (int64_t)g.col.size();
  p->unit_w = g.unit;
  p->int_w = g.integer;
  fem_status st;
  if ((st = upload(p, &p->row_ptr, g.row_ptr, s)) != FEM_OK) return st;
  if ((st = upload(p, &p->col, g.col, s)) != FEM_OK) return st;
  if (!g.unit && (st = upload(p, &p->w, g.wf, s)) != FEM_OK) return st;
  if (!g.integer && (st = upload(p, &p->w64, g.w64, s)) != FEM_OK) return st;
  if (!g.cnorm.empty() && (st = upload(p, &p->cnorm, g.cnorm, s)) != FEM_OK) return st;
  if (!g.cnorm2.empty() && (st = upload(p, &p->cnorm2, g.cnorm2, s)) != FEM_OK) return st;
  return FEM_OK;
}

// ---------------------------------------------------------------------------
// Clause builder: DIMACS-style clause list -> packed literals and the
// variable -> occurrence transpose (occurrences in clause order).  Host-only.
// ---------------------------------------------------------------------------
struct HostSat {
  int64_t n_clauses = 0;
  int32_t max_width = 0, min_width = 0;
  std::vector<int32_t> cl_ptr, cl_lit, occ_ptr, occ;
  // every clause has 3 literals: per occurrence (in occ order) the clause's other two
  // literals in clause order, the first with the occurrence's own negation in bit 31
  std::vector<int32_t> oth;
};

// The checks of a clause list that read only its header (the clause and literal counts).
static fem_status sat_basics(const fem_problem_desc* d) {
  const int64_t M = d->n_clauses;
  if (M < 0) return fail(FEM_ERR_INVALID_ARG, "n_clauses < 0");
  if (M > 0 && (!d->clause_ptr || !d->lits)) return fail(FEM_ERR_INVALID_ARG, "clause_ptr/lits must be non-NULL");
  if (M >= (1ll << 28)) return fail(FEM_ERR_UNSUPPORTED, "at most 2^28 - 1 clauses");
  const int64_t L = M > 0 ? d->clause_ptr[M] : 0;
  if (M > 0 && d->clause_ptr[0] != 0) return fail(FEM_ERR_INVALID_ARG, "clause_ptr[0] must be 0");
  if (L < 0 || L >= (int64_t)INT32_MAX) return fail(FEM_ERR_UNSUPPORTED, "literal count must be < 2^31");
  return FEM_OK;
}

static fem_status host_sat(const fem_problem_desc* d, HostSat& g) {
  const int32_t n = d->n;
  const int64_t M = d->n_clauses;
  if (fem_status st = sat_basics(d); st != FEM_OK) return st;
  const int64_t L = M > 0 ? d->clause_ptr[M] : 0;
  g.cl_ptr.assign(M + 1, 0);
  g.cl_lit.assign(L, 0);
  std::vector<int32_t> cnt(n + 1, 0);
  for (int64_t c = 0; c < M; ++c) {
    const int64_t b = d->clause_ptr[c], e = d->clause_ptr[c + 1];
    if (e < b || e > L) return fail(FEM_ERR_INVALID_ARG, "clause_ptr must be non-decreasing and end at the literal count");
    if (e - b > 8) return fail(FEM_ERR_UNSUPPORTED, "clause %lld has more than 8 literals", (long long)c);
    g.max_width = std::max<int32_t>(g.max_width, (int32_t)(e - b));
    g.cl_ptr[c + 1] = (int32_t)e;
    for (int64_t k = b; k < e; ++k) {
      const int32_t lit = d->lits[k];
      if (lit == 0 || lit > n || lit < -n)
        return fail(FEM_ERR_INVALID_ARG, "clause %lld: literal %d out of range", (long long)c, lit);
      const int32_t v = std::abs(lit) - 1;
      for (int64_t k2 = b; k2 < k; ++k2)
        if (std::abs(d->lits[k2]) - 1 == v)
          return fail(FEM_ERR_INVALID_ARG, "clause %lld repeats variable %d", (long long)c, v + 1);
      g.cl_lit[k] = (v << 1) | (lit < 0 ? 1 : 0);
      cnt[v]++;
    }
  }
  g.occ_ptr.assign(n + 1, 0);
  for (int32_t i = 0; i < n; ++i) g.occ_ptr[i + 1] = g.occ_ptr[i] + cnt[i];
  g.occ.assign(L, 0);
  std::vector<int32_t> fill(g.occ_ptr.begin(), g.occ_ptr.end() - 1);
  for (int64_t c = 0; c < M; ++c)
    for (int32_t k = g.cl_ptr[c]; k < g.cl_ptr[c + 1]; ++k)
      g.occ[fill[g.cl_lit[k] >> 1]++] = (int32_t)((c << 3) | (k - g.cl_ptr[c]));
  g.n_clauses = M;
  g.min_width = 8;
  for (int64_t c = 0; c < M; ++c) g.min_width = std::min<int32_t>(g.min_width, g.cl_ptr[c + 1] - g.cl_ptr[c]);
  if (M > 0 && g.min_width == 3 && g.max_width == 3) {
    g.oth.assign(2 * (size_t)L, 0);
    for (int64_t o = 0; o < L; ++o) {
      const int32_t c = g.occ[o] >> 3, pos = g.occ[o] & 7, b = g.cl_ptr[c];
      int32_t other[2], k2 = 0;
      for (int32_t k = 0; k < 3; ++k)
        if (k != pos) other[k2++] = g.cl_lit[b + k];
      const uint32_t own_neg = (uint32_t)(g.cl_lit[b + pos] & 1);
      g.oth[2 * o] = (int32_t)((uint32_t)other[0] | (own_neg << 31));
      g.oth[2 * o + 1] = other[1];
    }
  }
  return FEM_OK;
}

static fem_status upload_sat(Problem* p, const HostSat& g, cudaStream_t s) {
  p->n_clauses = g.n_clauses;
  p->n_occ = (int64_t)g.cl_lit.size();
  p->max_width = g.max_width;
  fem_status st;
  if ((st = upload(p, &p->cl_ptr, g.cl_ptr, s)) != FEM_OK) return st;
  if ((st = upload(p, &p->cl_lit, g.cl_lit, s)) != FEM_OK) return st;
  if ((st = upload(p, &p->occ_ptr, g.occ_ptr, s)) != FEM_OK) return st;
  if ((st = upload(p, &p->occ, g.occ, s)) != FEM_OK) return st;
  if (!g.oth.empty() && (st = upload(p, &p->oth, g.oth, s)) != FEM_OK) return st;
  return FEM_OK;
}

static void drop_step_graphs(Problem* p) {
  for (auto& g : p->step_graphs) cudaGraphExecDestroy(g.exec);
  p->step_graphs.clear();
}

static fem_status ensure_state(Problem* p, int32_t R, int32_t grad_mode, cudaStream_t s) {
  const size_t per = (size_t)p->n * R * (p->kind == FEM_BMINCUT ? p->q : 1);
  if (p->R == R && p->h[0]) {
    // bMinCut exact mode gathers its neighbours' centred marginals (first use)
    if (p->kind == FEM_BMINCUT && grad_mode == FEM_GRAD_EXACT && !p->mag[0])
      for (int b = 0; b < 2; ++b) {
        const fem_status st = dev_alloc_t(p, &p->mag[b], per);
        if (st != FEM_OK) return st;
      }
    return FEM_OK;
  }
  drop_step_graphs(p);  // the graphs name the buffers being replaced
  // the buffers sized for the previous R are released first (cudaFree waits for the
  // device, so no queued work still uses them)
  auto release = [p](auto*& ptr) {
    if (!ptr) return;
    cudaFree(ptr);
    p->allocs.erase(std::remove(p->allocs.begin(), p->allocs.end(), (void*)ptr), p->allocs.end());
    ptr = nullptr;
  };
  for (int b = 0; b < 2; ++b) {
    release(p->h[b]);
    release(p->words[b]);
    release(p->mag[b]);
    release(p->satP[b]);
  }
  release(p->m);
  release(p->v);
  for (int b = 0; b < 3; ++b) {
    release(p->cnt[b]);
    release(p->psum[b]);
  }
  release(p->part_i);
  release(p->part_f);
  release(p->part_cnt);
  release(p->energy_i);
  release(p->energy_f);
  release(p->best);
  release(p->states_dev);
  p->R = 0;  // no state until every buffer below is in place
  fem_status st;
  for (int b = 0; b < 2; ++b)
    if ((st = dev_alloc_t(p, &p->h[b], per)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->m, per)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->v, per)) != FEM_OK) return st;
  p->words_per_node = (p->kind == FEM_MAXCUT) ? R / 32
                      : (p->kind == FEM_BMINCUT) ? R * bmincut_bits(p->q) / 32 : (R + 31) / 32;
  for (int b = 0; b < 2; ++b)
    if ((st = dev_alloc_t(p, &p->words[b], (size_t)p->n * p->words_per_node)) != FEM_OK) return st;
  if (p->kind == FEM_MAXCUT || (p->kind == FEM_BMINCUT && grad_mode == FEM_GRAD_EXACT)) {
    for (int b = 0; b < 2; ++b) {
      if ((st = dev_alloc_t(p, &p->mag[b], per)) != FEM_OK) return st;
    }
  }
  if (p->kind == FEM_BMINCUT) {
    for (int b = 0; b < 3; ++b) {
      if ((st = dev_alloc_t(p, &p->cnt[b], (size_t)R * p->q)) != FEM_OK) return st;
      if ((st = dev_alloc_t(p, &p->psum[b], (size_t)R * p->q)) != FEM_OK) return st;
    }
  }
  if (p->kind == FEM_MAXKSAT)
    for (int b = 0; b < 2; ++b)
      if ((st = dev_alloc_t(p, &p->satP[b], per)) != FEM_OK) return st;
  p->part_blocks = std::max(1, std::min((p->n + 15) / 16, p->sm_count * 4));
  const size_t part = (size_t)p->part_blocks * R;
  if ((st = dev_alloc_t(p, &p->part_i, part)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->part_f, part)) != FEM_OK) return st;
  if (p->kind == FEM_BMINCUT && (st = dev_alloc_t(p, &p->part_cnt, part * p->q)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->energy_i, (size_t)R)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->energy_f, (size_t)R)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->best, 1)) != FEM_OK) return st;
  if ((st = dev_alloc_t(p, &p->states_dev, (size_t)p->n)) != FEM_OK) return st;
  p->R = R;
  (void)s;
  return FEM_OK;
}

static fem_status check_sticky(Problem* p, cudaStream_t s) {
  int32_t e = 0;
  FEM_CUDA(cudaMemcpyAsync(&e, p->err, sizeof(e), cudaMemcpyDeviceToHost, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  if (e & ERR_TIMEOUT) return fail(FEM_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (e & ERR_BOUNDS) return fail(FEM_ERR_DEVICE, "a device-side bounds check failed");
  return FEM_OK;
}

// fem_set_tma_gather: sparse MaxCut / QUBO steps on the staged tile kernels.
static std::atomic<int32_t> g_tma_gather{1};
bool tma_gather_enabled() { return g_tma_gather.load() != 0; }

}  // namespace fem

using namespace fem;

extern "C" {

const char* fem_status_string(fem_status s) {
  switch (s) {
    case FEM_OK: return "FEM_OK";
    case FEM_ERR_INVALID_ARG: return "FEM_ERR_INVALID_ARG";
    case FEM_ERR_UNSUPPORTED: return "FEM_ERR_UNSUPPORTED";
    case FEM_ERR_OOM: return "FEM_ERR_OOM";
    case FEM_ERR_CUDA: return "FEM_ERR_CUDA";
    case FEM_ERR_TIMEOUT: return "FEM_ERR_TIMEOUT";
    case FEM_ERR_STATE: return "FEM_ERR_STATE";
    case FEM_ERR_DEVICE: return "FEM_ERR_DEVICE";
  }
  return "FEM_ERR_UNKNOWN";
}

const char* fem_last_error(void) { return g_last_error.c_str(); }

int64_t fem_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void fem_destroy(fem_problem_t p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  drop_step_graphs(p);
  if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
  for (void* a : p->allocs) cudaFree(a);
  if (cur != p->device) cudaSetDevice(cur);
  delete p;
}

fem_status fem_create_problem(const fem_problem_desc* d, void* stream, fem_problem_t* out) {
  g_last_error.clear();
  if (!d || !out) return fail(FEM_ERR_INVALID_ARG, "desc and out must be non-NULL");
  *out = nullptr;
  if (d->kind < FEM_MAXCUT || d->kind > FEM_PSPIN) return fail(FEM_ERR_INVALID_ARG, "unknown kind %d", d->kind);
  if (d->n < 1) return fail(FEM_ERR_INVALID_ARG, "n must be >= 1");
  if ((d->kind == FEM_MAXCUT || d->kind == FEM_MAXKSAT || d->kind == FEM_QUBO || d->kind == FEM_PSPIN) && d->q != 2)
    return fail(FEM_ERR_INVALID_ARG, "q must be 2 for MaxCut, Max-k-SAT, QUBO and p-spin");
  if (d->linear && d->kind != FEM_QUBO && d->kind != FEM_PSPIN)
    return fail(FEM_ERR_INVALID_ARG, "linear applies to QUBO and p-spin problems only");
  if (d->term_weight && d->kind != FEM_PSPIN) return fail(FEM_ERR_INVALID_ARG, "term_weight applies to p-spin only");
  if (d->kind == FEM_PSPIN && d->n_clauses > 0 && !d->term_weight)
    return fail(FEM_ERR_INVALID_ARG, "p-spin needs term_weight");
  if (d->kind == FEM_QUBO && (d->dense_J || d->node_weight))
    return fail(FEM_ERR_INVALID_ARG, "QUBO takes a sparse graph of off-diagonal entries and optional linear terms");
  if ((d->kind == FEM_BMINCUT || d->kind == FEM_COLORING) && (d->q < 2 || d->q > 8))
    return fail(FEM_ERR_UNSUPPORTED, "bMinCut and colouring support 2 <= q <= 8");
  if (d->kind == FEM_COLORING && (d->dense_J || d->node_weight))
    return fail(FEM_ERR_INVALID_ARG, "colouring takes a sparse graph without node weights");
  // colouring runs on the bMinCut data path (same normalisers, counts and read-out)
  const int32_t kind = d->kind == FEM_COLORING ? FEM_BMINCUT
                       : d->kind == FEM_QUBO   ? FEM_MAXCUT
                       : d->kind == FEM_PSPIN  ? FEM_MAXKSAT
                                               : d->kind;
  cudaStream_t s = (cudaStream_t)stream;
  // 1. host-side validation and construction (no CUDA call yet)
  HostGraph hg;
  HostSat hs;
  fem_status st = FEM_OK;
  const int64_t dev_min = g_device_build_min_edges.load();
  bool sat_device = false;
  const bool device_build = !(d->kind == FEM_MAXCUT && d->dense_J) && kind != FEM_MAXKSAT && dev_min >= 0 &&
                            d->n_edges >= dev_min && d->n_edges > 0;
  if (d->kind == FEM_MAXCUT && d->dense_J) {
    // symmetric, zero diagonal, integers with |J_ij| <= 127 (exact in bf16 and int8):
    // checked on the device after one copy (dense_build)
  } else if (kind == FEM_MAXKSAT) {
    if ((st = sat_basics(d)) != FEM_OK) return st;
    // long clause lists are validated and built on the device (the literal count is
    // the size that decides, as the edge count does for graphs)
    sat_device = dev_min >= 0 && d->n_clauses > 0 && d->clause_ptr[d->n_clauses] >= dev_min;
    if (!sat_device && (st = host_sat(d, hs)) != FEM_OK) return st;
  } else {
    // the device builder validates the edges itself; QUBO reads them on the host first
    // (its per-node constants), so it validates them here as well
    if ((st = device_build && d->kind != FEM_QUBO ? edge_list_basics(d) : host_graph(kind, d->q, d, hg, !device_build)) !=
        FEM_OK)
      return st;
  }
  // QUBO: the gradient's per-node constant sum_j Q_ij + d_i and the linear terms
  std::vector<float> qoff;
  std::vector<double> qlin_f;
  std::vector<int64_t> qlin_i;
  bool qlin_int = true;
  if (d->kind == FEM_QUBO) {
    std::vector<double> rs(d->n, 0.0);
    for (int64_t e = 0; e < d->n_edges; ++e) {
      const double w = d->w ? d->w[e] : 1.0;
      rs[d->ei[e]] += w;
      rs[d->ej[e]] += w;
    }
    qoff.resize(d->n);
    qlin_f.resize(d->n);
    qlin_i.resize(d->n);
    for (int32_t i = 0; i < d->n; ++i) {
      const double li = d->linear ? d->linear[i] : 0.0;
      if (!std::isfinite(li)) return fail(FEM_ERR_INVALID_ARG, "linear[%d] must be finite", i);
      if (li != std::rint(li) || std::fabs(li) > 1e15) qlin_int = false;
      qlin_f[i] = li;
      qlin_i[i] = qlin_int ? (int64_t)li : 0;
      qoff[i] = (float)(rs[i] + li);
    }
  }
  // p-spin: term coefficients with the literals' negations folded in, and the fields
  std::vector<float> pj_f32;
  std::vector<double> pj_f64;
  std::vector<int64_t> pj_i64;
  bool pspin_int = true;
  if (d->kind == FEM_PSPIN) {
    const int64_t M = sat_device ? 0 : d->n_clauses;  // the device builder folds the terms
    pj_f32.resize(M);
    pj_f64.resize(M);
    pj_i64.resize(M);
    for (int64_t c = 0; c < M; ++c) {
      double J = d->term_weight[c];
      if (!std::isfinite(J)) return fail(FEM_ERR_INVALID_ARG, "term_weight[%lld] must be finite", (long long)c);
      for (int64_t k = d->clause_ptr[c]; k < d->clause_ptr[c + 1]; ++k)
        if (d->lits[k] < 0) J = -J;
      if (J != std::rint(J) || std::fabs(J) > 1099511627776.0) pspin_int = false;
      pj_f32[c] = (float)J;
      pj_f64[c] = J;
      pj_i64[c] = pspin_int ? (int64_t)J : 0;
    }
    qoff.resize(d->n);
    qlin_f.resize(d->n);
    qlin_i.resize(d->n);
    for (int32_t i = 0; i < d->n; ++i) {
      const double b = d->linear ? d->linear[i] : 0.0;
      if (!std::isfinite(b)) return fail(FEM_ERR_INVALID_ARG, "linear[%d] must be finite", i);
      if (b != std::rint(b) || std::fabs(b) > 1099511627776.0) pspin_int = false;
      qoff[i] = (float)b;
      qlin_f[i] = b;
      qlin_i[i] = pspin_int ? (int64_t)b : 0;
    }
  }
  std::vector<int32_t> nodew;
  int64_t nodew_sq = d->n;
  if (d->node_weight) {
    if (d->kind != FEM_BMINCUT || d->dense_J)
      return fail(FEM_ERR_INVALID_ARG, "node_weight applies to sparse bMinCut problems only");
    nodew.resize(d->n);
    int64_t tot = 0;
    nodew_sq = 0;
    for (int32_t i = 0; i < d->n; ++i) {
      const double v = d->node_weight[i];
      if (!(v >= 1.0 && v <= 1048576.0) || v != std::floor(v))
        return fail(FEM_ERR_INVALID_ARG, "node_weight[%d] must be an integer in [1, 2^20]", i);
      nodew[i] = (int32_t)v;
      tot += nodew[i];
      nodew_sq += (int64_t)nodew[i] * nodew[i];
    }
    if (tot >= (int64_t)INT32_MAX) return fail(FEM_ERR_INVALID_ARG, "the node weights must sum to less than 2^31");
  }
  // 2. device side
  std::unique_ptr<fem_problem> p(new fem_problem());
  p->kind = kind;
  p->coloring = d->kind == FEM_COLORING;
  p->qubo = d->kind == FEM_QUBO;
  p->qlin_int = qlin_int;
  p->pspin = d->kind == FEM_PSPIN;
  p->pspin_int = pspin_int;
  p->wtot_i = hg.wsum_i;
  p->wtot_f = hg.wsum_f;
  p->n = d->n;
  p->q = d->q;
  FEM_CUDA(cudaGetDevice(&p->device));
  FEM_CUDA(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device));
  if (d->kind == FEM_MAXCUT && d->dense_J) st = dense_upload(p.get(), d->dense_J, s);
  else if (kind == FEM_MAXKSAT && sat_device) {
    bool terms_int = true;
    st = device_sat_build(p.get(), d, p->pspin, &terms_int, s);
    p->pspin_int = p->pspin_int && terms_int;
  } else if (kind == FEM_MAXKSAT) st = upload_sat(p.get(), hs, s);  // internal kind
  else if (device_build) st = device_graph_build(p.get(), kind, d->q, d, s);  // sets the weight sums
  else st = upload_graph(p.get(), hg, s);
  p->nodew_sq = nodew_sq;
  if (st == FEM_OK && !nodew.empty()) st = upload(p.get(), &p->nodew, nodew, s);
  if (st == FEM_OK && p->qubo) st = upload(p.get(), &p->qoff, qoff, s);
  if (st == FEM_OK && p->qubo) st = upload(p.get(), &p->qlin_f, qlin_f, s);
  if (st == FEM_OK && p->qubo) st = upload(p.get(), &p->qlin_i, qlin_i, s);
  if (st == FEM_OK && p->pspin) st = upload(p.get(), &p->qoff, qoff, s);
  if (st == FEM_OK && p->pspin) st = upload(p.get(), &p->qlin_f, qlin_f, s);
  if (st == FEM_OK && p->pspin) st = upload(p.get(), &p->qlin_i, qlin_i, s);
  if (st == FEM_OK && p->pspin && !pj_f32.empty()) st = upload(p.get(), &p->pj, pj_f32, s);
  if (st == FEM_OK && p->pspin && !hs.oth.empty()) {  // 3-spin terms: the step reads J per occurrence
    std::vector<float> pjo(hs.occ.size());
    for (size_t o = 0; o < hs.occ.size(); ++o) pjo[o] = pj_f32[hs.occ[o] >> 3];
    st = upload(p.get(), &p->pjo, pjo, s);
  }
  if (st == FEM_OK && p->pspin && !pj_f64.empty()) st = upload(p.get(), &p->pj_f, pj_f64, s);
  if (st == FEM_OK && p->pspin && !pj_i64.empty()) st = upload(p.get(), &p->pj_i, pj_i64, s);
  if (st == FEM_OK) st = dev_alloc_t(p.get(), &p->err, 1);
  if (st == FEM_OK) {
    const cudaError_t e1 = cudaMemsetAsync(p->err, 0, sizeof(int32_t), s);
    const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamSynchronize(s) : e1;
    if (e2 != cudaSuccess) st = cuda_fail(e2, "fem_create_problem upload");
  }
  if (st != FEM_OK) {
    fem_destroy(p.release());
    return st;
  }
  *out = p.release();
  return FEM_OK;
}

fem_status fem_anneal(fem_problem_t p, const fem_anneal_params* a, void* stream) {
  g_last_error.clear();
  if (!p || !a) return fail(FEM_ERR_INVALID_ARG, "problem and params must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (a->n_steps < 1) return fail(FEM_ERR_INVALID_ARG, "n_steps must be >= 1");
  if (a->t_begin < 0 || a->t_end < a->t_begin || a->t_end > a->n_steps)
    return fail(FEM_ERR_INVALID_ARG, "need 0 <= t_begin <= t_end <= n_steps");
  if (!(a->beta_min > 0) || !(a->beta_max > 0) || !std::isfinite(a->beta_min) || !std::isfinite(a->beta_max))
    return fail(FEM_ERR_INVALID_ARG, "beta_min and beta_max must be finite and > 0");
  if (a->schedule != FEM_SCHED_EXPONENTIAL && a->schedule != FEM_SCHED_INVERSE_PROPORTIONAL)
    return fail(FEM_ERR_INVALID_ARG, "unknown schedule %d", a->schedule);
  if (a->optimizer < FEM_OPT_ADAM || a->optimizer > FEM_OPT_SGD)
    return fail(FEM_ERR_INVALID_ARG, "unknown optimizer %d", a->optimizer);
  if (a->grad_mode != FEM_GRAD_EXACT && a->grad_mode != FEM_GRAD_PAPER)
    return fail(FEM_ERR_INVALID_ARG, "unknown grad_mode %d", a->grad_mode);
  const int32_t R = a->replicas;
  if (R < 1) return fail(FEM_ERR_INVALID_ARG, "replicas must be >= 1");
  if (p->dense) {
    if (a->precision < FEM_PREC_FP32 || a->precision > FEM_PREC_FP8)
      return fail(FEM_ERR_INVALID_ARG, "unknown precision %d", a->precision);
    if (a->precision != FEM_PREC_FP32 && R % 128 != 0)
      return fail(FEM_ERR_UNSUPPORTED, "the tensor-core path needs replicas %% 128 == 0");
    if (a->precision == FEM_PREC_FP8 && (a->grad_mode != FEM_GRAD_PAPER || !p->dense_fp8_ok))
      return fail(FEM_ERR_UNSUPPORTED, "FP8 needs the paper-mode gradient and |J_ij| <= 16");
    if (a->t_begin > 0 && a->precision != p->precision)
      return fail(FEM_ERR_STATE, "a resumed call must keep the precision");
  } else if (p->kind == FEM_MAXCUT && R % 32 != 0) {
    return fail(FEM_ERR_UNSUPPORTED, "sparse MaxCut and QUBO need replicas %% 32 == 0");
  }
  if (p->qubo && a->grad_mode != FEM_GRAD_EXACT)
    return fail(FEM_ERR_UNSUPPORTED, "QUBO has the exact gradient only (the paper defines no discretised form)");
  if (p->kind == FEM_BMINCUT) {
    const int rpw = 32 / bmincut_bits(p->q);
    if (R % 16 != 0 || R % rpw != 0 || R > 1024)
      return fail(FEM_ERR_UNSUPPORTED, "bMinCut needs replicas %% 16 == 0, %% %d == 0 and <= 1024", rpw);
    if (!(a->lambda_max >= 0) || !std::isfinite(a->lambda_max))
      return fail(FEM_ERR_INVALID_ARG, "lambda_max must be finite and >= 0");
  }
  int cur_dev = 0;
  FEM_CUDA(cudaGetDevice(&cur_dev));
  if (cur_dev != p->device) return fail(FEM_ERR_STATE, "the current device is not the problem's device");

  // a fresh start also clears the sticky device error word of an earlier failed run
  if (a->t_begin == 0 && a->h_init) FEM_CUDA(cudaMemsetAsync(p->err, 0, sizeof(int32_t), s));
  if (a->t_begin == 0 && p->dense) {
    if (!a->h_init) return fail(FEM_ERR_INVALID_ARG, "h_init is required when t_begin == 0");
    fem_status st = FEM_OK;
    if (p->dense_R_alloc != R || p->dense_prec_alloc != a->precision) {
      if ((st = dense_state(p, R, a->precision, s)) != FEM_OK) return st;
    }
    p->R = R;
    p->cur = 0;
    p->steps_done = 0;
    p->n_steps = a->n_steps;
    p->grad_mode = a->grad_mode;
    p->optimizer = a->optimizer;
    p->precision = a->precision;
    p->lambda_max = a->lambda_max;
    const size_t per = (size_t)R * p->n_pad;
    FEM_CUDA(cudaMemsetAsync(p->h[0], 0, per * sizeof(float), s));
    FEM_CUDA(cudaMemsetAsync(p->m, 0, per * sizeof(float), s));
    FEM_CUDA(cudaMemsetAsync(p->v, 0, per * sizeof(float), s));
    if ((st = dense_set_fields(p, a->h_init, a->h_init_is_device != 0, s)) != FEM_OK) return st;
    if ((st = dense_operand(p, 0, s)) != FEM_OK) return st;
    if (!a->h_init_is_device) FEM_CUDA(cudaStreamSynchronize(s));
    p->initialised = true;
  } else if (a->t_begin == 0) {
    if (!a->h_init) return fail(FEM_ERR_INVALID_ARG, "h_init is required when t_begin == 0");
    fem_status st = ensure_state(p, R, a->grad_mode, s);
    if (st != FEM_OK) return st;
    const size_t per = (size_t)p->n * R * (p->kind == FEM_BMINCUT ? p->q : 1);
    // MaxCut fields on the device are copied by the sign-word pass below
    const bool fused_copy = p->kind == FEM_MAXCUT && a->h_init_is_device;
    if (!fused_copy)
      FEM_CUDA(cudaMemcpyAsync(p->h[0], a->h_init, per * sizeof(float),
                               a->h_init_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    FEM_CUDA(cudaMemsetAsync(p->m, 0, per * sizeof(float), s));
    FEM_CUDA(cudaMemsetAsync(p->v, 0, per * sizeof(float), s));
    p->cur = 0;
    p->steps_done = 0;
    p->n_steps = a->n_steps;
    p->grad_mode = a->grad_mode;
    p->optimizer = a->optimizer;
    p->precision = a->precision;
    p->lambda_max = a->lambda_max;
    if (p->kind == FEM_MAXCUT) {
      if ((st = maxcut_pack_words(p, 0, 0, s, fused_copy ? a->h_init : nullptr)) != FEM_OK) return st;
    } else if (p->kind == FEM_BMINCUT) {
      if ((st = bmincut_derive(p, 0, s)) != FEM_OK) return st;
    } else {
      if ((st = sat_marginals(p, 0, s)) != FEM_OK) return st;
    }
    if (!a->h_init_is_device) FEM_CUDA(cudaStreamSynchronize(s));  // h_init may be pageable
    p->initialised = true;
  } else {
    if (!p->initialised) return fail(FEM_ERR_STATE, "resume before the first anneal call");
    if (a->t_begin != p->steps_done)
      return fail(FEM_ERR_STATE, "t_begin (%d) must equal the steps already run (%d)", a->t_begin, p->steps_done);
    if (R != p->R || a->n_steps != p->n_steps || a->grad_mode != p->grad_mode || a->optimizer != p->optimizer)
      return fail(FEM_ERR_STATE, "a resumed call must keep replicas, n_steps, grad_mode and optimizer");
  }
  if (a->t_end == a->t_begin) return FEM_OK;
  // the device data every step kernel dereferences must exist (a guard against an
  // inconsistent problem, which would otherwise reach a kernel as null pointers)
  if (!p->dense && (p->kind == FEM_MAXKSAT ? (!p->occ_ptr || (p->n_clauses > 0 && (!p->cl_ptr || !p->occ)))
                                           : (!p->row_ptr || (p->nnz > 0 && !p->col))))
    return fail(FEM_ERR_STATE, "the problem's device data is incomplete");
  fem_anneal_params a_eff = *a;
  if (p->coloring) a_eff.lambda_max = 0.0;  // no balance term
  const std::vector<StepScalars> sc = make_step_scalars(a_eff, p->kind != FEM_BMINCUT);
  auto run = [&](cudaStream_t st_) -> fem_status {
    if (p->dense) return dense_steps(p, sc, a->t_begin, st_);
    if (p->kind == FEM_MAXCUT) return maxcut_sparse_steps(p, *a, sc, st_);
    if (p->kind == FEM_BMINCUT) return bmincut_sparse_steps(p, sc, a->t_begin, st_);
    if (p->kind == FEM_MAXKSAT) return sat_steps(p, sc, a->t_begin, st_);
    return fail(FEM_ERR_UNSUPPORTED, "problem kind not built in this library version");
  };
  // Small sparse problems step in a few microseconds, less than it takes the host to
  // submit a launch: windows of >= kGraphMinSteps steps then run as one CUDA graph,
  // captured once (on a private stream) and replayed for the same first step, buffer
  // parity, replica count, optimizer, mode and scalars.  The first window of a problem
  // always runs directly, so one-time setup calls never happen inside a capture.
  const long long elems = (long long)p->n * p->R * (p->kind == FEM_BMINCUT ? p->q : 1);
  const bool graph = !p->dense && p->stepped_uncaptured && elems <= kGraphMaxElems &&
                     (int64_t)sc.size() >= kGraphMinSteps;
  fem_status st = FEM_OK;
  if (!graph) {
    st = run(s);
    if (st != FEM_OK) return st;
    p->stepped_uncaptured = true;
  } else {
    Problem::StepGraph* hit = nullptr;
    for (auto& g : p->step_graphs)
      if (g.t_begin == a->t_begin && g.cur_before == p->cur && g.R == p->R && g.opt == p->optimizer &&
          g.mode == p->grad_mode && g.sc.size() == sc.size() &&
          std::memcmp(g.sc.data(), sc.data(), sc.size() * sizeof(StepScalars)) == 0)
        hit = &g;
    if (!hit) {
      if (p->step_graphs.size() >= 4) {
        cudaGraphExecDestroy(p->step_graphs.front().exec);
        p->step_graphs.erase(p->step_graphs.begin());
      }
      if (!p->capture_stream) FEM_CUDA(cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking));
      Problem::StepGraph g{a->t_begin, p->cur, 0, p->R, p->optimizer, p->grad_mode, sc, 0, nullptr};
      const int64_t l0 = fem_kernel_launches();
      FEM_CUDA(cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal));
      st = run(p->capture_stream);
      cudaGraph_t cg = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(p->capture_stream, &cg);
      g.launches = fem_kernel_launches() - l0;
      count_launches(-g.launches);  // captured, not run
      if (st != FEM_OK) {
        if (cg) cudaGraphDestroy(cg);
        return st;
      }
      if (ec != cudaSuccess) return cuda_fail(ec, "step graph capture");
      const cudaError_t ei = cudaGraphInstantiate(&g.exec, cg, 0);
      cudaGraphDestroy(cg);
      if (ei != cudaSuccess) return cuda_fail(ei, "step graph instantiate");
      g.cur_after = p->cur;
      p->step_graphs.push_back(std::move(g));
      hit = &p->step_graphs.back();
    }
    FEM_CUDA(cudaGraphLaunch(hit->exec, s));
    count_launches(hit->launches);
    p->cur = hit->cur_after;
  }
  p->steps_done = a->t_end;
  return FEM_OK;
}

fem_status fem_read_best(fem_problem_t p, int32_t* best_replica, int32_t* states,
                         int64_t* energy_i64, double* energy_f64, void* stream) {
  g_last_error.clear();
  if (!p) return fail(FEM_ERR_INVALID_ARG, "problem must be non-NULL");
  if (!p->initialised) return fail(FEM_ERR_STATE, "read-out before the first anneal call");
  cudaStream_t s = (cudaStream_t)stream;
  fem_status st = FEM_OK;
  if (p->dense) st = dense_readout(p, s);
  else if (p->kind == FEM_MAXCUT) st = maxcut_readout(p, s);
  else if (p->kind == FEM_BMINCUT) st = bmincut_readout(p, s);
  else if (p->kind == FEM_MAXKSAT) st = sat_readout(p, s);
  else st = fail(FEM_ERR_UNSUPPORTED, "problem kind not built");
  if (st != FEM_OK) return st;
  if (best_replica) FEM_CUDA(cudaMemcpyAsync(best_replica, p->best, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (states) FEM_CUDA(cudaMemcpyAsync(states, p->states_dev, (size_t)p->n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (energy_i64) FEM_CUDA(cudaMemcpyAsync(energy_i64, p->energy_i, (size_t)p->R * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (energy_f64) FEM_CUDA(cudaMemcpyAsync(energy_f64, p->energy_f, (size_t)p->R * sizeof(double), cudaMemcpyDeviceToHost, s));
  return check_sticky(p, s);
}

fem_status fem_schedule_value(const fem_anneal_params* a, int32_t t, double* beta, double* lambda) {
  g_last_error.clear();
  if (!a) return fail(FEM_ERR_INVALID_ARG, "params must be non-NULL");
  if (a->n_steps < 1 || t < 0 || t >= a->n_steps) return fail(FEM_ERR_INVALID_ARG, "need 0 <= t < n_steps");
  if (!(a->beta_min > 0) || !(a->beta_max > 0) || !std::isfinite(a->beta_min) || !std::isfinite(a->beta_max))
    return fail(FEM_ERR_INVALID_ARG, "beta_min and beta_max must be finite and > 0");
  if (a->schedule != FEM_SCHED_EXPONENTIAL && a->schedule != FEM_SCHED_INVERSE_PROPORTIONAL)
    return fail(FEM_ERR_INVALID_ARG, "unknown schedule %d", a->schedule);
  if (beta) *beta = beta_at(*a, t);
  if (lambda) *lambda = lambda_at(*a, t);
  return FEM_OK;
}

fem_status fem_set_step_barrier_timeout(fem_problem_t p, int64_t ns) {
  if (!p || ns < 0) return fail(FEM_ERR_INVALID_ARG, "fem_set_step_barrier_timeout: problem and ns >= 0 required");
  p->barrier_wait_ns = ns;
  return FEM_OK;
}

fem_status fem_inject_step_stall(fem_problem_t p, int32_t row_tile) {
  if (!p || row_tile < -1) return fail(FEM_ERR_INVALID_ARG, "fem_inject_step_stall: problem and row_tile >= -1 required");
  p->stall_tile = row_tile;
  return FEM_OK;
}

void fem_set_device_graph_build(int64_t min_edges) { g_device_build_min_edges.store(min_edges); }

void fem_set_tma_gather(int32_t on) { fem::g_tma_gather.store(on ? 1 : 0); }

void fem_inject_allocation_failure(int64_t after) { g_fail_alloc_after.store(after < 0 ? -1 : after); }

fem_status fem_set_dense_launch(fem_problem_t p, int32_t mode) {
  if (!p || !p->dense) return fail(FEM_ERR_INVALID_ARG, "fem_set_dense_launch: not a dense problem");
  if (mode < FEM_DENSE_AUTO || mode > FEM_DENSE_PERSISTENT_SINGLE)
    return fail(FEM_ERR_INVALID_ARG, "fem_set_dense_launch: mode %d", (int)mode);
  p->dense_launch = mode;
  return FEM_OK;
}

fem_status fem_read_fields(fem_problem_t p, float* h_host, void* stream) {
  g_last_error.clear();
  if (!p || !h_host) return fail(FEM_ERR_INVALID_ARG, "problem and h_host must be non-NULL");
  if (!p->initialised) return fail(FEM_ERR_STATE, "no fields before the first anneal call");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t per = (size_t)p->n * p->R * (p->kind == FEM_BMINCUT ? p->q : 1);
  if (p->dense) {
    const fem_status st = dense_get(p, p->h[0], h_host, s);
    if (st != FEM_OK) return st;
    return check_sticky(p, s);
  }
  const float* src = current_fields(p);
  FEM_CUDA(cudaMemcpyAsync(h_host, src, per * sizeof(float), cudaMemcpyDefault, s));  // host or device
  return check_sticky(p, s);
}

fem_status fem_read_states(fem_problem_t p, int32_t* states_host, void* stream) {
  g_last_error.clear();
  if (!p || !states_host) return fail(FEM_ERR_INVALID_ARG, "problem and states_host must be non-NULL");
  if (!p->initialised) return fail(FEM_ERR_STATE, "no states before the first anneal call");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* tmp = nullptr;
  const size_t total = (size_t)p->n * p->R;
  FEM_CUDA(cudaMallocAsync((void**)&tmp, total * sizeof(int32_t), s));
  fem_status st = FEM_OK;
  if (p->dense) st = dense_states_all(p, tmp, s);
  else if (p->kind == FEM_MAXCUT) st = maxcut_states_all(p, tmp, s);
  else if (p->kind == FEM_BMINCUT) st = bmincut_states_all(p, tmp, s);
  else if (p->kind == FEM_MAXKSAT) st = sat_states_all(p, tmp, s);
  else st = fail(FEM_ERR_UNSUPPORTED, "problem kind not built");
  if (st == FEM_OK) {
    const cudaError_t e = cudaMemcpyAsync(states_host, tmp, total * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_fail(e, "fem_read_states copy");
  }
  cudaFreeAsync(tmp, s);
  if (st != FEM_OK) return st;
  return check_sticky(p, s);
}

fem_status fem_read_state(fem_problem_t p, float* h, float* m, float* v, void* stream) {
  g_last_error.clear();
  if (!p) return fail(FEM_ERR_INVALID_ARG, "problem must be non-NULL");
  if (!p->initialised) return fail(FEM_ERR_STATE, "no state before the first anneal call");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)p->n * p->R * (p->kind == FEM_BMINCUT ? p->q : 1) * sizeof(float);
  if (p->dense) {
    fem_status st = FEM_OK;
    if (h && (st = dense_get(p, p->h[0], h, s)) != FEM_OK) return st;
    if (m && (st = dense_get(p, p->m, m, s)) != FEM_OK) return st;
    if (v && (st = dense_get(p, p->v, v, s)) != FEM_OK) return st;
    return check_sticky(p, s);
  }
  const float* src = current_fields(p);
  if (h) FEM_CUDA(cudaMemcpyAsync(h, src, bytes, cudaMemcpyDeviceToHost, s));
  if (m) FEM_CUDA(cudaMemcpyAsync(m, p->m, bytes, cudaMemcpyDeviceToHost, s));
  if (v) FEM_CUDA(cudaMemcpyAsync(v, p->v, bytes, cudaMemcpyDeviceToHost, s));
  return check_sticky(p, s);
}

fem_status fem_write_state(fem_problem_t p, const float* h, const float* m, const float* v,
                           int32_t steps_done, void* stream) {
  g_last_error.clear();
  if (!p || !h) return fail(FEM_ERR_INVALID_ARG, "problem and h must be non-NULL");
  if (!p->initialised) return fail(FEM_ERR_STATE, "fem_write_state needs an initialised problem");
  if (steps_done < 0 || steps_done > p->n_steps)
    return fail(FEM_ERR_INVALID_ARG, "steps_done must be in [0, n_steps]");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)p->n * p->R * (p->kind == FEM_BMINCUT ? p->q : 1) * sizeof(float);
  const int t = steps_done;
  if (p->dense) {
    const size_t per = (size_t)p->R * p->n_pad * sizeof(float);
    FEM_CUDA(cudaMemsetAsync(p->m, 0, per, s));
    FEM_CUDA(cudaMemsetAsync(p->v, 0, per, s));
    fem_status st = dense_put(p, p->h[0], h, s);
    if (st == FEM_OK && m) st = dense_put(p, p->m, m, s);
    if (st == FEM_OK && v) st = dense_put(p, p->v, v, s);
    if (st == FEM_OK) st = dense_operand(p, t, s);
    if (st != FEM_OK) return st;
    FEM_CUDA(cudaStreamSynchronize(s));
    p->steps_done = steps_done;
    return check_sticky(p, s);
  }
  float* dst = fields_for_step(p, t);
  FEM_CUDA(cudaMemcpyAsync(dst, h, bytes, cudaMemcpyHostToDevice, s));
  if (m) FEM_CUDA(cudaMemcpyAsync(p->m, m, bytes, cudaMemcpyHostToDevice, s));
  else FEM_CUDA(cudaMemsetAsync(p->m, 0, bytes, s));
  if (v) FEM_CUDA(cudaMemcpyAsync(p->v, v, bytes, cudaMemcpyHostToDevice, s));
  else FEM_CUDA(cudaMemsetAsync(p->v, 0, bytes, s));
  fem_status st = FEM_OK;
  if (p->kind == FEM_MAXCUT) {
    p->cur = t & 1;
    st = maxcut_pack_words(p, p->grad_mode == FEM_GRAD_PAPER ? 0 : (t & 1), t & 1, s);
  } else if (p->kind == FEM_BMINCUT) {
    st = bmincut_derive(p, t, s);
  } else {
    st = sat_marginals(p, t, s);
  }
  if (st != FEM_OK) return st;
  FEM_CUDA(cudaStreamSynchronize(s));
  p->steps_done = steps_done;
  return check_sticky(p, s);
}

fem_status fem_problem_info(fem_problem_t p, int32_t* steps_done, int32_t* n, int32_t* q,
                            int32_t* replicas, int64_t* units_per_replica) {
  if (!p) return fail(FEM_ERR_INVALID_ARG, "problem must be non-NULL");
  if (steps_done) *steps_done = p->steps_done;
  if (n) *n = p->n;
  if (q) *q = p->q;
  if (replicas) *replicas = p->R;
  if (units_per_replica) {
    if (p->dense) *units_per_replica = (int64_t)p->n * (p->n - 1) / 2;
    else if (p->kind == FEM_MAXKSAT) *units_per_replica = p->n_occ;
    else *units_per_replica = p->n_edges;
  }
  return FEM_OK;
}

fem_status fem_dense_last_launch(fem_problem_t p, int32_t* mode) {
  if (!p || !mode) return fail(FEM_ERR_INVALID_ARG, "problem and mode must be non-NULL");
  *mode = p->dense ? p->dense_last_launch : 0;
  return FEM_OK;
}

fem_status fem_sync(fem_problem_t p, void* stream) {
  g_last_error.clear();
  if (!p) return fail(FEM_ERR_INVALID_ARG, "problem must be non-NULL");
  return check_sticky(p, (cudaStream_t)stream);
}

}  // extern "C"
