// Batched anneal: many bMinCut and Max-k-SAT problems advanced together, two
// persistent launches per step over a work list (one for the q-state members, one
// for the clause-shaped members, so that each kernel gets the registers of its own
// element code), the step loop captured in a CUDA graph, and the work-item size
// chosen by timing (a small autotuner).
//
// Every member keeps its own state buffers; the batch only adds a device table of
// per-member descriptors and a list of work items (member, element range), the
// q-state members' items first.  A block takes items in a grid-stride loop; a
// bMinCut item accumulates its group counts in shared memory and adds them to its
// member's counts once, so the per-member results are bit-identical to running
// the members one by one (integer counts and fixed-point sums do not depend on the
// order of the additions).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "bmincut_core.cuh"
#include "fem_internal.h"
#include "sat_core.cuh"

namespace fem {

struct BatchMember {
  int32_t kind, n, R, q, wpn, mode, opt;
  const int32_t* row_ptr;
  const uint32_t* col;
  const float* w;
  const float* cf;
  const float* ca;
  const int32_t* nodew;
  float cw, lam_scale;  // see BmcArgs
  float* h0;
  float* h1;
  float* m;
  float* v;
  float* dq[2];  // exact mode: the centred marginals the neighbour terms gather
  uint32_t* words[2];
  int32_t* cnt[3];
  unsigned long long* psum[3];
  float* satP[2];
  const int32_t* cl_ptr;
  const int32_t* cl_lit;
  const int32_t* occ_ptr;
  const int32_t* occ;
  const int2* oth;
  const float* jw;   // p-spin members: term coefficients, NULL for Max-k-SAT
  const float* jwo;  // p-spin members with 3-spin terms: J per occurrence
  const float* lin;  // p-spin members: fields b_i
};

struct BatchItem {
  int32_t member;
  int32_t first;     // the member's first item zeroes its count buffer for step t+2
  long long e0, e1;  // element range [e0, e1), e = node * R + replica; e0 % 32 == 0
};

namespace {

// The element code reads its arguments from a block-shared copy, written by thread 0
// per item: values the compiler would otherwise hold in registers for the whole item
// (and spill) are re-read from shared memory where they are used.
template <int Q, int MODE, int RC = 0>
__device__ void run_bmincut_item(const BatchMember& b, const BatchItem& it, const StepScalars& s, int t,
                                 int32_t* scnt, unsigned long long* sps, BmcArgs& a) {
  if (threadIdx.x == 0) {
    a = BmcArgs{};
    a.row_ptr = b.row_ptr;
    a.col = b.col;
    a.w = b.w;
    a.cf = b.cf;
    a.ca = b.ca;
    a.nodew = b.nodew;
    a.cw = b.cw;
    a.lam_scale = b.lam_scale;
    a.n = b.n;
    a.R = b.R;
    a.wpn = b.wpn;
    a.opt = b.opt;
    a.h_in = MODE == FEM_GRAD_PAPER ? b.h0 : ((t & 1) ? b.h1 : b.h0);
    a.h_out = MODE == FEM_GRAD_PAPER ? b.h0 : ((t & 1) ? b.h0 : b.h1);
    a.d_in = MODE == FEM_GRAD_PAPER ? nullptr : b.dq[t & 1];
    a.d_out = MODE == FEM_GRAD_PAPER ? nullptr : b.dq[(t + 1) & 1];
    a.m = b.m;
    a.v = b.v;
    a.words_in = b.words[t & 1];
    a.words_out = b.words[(t + 1) & 1];
    a.cnt_in = b.cnt[t % 3];
    a.cnt_out = b.cnt[(t + 1) % 3];
    a.cnt_zero = b.cnt[(t + 2) % 3];
    a.ps_in = b.psum[t % 3];
    a.ps_out = b.psum[(t + 1) % 3];
    a.ps_zero = b.psum[(t + 2) % 3];
  }
  __syncthreads();
  const int RQ = (RC ? RC : a.R) * Q;
  for (int x = threadIdx.x; x < RQ; x += blockDim.x) {
    scnt[x] = 0;
    if (MODE == FEM_GRAD_EXACT) sps[x] = 0ull;
    if (it.first) {
      a.cnt_zero[x] = 0;
      if (MODE == FEM_GRAD_EXACT) a.ps_zero[x] = 0ull;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (long long base = it.e0 + (threadIdx.x & ~31); base < it.e1; base += blockDim.x) {
    const long long e = base + lane;
    bmincut_element<Q, MODE, RC>(a, s, e, e < it.e1, lane, scnt, sps);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < RQ; x += blockDim.x) {
    if (scnt[x]) atomicAdd(&a.cnt_out[x], scnt[x]);
    if (MODE == FEM_GRAD_EXACT && sps[x]) atomicAdd(&a.ps_out[x], sps[x]);
  }
  __syncthreads();
}

template <int RC = 0>
__device__ void run_sat_item(const BatchMember& b, const BatchItem& it, const StepScalars& s, int t, SatArgs& a) {
  if (threadIdx.x == 0) {
    a = SatArgs{};
    a.cl_ptr = b.cl_ptr;
    a.cl_lit = b.cl_lit;
    a.occ_ptr = b.occ_ptr;
    a.occ = b.occ;
    a.oth = b.oth;
    a.jw = b.jw;
    a.jwo = b.jwo;
    a.lin = b.lin;
    a.n = b.n;
    a.R = b.R;
    a.opt = b.opt;
    a.h = b.h0;
    a.m = b.m;
    a.v = b.v;
    a.P_in = b.satP[t & 1];
    a.P_out = b.satP[(t + 1) & 1];
  }
  __syncthreads();
  // four replicas per thread (e0 and e1 are multiples of R), two occurrences at a time;
  // p-spin members take the per-element path, which gives the same bits, since the
  // four-replica p-spin code would spill in this kernel
  if (sat_k3_shape(a) && !a.jw) {
    for (long long e = it.e0 + threadIdx.x * 4; e < it.e1; e += blockDim.x * 4) sat_element_k3<2, false, RC>(a, s, e);
  } else {
    for (long long e = it.e0 + threadIdx.x; e < it.e1; e += blockDim.x) sat_element(a, s, e);
  }
  __syncthreads();  // the next item's arguments overwrite a
}

// The q-state members' step: blocks walk their items (the first n_items of the list).
// Q and MODE are shared by all of them; s carries the q-state gradient scale (gamma).  RC: the
// members' replica count as a compile-time constant (0: run time).  Resident blocks per SM:
// five for paper mode with q <= 4 at R = 16 (measured faster than four), three for q >= 7,
// else four.
template <int Q, int MODE, int RC = 0>
__global__ void __launch_bounds__(256, Q >= 7 ? 3 : ((Q <= 4 && MODE == FEM_GRAD_PAPER && RC == 16) ? 5 : 4))
    k_batch_bmincut(const BatchMember* __restrict__ members, const BatchItem* __restrict__ items, int32_t n_items,
                    int32_t max_rq, StepScalars s, int32_t t) {
  extern __shared__ unsigned long long smem_b[];
  unsigned long long* sps = smem_b;
  int32_t* scnt = reinterpret_cast<int32_t*>(smem_b + (MODE == FEM_GRAD_EXACT ? max_rq : 0));
  __shared__ BmcArgs args;
  for (int k = blockIdx.x; k < n_items; k += gridDim.x) {
    const BatchItem it = items[k];
    run_bmincut_item<Q, MODE, RC>(members[it.member], it, s, t, scnt, sps, args);
  }
}

// The clause-shaped members' step (Max-k-SAT and p-spin); s carries the single-field
// gradient scale (gamma/4).  RC: the members' replica count at compile time (0: run time).
template <int RC = 0>
__global__ void __launch_bounds__(256, 4) k_batch_sat(const BatchMember* __restrict__ members,
                                                   const BatchItem* __restrict__ items, int32_t n_items,
                                                   StepScalars s, int32_t t) {
  __shared__ SatArgs args;
  for (int k = blockIdx.x; k < n_items; k += gridDim.x) {
    const BatchItem it = items[k];
    run_sat_item<RC>(members[it.member], it, s, t, args);
  }
}

using BatchKernel = void (*)(const BatchMember*, const BatchItem*, int32_t, int32_t, StepScalars, int32_t);

// r16: every member has R = 16 (one or two packed words per node from q = 3 on)
template <int MODE>
BatchKernel pick_q(int q, bool r16) {
  switch (q) {
    case 2: return k_batch_bmincut<2, MODE>;
    case 3: return r16 ? k_batch_bmincut<3, MODE, 16> : k_batch_bmincut<3, MODE>;
    case 4: return r16 ? k_batch_bmincut<4, MODE, 16> : k_batch_bmincut<4, MODE>;
    case 5: return r16 ? k_batch_bmincut<5, MODE, 16> : k_batch_bmincut<5, MODE>;
    case 6: return r16 ? k_batch_bmincut<6, MODE, 16> : k_batch_bmincut<6, MODE>;
    case 7: return r16 ? k_batch_bmincut<7, MODE, 16> : k_batch_bmincut<7, MODE>;
    default: return r16 ? k_batch_bmincut<8, MODE, 16> : k_batch_bmincut<8, MODE>;
  }
}

// Process-wide tuning cache: (bMinCut elements, SAT elements, R, q, mode) -> nodes per item.
std::mutex g_tune_mutex;
std::map<std::tuple<long long, long long, int, int, int>, int> g_tune_cache;

}  // namespace

struct Batch {
  std::vector<Problem*> members;
  int device = 0, sm_count = 148;
  int R = 0, q = 4, mode = FEM_GRAD_PAPER, opt = FEM_OPT_ADAM;
  long long elems_bmc = 0, elems_sat = 0;
  BatchMember* d_members = nullptr;
  BatchItem* d_items = nullptr;  // the q-state members' items, then the clause-shaped ones
  int n_bmc = 0, n_sat = 0, nodes_per_item = 0, max_rq = 0;
  bool ready = false;
  std::vector<uint64_t> sig;     // members' allocation generations the descriptors were built from
  cudaStream_t capture_stream = nullptr;
  // captured step loops, keyed by (first step, item size, the steps' scalars)
  struct Graph {
    int t0, npi;
    std::vector<StepScalars> sq, s1;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  std::vector<void*> allocs;
};

static void batch_drop_graphs(Batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

static fem_status batch_free_plan(Batch* b) {
  batch_drop_graphs(b);
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
  b->d_members = nullptr;
  b->d_items = nullptr;
  b->n_bmc = b->n_sat = 0;
  b->nodes_per_item = 0;
  b->ready = false;
  return FEM_OK;
}

// Work items: every member's nodes in runs of `npi` nodes (npi even, so that
// e0 = node0 * R is a multiple of 32 for R % 16 == 0), the q-state members' items
// first.
static fem_status batch_build_items(Batch* b, int npi, std::vector<BatchItem>& items) {
  items.clear();
  b->n_bmc = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (size_t k = 0; k < b->members.size(); ++k) {
      const Problem* p = b->members[k];
      if ((p->kind == FEM_BMINCUT) != (pass == 0)) continue;
      bool first = true;
      for (long long i0 = 0; i0 < p->n; i0 += npi) {
        const long long i1 = std::min<long long>(p->n, i0 + npi);
        items.push_back(BatchItem{(int32_t)k, first ? 1 : 0, i0 * p->R, i1 * p->R});
        first = false;
      }
    }
    if (pass == 0) b->n_bmc = (int)items.size();
  }
  b->n_sat = (int)items.size() - b->n_bmc;
  return FEM_OK;
}

static fem_status batch_upload_items(Batch* b, int npi, cudaStream_t s) {
  std::vector<BatchItem> items;
  batch_build_items(b, npi, items);
  if (b->d_items) {
    cudaFree(b->d_items);
    b->allocs.erase(std::remove(b->allocs.begin(), b->allocs.end(), (void*)b->d_items), b->allocs.end());
  }
  void* p = nullptr;
  FEM_CUDA(cudaMalloc(&p, items.size() * sizeof(BatchItem)));
  b->allocs.push_back(p);
  b->d_items = (BatchItem*)p;
  FEM_CUDA(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, s));
  FEM_CUDA(cudaStreamSynchronize(s));
  b->nodes_per_item = npi;
  return FEM_OK;
}

static fem_status batch_prepare(Batch* b, cudaStream_t s) {
  batch_free_plan(b);
  std::vector<BatchMember> dm;
  b->elems_bmc = b->elems_sat = 0;
  b->max_rq = 1;
  for (Problem* p : b->members) {
    BatchMember m{};
    m.kind = p->kind;
    m.n = p->n;
    m.R = p->R;
    m.q = p->q;
    m.wpn = p->words_per_node;
    m.mode = p->grad_mode;
    m.opt = p->optimizer;
    m.row_ptr = p->row_ptr;
    m.col = p->col;
    m.w = p->unit_w ? nullptr : p->w;
    m.cf = p->cnorm;
    m.ca = p->cnorm2;
    m.nodew = p->nodew;
    m.cw = p->coloring ? 1.f : (p->grad_mode == FEM_GRAD_EXACT ? -2.f : -1.f);
    m.lam_scale = p->coloring ? 0.f : 1.f;
    m.h0 = p->h[0];
    m.h1 = p->h[1];
    m.m = p->m;
    m.v = p->v;
    for (int k = 0; k < 2; ++k) {
      m.words[k] = p->words[k];
      m.satP[k] = p->satP[k];
      m.dq[k] = p->kind == FEM_BMINCUT ? p->mag[k] : nullptr;
    }
    for (int k = 0; k < 3; ++k) {
      m.cnt[k] = p->cnt[k];
      m.psum[k] = p->psum[k];
    }
    m.cl_ptr = p->cl_ptr;
    m.cl_lit = p->cl_lit;
    m.occ_ptr = p->occ_ptr;
    m.occ = p->occ;
    m.oth = reinterpret_cast<const int2*>(p->oth);
    m.jw = p->pspin ? p->pj : nullptr;
    m.jwo = p->pspin ? p->pjo : nullptr;
    m.lin = p->pspin ? p->qoff : nullptr;
    dm.push_back(m);
    if (p->kind == FEM_BMINCUT) {
      if (p->grad_mode == FEM_GRAD_EXACT && (!p->mag[0] || !p->mag[1]))
        return fail(FEM_ERR_STATE, "exact-mode buffers of a member are not allocated");
      b->elems_bmc += (long long)p->n * p->R;
      b->max_rq = std::max(b->max_rq, p->R * p->q);
    } else {
      b->elems_sat += (long long)p->n * p->R;
    }
  }
  void* p = nullptr;
  FEM_CUDA(cudaMalloc(&p, dm.size() * sizeof(BatchMember)));
  b->allocs.push_back(p);
  b->d_members = (BatchMember*)p;
  FEM_CUDA(cudaMemcpyAsync(b->d_members, dm.data(), dm.size() * sizeof(BatchMember), cudaMemcpyHostToDevice, s));
  b->ready = true;
  return FEM_OK;
}

static size_t batch_smem(const Batch* b) {
  return (size_t)b->max_rq * (b->mode == FEM_GRAD_EXACT ? 12 : 4);
}

// Resident blocks of a grid-stride launch over n items (at least one block).
template <typename K>
static int batch_grid(const Batch* b, K k, size_t smem, int n) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return std::max(1, std::min(n, per_sm * b->sm_count));
}

// One step: the q-state members' launch, then the clause-shaped members' launch.
// Returns the number of launches.
static int batch_launch(Batch* b, BatchKernel k, const StepScalars& sq, const StepScalars& s1, int t,
                        cudaStream_t s) {
  int n = 0;
  if (b->n_bmc > 0) {
    k<<<batch_grid(b, k, batch_smem(b), b->n_bmc), 256, batch_smem(b), s>>>(b->d_members, b->d_items, b->n_bmc,
                                                                              b->max_rq, sq, t);
    ++n;
  }
  if (b->n_sat > 0) {
    const auto ks = b->R == 16 ? k_batch_sat<16> : k_batch_sat<0>;
    ks<<<batch_grid(b, ks, 0, b->n_sat), 256, 0, s>>>(b->d_members, b->d_items + b->n_bmc, b->n_sat, s1, t);
    ++n;
  }
  return n;
}

}  // namespace fem

struct fem_batch : public fem::Batch {};

using namespace fem;

extern "C" {

fem_status fem_batch_create(fem_problem_t const* probs, int32_t count, fem_batch_t* out) {
  if (!probs || !out || count < 1) return fail(FEM_ERR_INVALID_ARG, "probs, out and count >= 1 are required");
  *out = nullptr;
  int q = -1;
  for (int32_t k = 0; k < count; ++k) {
    const Problem* p = probs[k];
    if (!p) return fail(FEM_ERR_INVALID_ARG, "member %d is NULL", k);
    if (p->dense || (p->kind != FEM_BMINCUT && p->kind != FEM_MAXKSAT))
      return fail(FEM_ERR_UNSUPPORTED, "batches hold sparse bMinCut and Max-k-SAT problems");
    if (p->kind == FEM_BMINCUT) {
      if (q >= 0 && p->q != q) return fail(FEM_ERR_UNSUPPORTED, "bMinCut members of a batch must share q");
      q = p->q;
    }
    if (k > 0 && p->device != probs[0]->device) return fail(FEM_ERR_INVALID_ARG, "members on different devices");
  }
  fem_batch* b = new fem_batch();
  b->members.assign(probs, probs + count);
  b->device = probs[0]->device;
  b->sm_count = probs[0]->sm_count;
  b->q = q < 0 ? 2 : q;
  *out = b;
  return FEM_OK;
}

void fem_batch_destroy(fem_batch_t b) {
  if (!b) return;
  batch_free_plan(b);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
}

fem_status fem_batch_anneal(fem_batch_t b, const fem_anneal_params* a, const float* const* h_init, void* stream) {
  if (!b || !a) return fail(FEM_ERR_INVALID_ARG, "batch and params must be non-NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (a->replicas % 16 != 0) return fail(FEM_ERR_UNSUPPORTED, "batched members need replicas %% 16 == 0");
  // initialise (or check the resume state of) every member with the single-problem path
  for (size_t k = 0; k < b->members.size(); ++k) {
    fem_anneal_params pk = *a;
    pk.t_end = a->t_begin;
    if (a->t_begin == 0) {
      if (!h_init || !h_init[k]) return fail(FEM_ERR_INVALID_ARG, "h_init[%zu] is required", k);
      pk.h_init = h_init[k];
    }
    const fem_status st = fem_anneal(static_cast<fem_problem_t>(b->members[k]), &pk, stream);
    if (st != FEM_OK) return st;
  }
  if (a->t_end == a->t_begin) return FEM_OK;
  const int R = a->replicas;
  // the descriptors hold member device pointers: rebuild them when any member has
  // allocated since (a fresh start or a new replica count or mode reallocates buffers,
  // and a new buffer may reuse a freed address, so pointers alone cannot tell)
  std::vector<uint64_t> sig;
  for (const Problem* p : b->members) sig.push_back(p->alloc_gen);
  const bool changed = !b->ready || b->R != R || b->mode != a->grad_mode || b->opt != a->optimizer || sig != b->sig;
  if (changed) {
    b->sig = sig;
    b->R = R;
    b->mode = a->grad_mode;
    b->opt = a->optimizer;
    fem_status st = batch_prepare(b, s);
    if (st != FEM_OK) return st;
  }
  const BatchKernel k = b->mode == FEM_GRAD_EXACT ? pick_q<FEM_GRAD_EXACT>(b->q, R == 16)
                                                 : pick_q<FEM_GRAD_PAPER>(b->q, R == 16);
  if (batch_smem(b) > 48 * 1024)
    FEM_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem(b)));
  const std::vector<StepScalars> sc = make_step_scalars(*a, 0);      // q-state scale
  const std::vector<StepScalars> sc1 = make_step_scalars(*a, 1);     // single-field scale
  int t = a->t_begin;
  size_t done = 0;
  // ---- autotune the item size on the first steps (the result is bit-identical for
  // every candidate; only the timing differs)
  const auto key = std::make_tuple(b->elems_bmc, b->elems_sat, R, b->q, b->mode);
  int npi = 0;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto f = g_tune_cache.find(key);
    if (f != g_tune_cache.end()) npi = f->second;
  }
  if (npi == 0) {
    const int cands[3] = {64, 256, 1024};
    float best_ms = 1e30f;
    int64_t launches = 0;
    cudaEvent_t e0, e1;
    FEM_CUDA(cudaEventCreate(&e0));
    FEM_CUDA(cudaEventCreate(&e1));
    for (int c : cands) {
      if (done + 2 > sc.size()) break;
      fem_status st = batch_upload_items(b, c, s);
      if (st != FEM_OK) return st;
      launches += batch_launch(b, k, sc[done], sc1[done], t, s);  // a warm step, not timed
      ++t;
      ++done;
      FEM_CUDA(cudaEventRecord(e0, s));
      launches += batch_launch(b, k, sc[done], sc1[done], t, s);
      FEM_CUDA(cudaEventRecord(e1, s));
      FEM_CUDA(cudaEventSynchronize(e1));
      ++t;
      ++done;
      float ms = 0.f;
      FEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        npi = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (npi == 0) npi = 256;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = npi;
    count_launches(launches);
  }
  if (b->nodes_per_item != npi) {
    fem_status st = batch_upload_items(b, npi, s);
    if (st != FEM_OK) return st;
    batch_drop_graphs(b);
  }
  // ---- the remaining steps as one CUDA graph (captured on a private stream, replayed
  // on the caller's stream; cached for the same first step, item size and scalars)
  if (done < sc.size()) {
    const int t0 = t;
    const std::vector<StepScalars> sq(sc.begin() + done, sc.end()), s1(sc1.begin() + done, sc1.end());
    auto same = [](const std::vector<StepScalars>& x, const std::vector<StepScalars>& y) {
      return x.size() == y.size() && std::memcmp(x.data(), y.data(), x.size() * sizeof(StepScalars)) == 0;
    };
    Batch::Graph* hit = nullptr;
    for (auto& g : b->graphs)
      if (g.t0 == t0 && g.npi == npi && same(g.sq, sq) && same(g.s1, s1)) hit = &g;
    if (!hit) {
      if (b->graphs.size() >= 4) {
        cudaGraphExecDestroy(b->graphs.front().exec);
        b->graphs.erase(b->graphs.begin());
      }
      if (!b->capture_stream) FEM_CUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
      FEM_CUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
      for (size_t j = 0; j < sq.size(); ++j) batch_launch(b, k, sq[j], s1[j], t0 + (int)j, b->capture_stream);
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(b->capture_stream, &g);
      if (ec != cudaSuccess) return cuda_fail(ec, "batch graph capture");
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) return cuda_fail(ei, "batch graph instantiate");
      b->graphs.push_back(Batch::Graph{t0, npi, sq, s1, exec});
      hit = &b->graphs.back();
    }
    FEM_CUDA(cudaGraphLaunch(hit->exec, s));
    count_launches((int64_t)sq.size() * ((b->n_bmc > 0) + (b->n_sat > 0)));
  }
  FEM_CUDA(cudaGetLastError());
  for (Problem* p : b->members) p->steps_done = a->t_end;
  return FEM_OK;
}

fem_status fem_anneal_batch(fem_problem_t const* probs, int32_t count, const fem_anneal_params* prm,
                            const float* const* h_init, void* stream) {
  fem_batch_t b = nullptr;
  fem_status st = fem_batch_create(probs, count, &b);
  if (st != FEM_OK) return st;
  st = fem_batch_anneal(b, prm, h_init, stream);
  // the work list and the graph must outlive the work queued on the stream
  const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (st == FEM_OK && e != cudaSuccess) st = cuda_fail(e, "fem_anneal_batch");
  fem_batch_destroy(b);
  return st;
}

}  // extern "C"
