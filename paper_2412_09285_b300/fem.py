"""Thin ctypes binding of libfem's C ABI (``include/fem.h``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  The functions keep the C names (``fem_create_problem``, ``fem_anneal``,
``fem_read_best`` ...); ``Problem`` is a small convenience wrapper over them that
takes numpy arrays or torch tensors.  Importing this module loads the in-tree
``libfem.so``; if it is missing, the import fails loudly - there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfem.so")

FEM_OK, FEM_ERR_INVALID_ARG, FEM_ERR_UNSUPPORTED, FEM_ERR_OOM = 0, 1, 2, 3
FEM_ERR_CUDA, FEM_ERR_TIMEOUT, FEM_ERR_STATE, FEM_ERR_DEVICE = 4, 5, 6, 7
FEM_MAXCUT, FEM_BMINCUT, FEM_MAXKSAT = 0, 1, 2
FEM_SCHED_EXPONENTIAL, FEM_SCHED_INVERSE_PROPORTIONAL = 0, 1
FEM_OPT_ADAM, FEM_OPT_RMSPROP, FEM_OPT_SGD = 0, 1, 2
FEM_GRAD_EXACT, FEM_GRAD_PAPER = 0, 1
FEM_PREC_FP32, FEM_PREC_BF16, FEM_PREC_BF16X2, FEM_PREC_FP8 = 0, 1, 2, 3

FEM_COLORING, FEM_QUBO, FEM_PSPIN = 3, 4, 5
KINDS = {"maxcut": FEM_MAXCUT, "bmincut": FEM_BMINCUT, "sat": FEM_MAXKSAT, "coloring": FEM_COLORING,
         "qubo": FEM_QUBO, "pspin": FEM_PSPIN}
Q_STATE_KINDS = ("bmincut", "coloring")
SCHEDULES = {"exponential": FEM_SCHED_EXPONENTIAL, "inverse_proportional": FEM_SCHED_INVERSE_PROPORTIONAL}
OPTIMIZERS = {"adam": FEM_OPT_ADAM, "rmsprop": FEM_OPT_RMSPROP, "sgd": FEM_OPT_SGD}
GRAD_MODES = {"exact": FEM_GRAD_EXACT, "paper": FEM_GRAD_PAPER}
PRECISIONS = {"fp32": FEM_PREC_FP32, "bf16": FEM_PREC_BF16, "bf16x2": FEM_PREC_BF16X2, "fp8": FEM_PREC_FP8}


class fem_problem_desc(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("n", C.c_int32), ("q", C.c_int32),
        ("n_edges", C.c_int64), ("ei", C.c_void_p), ("ej", C.c_void_p), ("w", C.c_void_p),
        ("dense_J", C.c_void_p),
        ("n_clauses", C.c_int64), ("clause_ptr", C.c_void_p), ("lits", C.c_void_p),
        ("node_weight", C.c_void_p), ("linear", C.c_void_p), ("term_weight", C.c_void_p),
    ]


class fem_anneal_params(C.Structure):
    _fields_ = [
        ("replicas", C.c_int32), ("n_steps", C.c_int32), ("t_begin", C.c_int32), ("t_end", C.c_int32),
        ("schedule", C.c_int32), ("beta_min", C.c_double), ("beta_max", C.c_double),
        ("optimizer", C.c_int32), ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
        ("eps", C.c_double), ("weight_decay", C.c_double), ("momentum", C.c_double),
        ("alpha", C.c_double), ("dampening", C.c_double), ("gamma_grad", C.c_double),
        ("lambda_max", C.c_double), ("grad_mode", C.c_int32), ("precision", C.c_int32),
        ("h_init", C.c_void_p), ("h_init_is_device", C.c_int32),
    ]


class FemError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {status_string(status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfem.so not built at {LIB_PATH}; run python -m paper_2412_09285_b300.build")
    lib = C.CDLL(LIB_PATH)
    P, S = C.c_void_p, C.c_int
    sig = {
        "fem_create_problem": (S, [C.POINTER(fem_problem_desc), P, C.POINTER(P)]),
        "fem_anneal": (S, [P, C.POINTER(fem_anneal_params), P]),
        "fem_read_best": (S, [P, P, P, P, P, P]),
        "fem_read_fields": (S, [P, P, P]),
        "fem_read_states": (S, [P, P, P]),
        "fem_read_state": (S, [P, P, P, P, P]),
        "fem_write_state": (S, [P, P, P, P, C.c_int32, P]),
        "fem_problem_info": (S, [P, P, P, P, P, P]),
        "fem_sync": (S, [P, P]),
        "fem_set_dense_launch": (S, [P, C.c_int32]),
        "fem_dense_last_launch": (S, [P, C.POINTER(C.c_int32)]),
        "fem_set_step_barrier_timeout": (S, [P, C.c_int64]),
        "fem_inject_step_stall": (S, [P, C.c_int32]),
        "fem_anneal_batch": (S, [P, C.c_int32, C.POINTER(fem_anneal_params), P, P]),
        "fem_inject_allocation_failure": (None, [C.c_int64]),
        "fem_set_device_graph_build": (None, [C.c_int64]),
        "fem_set_tma_gather": (None, [C.c_int32]),
        "fem_destroy": (None, [P]),
        "fem_status_string": (C.c_char_p, [S]),
        "fem_last_error": (C.c_char_p, []),
        "fem_kernel_launches": (C.c_int64, []),
        "fem_schedule_value": (S, [C.POINTER(fem_anneal_params), C.c_int32, P, P]),
        "fem_batch_create": (S, [P, C.c_int32, C.POINTER(P)]),
        "fem_batch_anneal": (S, [P, C.POINTER(fem_anneal_params), P, P]),
        "fem_batch_destroy": (None, [P]),
        "fem_mpnn_num_params": (C.c_int32, []),
        "fem_mpnn_create": (S, [P, C.POINTER(P)]),
        "fem_mpnn_get_params": (S, [P, P]),
        "fem_mpnn_predict": (S, [P, P, P, C.c_int32, C.c_float, P, P]),
        "fem_mpnn_grad": (S, [P, P, P, P, C.c_int32, P, C.POINTER(C.c_double), P]),
        "fem_mpnn_train_step": (S, [P, P, P, P, C.c_int32, C.c_double, C.POINTER(C.c_double), P]),
        "fem_mpnn_destroy": (None, [P]),
        "fem_maxcut_energies_noalloc": (S, [P, P, C.c_int32, P, C.c_int32, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


_lib = _load()


def status_string(s: int) -> str:
    return _lib.fem_status_string(int(s)).decode()


def _check(status, where):
    if status != FEM_OK:
        raise FemError(status, where, _lib.fem_last_error().decode())


def _ptr(a):
    """Address of a numpy array's or torch tensor's data (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ----------------------------------------------------------------- C-named calls

def fem_create_problem(desc: fem_problem_desc, stream=None) -> int:
    h = C.c_void_p()
    _check(_lib.fem_create_problem(C.byref(desc), _stream(stream), C.byref(h)), "fem_create_problem")
    return h.value


def fem_anneal(handle: int, params: fem_anneal_params, stream=None) -> None:
    _check(_lib.fem_anneal(handle, C.byref(params), _stream(stream)), "fem_anneal")


def fem_read_best(handle, best_replica=None, states=None, energy_i64=None, energy_f64=None, stream=None):
    _check(_lib.fem_read_best(handle, _ptr(best_replica), _ptr(states), _ptr(energy_i64),
                              _ptr(energy_f64), _stream(stream)), "fem_read_best")


def fem_read_fields(handle, h_host, stream=None):
    _check(_lib.fem_read_fields(handle, _ptr(h_host), _stream(stream)), "fem_read_fields")


def fem_read_states(handle, states_host, stream=None):
    _check(_lib.fem_read_states(handle, _ptr(states_host), _stream(stream)), "fem_read_states")


def fem_read_state(handle, h=None, m=None, v=None, stream=None):
    _check(_lib.fem_read_state(handle, _ptr(h), _ptr(m), _ptr(v), _stream(stream)), "fem_read_state")


def fem_write_state(handle, h, m=None, v=None, steps_done=0, stream=None):
    _check(_lib.fem_write_state(handle, _ptr(h), _ptr(m), _ptr(v), int(steps_done), _stream(stream)),
           "fem_write_state")


def fem_problem_info(handle):
    vals = [C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64()]
    _check(_lib.fem_problem_info(handle, *[C.byref(v) for v in vals]), "fem_problem_info")
    return dict(steps_done=vals[0].value, n=vals[1].value, q=vals[2].value,
                replicas=vals[3].value, units_per_replica=vals[4].value)


def fem_sync(handle, stream=None):
    _check(_lib.fem_sync(handle, _stream(stream)), "fem_sync")


def fem_dense_last_launch(handle):
    out = C.c_int32()
    _check(_lib.fem_dense_last_launch(handle, C.byref(out)), "fem_dense_last_launch")
    return out.value


def fem_set_dense_launch(handle, mode):
    """mode: 0 auto, 1 one kernel per step, 2 persistent, 3 persistent without CTA
    pairs (fem_dense_launch)."""
    _check(_lib.fem_set_dense_launch(handle, int(mode)), "fem_set_dense_launch")


def fem_set_step_barrier_timeout(handle, ns):
    _check(_lib.fem_set_step_barrier_timeout(handle, int(ns)), "fem_set_step_barrier_timeout")


def fem_inject_step_stall(handle, row_tile):
    """The persistent dense kernel's CTAs of `row_tile` stop reporting ready (-1: off)."""
    _check(_lib.fem_inject_step_stall(handle, int(row_tile)), "fem_inject_step_stall")


def fem_set_device_graph_build(min_edges):
    """Graphs with at least min_edges edges build their CSR on the device (< 0: never)."""
    _lib.fem_set_device_graph_build(int(min_edges))


def fem_set_tma_gather(on):
    """Sparse MaxCut / QUBO steps on the staged tile kernels (True, the default: exact mode
    with TMA gather4 copies, paper mode with bulk-copied state) or the direct kernels
    (False); both give the same bits."""
    _lib.fem_set_tma_gather(1 if on else 0)


def fem_inject_allocation_failure(after):
    """The device allocation after `after` successful ones fails with FEM_ERR_OOM (-1: off)."""
    _lib.fem_inject_allocation_failure(int(after))


def fem_destroy(handle):
    _lib.fem_destroy(handle)


def fem_schedule_value(t, n_steps, **kw):
    """(beta_t, lambda_t) of step t of an anneal of n_steps steps with the schedule
    settings in kw (the library's own schedule)."""
    p = make_params(1, n_steps, **kw)
    beta, lam = C.c_double(), C.c_double()
    _check(_lib.fem_schedule_value(C.byref(p), int(t), C.byref(beta), C.byref(lam)), "fem_schedule_value")
    return beta.value, lam.value


def fem_kernel_launches() -> int:
    return int(_lib.fem_kernel_launches())


def fem_maxcut_energies_noalloc(row_ptr, col, n, words, replicas, energy, best_replica, stream=None):
    """All array arguments are CUDA tensors (device pointers); nothing is allocated."""
    _check(_lib.fem_maxcut_energies_noalloc(_ptr(row_ptr), _ptr(col), int(n), _ptr(words),
                                            int(replicas), _ptr(energy), _ptr(best_replica),
                                            _stream(stream)), "fem_maxcut_energies_noalloc")


# ----------------------------------------------------------------- convenience

DEFAULTS = dict(schedule="exponential", beta_min=0.05, beta_max=5.0, optimizer="adam", lr=0.1,
                beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, momentum=0.0, alpha=0.99,
                dampening=0.0, gamma_grad=1.0, lambda_max=1.0, grad_mode="paper", precision="bf16")


def make_params(replicas, n_steps, t_begin=0, t_end=None, h_init=None, **kw) -> fem_anneal_params:
    o = dict(DEFAULTS)
    o.update(kw)
    p = fem_anneal_params()
    p.replicas, p.n_steps = int(replicas), int(n_steps)
    p.t_begin = int(t_begin)
    p.t_end = int(n_steps if t_end is None else t_end)
    p.schedule = SCHEDULES[o["schedule"]]
    p.beta_min, p.beta_max = float(o["beta_min"]), float(o["beta_max"])
    p.optimizer = OPTIMIZERS[o["optimizer"]]
    for k in ("lr", "beta1", "beta2", "eps", "weight_decay", "momentum", "alpha", "dampening",
              "gamma_grad", "lambda_max"):
        setattr(p, k, float(o[k]))
    p.grad_mode = GRAD_MODES[o["grad_mode"]]
    p.precision = PRECISIONS[o["precision"]]
    p.h_init = _ptr(h_init)
    p.h_init_is_device = int(bool(h_init is not None and hasattr(h_init, "is_cuda") and h_init.is_cuda))
    return p


class Problem:
    """Owns one libfem problem handle.  Inputs are host numpy arrays (or objects
    from ``instances``); h_init may also be a CUDA torch tensor."""

    def __init__(self, kind="maxcut", graph=None, clauses=None, dense=None, q=2, stream=None, node_weight=None,
                 linear=None, term_weight=None):
        self.kind = kind
        self.stream = stream
        d = fem_problem_desc()
        d.kind = KINDS[kind]
        d.q = int(q)
        self._keep = []
        if graph is not None:
            d.n = graph.n
            ei = np.ascontiguousarray(graph.ei, np.int32)
            ej = np.ascontiguousarray(graph.ej, np.int32)
            w = np.ascontiguousarray(graph.w, np.float64)
            self._keep += [ei, ej, w]
            d.n_edges, d.ei, d.ej, d.w = ei.shape[0], _ptr(ei), _ptr(ej), _ptr(w)
        if term_weight is not None:
            T = np.ascontiguousarray(term_weight, np.float64)
            self._keep.append(T)
            d.term_weight = _ptr(T)
        if linear is not None:
            L = np.ascontiguousarray(linear, np.float64)
            self._keep.append(L)
            d.linear = _ptr(L)
        if node_weight is not None:
            V = np.ascontiguousarray(node_weight, np.float64)
            self._keep.append(V)
            d.node_weight = _ptr(V)
        if dense is not None:
            J = np.ascontiguousarray(dense, np.float32)
            self._keep.append(J)
            d.n = J.shape[0]
            d.dense_J = _ptr(J)
        if clauses is not None:
            d.n = clauses.n
            ptr = np.ascontiguousarray(clauses.ptr, np.int64)
            lits = np.ascontiguousarray(clauses.lits, np.int32)
            self._keep += [ptr, lits]
            d.n_clauses, d.clause_ptr, d.lits = ptr.shape[0] - 1, _ptr(ptr), _ptr(lits)
        self.n, self.q = d.n, d.q
        self.handle = fem_create_problem(d, stream)
        self._keep = []
        self.replicas = 0

    def anneal(self, h_init=None, replicas=None, n_steps=1000, t_begin=0, t_end=None, **kw):
        if h_init is not None and not hasattr(h_init, "data_ptr"):
            h_init = np.ascontiguousarray(h_init, np.float32)
        if replicas is None:
            replicas = h_init.shape[1] if h_init is not None else self.replicas
        self.replicas = int(replicas)
        p = make_params(replicas, n_steps, t_begin, t_end, h_init, **kw)
        fem_anneal(self.handle, p, self.stream)
        return self

    def fields(self):
        shape = (self.n, self.replicas) if self.kind not in Q_STATE_KINDS else (self.n, self.replicas, self.q)
        out = np.empty(shape, np.float32)
        fem_read_fields(self.handle, out, self.stream)
        return out

    def _shape(self):
        return (self.n, self.replicas) if self.kind not in Q_STATE_KINDS else (self.n, self.replicas, self.q)

    def state(self):
        """(h, m, v) as float32 host arrays (a checkpoint, with info()['steps_done'])."""
        h, m, v = (np.empty(self._shape(), np.float32) for _ in range(3))
        fem_read_state(self.handle, h, m, v, self.stream)
        return h, m, v

    def set_state(self, h, m=None, v=None, steps_done=0):
        conv = lambda x: None if x is None else np.ascontiguousarray(x, np.float32)
        h, m, v = conv(h), conv(m), conv(v)
        fem_write_state(self.handle, h, m, v, steps_done, self.stream)

    def states(self):
        out = np.empty((self.n, self.replicas), np.int32)
        fem_read_states(self.handle, out, self.stream)
        return out

    def best(self, states=True):
        """Best replica, every replica's energy and (unless states=False) the best
        replica's states copied to the host."""
        br = np.zeros(1, np.int32)
        st = np.empty(self.n, np.int32) if states else None
        ei = np.empty(self.replicas, np.int64)
        ef = np.empty(self.replicas, np.float64)
        fem_read_best(self.handle, br, st, ei, ef, self.stream)
        return dict(best_replica=int(br[0]), states=st, energy_i64=ei, energy_f64=ef)

    def info(self):
        return fem_problem_info(self.handle)

    def set_dense_launch(self, mode):
        """'auto', 'per_step', 'persistent' or 'persistent_single' (dense problems)."""
        fem_set_dense_launch(self.handle, {"auto": 0, "per_step": 1, "persistent": 2, "persistent_single": 3}[mode])

    def dense_last_launch(self):
        """The kernel the last window ran on: None, 'per_step', 'persistent' (CTA pairs)
        or 'persistent_single'."""
        return {0: None, 1: "per_step", 2: "persistent", 3: "persistent_single"}[fem_dense_last_launch(self.handle)]

    def sync(self):
        fem_sync(self.handle, self.stream)

    def close(self):
        if getattr(self, "handle", None):
            fem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- batches

def fem_batch_create(handles) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    out = C.c_void_p()
    _check(_lib.fem_batch_create(C.cast(arr, C.c_void_p), len(handles), C.byref(out)), "fem_batch_create")
    return out.value


def fem_batch_anneal(batch, params, h_inits=None, stream=None):
    ptrs = None
    if h_inits is not None:
        ptrs = (C.c_void_p * len(h_inits))(*[_ptr(h) for h in h_inits])
    _check(_lib.fem_batch_anneal(batch, C.byref(params), C.cast(ptrs, C.c_void_p) if ptrs else None,
                                 _stream(stream)), "fem_batch_anneal")


def anneal_batch(problems, h_inits, replicas=None, n_steps=1000, t_begin=0, t_end=None, stream=None, **kw):
    """One call for several problems (fem_anneal_batch): the batch is built for the
    call and released after it; synchronises the stream."""
    on_device = all(getattr(h, "is_cuda", False) for h in h_inits) if h_inits is not None else False
    if h_inits is not None and not on_device:
        h_inits = [np.ascontiguousarray(h, np.float32) for h in h_inits]
    if replicas is None:
        replicas = h_inits[0].shape[1]
    for p in problems:
        p.replicas = int(replicas)
    params = make_params(replicas, n_steps, t_begin, t_end, None, **kw)
    params.h_init_is_device = int(on_device)
    handles = (C.c_void_p * len(problems))(*[p.handle for p in problems])
    ptrs = (C.c_void_p * len(h_inits))(*[_ptr(h) for h in h_inits]) if h_inits is not None else None
    _check(_lib.fem_anneal_batch(C.cast(handles, C.c_void_p), len(problems), C.byref(params),
                                 C.cast(ptrs, C.c_void_p) if ptrs else None, _stream(stream)), "fem_anneal_batch")


def fem_batch_destroy(batch):
    _lib.fem_batch_destroy(batch)


class Batch:
    """Several Problem objects advanced together by fem_batch_anneal."""

    def __init__(self, problems, stream=None):
        self.problems = list(problems)
        self.stream = stream
        self.handle = fem_batch_create([p.handle for p in self.problems])

    def anneal(self, h_inits=None, replicas=None, n_steps=1000, t_begin=0, t_end=None, **kw):
        on_device = False
        if h_inits is not None:
            on_device = all(getattr(h, "is_cuda", False) for h in h_inits)
            if not on_device:
                h_inits = [np.ascontiguousarray(h, np.float32) for h in h_inits]
            replicas = h_inits[0].shape[1] if replicas is None else replicas
        for p in self.problems:
            p.replicas = int(replicas)
        params = make_params(replicas, n_steps, t_begin, t_end, None, **kw)
        params.h_init_is_device = int(on_device)
        fem_batch_anneal(self.handle, params, h_inits, self.stream)
        return self

    def close(self):
        if getattr(self, "handle", None):
            fem_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
