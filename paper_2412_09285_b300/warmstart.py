"""Learned warm start for sparse MaxCut FEM: the network binding, training on FEM's
own converged fields, and the warm-started anneal.

The network (C ABI ``fem_mpnn_*``, kernels in csrc/mpnn.cu) predicts local fields
y = sum_k theta_k(i) (P^k z)_i from the graph and a replica's random initial fields
z (units of 0.001).  It is trained on the fields plain FEM converges to (loss on
tanh(y/2) against tanh(h/2)); since those depend only weakly on z the least-squares
optimum is small in magnitude, so at inference the prediction is rescaled per replica
to a chosen root-mean-square (the network fixes the direction, the caller the
magnitude).  A warm-started anneal then runs a shortened schedule that starts at
beta(t_start) of the full schedule.  Plain random-initialised FEM is both the fallback
and the judge: the comparison is the best cut of the warm-started anneal against plain
FEM at the same and at the full budget, and against the same shortened schedule
started from rescaled noise instead of the prediction (which isolates what the network
adds beyond the shorter schedule).

Every computation runs in the library's kernels; torch only holds device buffers.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import fem as F
from . import instances as I

__all__ = ["Mpnn", "beta_at", "fem_fields_at", "warm_anneal", "train", "make_graphs"]


class Mpnn:
    """Owns a fem_mpnn handle (fp32 master weights, Adam state, bf16 copy)."""

    def __init__(self, params: dict | None = None, seed: int = 0):
        flat = I.mpnn_flatten(params if params is not None else I.mpnn_init(seed))
        assert flat.size == F._lib.fem_mpnn_num_params()
        h = C.c_void_p()
        F._check(F._lib.fem_mpnn_create(flat.ctypes.data, C.byref(h)), "fem_mpnn_create")
        self.handle = h.value

    def params(self) -> dict:
        flat = np.empty(F._lib.fem_mpnn_num_params(), np.float32)
        F._check(F._lib.fem_mpnn_get_params(self.handle, flat.ctypes.data), "fem_mpnn_get_params")
        return I.mpnn_unflatten(flat)

    def predict(self, problem, z, R, y, rms=0.0, stream=None):
        """y = the network's fields for initial fields z; rms > 0 rescales every replica's
        column to that root-mean-square."""
        F._check(F._lib.fem_mpnn_predict(self.handle, problem.handle, F._ptr(z), int(R), float(rms), F._ptr(y),
                                         F._stream(stream)), "fem_mpnn_predict")

    def grad(self, problem, z, h_target, R, stream=None):
        g = np.empty(F._lib.fem_mpnn_num_params(), np.float32)
        loss = C.c_double()
        F._check(F._lib.fem_mpnn_grad(self.handle, problem.handle, F._ptr(z), F._ptr(h_target), int(R),
                                      g.ctypes.data, C.byref(loss), F._stream(stream)), "fem_mpnn_grad")
        return I.mpnn_unflatten(g), loss.value

    def train_step(self, problem, z, h_target, R, lr, stream=None) -> float:
        loss = C.c_double()
        F._check(F._lib.fem_mpnn_train_step(self.handle, problem.handle, F._ptr(z), F._ptr(h_target), int(R),
                                            float(lr), C.byref(loss), F._stream(stream)), "fem_mpnn_train_step")
        return loss.value

    def close(self):
        if getattr(self, "handle", None):
            F._lib.fem_mpnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def beta_at(t, n_steps, beta_min=0.05, beta_max=5.0):
    """The exponential schedule's beta at step t, from the library (fem_schedule_value)."""
    return F.fem_schedule_value(t, n_steps, beta_min=beta_min, beta_max=beta_max)[0]


def fem_fields_at(problem, h0, n_steps, t_end, out, **kw):
    """Plain FEM from h0 (device [n][R]) for t_end of n_steps steps; its fields into out
    (device).  t_end = n_steps gives the converged fields the network is trained on."""
    R = h0.shape[1]
    problem.anneal(h_init=h0, replicas=R, n_steps=n_steps, t_end=t_end, **kw)
    F.fem_read_fields(problem.handle, out, problem.stream)


def warm_anneal(problem, y, budget, n_full, t_start, beta_min=0.05, beta_max=5.0, **kw):
    """A shortened anneal of `budget` steps from fields y (device [n][R]); beta runs from
    beta(t_start) of the full n_full-step schedule to beta_max."""
    R = y.shape[1]
    problem.anneal(h_init=y, replicas=R, n_steps=budget, beta_min=beta_at(t_start, n_full, beta_min, beta_max),
                   beta_max=beta_max, **kw)


def train(net, graphs, epochs, R, n_steps, lr, seed=0, device="cuda"):
    """One Adam step per graph and epoch on FEM's converged fields from fresh random
    initial fields; returns the mean loss of every epoch."""
    import torch
    from . import instances as I
    out = []
    for epoch in range(epochs):
        losses = []
        for k, g in enumerate(graphs):
            prob = F.Problem("maxcut", graph=g)
            z = torch.from_numpy(I.initial_fields(g.n, R, seed=seed + 100003 * epoch + k) * np.float32(1000.0)).to(device)
            target = torch.empty_like(z)
            fem_fields_at(prob, z * 0.001, n_steps, n_steps, target)
            losses.append(net.train_step(prob, z, target, R, lr=lr))
            prob.close()
        out.append(float(np.mean(losses)))
    return out


def _gen(args):
    n, m, seed = args
    g = I.er_gnm(int(n), int(m), seed=int(seed), weights="pm1")
    return g.n, g.ei, g.ej, g.w


def make_graphs(count, lo, hi, mean_degree, seed, pool=None):
    """ER graphs with n log-uniform in [lo, hi], m = n * mean_degree / 2, +-1 weights."""
    sizes = I.loguniform_sizes(count, lo, hi, seed=seed)
    jobs = [(n, int(n * mean_degree / 2), seed * 100003 + k) for k, n in enumerate(sizes)]
    res = pool.map(_gen, jobs) if pool is not None else [_gen(j) for j in jobs]
    return [I.Graph(n, ei, ej, w) for n, ei, ej, w in res]
