#!/usr/bin/env python3
"""Benchmark of the FEM per-step replica update on B300 (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload W] [--precision bf16|fp8|bf16x2|fp32] [--grad-mode paper|exact]

Workloads (synthetic, seeded; the paper's data sets are not available; the batched, warm-start
and single-problem workloads bmincut, bmincut_weighted, coloring, qubo, sat and pspin are
described in WORKLOADS below):
  sparse (default)  sparse MaxCut at scale: ER G(n, m), n = 2^20, m = 3n, +-1 weights,
                    R = 32, 2000-step exponential beta 0.05 -> 5, Adam lr 0.1, paper-mode
                    gradient.  Units: |E| undirected edges x replicas x steps.
  small             ER G(800, 0.06), unit weights, R = 32, 1000 steps (latency-bound).
  dense             SK complete graph n = 2000, J = +-1, R = 1024, 1000 steps, the J.M
                    contraction on the tensor cores (--precision).  Units: n(n-1)/2 edges.

A "step" is one anneal step of all replicas (schedule, contraction, gradient,
optimizer).  The timed region runs K steps from freshly initialised fields
resident in HBM (chained anneals of the workload's length) and ends each anneal
with the read-out (argmax, exact int64 objective, argmin over replicas).

Under torchrun the global replica set is R per rank and every rank runs its block of
it (sharding.shard_fields; no data-path collective, weak scaling); the best replica
over ranks is gathered after timing, and rank 0 prints the line.  ``--impl reference``
times the FP64 CPU oracle (there is no other implementation of the method to run) on
all host cores, one single-threaded process per block of replicas.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge*replica*steps/s"
WORKLOADS = {
    "sparse": dict(kind="sparse", name="sparse MaxCut at scale: ER G(n,m) n=2^20, m=3n, +-1 weights, R=32, "
                                      "2000-step exponential beta 0.05->5, Adam lr 0.1, paper-mode gradient",
                   n=1 << 20, m=3 << 20, weights="pm1", R=32, n_steps=2000, graph_seed=2024, h_seed=2025,
                   cpu_steps=6),
    "small": dict(kind="sparse", name="plain MaxCut: ER G(800, 0.06), unit weights, R=32, 1000-step "
                                     "exponential beta 0.05->5, Adam lr 0.1, paper-mode gradient",
                  n=800, p=0.06, weights="unit", R=32, n_steps=1000, graph_seed=1, h_seed=2, cpu_steps=1000),
    "dense": dict(kind="dense", name="dense SK MaxCut: complete graph n=2000, J=+-1, R=1024, 1000-step "
                                    "exponential beta 0.05->5, Adam lr 0.1, paper-mode gradient",
                  n=2000, R=1024, n_steps=1000, graph_seed=3, h_seed=4, cpu_steps=4),
    "batched": dict(kind="batched", name="batched heterogeneous: 256 bMinCut (random geometric graphs, n "
                                        "log-uniform 1k-64k, mean degree 10, unit weights, q=4, lambda_max=1) + "
                                        "64 random Max-3-SAT (n log-uniform 5k-50k, M=4.2n), R=16 each, 1000-step "
                                        "exponential beta 0.05->5, Adam lr 0.1, paper-mode gradient, two launches "
                                        "per step (bMinCut and SAT members), CUDA-graph step loop, autotuned "
                                        "work items",
                    n_bmc=256, bmc_lo=1000, bmc_hi=64000, deg=10.0, q=4, n_sat=64, sat_lo=5000, sat_hi=50000,
                    ratio=4.2, R=16, n_steps=1000, graph_seed=5, h_seed=6, cpu_steps=2),
    # learned warm start (time to target only): ER graphs, n log-uniform 20k-200k, mean
    # degree 8, +-1 weights, R = 32, full budget 2000 steps; the network is trained here
    # on FEM's converged fields of the training graphs (disjoint seeds from the held-out)
    "warmstart": dict(kind="warmstart", name="learned warm start: MaxCut on ER graphs, n log-uniform 20k-200k, "
                                             "mean degree 8, +-1 weights, R=32, 2000-step exponential beta "
                                             "0.05->5, Adam lr 0.1, paper-mode gradient",
                      n_lo=20000, n_hi=200000, deg=8.0, R=32, n_steps=2000, n_train=64, n_held=16, epochs=3,
                      lr=3e-3, rms=0.1, train_seed=31, held_seed=32, h_seed=33),
    # the learned warm start at the full configuration: 2000 training and 100 held-out graphs
    "warmstart_full": dict(kind="warmstart", name="learned warm start, full configuration: MaxCut on ER graphs, n "
                                                  "log-uniform 20k-200k, mean degree 8, +-1 weights, R=32, 2000-step "
                                                  "exponential beta 0.05->5, Adam lr 0.1, paper-mode gradient; 2000 "
                                                  "training and 100 held-out graphs",
                           n_lo=20000, n_hi=200000, deg=8.0, R=32, n_steps=2000, n_train=2000, n_held=100, epochs=2,
                           lr=3e-3, rms=0.1, train_seed=31, held_seed=32, h_seed=33),
    # the warm-start network's inference (fem_mpnn_predict) on the largest graph of the range
    "mpnn": dict(kind="mpnn", name="warm-start network inference: 3 message-passing layers of width 64 (bf16 weights, "
                                   "fp32 activations) and a 4-tap head on ER n=200000, mean degree 8, +-1 weights, "
                                   "R=32 replicas of initial fields, rescaled to rms 0.1",
                 n=200000, m=800000, R=32, graph_seed=34, h_seed=35, n_steps=1),
    # the batched workload at 1/8 scale (same size distributions): the case profiled in detail
    "batched_small": dict(kind="batched", name="batched heterogeneous at 1/8 scale: 32 bMinCut (random geometric "
                                              "graphs, n log-uniform 1k-64k, mean degree 10, unit weights, q=4) + 8 "
                                              "random Max-3-SAT (n log-uniform 5k-50k, M=4.2n), R=16 each, 1000-step "
                                              "exponential beta 0.05->5, Adam lr 0.1, paper-mode gradient",
                          n_bmc=32, bmc_lo=1000, bmc_hi=64000, deg=10.0, q=4, n_sat=8, sat_lo=5000, sat_hi=50000,
                          ratio=4.2, R=16, n_steps=1000, graph_seed=5, h_seed=6, cpu_steps=2),
}

# One problem per kind of the widened rows (balanced MinCut with and without node weights,
# colouring, QUBO, Max-3-SAT, higher-order p-spin terms), each at a size whose state is
# larger than L2.  The CPU oracle baseline of these runs on an instance of the same
# generator at 1/cpu_div of the size (a full oracle step at this size takes minutes).
_SINGLE = dict(n=1 << 20, n_steps=1000, cpu_div=16, cpu_steps=4)
_SCHED = "1000-step exponential beta 0.05->5, Adam lr 0.1"
WORKLOADS.update({
    "bmincut": dict(_SINGLE, kind="single", problem="bmincut", graph="rgg", deg=10.0, q=4, R=16, graph_seed=41,
                    h_seed=42, name=f"balanced 4-way MinCut: random geometric graph n=2^20, mean degree 10, unit "
                                    f"weights, lambda_max=1, R=16, {_SCHED}, paper-mode gradient"),
    "bmincut_q8": dict(_SINGLE, kind="single", problem="bmincut", graph="rgg", deg=10.0, q=8, R=16, graph_seed=41,
                       h_seed=42, name=f"balanced 8-way MinCut: random geometric graph n=2^20, mean degree 10, unit "
                                       f"weights, lambda_max=1, R=16, {_SCHED}, paper-mode gradient"),
    "bmincut_weighted": dict(_SINGLE, kind="single", problem="bmincut", graph="rgg", deg=10.0, q=4, R=16,
                             node_weights=(1, 4), graph_seed=41, h_seed=42,
                             name=f"node-weighted balanced 4-way MinCut: random geometric graph n=2^20, mean degree "
                                  f"10, node weights uniform in 1..4, lambda_max=1, R=16, {_SCHED}, paper-mode "
                                  f"gradient"),
    "coloring": dict(_SINGLE, kind="single", problem="coloring", graph="rgg", deg=10.0, q=4, R=16, graph_seed=43,
                     h_seed=44, name=f"4-colouring: random geometric graph n=2^20, mean degree 10, R=16, {_SCHED}, "
                                     f"paper-mode gradient"),
    "qubo": dict(_SINGLE, kind="single", problem="qubo", graph="er", m=3 << 20, R=32, linear=(-2, 2),
                 grad_mode="exact", graph_seed=45, h_seed=46,
                 name=f"QUBO: ER G(n,m) n=2^20, m=3n, couplings +-1, linear terms uniform in -2..2, R=32, "
                      f"{_SCHED}, exact gradient"),
    "sat": dict(_SINGLE, kind="single", problem="sat", ratio=4.2, k=3, R=16, graph_seed=47, h_seed=48,
                name=f"random Max-3-SAT: n=2^20 variables, M=4.2n clauses, uniform literal signs, R=16, {_SCHED}"),
    "pspin": dict(_SINGLE, kind="single", problem="pspin", ratio=4.2, k=3, R=16, linear=(-1, 1), graph_seed=49,
                  cpu_div=32, cpu_steps=1,
                  h_seed=50, name=f"3-spin interactions: n=2^20 spins, 4.2n random 3-spin terms, J=+-1, fields "
                                  f"uniform in -1..1, R=16, {_SCHED}"),
})


class _SingleInstance:
    """One problem of a widened row (graph or clause list plus node weights, linear
    terms or term couplings), at 1/scale of the workload's size."""

    def __init__(self, wl, scale=1):
        from paper_2412_09285_b300 import instances as I
        n, s = wl["n"] // scale, wl["graph_seed"]
        rng = np.random.Generator(np.random.PCG64(s + 7))
        self.problem, self.graph, self.clauses = wl["problem"], None, None
        self.node_weight = self.linear = self.term_weight = None
        if wl["problem"] in ("sat", "pspin"):
            self.clauses = I.random_ksat(n, int(round(wl["ratio"] * n)), wl["k"], seed=s)
            if wl["problem"] == "pspin":  # terms of distinct spins; the sign lives in J
                self.clauses = I.Clauses(n, self.clauses.ptr, np.abs(self.clauses.lits))
                self.term_weight = rng.choice([-1.0, 1.0], size=self.clauses.n_clauses)
            self.n, self.units = n, int(self.clauses.ptr[-1])
        else:
            self.graph = (I.rgg(n, wl["deg"], seed=s) if wl["graph"] == "rgg"
                          else I.er_gnm(n, wl["m"] // scale, seed=s, weights="pm1"))
            self.n, self.units = n, self.graph.n_edges
        if "node_weights" in wl:
            lo, hi = wl["node_weights"]
            self.node_weight = rng.integers(lo, hi + 1, size=n).astype(np.int32)
        if "linear" in wl:
            lo, hi = wl["linear"]
            self.linear = rng.integers(lo, hi + 1, size=n).astype(np.float64)

    def problem_obj(self, fem, wl, stream):
        return fem.Problem(self.problem, graph=self.graph, clauses=self.clauses, q=wl.get("q", 2), stream=stream,
                           node_weight=self.node_weight, linear=self.linear, term_weight=self.term_weight)

    def oracle_problem(self):
        import oracle as O
        if self.clauses is not None:
            c = self.clauses
            if self.problem == "sat":
                return ("sat", O.sat_arrays(c.ptr, c.lits))
            return ("pspin", (c.ptr, np.abs(c.lits) - 1, self.term_weight, self.linear))
        g = self.graph
        W = O.coupling_matrix(g.n, g.ei, g.ej, g.w)
        if self.problem == "qubo":
            return ("qubo", (W, self.linear))
        if self.problem == "bmincut" and self.node_weight is not None:
            return ("bmincut", W, self.node_weight.astype(np.float64))
        return (self.problem, W)

    def host_bytes(self):
        """Bytes of the problem description a user passes from host memory."""
        b = 0
        if self.graph is not None:
            b += 8 * self.graph.n_edges + 4 * (self.n + 1)
        if self.clauses is not None:
            b += 8 * (self.clauses.n_clauses + 1) + 4 * int(self.clauses.ptr[-1])
        for x in (self.node_weight, self.linear, self.term_weight):
            b += 0 if x is None else x.nbytes
        return b


class _BatchInstance:
    """The members of the batched workload (graphs and clause lists)."""

    def __init__(self, wl):
        from paper_2412_09285_b300 import instances as I
        s = wl["graph_seed"]
        self.graphs = [I.rgg(int(n), wl["deg"], seed=1000 * s + k)
                       for k, n in enumerate(I.loguniform_sizes(wl["n_bmc"], wl["bmc_lo"], wl["bmc_hi"], seed=s))]
        self.sats = [I.random_ksat(int(n), int(round(wl["ratio"] * n)), 3, seed=2000 * s + k)
                     for k, n in enumerate(I.loguniform_sizes(wl["n_sat"], wl["sat_lo"], wl["sat_hi"], seed=s + 1))]
        self.n = sum(g.n for g in self.graphs) + sum(c.n for c in self.sats)
        self.units = sum(g.n_edges for g in self.graphs) + sum(int(c.ptr[-1]) for c in self.sats)

    def h0(self, wl, replicas=None):
        from paper_2412_09285_b300 import instances as I
        base, R = wl["h_seed"], replicas or wl["R"]
        return ([I.initial_fields(g.n, R, seed=base * 100000 + k, q=wl["q"]) for k, g in enumerate(self.graphs)]
                + [I.initial_fields(c.n, R, seed=base * 100000 + 50000 + k) for k, c in enumerate(self.sats)])


class _BatchRunner:
    """Adapter with the single-problem interface the timing loop uses."""

    def __init__(self, fem, wl, inst, stream):
        self.probs = ([fem.Problem("bmincut", graph=g, q=wl["q"], stream=stream) for g in inst.graphs]
                      + [fem.Problem("sat", clauses=c, stream=stream) for c in inst.sats])
        self.batch = fem.Batch(self.probs, stream=stream)
        self.h0 = None

    def anneal(self, h_init=None, replicas=None, n_steps=1000, t_begin=0, t_end=None, **kw):
        kw.pop("precision", None)
        self.batch.anneal(h_inits=h_init if t_begin == 0 else None, replicas=replicas, n_steps=n_steps,
                          t_begin=t_begin, t_end=t_end, lambda_max=1.0, **kw)

    def best(self, states=True):
        """Sum over members of each member's best energy (one read-out per member)."""
        tot = 0.0
        for p in self.probs:
            r = p.best(states=states)
            tot += float(r["energy_f64"][r["best_replica"]])
        return {"energy_f64": np.array([tot]), "best_replica": 0, "energy_i64": np.array([int(tot)])}

    def close(self):
        self.batch.close()
        for p in self.probs:
            p.close()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def _instance(wl):
    from paper_2412_09285_b300 import instances as I
    if wl["kind"] == "batched":
        return _BatchInstance(wl)
    if wl["kind"] == "single":
        return _SingleInstance(wl)
    if wl["kind"] == "dense":
        return I.sk_dense(wl["n"], seed=wl["graph_seed"])
    if "m" in wl:
        return I.er_gnm(wl["n"], wl["m"], seed=wl["graph_seed"], weights=wl["weights"])
    return I.er_gnp(wl["n"], wl["p"], seed=wl["graph_seed"], weights=wl["weights"])


def _pinned_instance(inst, torch):
    """The same instance with its host arrays in pinned (page-locked) memory, so the
    end-to-end run copies its inputs from pinned host buffers."""
    import copy
    from paper_2412_09285_b300 import instances as I

    def pin(x):
        return None if x is None else torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()

    def pin_graph(g):
        return I.Graph(g.n, pin(g.ei), pin(g.ej), pin(g.w),
                       dense=None if g.dense is None else pin(g.dense.astype(np.float32)))

    def pin_clauses(c):
        return I.Clauses(c.n, pin(np.asarray(c.ptr, np.int64)), pin(np.asarray(c.lits, np.int32)))
    if isinstance(inst, I.Graph):
        return pin_graph(inst)
    out = copy.copy(inst)
    if isinstance(inst, _SingleInstance):
        out.graph = None if inst.graph is None else pin_graph(inst.graph)
        out.clauses = None if inst.clauses is None else pin_clauses(inst.clauses)
        out.node_weight, out.linear, out.term_weight = pin(inst.node_weight), pin(inst.linear), pin(inst.term_weight)
    elif isinstance(inst, _BatchInstance):
        out.graphs = [pin_graph(g) for g in inst.graphs]
        out.sats = [pin_clauses(c) for c in inst.sats]
    return out


def _make_problem(fem, wl, inst, stream, dense_launch="auto"):
    if wl["kind"] == "batched":
        return _BatchRunner(fem, wl, inst, stream)
    if wl["kind"] == "single":
        return inst.problem_obj(fem, wl, stream)
    if wl["kind"] == "dense":
        P = fem.Problem("maxcut", dense=inst.dense, stream=stream)
        P.set_dense_launch(dense_launch)
        return P
    return fem.Problem("maxcut", graph=inst, stream=stream)


# The source files each profiled kernel is compiled from (its .cu and the local headers
# with device code it includes; the host-side problem record is not part of it); a
# summary's traffic figure counts only while they are unchanged.
KERNEL_SOURCES = {
    "sparse": ["maxcut_sparse.cu", "step_common.cuh", "step_scalars.h"],
    "exact": ["maxcut_gather.cu", "step_common.cuh", "step_scalars.h"],
    "paper_tile": ["maxcut_paper_tile.cu", "step_common.cuh", "step_scalars.h"],
    "dense": ["dense_tc.cu", "step_common.cuh", "step_scalars.h"],
    "batched": ["batch.cu", "bmincut_core.cuh", "sat_core.cuh", "step_common.cuh", "step_scalars.h"],
    "bmincut": ["bmincut_sparse.cu", "bmincut_core.cuh", "step_common.cuh", "step_scalars.h"],
    "sat": ["sat.cu", "sat_core.cuh", "step_common.cuh", "step_scalars.h"],
}
# the committed ncu summary of each single-problem workload whose traffic is reported
_SINGLE_PROFILES = {"bmincut": ("bmincut_step_rgg1M_q4_R16.md", "bmincut"), "sat": ("sat_step_3sat1M_R16.md", "sat"),
                    "pspin": ("pspin_step_3spin1M_R16.md", "sat"),
                    "qubo": ("maxcut_step_exact_n1M_R32.md", "exact", "qubo_traffic_bytes_per_launch")}


def source_sha256(kind):
    """sha256 over the code-generation flags and the concatenated sources of one kernel
    family (see KERNEL_SOURCES)."""
    from paper_2412_09285_b300 import build as B
    csrc = os.path.join(ROOT, "paper_2412_09285_b300", "csrc")
    h = hashlib.sha256()
    h.update(" ".join(B.ARCH + B.CODEGEN).encode())
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic_from_profile(name, kind, key="traffic_bytes_per_launch"):
    """DRAM bytes per launch from a committed ncu summary, if the kernel's sources are
    unchanged since the capture (else None)."""
    try:
        txt = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    m1 = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    m2 = re.search(r"(?m)^" + key + r":\s*([0-9]+)", txt)
    if not (m1 and m2):
        return None
    return int(m2.group(1)) if source_sha256(kind) == m1.group(1) else None


def _roofline(wl, inst, step_ms, precision, dense_launch=None, grad_mode="paper", opt="adam"):
    """Algorithmic work of one step launch / its measured duration, against the peak."""
    peaks, src = _peaks()
    R = wl["R"]
    sb = 16 if opt == "sgd" else 24  # state bytes per element: h and m (+ v) read and written
    if wl["kind"] == "batched":
        q = wl["q"]
        alg = 0
        for g in inst.graphs:
            n, nnz = g.n, 2 * g.n_edges
            # h, m, v read + written, col, row_ptr, c^f and c^a, argmax words read once + written once
            alg += 24 * q * n * R + 4 * nnz + 4 * (n + 1) + 8 * n + 8 * n * (R * 2 // 32)
        for c in inst.sats:
            n, L, M = c.n, int(c.ptr[-1]), c.n_clauses
            # h, m, v read + written, marginals read once + written once, clause lists and transpose
            alg += 24 * n * R + 8 * n * R + 4 * (n + 1) + 4 * L + 4 * (M + 1) + 4 * L
        ach = alg / (step_ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"],
                "traffic": (_traffic_from_profile("batch_step_bmc256_sat64_R16.md", "batched")
                            if wl is WORKLOADS["batched"] else None),
                "kernel": "k_batch_bmincut<4, paper> + k_batch_sat (the two launches of one step)",
                "algorithmic_bytes_per_launch": alg, "launch_ms": step_ms,
                "peak_source": f"{src} hbm_gbs (copy), of {src}", "frac_of_8TBs": ach / 8000.0}
    if wl["kind"] == "single":
        n, R_, pr = inst.n, R, wl["problem"]
        if pr in ("bmincut", "coloring"):
            q, nnz = wl["q"], 2 * inst.graph.n_edges
            bits = max(1, (q - 1).bit_length())
            wpn = max(1, R_ * bits // 32)
            if grad_mode == "paper":
                # h, m, v read + written, col, row_ptr, c^f and c^a, argmax words read once
                # and written once (+ node weights)
                alg = 24 * q * n * R_ + 4 * nnz + 4 * (n + 1) + 8 * n + 8 * n * wpn
            else:
                # h, m, v read + written, the gathered centred marginals read once and
                # written once, col, row_ptr, argmax words written (+ node weights)
                alg = 24 * q * n * R_ + 8 * q * n * R_ + 4 * nnz + 4 * (n + 1) + 4 * n * wpn
            alg += 4 * n if inst.node_weight is not None else 0
            kernel = f"k_bmincut_step<{q}, {grad_mode}>"
        elif pr == "qubo":
            nnz = 2 * inst.graph.n_edges
            # the exact-mode MaxCut step: h, m, v, the gathered marginals m = tanh(h/2) read
            # once and written once, CSR, sign words, per-node offsets
            alg = 24 * n * R_ + 8 * n * R_ + 4 * nnz + 4 * (n + 1) + 4 * n * (R_ // 32) + 4 * n
            kernel = "k_exact_gather<adam, unit> (QUBO offsets)"
        elif pr == "sat":
            L = inst.units
            # h, m, v, the marginals read once and written once, occurrence pointers and
            # the other-literal table (8 B per occurrence)
            alg = 24 * n * R_ + 8 * n * R_ + 4 * (n + 1) + 8 * L
            kernel = "k_sat_step (four replicas per thread)"
        else:
            L, M = inst.units, inst.clauses.n_clauses
            # h, m, v, the marginals, occurrences, clause pointers and literals, term
            # couplings and fields, each read once
            alg = 24 * n * R_ + 8 * n * R_ + 4 * (n + 1) + 8 * L + 8 * M + 4 * n
            kernel = "k_sat_step (p-spin terms)"
        ach = alg / (step_ms / 1e3) / 1e9
        prof = next((v for k, v in _SINGLE_PROFILES.items() if WORKLOADS.get(k) is wl), None)
        if grad_mode != (wl.get("grad_mode") or "paper"):
            prof = None  # the committed captures are of the workload's own gradient mode
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": _traffic_from_profile(*prof) if prof else None,
                "kernel": kernel,
                "algorithmic_bytes_per_launch": alg, "launch_ms": step_ms,
                "peak_source": f"{src} hbm_gbs (copy), of {src}", "frac_of_8TBs": ach / 8000.0}
    if wl["kind"] == "sparse" and grad_mode == "exact":
        n, nnz = inst.n, 2 * inst.n_edges
        # h, m, v read + written, m = tanh(h/2) read once (its gathers beyond that are
        # traffic, not algorithm) and written once, CSR, sign words written
        alg = sb * n * R + 8 * n * R + 4 * nnz + 4 * (n + 1) + 4 * n * (R // 32)
        ach = alg / (step_ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"],
                "traffic": (_traffic_from_profile("maxcut_step_exact_n1M_R32.md", "exact")
                            if wl is WORKLOADS["sparse"] and opt == "adam" else None),
                "kernel": f"k_exact_gather<{opt}, unit>", "algorithmic_bytes_per_launch": alg,
                "launch_ms": step_ms, "peak_source": f"{src} hbm_gbs (copy), of {src}",
                "frac_of_8TBs": ach / 8000.0}
    if wl["kind"] == "sparse":
        n, nnz = inst.n, 2 * inst.n_edges
        # h, m, v read + written (24 B per node*replica), CSR col (4 B per directed entry),
        # row_ptr, the sign words read once and written once (4 B per node per 32 replicas)
        alg = sb * n * R + 4 * nnz + 4 * (n + 1) + 8 * n * (R // 32)
        ach = alg / (step_ms / 1e3) / 1e9
        # the staged tile kernel runs graphs of >= 4096 groups of four nodes
        groups4 = (n + 3) // 4
        tile = groups4 >= 4096
        kernel = (f"k_paper_tile<{opt}, unit>" if tile
                  else f"k_maxcut_step_paper<{opt}, unit, {4 if groups4 >= 4096 else 1}>")
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"],
                "traffic": (_traffic_from_profile("maxcut_step_sparse_n1M_R32.md", "paper_tile")
                            if wl is WORKLOADS["sparse"] and opt == "adam" else None),
                "kernel": kernel, "algorithmic_bytes_per_launch": alg,
                "launch_ms": step_ms, "peak_source": f"{src} hbm_gbs (copy), of {src}",
                "frac_of_8TBs": ach / 8000.0}
    n = inst.n
    flops = 2.0 * n * n * R * (2 if precision == "bf16x2" else 1)
    ach = flops / (step_ms / 1e3) / 1e12
    if precision == "fp32":
        # CUDA-core fp32: 148 SMs x 128 lanes x 2 flop x 2.032 GHz
        peak, bound, psrc = 148 * 128 * 2 * 2.032e9 / 1e12, "alu", "derived fp32 FMA peak at 2032 MHz"
    else:
        base = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        peak = base * (2.0 if precision == "fp8" else 1.0)
        bound = "tensor"
        psrc = (f"{src} bf16_tflops_sustained" + (" x 2 (nominal fp8/bf16 ratio)" if precision == "fp8" else "")
                + f", of {src}")
    persistent = dense_launch in ("persistent", "persistent_single")
    if dense_launch == "persistent":
        # one launch of CTA pairs runs the whole timed window; figures are per step
        kernel, prof = f"k_dense_anneal_tc<{precision}, pair>", f"dense_anneal_{precision}_pair_sk2000_R1024.md"
    elif persistent:
        kernel, prof = f"k_dense_anneal_tc<{precision}>", f"dense_anneal_{precision}_sk2000_R1024.md"
    else:
        kernel = f"k_dense_step_{'fp32' if precision == 'fp32' else 'tc<' + precision + '>'}"
        prof = f"dense_step_{precision}_sk2000_R1024.md"
    return {"bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": _traffic_from_profile(prof, "dense"),
            "kernel": kernel, "algorithmic_flops_per_step": flops, "step_ms": step_ms,
            "launch": "persistent (one launch per anneal window)" if persistent else "one launch per step",
            "peak_source": psrc}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        """Median SM clock over the samples taken while the GPU was busy (utilisation
        >= 50%; all samples if none was), the maximum clock, and every throttle reason
        seen in any sample."""
        sm, busy, mx, reasons = [], [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                clk = float(f[1])
                mx = float(f[2])
                util = float(f[9])
            except ValueError:
                continue
            sm.append(clk)
            if util >= 50.0:
                busy.append(clk)
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        pick = busy or sm
        return {"sm_mhz": statistics.median(pick) if pick else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm), "samples_busy": len(busy)}


def _dist():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _oracle_problem(wl, inst):
    import oracle as O
    if wl["kind"] == "dense":
        return ("maxcut", inst.dense.astype(np.float64))
    return ("maxcut", O.coupling_matrix(inst.n, inst.ei, inst.ej, inst.w))


def _units_per_replica(wl, inst):
    if wl["kind"] in ("batched", "single"):
        return inst.units
    return inst.n * (inst.n - 1) // 2 if wl["kind"] == "dense" else inst.n_edges


def _host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_part(wl_name, part, nparts, steps, warmup, barrier, queue):
    """One process of the CPU sample: the oracle, unchanged, on this part's share of the
    sample (a block of replicas; for the batched workload every nparts-th member).  The
    processes start their timed region together at the barrier."""
    import oracle as O
    from paper_2412_09285_b300 import instances as I
    from paper_2412_09285_b300.sharding import shard_replicas
    wl = WORKLOADS[wl_name]
    R = wl["R"]
    jobs = []   # (problem, h0 float64, units per replica and step, mode, extra kw)
    if wl["kind"] == "batched":
        inst = _BatchInstance(wl)
        for k, g in enumerate(inst.graphs[:8]):
            if k % nparts == part:
                jobs.append((("bmincut", O.coupling_matrix(g.n, g.ei, g.ej, g.w)),
                             I.initial_fields(g.n, R, seed=k, q=wl["q"]).astype(np.float64), g.n_edges, "paper",
                             dict(lambda_max=1.0)))
        for k, c in enumerate(inst.sats[:4]):
            if (8 + k) % nparts == part:
                jobs.append((("sat", O.sat_arrays(c.ptr, c.lits)), I.initial_fields(c.n, R, seed=k).astype(np.float64),
                             int(c.ptr[-1]), "paper", {}))
    else:
        off, cnt = shard_replicas(R, nparts, part, multiple=1)
        if wl["kind"] == "single":
            small = _SingleInstance(wl, scale=wl["cpu_div"])
            qh = wl["q"] if wl["problem"] in ("bmincut", "coloring") else 1
            h = I.initial_fields(small.n, R, seed=wl["h_seed"], q=qh).astype(np.float64)
            jobs.append((small.oracle_problem(), h[:, off:off + cnt].copy(), small.units,
                         wl.get("grad_mode", "paper"), {}))
        else:
            inst = _instance(wl)
            h = I.initial_fields(inst.n, R, seed=wl["h_seed"]).astype(np.float64)
            jobs.append((_oracle_problem(wl, inst), h[:, off:off + cnt].copy(), _units_per_replica(wl, inst),
                         "paper", {}))
    runs = []
    for prob, h0, units, mode, kw in jobs:
        opt = None
        if warmup:
            h0, opt = O.anneal(prob, h0, max(wl["n_steps"], warmup + steps), t_end=warmup, mode=mode, **kw)
        runs.append((prob, h0, units, mode, kw, opt))
    barrier.wait()
    c0, t0 = time.process_time(), time.perf_counter()
    units_done = 0
    for prob, h0, units, mode, kw, opt in runs:
        O.anneal(prob, h0, max(wl["n_steps"], warmup + steps), t_begin=warmup, t_end=warmup + steps, mode=mode,
                 opt=opt, **kw)
        units_done += units * h0.shape[1] * steps
    queue.put((part, units_done, time.perf_counter() - t0, time.process_time() - c0))


def oracle_on_host_cores(wl_name, steps, warmup=0):
    """The FP64 oracle timed on every host core: one spawned process per core (at most
    one per replica, or per member of the batched sample), each single-threaded and
    running the oracle unchanged on its share; the processes start together.  Returns
    (units, wall of the slowest process, processes)."""
    import multiprocessing as mp
    wl = WORKLOADS[wl_name]
    limit = 12 if wl["kind"] == "batched" else wl["R"]
    nparts = max(1, min(_host_cores(), limit))
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(nparts), ctx.Queue()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:   # one thread per process: the processes are the parallelism
        os.environ[k] = "1"
    try:
        procs = [ctx.Process(target=_oracle_part, args=(wl_name, k, nparts, steps, warmup, barrier, queue))
                 for k in range(nparts)]
        for pr in procs:
            pr.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    res = [queue.get() for _ in procs]
    for pr in procs:
        pr.join()
    return sum(r[1] for r in res), max(r[2] for r in res), nparts


def cpu_baseline(wl, inst):
    """The FP64 oracle as it stands, timed on this host's cores on a bounded sample."""
    name = next(k for k, v in WORKLOADS.items() if v is wl)
    steps = wl["cpu_steps"]
    units, wall, procs = oracle_on_host_cores(name, steps)
    if wl["kind"] == "batched":
        sample = f"first {steps} steps of the first 8 bMinCut and 4 SAT members, all {wl['R']} replicas"
    elif wl["kind"] == "single":
        sample = (f"the same generator at n/{wl['cpu_div']} (n={wl['n'] // wl['cpu_div']}), first {steps} steps, "
                  f"all {wl['R']} replicas")
    else:
        sample = f"first {steps} of {wl['n_steps']} steps, all {wl['R']} replicas, same instance"
    return {"value": units / wall, "unit": METRIC, "cores": procs, "kind": "oracle",
            "sample": f"{sample}; {procs} single-threaded processes on {_host_cores()} host cores, "
                      f"{wall:.1f} s wall"}


def run_reference(args, wl):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    name = next(k for k, v in WORKLOADS.items() if v is wl)
    units, wall, procs = oracle_on_host_cores(name, args.steps, warmup=args.warmup)
    value = units / wall
    if wl["kind"] == "batched":
        sample = "every replica of the first 8 bMinCut and 4 SAT members per step"
    elif wl["kind"] == "single":
        sample = f"the same generator at n/{wl['cpu_div']}, all {wl['R']} replicas per step"
    else:
        sample = f"all {wl['R']} replicas per step, same instance"
    line = {"metric": METRIC, "value": value, "unit": METRIC, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl["name"]},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": procs, "kind": "oracle",
                             "sample": f"{sample}; {procs} single-threaded processes on {_host_cores()} host "
                                       f"cores"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, wl):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2412_09285_b300 import fem
    from paper_2412_09285_b300 import instances as I

    inst = _instance(wl)
    R, n_steps = wl["R"], wl["n_steps"]
    K, Wm = args.steps, args.warmup
    precision = args.precision if wl["kind"] == "dense" else "bf16"
    # weak scaling: the global replica set is R per rank; each rank runs its block of it
    # (shard_fields), and the only exchange is the final best over ranks
    from paper_2412_09285_b300.sharding import shard_fields, shard_replicas
    mult = 128 if wl["kind"] == "dense" else (16 if wl["kind"] == "batched" or wl.get("problem") in
                                              ("bmincut", "coloring", "sat", "pspin") else 32)
    rep_off, _ = shard_replicas(R * ws, ws, rank, multiple=mult)
    if wl["kind"] == "batched":
        h0_host = [shard_fields(x, ws, rank, multiple=mult) for x in inst.h0(wl, replicas=R * ws)]
        h0 = [torch.from_numpy(x).to(dev) for x in h0_host]
        Wm = max(Wm, 8)   # the first call also tunes the work-item size (two steps per candidate)
    else:
        qh = wl["q"] if wl.get("problem") in ("bmincut", "coloring") else 1
        h0_host = shard_fields(I.initial_fields(inst.n, R * ws, seed=wl["h_seed"], q=qh), ws, rank, multiple=mult)
        h0 = torch.from_numpy(h0_host).to(dev)
    stream = torch.cuda.current_stream()
    prob = _make_problem(fem, wl, inst, stream, args.dense_launch)
    grad_mode = args.grad_mode or wl.get("grad_mode") or ("exact" if precision == "bf16x2" else "paper")
    kw = dict(grad_mode=grad_mode, optimizer=args.optimizer, lr=args.lr or {"adam": 0.1, "rmsprop": 0.01, "sgd": 0.05}[
        args.optimizer], precision=precision, schedule=args.schedule)
    if args.optimizer == "sgd":
        kw.update(momentum=0.9)

    def one_anneal(k, events):
        """Fresh fields from the resident h0, then k steps, then the read-out (best
        replica and every replica's energy to the host; the best states stay on the
        device).  Events bracket steps 1..k-1 so the per-launch step time excludes the
        initialisation."""
        prob.anneal(h_init=h0, replicas=R, n_steps=n_steps, t_begin=0, t_end=1, **kw)
        if k > 1:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            prob.anneal(replicas=R, n_steps=n_steps, t_begin=1, t_end=k, **kw)
            e1.record(stream)
            events.append((e0, e1, k - 1))
        return prob.best(states=False)

    # warm-up (untimed): W steps, then one anneal of the timed length, so that the
    # one-time work of a window shape (CUDA-graph capture, first-call tuning) is done
    one_anneal(Wm, [])
    one_anneal(min(K, n_steps), [])
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k_ev = []
    launches0 = fem.fem_kernel_launches()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        done, best = 0, None
        while done < K:
            k = min(n_steps, K - done)
            best = one_anneal(k, k_ev)
            done += k
        end.record(stream)
        torch.cuda.synchronize()
    launches = fem.fem_kernel_launches() - launches0
    t_ms = start.elapsed_time(end)
    step_ms = sum(a.elapsed_time(b) for a, b, _ in k_ev) / max(1, sum(k for _, _, k in k_ev))
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([t_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
        from paper_2412_09285_b300.sharding import best_over_ranks
        # the best replica over all ranks (after timing; one small all_gather)
        g_best = best_over_ranks(float(best["energy_f64"][best["best_replica"]]), rep_off + best["best_replica"],
                                 rank, ws, device=dev)
        best = dict(best, energy_f64=np.array([g_best[0]]), best_replica=0)
    units_per_step = _units_per_replica(wl, inst) * R
    value = units_per_step * K * ws / (t_ms / 1e3)

    # end to end through the public API from host buffers (create + anneal + read-out)
    if wl["kind"] == "batched":
        h0_pinned = [torch.from_numpy(x).pin_memory().numpy() for x in h0_host]
        h0_bytes = sum(x.nbytes for x in h0_host)
    else:
        h0_pinned = torch.from_numpy(h0_host).pin_memory().numpy()
        h0_bytes = h0_host.nbytes
    e2e_steps = min(K, n_steps)
    inst_pinned = _pinned_instance(inst, torch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p2 = _make_problem(fem, wl, inst_pinned, stream, args.dense_launch)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    p2.anneal(h_init=h0_pinned, replicas=R, n_steps=n_steps, t_end=e2e_steps, **kw)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    p2.best()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    phases = {"create": (t1 - t0) * 1e3, "anneal_with_h_init": (t2 - t1) * 1e3, "read_best": (t0 + e2e_s - t2) * 1e3}
    p2.close()
    if wl["kind"] == "dense":
        h2d = h0_bytes + 4 * inst.n * inst.n
    elif wl["kind"] == "single":
        h2d = h0_bytes + inst.host_bytes()
    elif wl["kind"] == "batched":
        h2d = h0_bytes + sum(4 * (g.n + 1) + 8 * g.n_edges for g in inst.graphs) \
            + sum(8 * (c.n_clauses + 1) + 8 * int(c.ptr[-1]) for c in inst.sats)
    else:
        h2d = h0_bytes + 4 * (inst.n + 1) + 8 * inst.n_edges
    d2h = 4 * inst.n + 16 * R + 4
    e2e = {"value": units_per_step * e2e_steps / e2e_s, "unit": METRIC,
           "h2d_bytes_per_step": int(round(h2d / e2e_steps)), "d2h_bytes_per_step": int(round(d2h / e2e_steps)),
           "phases_ms": {k: round(v, 3) for k, v in phases.items()},
           "note": f"one full user call sequence per {e2e_steps} steps: fem_create_problem from pinned host arrays "
                   "(graphs of >= 65536 edges validated and built into CSR on the device), h_init "
                   "from pinned host memory, anneal, fem_read_best (best states and energies) to host"}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": K, "warmup": Wm,
            "ms_per_step": t_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"bf16": "bf16", "fp8": "e4m3", "bf16x2": "bf16x2", "fp32": "f32"}[precision]
            if wl["kind"] == "dense" else "f32",
            "data": "synthetic",
            "config": {"workload": wl["name"] if grad_mode == "paper" or wl["kind"] != "sparse"
                       else wl["name"].replace("paper-mode gradient", "exact gradient"), "n": inst.n, "units_per_replica": _units_per_replica(wl, inst),
                       "replicas_per_gpu": R, "anneal_steps": n_steps,
                       **({"precision": precision} if wl["kind"] == "dense" else {}),
                       "optimizer": f"{kw['optimizer']} lr {kw['lr']}" + (" momentum 0.9" if kw["optimizer"] == "sgd"
                                                                           else ""),
                       "schedule": kw["schedule"],
                       "parallelism": f"replica-sharded x{ws}",
                       "l2": ("working set L2-resident (latency/compute-bound workload)"
                              if wl["kind"] == "dense" or (wl["kind"] == "sparse" and inst.n <= 100000)
                              else "inputs larger than L2")},
            "roofline": _roofline(wl, inst, step_ms, precision,
                                  dense_launch=prob.dense_last_launch() if wl["kind"] == "dense" else None,
                                  grad_mode=grad_mode, opt=kw["optimizer"]), "gpu_launches": int(launches), "e2e": e2e,
            "clocks": clk.summary(),
            "best_energy": float(best["energy_f64"][best["best_replica"]])}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, inst)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _timed(fn):
    """Wall time of fn() in ms with the device drained before and after."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) * 1e3, out


def _ttt_summary(plain, fast, budgets):
    """Per instance: target = plain's best at the full budget; time to target = the
    fastest run (of the budgets tried) whose best is within 0.1% of it."""
    out = []
    for p, f in zip(plain, fast):
        target = p[budgets[-1]][1]
        thr = target - 0.001 * abs(target)
        tp = min(t for b, (t, c) in p.items() if c >= thr)
        tf = [t for b, (t, c) in f.items() if c >= thr]
        out.append((tp, min(tf) if tf else None))
    reached = [x for x in out if x[1] is not None]
    return {"instances": len(out), "reached": len(reached),
            "plain_ms_mean": float(np.mean([x[0] for x in out])),
            "fast_ms_mean_over_reached": float(np.mean([x[1] for x in reached])) if reached else None,
            "speedup_over_reached": float(np.mean([x[0] / x[1] for x in reached])) if reached else None}


def run_ttt(args, wl):
    """Time to target cut (the metric's second part): the reduced-precision (dense), batched
    and warm-started forms against plain FP32 FEM on the same GPU, target = plain FEM's best
    cut at its full budget, within 0.1%.  One JSON line."""
    import torch
    from paper_2412_09285_b300 import fem
    from paper_2412_09285_b300 import instances as I
    dev = torch.device("cuda")
    N = wl["n_steps"]
    line = {"metric": "time-to-target-cut", "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "data": "synthetic", "config": {"workload": wl["name"], "target": "plain FP32 FEM best cut at the full "
                                            "budget, within 0.1%"}}
    pool = None
    if wl["kind"] == "warmstart" and wl["n_train"] + wl["n_held"] > 200:
        import multiprocessing as mp   # graph generation on every host core (spawned processes)
        pool = mp.get_context("spawn").Pool(_host_cores())
    clk = ClockSampler(0)
    clk.__enter__()
    if wl["kind"] == "dense":
        inst = _instance(wl)
        R = wl["R"]
        # end to end: initial fields from pinned host memory, the best replica's states to the host
        h0 = torch.from_numpy(I.initial_fields(inst.n, R, seed=wl["h_seed"])).pin_memory().numpy()
        budgets = [N // 4, N // 2, N]

        def run(prec, b):
            P = fem.Problem("maxcut", dense=inst.dense)
            P.anneal(h_init=h0, replicas=R, n_steps=b, precision=prec)   # compile / first-call effects
            t, r = _timed(lambda: P.anneal(h_init=h0, replicas=R, n_steps=b, precision=prec).best())
            P.close()
            return t, -float(r["energy_f64"][r["best_replica"]])
        plain = {b: run("fp32", b) for b in budgets}
        res = {"fp32": plain}
        for prec in ("bf16", "fp8"):
            res[prec] = {b: run(prec, b) for b in budgets}
        line["time_to_target"] = {prec: _ttt_summary([plain], [res[prec]], budgets) for prec in ("bf16", "fp8")}
        line["best_cut"] = {prec: {str(b): c for b, (t, c) in v.items()} for prec, v in res.items()}
        line["ms"] = {prec: {str(b): t for b, (t, c) in v.items()} for prec, v in res.items()}
        line["value"] = line["time_to_target"]["fp8"]["fast_ms_mean_over_reached"]
        # the plain FP32 FEM that anchors the speed-ups, against the CUDA-core FMA peak
        flops = 2.0 * inst.n * inst.n * R * N
        fma_peak = 148 * 128 * 2 * 2.032e9 / 1e12
        ach = flops / (plain[N][0] / 1e3) / 1e12
        line["plain_fp32_roofline"] = {"bound": "alu", "achieved": ach, "peak": fma_peak, "unit": "TFLOP/s",
                                       "frac": ach / fma_peak, "kernel": "k_dense_step_fp32",
                                       "note": "whole anneal incl. read-out; peak = 148 SMs x 128 FP32 lanes x 2 "
                                               "flop x 2.032 GHz (derived)"}
    elif wl["kind"] == "batched":
        inst = _instance(wl)
        h0 = [torch.from_numpy(x).pin_memory().numpy() for x in inst.h0(wl)]
        R = wl["R"]
        probs = ([fem.Problem("bmincut", graph=g, q=wl["q"]) for g in inst.graphs]
                 + [fem.Problem("sat", clauses=c) for c in inst.sats])
        kw = dict(replicas=R, n_steps=N, lambda_max=1.0)

        def one_by_one():
            out = []
            for p, h in zip(probs, h0):
                p.anneal(h_init=h, **kw)
                r = p.best()
                out.append(float(r["energy_f64"][r["best_replica"]]))
            return out
        B = fem.Batch(probs)

        def batched():
            B.anneal(h_inits=h0, **kw)
            out = []
            for p in probs:
                r = p.best()
                out.append(float(r["energy_f64"][r["best_replica"]]))
            return out
        B.anneal(h_inits=h0, replicas=R, n_steps=N, t_end=20, lambda_max=1.0)  # first-call tuning
        t_plain, e_plain = _timed(one_by_one)
        t_batch, e_batch = _timed(batched)
        line["time_to_target"] = {"plain_ms": t_plain, "batched_ms": t_batch, "speedup": t_plain / t_batch,
                                  "same_best_energies": bool(e_plain == e_batch), "members": len(probs)}
        line["value"] = t_batch
    else:
        from paper_2412_09285_b300 import warmstart as ws
        R, rms = wl["R"], wl["rms"]
        gen = lambda cnt, seed: ws.make_graphs(cnt, wl["n_lo"], wl["n_hi"], wl["deg"], seed=seed, pool=pool)
        t_gen, (train, held) = _timed(lambda: (gen(wl["n_train"], wl["train_seed"]), gen(wl["n_held"], wl["held_seed"])))
        net = ws.Mpnn(seed=1)
        t_train, losses = _timed(lambda: ws.train(net, train, wl["epochs"], R, N, lr=wl["lr"], seed=wl["h_seed"]))
        budgets = [N // 8, N // 4, N // 2, N]
        noise = ws.Mpnn({**I.mpnn_init(0), "C": np.zeros((64, 4)), "c": np.array([1.0, 0.0, 0.0, 0.0])})
        plain, warm, ctrl = [], [], []
        for k, g in enumerate(held):
            z = torch.from_numpy(I.initial_fields(g.n, R, seed=wl["h_seed"] * 1000 + k) * np.float32(1000.0)).to(dev)
            probs = [fem.Problem("maxcut", graph=g) for _ in range(2)]

            def plain_run(b):
                return _timed(lambda: -float(probs[0].anneal(h_init=z * 0.001, replicas=R, n_steps=b)
                                             .best()["energy_f64"].min()))
            y = torch.empty_like(z)

            def warm_run(b, model):
                def go():
                    model.predict(probs[1], z, R, y, rms=rms)
                    ws.warm_anneal(probs[1], y, b, N, N // 4)
                    return -float(probs[1].best()["energy_f64"].min())
                return _timed(go)
            plain_run(budgets[0])  # first-call effects
            plain.append({b: plain_run(b) for b in budgets})
            warm.append({b: warm_run(b, net) for b in budgets})
            ctrl.append({b: warm_run(b, noise) for b in budgets})
            for p in probs:
                p.close()
        gap = lambda runs: {str(b): float(np.mean([(r[b][1] - p[N][1]) / abs(p[N][1]) for r, p in zip(runs, plain)]))
                            for b in budgets}
        line["time_to_target"] = {"warm": _ttt_summary(plain, warm, budgets),
                                  "noise_control": _ttt_summary(plain, ctrl, budgets)}
        line["relative_cut_gap_vs_plain_full"] = {"plain": gap(plain), "warm": gap(warm), "noise_control": gap(ctrl)}
        line["ms_per_budget"] = {"plain": {str(b): float(np.mean([r[b][0] for r in plain])) for b in budgets},
                                 "warm": {str(b): float(np.mean([r[b][0] for r in warm])) for b in budgets}}
        line["train"] = {"graphs": len(train), "epochs": wl["epochs"], "loss_by_epoch": losses,
                         "train_s": t_train / 1e3, "generate_s": t_gen / 1e3, "held_out": len(held)}
        line["value"] = line["time_to_target"]["warm"]["fast_ms_mean_over_reached"]
    clk.__exit__(None, None, None)
    if pool is not None:
        pool.close()
    line["clocks"] = clk.summary()
    line["e2e"] = {"note": "every time is the wall time of the user calls (fem_anneal + fem_read_best) with "
                           + ("initial fields from pinned host memory and the best states read to the host"
                              if wl["kind"] != "warmstart" else "fields on the device and the best energy to the host")}
    print(json.dumps(line))


def mpnn_algorithmic_bytes(n, nnz, R, width=64, feats=4, taps=4):
    """Bytes of one fem_mpnn_predict when every array is read or written once: the CSR
    (once per propagation), the features, three layers (propagation + dense update),
    the head, the taps of P^k z and the output with its rescaling."""
    csr = 4 * (n + 1) + 4 * nnz
    b = csr + 4 * n * feats                                   # features
    for din in (feats, width, width):
        b += csr + 4 * n * din + 4 * n * din                  # a = P x: read x, write a
        b += 4 * n * din * 2 + 4 * n * width                  # x' = tanh(x A + a B + b)
    b += 4 * n * width + 4 * n * taps                         # head
    b += 8 * n * R                                            # u_0 = z
    b += (taps - 1) * (csr + 8 * n * R)                       # u_k = P u_(k-1)
    b += 4 * n * taps + taps * 4 * n * R + 4 * n * R          # y = sum_k theta_k u_k
    b += 3 * 4 * n * R                                        # rms rescaling
    return b


def run_mpnn(args, wl):
    """Inference time of the warm-start network, against the HBM roofline of its
    algorithmic bytes (one JSON line)."""
    import torch
    from paper_2412_09285_b300 import fem
    from paper_2412_09285_b300 import instances as I
    from paper_2412_09285_b300 import warmstart as ws
    dev = torch.device("cuda")
    g = I.er_gnm(wl["n"], wl["m"], seed=wl["graph_seed"], weights="pm1")
    R = wl["R"]
    P = fem.Problem("maxcut", graph=g)
    net = ws.Mpnn(seed=1)
    z = torch.from_numpy(I.initial_fields(g.n, R, seed=wl["h_seed"]) * np.float32(1000.0)).to(dev)
    y = torch.empty_like(z)
    stream = torch.cuda.current_stream()
    K = args.steps or 50
    for _ in range(max(3, args.warmup)):
        net.predict(P, z, R, y, rms=0.1)
    torch.cuda.synchronize()
    l0 = fem.fem_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(K):
            net.predict(P, z, R, y, rms=0.1)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    launches = fem.fem_kernel_launches() - l0
    # end to end: the graph from pinned host arrays, z from pinned memory, the prediction
    # back to pinned host memory
    g_pin = _pinned_instance(g, torch)
    z_host = torch.from_numpy(z.cpu().numpy()).pin_memory()
    y_host = torch.empty(z_host.shape, dtype=z_host.dtype, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P2 = fem.Problem("maxcut", graph=g_pin)
    zd = z_host.to(dev, non_blocking=True)
    yd = torch.empty_like(zd)
    net.predict(P2, zd, R, yd, rms=0.1)
    y_host.copy_(yd, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    P2.close()
    e2e = {"value": g.n_edges * R / e2e_s, "unit": "edge*replica/s",
           "h2d_bytes_per_step": int(12 * g.n_edges + z_host.numel() * 4), "d2h_bytes_per_step": int(y_host.numel() * 4),
           "note": "one call sequence: fem_create_problem from pinned host arrays, z copied from pinned memory, "
                   "fem_mpnn_predict, the prediction copied to pinned host memory"}
    peaks, src = _peaks()
    alg = mpnn_algorithmic_bytes(g.n, 2 * g.n_edges, R)
    ach = alg / (ms / 1e3) / 1e9
    flops = 2 * g.n * (4 * 64 * 2 + 64 * 64 * 2 * 2) + 2 * g.n * 64 * 4
    line = {"metric": "mpnn-predict edge*replica/s", "value": g.n_edges * R / (ms / 1e3),
            "unit": "edge*replica/s", "n_gpus": 1, "steps": K, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "dtype": "bf16 weights, f32 activations", "data": "synthetic",
            "config": {"workload": wl["name"], "n": g.n, "edges": g.n_edges, "replicas": R},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": "fem_mpnn_predict (all launches)",
                         "algorithmic_bytes_per_call": alg, "dense_flops_per_call": flops,
                         "peak_source": f"{src} hbm_gbs (copy), of {src}",
                         "note": "the layer products are n x 64 x 64 (about 7 GFLOP per call at n = 2e5, "
                                 "90 us at the CUDA cores' FP32 FMA peak, 4 us on the tensor cores) against "
                                 "about 1.1 GB of memory passes (170 us at the copy peak): memory-bound"},
            "gpu_launches": int(launches), "launches_per_call": launches / K, "e2e": e2e, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sparse", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp8", "bf16x2", "fp32"])
    ap.add_argument("--grad-mode", default=None, choices=["paper", "exact"],
                    help="sparse workloads: the discretised (paper) or exact gradient (default paper)")
    ap.add_argument("--dense-launch", default="auto", choices=["auto", "per_step", "persistent", "persistent_single"],
                    help="dense workload: persistent (state in tensor memory; CTA pairs where the row tiles "
                         "pair up, persistent_single without pairs) or one kernel per step")
    ap.add_argument("--optimizer", default="adam", choices=["adam", "rmsprop", "sgd"],
                    help="the optimizer of the step (adam lr 0.1, rmsprop lr 0.01, sgd lr 0.05 momentum 0.9)")
    ap.add_argument("--lr", type=float, default=None)
    ap.add_argument("--schedule", default="exponential", choices=["exponential", "inverse_proportional"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ttt", action="store_true",
                    help="time to target cut of the dense, batched or warmstart workload against plain FP32 FEM")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.ttt or wl["kind"] == "warmstart":
        run_ttt(args, wl)
        return
    if wl["kind"] == "mpnn":
        run_mpnn(args, wl)
        return
    if args.steps is None:
        args.steps = wl["n_steps"]
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
