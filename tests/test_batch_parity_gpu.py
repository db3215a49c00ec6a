"""Batched members against the FP64 oracle directly, not only through the same members
annealed alone.

* A small batch (bMinCut on random geometric graphs, q = 4, and random Max-3-SAT, R = 16):
  every member's marginals over the first 50 fp32 steps, with the gates of
  tests/parity.py; the one-step checks of excluded elements run through the batch (every
  member's state written back, one batched step).
* The batched workload at full size, as the benchmark times it (256 bMinCut members with
  n log-uniform in 1k-64k, 64 Max-3-SAT members with n log-uniform in 5k-50k and
  M = 4.2 n, R = 16, paper-mode gradient, lambda_max = 1, generated with the benchmark's
  seeds): after 20 batched steps, one batched step of sampled members (the largest and a
  middle-sized member of each kind) from the GPU's own state against the oracle's step
  from the same state, then the int64 objectives of every member against the oracle's
  recomputation from the GPU's states.
"""
import numpy as np
import pytest

import oracle as O
import parity
from paper_2412_09285_b300 import instances as I

pytestmark = pytest.mark.gpu

CHECK = [1, 2, 5, 10, 20, 35, 50]
N_STEPS = 1000
R = 16
Q = 4
LAM = 1.0


@pytest.fixture(scope="module")
def fem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2412_09285_b300 import build
    build.build()
    from paper_2412_09285_b300 import fem as F
    return F


def _sched(kind):
    s = dict(schedule="exponential", beta_min=0.05, beta_max=5.0, gamma=1.0)
    if kind == "bmincut":
        s["lambda_max"] = LAM
    return s


def _oracle_problem(kind, x):
    if kind == "bmincut":
        return ("bmincut", O.coupling_matrix(x.n, x.ei, x.ej, x.w))
    return ("sat", O.sat_arrays(x.ptr, x.lits))


def _marg(kind):
    return parity.softmax if kind == "bmincut" else parity.sigmoid


class _BatchRun:
    """One batch of members, annealed in windows; keeps every member's state at each
    checkpoint so that a one-step check can restart the whole batch from it."""

    def __init__(self, fem, members, h0s, mode):
        self.members = members
        self.probs = [fem.Problem("bmincut", graph=x, q=Q) if k == "bmincut" else fem.Problem("sat", clauses=x)
                      for k, x in members]
        self.batch = fem.Batch(self.probs)
        self.h0s = h0s
        self.mode = mode
        self.states = {0: [(h, np.zeros_like(h), np.zeros_like(h)) for h in h0s]}

    def anneal(self, t_begin, t_end, h_inits=None):
        self.batch.anneal(h_inits=h_inits, replicas=R, n_steps=N_STEPS, t_begin=t_begin, t_end=t_end,
                          grad_mode=self.mode, lambda_max=LAM)

    def windows(self, checkpoints):
        got, t = {}, 0
        for T in checkpoints:
            self.anneal(t, T, self.h0s if t == 0 else None)
            got[T] = [p.fields() for p in self.probs]
            self.states[T] = [p.state() for p in self.probs]
            t = T
        return got

    def gpu_step(self, k):
        """parity.one_step_from's GPU side for member k: every member restarted from its
        checkpointed state (member k from the given one), then one batched step."""
        def step(T, h, m, v):
            if T == 0:
                h0s = list(self.h0s)
                h0s[k] = h
                self.anneal(0, 1, h0s)
            else:
                for j, p in enumerate(self.probs):
                    hj, mj, vj = (h, m, v) if j == k else self.states[T][j]
                    p.set_state(hj, mj, vj, steps_done=T)
                self.anneal(T, T + 1)
            g, mg, _ = self.probs[k].state()
            return g, mg
        return step

    def forced(self, k):
        kind, x = self.members[k]
        return parity.one_step_from(self.gpu_step(k), _oracle_problem(kind, x), N_STEPS,
                                    mode=self.mode if kind == "bmincut" else "exact", sched=_sched(kind))

    def close(self):
        self.batch.close()
        for p in self.probs:
            p.close()


def _small_members(seed):
    graphs = [I.rgg(int(n), 10.0, seed=seed + 10 + k) for k, n in enumerate(I.loguniform_sizes(3, 300, 1200, seed=seed))]
    sats = [I.random_ksat(int(n), int(4.2 * n), 3, seed=seed + 30 + k)
            for k, n in enumerate(I.loguniform_sizes(2, 400, 1500, seed=seed + 1))]
    members = [("bmincut", g) for g in graphs] + [("sat", c) for c in sats]
    h0s = ([I.initial_fields(g.n, R, seed=seed + 50 + k, q=Q) for k, g in enumerate(graphs)]
           + [I.initial_fields(c.n, R, seed=seed + 70 + k) for k, c in enumerate(sats)])
    return members, h0s


def _agree(got, ref, checkpoints):
    a = np.ones(got[checkpoints[0]].shape[1], bool)
    for t in checkpoints:
        a &= np.all(np.argmax(got[t], axis=2) == np.argmax(ref[t], axis=2), axis=0)
    return a


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_batched_members_first_50_steps(fem, mode):
    members, h0s = _small_members(700)
    run = _BatchRun(fem, members, h0s, mode)
    got = run.windows(CHECK)
    for k, (kind, x) in enumerate(members):
        tr = {t: None for t in CHECK}
        cd = {t: None for t in CHECK}
        mk = mode if kind == "bmincut" else "exact"
        O.anneal(_oracle_problem(kind, x), h0s[k].astype(np.float64), N_STEPS, t_end=max(CHECK),
                 opt_kw=dict(lr=0.1), mode=mk, trace=tr, cond=cd, **_sched(kind))
        gk = {t: got[t][k] for t in CHECK}
        agree = None
        if kind == "bmincut" and mode == "paper":
            agree = _agree(gk, tr, CHECK)
            assert agree.sum() >= R - 2, (k, agree.sum())
        parity.compare_trajectory(gk, tr, cd, CHECK, (mode, kind, k, x.n), marg=_marg(kind), agree=agree,
                                  forced=run.forced(k), state={t: run.states[t][k] for t in [0] + CHECK})
    run.close()


def test_full_size_batch_sampled_members_and_objectives(fem):
    # the batched benchmark workload, with its seeds
    graphs = [I.rgg(int(n), 10.0, seed=5000 + k) for k, n in enumerate(I.loguniform_sizes(256, 1000, 64000, seed=5))]
    sats = [I.random_ksat(int(n), int(round(4.2 * n)), 3, seed=10000 + k)
            for k, n in enumerate(I.loguniform_sizes(64, 5000, 50000, seed=6))]
    members = [("bmincut", g) for g in graphs] + [("sat", c) for c in sats]
    h0s = ([I.initial_fields(g.n, R, seed=600000 + k, q=Q) for k, g in enumerate(graphs)]
           + [I.initial_fields(c.n, R, seed=650000 + k) for k, c in enumerate(sats)])
    run = _BatchRun(fem, members, h0s, "paper")
    T = 20
    run.windows([T])
    nb = len(graphs)
    by_n = lambda ks: sorted(ks, key=lambda k: members[k][1].n)
    bmc, sat = by_n(range(nb)), by_n(range(nb, len(members)))
    for k in (bmc[-1], bmc[len(bmc) // 2], sat[-1], sat[len(sat) // 2]):
        kind, x = members[k]
        step = run.forced(k)
        g1, r1, extra = step(T, run.states[T][k])
        # from the same state the discretised states agree, so every replica is compared
        parity.compare(g1, r1, extra["cond"], ("full size", kind, k, x.n), marg=_marg(kind),
                       forced=lambda _t, _s: (g1, r1, extra), prev=T, prev_state=run.states[T][k])
    # every member's objective of the GPU's own states (all members are now at step T + 1)
    for k, (kind, x) in enumerate(members):
        P = run.probs[k]
        best = P.best()
        if kind == "bmincut":
            E, _, _ = O.bmincut_objective(x.ei, x.ej, x.w, P.states(), Q, LAM)
        else:
            E = O.sat_unsat(x.ptr, x.lits, P.states().astype(np.int8))
        assert np.array_equal(best["energy_i64"], E), (kind, k)
        assert best["best_replica"] == int(np.argmin(E)), (kind, k)
    print(f"PARITY test_batch_parity_gpu::full size objectives: {len(members)} members "
          f"({nb} bMinCut, {len(members) - nb} Max-3-SAT), int64 energies bit-exact")
    run.close()
