"""GPU vs oracle parity for sparse MaxCut, through the C ABI.

Two kinds of field comparison:

* Trajectories (the gate for the workloads' settings: Adam, lr 0.1, beta
  0.05 -> 5): sigmoid(h) within 1e-4 max-abs over the first 50 fp32 steps from
  the same h0 - in exact mode on every well-conditioned element, in paper mode on
  every replica whose discrete trajectory agrees with the oracle's.
* Teacher-forced windows (every optimizer and schedule): the oracle's fp64 state
  at step t0, rounded to fp32, is written into the GPU problem; both sides then
  run 3 steps and must agree within 1e-4.  With the paper's aggressive RMSprop /
  SGD settings the fp32-vs-fp64 trajectory itself diverges (the dynamics amplify
  a 1e-8 rounding difference by orders of magnitude over tens of steps), so
  comparing whole trajectories there would test chaos, not the kernel.

Conditioning (tests/parity.py): elements whose oracle optimizer denominator fell
below 1e-6 are capped in number, loosely bounded along the trajectory, and checked at
1e-4 by one step from the GPU's own state at the previous checkpoint.

Objectives: bit-exact (int64) for the GPU's own discrete states.
"""
import numpy as np
import pytest

import oracle as O
import parity
from paper_2412_09285_b300 import instances as I

pytestmark = pytest.mark.gpu

CHECK = [1, 2, 5, 10, 20, 35, 50]


@pytest.fixture(scope="module")
def fem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2412_09285_b300 import build
    build.build()
    from paper_2412_09285_b300 import fem as F
    return F


def _check_marginals(got, ref, cond, where, agree=None, forced=None, prev=None, prev_state=None):
    return parity.compare(got, ref, cond, where, agree=agree, forced=forced, prev=prev,
                          prev_state=prev_state)


def _okw(kw):
    return {k: kw[k] for k in ("lr", "beta1", "beta2", "eps", "weight_decay", "momentum", "alpha",
                               "dampening") if k in kw} or dict(lr=0.1)


def _sched(kw):
    return dict(schedule=kw.get("schedule", "exponential"), beta_min=kw.get("beta_min", 0.05),
                beta_max=kw.get("beta_max", 5.0), gamma=kw.get("gamma_grad", 1.0))


def _gpu_trace(fem, graph, h0, checkpoints, n_steps, **kw):
    P = fem.Problem("maxcut", graph=graph)
    got, state = parity.gpu_windows(P, h0, checkpoints, n_steps, **kw)
    return P, got, state


def _forced(P, graph, n_steps, mode, **kw):
    """One step on both sides from a given fp32 state (parity.one_step)."""
    W = O.coupling_matrix(graph.n, graph.ei, graph.ej, graph.w)
    run = {k: v for k, v in kw.items() if k != "optimizer"}
    return parity.one_step(P, ("maxcut", W), n_steps, optimizer=kw.get("optimizer", "adam"),
                           opt_kw=_okw(kw), mode=mode, sched=_sched(kw), grad_mode=mode, **run)


def _oracle_trace(graph, h0, checkpoints, n_steps, mode, **kw):
    W = O.coupling_matrix(graph.n, graph.ei, graph.ej, graph.w)
    tr = {t: None for t in checkpoints}
    cd = {t: None for t in checkpoints}
    O.anneal(("maxcut", W), h0.astype(np.float64), n_steps, t_end=max(checkpoints),
             optimizer=kw.get("optimizer", "adam"), opt_kw=_okw(kw), mode=mode, trace=tr, cond=cd,
             **_sched(kw))
    return tr, cd


def _agreeing_replicas(got, ref, checkpoints):
    agree = np.ones(got[checkpoints[0]].shape[1], bool)
    for t in checkpoints:
        agree &= np.all((got[t] >= 0) == (ref[t] >= 0), axis=0)
    return agree


# ------------------------------------------------------------ trajectories

@pytest.mark.parametrize("weights", ["unit", "pm1", "real"])
def test_exact_mode_marginals_first_50_steps(fem, weights):
    g = I.er_gnp(800, 0.06, seed=1, weights=weights)
    h0 = I.initial_fields(800, 32, seed=2)
    P, got, st = _gpu_trace(fem, g, h0, CHECK, 1000, grad_mode="exact", lr=0.1)
    ref, cd = _oracle_trace(g, h0, CHECK, 1000, "exact", lr=0.1)
    parity.compare_trajectory(got, ref, cd, CHECK, weights, state=st,
                              forced=_forced(P, g, 1000, "exact", lr=0.1))


@pytest.mark.parametrize("weights", ["unit", "pm1", "real"])
def test_paper_mode_marginals_first_50_steps(fem, weights):
    g = I.er_gnp(800, 0.06, seed=3, weights=weights)
    h0 = I.initial_fields(800, 32, seed=4)
    P, got, st = _gpu_trace(fem, g, h0, CHECK, 1000, grad_mode="paper", lr=0.1)
    ref, cd = _oracle_trace(g, h0, CHECK, 1000, "paper", lr=0.1)
    agree = _agreeing_replicas(got, ref, CHECK)
    assert agree.sum() >= 30, agree.sum()      # sign disagreements are rare near-ties
    parity.compare_trajectory(got, ref, cd, CHECK, weights, agree=agree, state=st,
                              forced=_forced(P, g, 1000, "paper", lr=0.1))


# ------------------------------------------------ teacher-forced step windows

OPTIMIZER_CASES = [
    ("rmsprop", dict(lr=0.03, alpha=0.56, momentum=0.63, weight_decay=0.013,
                     schedule="inverse_proportional", beta_min=1 / 1.16, beta_max=1 / 6e-5)),
    ("rmsprop", dict(lr=0.01, alpha=0.99, momentum=0.0)),
    ("sgd", dict(lr=0.5, momentum=0.71, dampening=0.11, weight_decay=0.018, gamma_grad=6.0,
                 schedule="inverse_proportional", beta_min=1 / 0.63, beta_max=1e5)),
    # lr * gamma / (4 beta_min) != 1: at exactly 1 the first step maps h to h * m^2 ~ 0 on
    # nodes whose discretised neighbourhood sums to 0, a sign decided by rounding alone
    ("sgd", dict(lr=0.13, momentum=0.0)),
    ("adam", dict(lr=0.05, beta1=0.8, beta2=0.99, eps=1e-6, weight_decay=0.01, gamma_grad=2.0)),
    ("adam", dict(lr=0.1)),
]


@pytest.mark.parametrize("mode", ["exact", "paper"])
@pytest.mark.parametrize("opt,kw", OPTIMIZER_CASES)
def test_teacher_forced_windows(fem, opt, kw, mode):
    g = I.er_gnp(500, 0.05, seed=5, weights="pm1")
    W = O.coupling_matrix(g.n, g.ei, g.ej, g.w)
    h0 = I.initial_fields(500, 64, seed=6)
    n_steps = 1000
    P = fem.Problem("maxcut", graph=g)
    P.anneal(h_init=h0, n_steps=n_steps, t_end=0, grad_mode=mode, optimizer=opt, **kw)
    h, o = O.anneal(("maxcut", W), h0.astype(np.float64), n_steps, t_end=0, optimizer=opt,
                    opt_kw=_okw(kw), mode=mode, **_sched(kw))
    t = 0
    for t0 in (0, 7, 30, 120, 600):
        if t0 > t:
            h, o = O.anneal(("maxcut", W), h, n_steps, t_begin=t, t_end=t0, optimizer=opt, opt=o,
                            mode=mode, **_sched(kw))
        # round the oracle's state to fp32, give the same state to both sides
        m, v = parity.opt_state(o)
        h32, m32, v32 = (x.astype(np.float32) for x in (h, m, v))
        h = h32.astype(np.float64)
        parity.set_opt_state(o, m32.astype(np.float64), v32.astype(np.float64))
        cd = {t0 + 3: None}
        h, o = O.anneal(("maxcut", W), h, n_steps, t_begin=t0, t_end=t0 + 3, optimizer=opt, opt=o,
                        mode=mode, cond=cd, **_sched(kw))
        if t0 == 0:   # a step count of 0 is a fresh start: fields from h_init, zero state
            P.anneal(h_init=h32, n_steps=n_steps, t_end=3, grad_mode=mode, optimizer=opt, **kw)
        else:
            P.set_state(h32, m32, v32, steps_done=t0)
            P.anneal(n_steps=n_steps, t_begin=t0, t_end=t0 + 3, grad_mode=mode, optimizer=opt,
                     replicas=64, **kw)
        got = P.fields()
        agree = np.all((got >= 0) == (h >= 0), axis=0) if mode == "paper" else None
        if agree is not None:
            assert agree.sum() >= 56, (t0, agree.sum())
        # a fresh conditioning record for the window (denominators of the 3 steps)
        _check_marginals(got, h, cd[t0 + 3], (opt, mode, t0), agree,
                         forced=_forced(P, g, n_steps, mode, optimizer=opt, **kw), prev=t0,
                         prev_state=(h32, m32, v32))
        t = t0 + 3


# ------------------------------------------------------------- objectives

@pytest.mark.parametrize("weights", ["unit", "pm1", "int3", "real"])
def test_objectives_bit_exact_after_full_anneal(fem, weights):
    wk = "real" if weights == "real" else ("unit" if weights == "int3" else weights)
    g = I.er_gnp(800, 0.06, seed=7, weights=wk)
    if weights == "int3":
        g.w = np.random.Generator(np.random.PCG64(8)).integers(1, 4, g.n_edges).astype(np.float64)
    h0 = I.initial_fields(800, 32, seed=9)
    P = fem.Problem("maxcut", graph=g)
    P.anneal(h_init=h0, n_steps=1000, grad_mode="paper")
    states = P.states()
    h = P.fields()
    assert np.array_equal(states, np.where(h >= 0, 1, -1))
    res = P.best()
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, states.astype(np.int8))
    if weights == "real":
        assert np.allclose(-res["energy_f64"], cut, rtol=1e-12)
    else:
        assert np.array_equal(-res["energy_i64"], cut)
        assert np.array_equal(res["energy_f64"], res["energy_i64"].astype(np.float64))
    best = O.best_replica(-cut)
    assert res["best_replica"] == best
    assert np.array_equal(res["states"], states[:, best])
    # the anneal actually solves something: the best cut beats a random partition clearly
    assert cut.max() > 0.55 * g.w.sum()


@pytest.mark.parametrize("mode", ["paper", "exact"])
def test_resume_and_checkpoint_are_bit_identical(fem, mode):
    g = I.er_gnp(600, 0.05, seed=10, weights="pm1")
    h0 = I.initial_fields(600, 32, seed=11)
    a = fem.Problem("maxcut", graph=g).anneal(h_init=h0, n_steps=400, grad_mode=mode)
    b = fem.Problem("maxcut", graph=g)
    b.anneal(h_init=h0, n_steps=400, t_end=123, grad_mode=mode)
    b.anneal(n_steps=400, t_begin=123, t_end=400, grad_mode=mode, replicas=32)
    assert np.array_equal(a.fields(), b.fields())
    # checkpoint at 201, restore into a fresh problem, finish there
    c = fem.Problem("maxcut", graph=g)
    c.anneal(h_init=h0, n_steps=400, t_end=201, grad_mode=mode)
    ck = c.state()
    assert c.info()["steps_done"] == 201
    d = fem.Problem("maxcut", graph=g)
    d.anneal(h_init=h0, n_steps=400, t_end=0, grad_mode=mode)
    d.set_state(*ck, steps_done=201)
    d.anneal(n_steps=400, t_begin=201, grad_mode=mode, replicas=32)
    assert np.array_equal(a.fields(), d.fields())
    assert np.array_equal(a.best()["energy_i64"], d.best()["energy_i64"])


@pytest.mark.parametrize("n,p,R", [(1, 0.0, 32), (37, 0.0, 32), (300, 0.004, 64), (257, 0.03, 96)])
def test_edge_cases_isolated_empty_multiword(fem, n, p, R):
    g = I.er_gnp(n, p, seed=12, weights="pm1")
    h0 = I.initial_fields(n, R, seed=13)
    P, got, st = _gpu_trace(fem, g, h0, [1, 10, 50], 200, grad_mode="exact")
    ref, cd = _oracle_trace(g, h0, [1, 10, 50], 200, "exact", lr=0.1)
    parity.compare_trajectory(got, ref, cd, [1, 10, 50], n, state=st,
                              forced=_forced(P, g, 200, "exact", lr=0.1))
    P = fem.Problem("maxcut", graph=g).anneal(h_init=h0, n_steps=200, grad_mode="paper")
    res = P.best()
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, P.states().astype(np.int8))
    assert np.array_equal(-res["energy_i64"], cut)


def test_error_paths(fem):
    g = I.er_gnp(100, 0.05, seed=14, weights="pm1")
    P = fem.Problem("maxcut", graph=g)
    with pytest.raises(fem.FemError) as e:
        P.best()
    assert e.value.status == fem.FEM_ERR_STATE
    with pytest.raises(fem.FemError) as e:
        P.set_state(np.zeros((100, 32), np.float32))
    assert e.value.status == fem.FEM_ERR_STATE
    with pytest.raises(fem.FemError) as e:
        P.anneal(h_init=I.initial_fields(100, 48, seed=1), n_steps=10)
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    P.anneal(h_init=I.initial_fields(100, 32, seed=1), n_steps=10, t_end=5)
    with pytest.raises(fem.FemError) as e:
        P.anneal(n_steps=10, t_begin=4, replicas=32)
    assert e.value.status == fem.FEM_ERR_STATE
    with pytest.raises(fem.FemError) as e:
        P.set_state(np.zeros((100, 32), np.float32), steps_done=11)
    assert e.value.status == fem.FEM_ERR_INVALID_ARG
    P.sync()


def _with_hubs(g, hubs, width, seed):
    """g plus `hubs` nodes each joined to `width` random others with +-1 weights."""
    rng = np.random.Generator(np.random.PCG64(seed))
    have = {(a, b): x for a, b, x in zip(g.ei.tolist(), g.ej.tolist(), g.w.tolist())}
    for h in rng.choice(g.n, hubs, replace=False).tolist():
        for j in rng.choice(g.n, width, replace=False).tolist():
            if j != h:
                have.setdefault((min(h, j), max(h, j)), float(rng.choice([-1.0, 1.0])))
    e = sorted(have)
    return I.Graph(g.n, [a for a, _ in e], [b for _, b in e], [have[k] for k in e])


@pytest.mark.parametrize("R", [32, 64])
def test_exact_mode_grouped_nodes_with_hubs(fem, R):
    """Exact mode at mid size (n = 20000, mean degree 6) with 40 hubs of degree ~100,
    whose neighbour lists span several 32-entry chunks; R = 64 gives two replica words
    per node."""
    g = _with_hubs(I.er_gnm(20000, 60000, seed=31, weights="pm1"), 40, 100, seed=32)
    h0 = I.initial_fields(g.n, R, seed=33)
    P, got, st = _gpu_trace(fem, g, h0, [1, 10, 50], 1000, grad_mode="exact")
    ref, cd = _oracle_trace(g, h0, [1, 10, 50], 1000, "exact", lr=0.1)
    parity.compare_trajectory(got, ref, cd, [1, 10, 50], R, state=st,
                              forced=_forced(P, g, 1000, "exact", lr=0.1))


def test_full_size_sparse_steps_match_oracle(fem):
    """N = 2^20, mean degree 6, +-1 weights, R = 32 (the sparse-at-scale
    workload) in the launch configuration the benchmark times: every element
    of the first 3 steps against the oracle, then exact objectives after 30."""
    n = 1 << 20
    g = I.er_gnm(n, 3 * n, seed=2024, weights="pm1")
    h0 = I.initial_fields(n, 32, seed=2025)
    for mode in ("paper", "exact"):
        P, got, st = _gpu_trace(fem, g, h0, [1, 2, 3], 2000, grad_mode=mode)
        ref, cd = _oracle_trace(g, h0, [1, 2, 3], 2000, mode, lr=0.1)
        agree = _agreeing_replicas(got, ref, [1, 2, 3]) if mode == "paper" else None
        if agree is not None:
            assert agree.sum() >= 28
        parity.compare_trajectory(got, ref, cd, [1, 2, 3], mode, agree=agree, state=st,
                                  forced=_forced(P, g, 2000, mode, lr=0.1))
        del P, st
    P = fem.Problem("maxcut", graph=g).anneal(h_init=h0, n_steps=2000, t_end=30)
    st = P.states()
    res = P.best()
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, st.astype(np.int8))
    assert np.array_equal(-res["energy_i64"], cut)
