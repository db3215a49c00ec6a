"""GPU vs oracle parity for balanced q-way MinCut (softmax fields), through the C ABI.

Same gates as the MaxCut tests: softmax marginals within 1e-4 max-abs over the
first 50 fp32 steps (the workloads' Adam settings; well-conditioned elements;
paper mode on replicas whose discrete trajectory agrees), teacher-forced 3-step
windows for the other optimizers, and bit-exact int64 energies
E = cut + lambda_max * sum_s n_s (n_s - 1) for the GPU's own states.
"""
import numpy as np
import pytest

import oracle as O
import parity
from paper_2412_09285_b300 import instances as I

pytestmark = pytest.mark.gpu

# The kernel evaluates every difference of the centred gradient without cancellation
# (integer counts, fixed-point column sums, expm1 deviations), so its gradient error is
# ~1e-9; conditioning and the one-step check of excluded elements: tests/parity.py.
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


def _check(got, ref, cond, where, agree=None, mode="paper", forced=None, prev=None, prev_state=None):
    return parity.compare(got, ref, cond, where, marg=parity.softmax, agree=agree, forced=forced,
                          prev=prev, prev_state=prev_state)


def _okw(kw):
    return {k: kw[k] for k in ("lr", "beta1", "beta2", "eps", "weight_decay", "momentum", "alpha",
                               "dampening") if k in kw} or dict(lr=0.1)


def _sched(kw):
    return dict(schedule=kw.get("schedule", "exponential"), beta_min=kw.get("beta_min", 0.05),
                beta_max=kw.get("beta_max", 5.0), gamma=kw.get("gamma_grad", 1.0),
                lambda_max=kw.get("lambda_max", 1.0))


def _problem(g, V=None):
    W = O.coupling_matrix(g.n, g.ei, g.ej, g.w)
    return ("bmincut", W) if V is None else ("bmincut", W, V)


def _forced(P, g, n_steps, mode, V=None, **kw):
    """One step on both sides from a given fp32 state (parity.one_step)."""
    run = {k: v for k, v in kw.items() if k != "optimizer"}
    return parity.one_step(P, _problem(g, V), n_steps, optimizer=kw.get("optimizer", "adam"),
                           opt_kw=_okw(kw), mode=mode, sched=_sched(kw), grad_mode=mode, **run)


def _traces(fem, g, h0, q, checkpoints, n_steps, mode, V=None, **kw):
    P = fem.Problem("bmincut", graph=g, q=q, node_weight=V)
    got, st = parity.gpu_windows(P, h0, checkpoints, n_steps, grad_mode=mode, **kw)
    tr = {t: None for t in checkpoints}
    cd = {t: None for t in checkpoints}
    O.anneal(_problem(g, V), h0.astype(np.float64), n_steps, t_end=max(checkpoints),
             optimizer=kw.get("optimizer", "adam"), opt_kw=_okw(kw), mode=mode, trace=tr, cond=cd,
             **_sched(kw))
    return P, got, tr, cd, st


def _agree(got, ref, checkpoints):
    a = np.ones(got[checkpoints[0]].shape[1], bool)
    for t in checkpoints:
        a &= np.all(np.argmax(got[t], axis=2) == np.argmax(ref[t], axis=2), axis=0)
    return a


@pytest.mark.parametrize("q", [4, 2, 3, 5, 6, 8])
def test_exact_mode_marginals_first_50_steps(fem, q):
    g = I.rgg(1000, 10.0, seed=21)
    R = 32 if q == 2 else 16
    h0 = I.initial_fields(1000, R, seed=22, q=q)
    P, got, ref, cd, st = _traces(fem, g, h0, q, CHECK, 1000, "exact", lr=0.1)
    parity.compare_trajectory(got, ref, cd, CHECK, q, marg=parity.softmax, state=st,
                              forced=_forced(P, g, 1000, "exact", lr=0.1))


@pytest.mark.parametrize("q,lam", [(4, 1.0), (4, 0.05), (8, 0.2)])
def test_paper_mode_marginals_first_50_steps(fem, q, lam):
    g = I.rgg(1200, 10.0, seed=23)
    R = 16 if q <= 4 else 32
    h0 = I.initial_fields(1200, R, seed=24, q=q)
    P, got, ref, cd, st = _traces(fem, g, h0, q, CHECK, 1000, "paper", lr=0.1, lambda_max=lam)
    agree = _agree(got, ref, CHECK)
    assert agree.sum() >= R - 2, agree.sum()
    parity.compare_trajectory(got, ref, cd, CHECK, (q, lam), marg=parity.softmax, agree=agree, state=st,
                              forced=_forced(P, g, 1000, "paper", lr=0.1, lambda_max=lam))


@pytest.mark.parametrize("q", [5, 6, 8])
def test_paper_mode_two_word_states(fem, q):
    """q = 5..8 at R = 16: four bits per replica, two packed words per node, neighbour
    counts from the bit planes of each word; q = 6 and 8 move their fields as float2 /
    float4.  Marginals against the oracle over 50 steps, then int64 energies of the
    GPU's own states after an anneal."""
    g = I.rgg(1200, 10.0, seed=25)
    R = 16
    h0 = I.initial_fields(1200, R, seed=26, q=q)
    P, got, ref, cd, st = _traces(fem, g, h0, q, CHECK, 1000, "paper", lr=0.1, lambda_max=0.2)
    agree = _agree(got, ref, CHECK)
    assert agree.sum() >= R - 2, agree.sum()
    parity.compare_trajectory(got, ref, cd, CHECK, q, marg=parity.softmax, agree=agree, state=st,
                              forced=_forced(P, g, 1000, "paper", lr=0.1, lambda_max=0.2))
    P = fem.Problem("bmincut", graph=g, q=q).anneal(h_init=h0, n_steps=300, lambda_max=1.0)
    st = P.states()
    assert np.array_equal(st, np.argmax(P.fields(), axis=2))
    E, _, _ = O.bmincut_objective(g.ei, g.ej, g.w, st, q, 1.0)
    assert np.array_equal(P.best()["energy_i64"], E)


@pytest.mark.parametrize("mode", ["exact", "paper"])
@pytest.mark.parametrize("opt,kw", [
    ("adam", dict(lr=0.1)),
    ("rmsprop", dict(lr=0.02, alpha=0.9, momentum=0.5, weight_decay=0.01)),
    ("sgd", dict(lr=0.5, momentum=0.6, dampening=0.1, schedule="inverse_proportional",
                 beta_min=0.1, beta_max=20.0, gamma_grad=3.0)),
])
def test_teacher_forced_windows(fem, opt, kw, mode):
    q = 4
    g = I.rgg(800, 10.0, seed=25)
    W = O.coupling_matrix(g.n, g.ei, g.ej, g.w)
    h0 = I.initial_fields(800, 16, seed=26, q=q)
    n_steps = 1000
    P = fem.Problem("bmincut", graph=g, q=q)
    P.anneal(h_init=h0, n_steps=n_steps, t_end=0, grad_mode=mode, optimizer=opt, **kw)
    h, o = O.anneal(("bmincut", W), h0.astype(np.float64), n_steps, t_end=0, optimizer=opt,
                    opt_kw=_okw(kw), mode=mode, **_sched(kw))
    t = 0
    for t0 in (0, 9, 40, 300, 800):
        if t0 > t:
            h, o = O.anneal(("bmincut", W), h, n_steps, t_begin=t, t_end=t0, optimizer=opt, opt=o,
                            mode=mode, **_sched(kw))
        m, v = parity.opt_state(o)
        h32, m32, v32 = (x.astype(np.float32) for x in (h, m, v))
        h = h32.astype(np.float64)
        parity.set_opt_state(o, m32.astype(np.float64), v32.astype(np.float64))
        cd = {t0 + 3: None}
        h, o = O.anneal(("bmincut", W), h, n_steps, t_begin=t0, t_end=t0 + 3, optimizer=opt, opt=o,
                        mode=mode, cond=cd, **_sched(kw))
        if t0 == 0:   # a step count of 0 is a fresh start: fields from h_init, zero state
            P.anneal(h_init=h32, n_steps=n_steps, t_end=3, grad_mode=mode, optimizer=opt, **kw)
        else:
            P.set_state(h32, m32, v32, steps_done=t0)
            P.anneal(n_steps=n_steps, t_begin=t0, t_end=t0 + 3, grad_mode=mode, optimizer=opt,
                     replicas=16, **kw)
        got = P.fields()
        agree = (np.all(np.argmax(got, 2) == np.argmax(h, 2), axis=0) if mode == "paper" else None)
        if agree is not None:
            assert agree.sum() >= 14, (t0, agree.sum())
        _check(got, h, cd[t0 + 3], (opt, mode, t0), agree, mode=mode,
               forced=_forced(P, g, n_steps, mode, optimizer=opt, **kw), prev=t0,
               prev_state=(h32, m32, v32))
        t = t0 + 3


@pytest.mark.parametrize("q,R,lam,weights", [(4, 16, 1.0, "unit"), (4, 32, 0.5, "int"),
                                             (2, 32, 1.0, "unit"), (3, 16, 2.0, "real"),
                                             (8, 16, 1.0, "unit")])
def test_objectives_bit_exact_after_full_anneal(fem, q, R, lam, weights):
    g = I.rgg(1500, 8.0, seed=27)
    if weights == "int":
        g.w = np.random.Generator(np.random.PCG64(28)).integers(1, 5, g.n_edges).astype(np.float64)
    elif weights == "real":
        g.w = np.random.Generator(np.random.PCG64(28)).uniform(0.5, 2.0, g.n_edges)
    h0 = I.initial_fields(1500, R, seed=29, q=q)
    P = fem.Problem("bmincut", graph=g, q=q)
    P.anneal(h_init=h0, n_steps=600, grad_mode="paper", lambda_max=lam)
    st = P.states()
    assert np.array_equal(st, np.argmax(P.fields(), axis=2))
    E, cut, sizes = O.bmincut_objective(g.ei, g.ej, g.w, st, q, lam)
    res = P.best()
    if weights != "real" and float(lam).is_integer():
        assert np.array_equal(res["energy_i64"], E)
    else:
        assert np.allclose(res["energy_f64"], E, rtol=1e-12)
    b = O.best_replica(E)
    assert res["best_replica"] == b
    assert np.array_equal(res["states"], st[:, b])


@pytest.mark.parametrize("mode", ["paper", "exact"])
def test_resume_and_checkpoint_bit_identical(fem, mode):
    q = 4
    g = I.rgg(700, 9.0, seed=30)
    h0 = I.initial_fields(700, 16, seed=31, q=q)
    a = fem.Problem("bmincut", graph=g, q=q).anneal(h_init=h0, n_steps=300, grad_mode=mode)
    b = fem.Problem("bmincut", graph=g, q=q)
    b.anneal(h_init=h0, n_steps=300, t_end=101, grad_mode=mode)
    b.anneal(n_steps=300, t_begin=101, grad_mode=mode, replicas=16)
    assert np.array_equal(a.fields(), b.fields())
    c = fem.Problem("bmincut", graph=g, q=q)
    c.anneal(h_init=h0, n_steps=300, t_end=157, grad_mode=mode)
    ck = c.state()
    d = fem.Problem("bmincut", graph=g, q=q)
    d.anneal(h_init=h0, n_steps=300, t_end=0, grad_mode=mode)
    d.set_state(*ck, steps_done=157)
    d.anneal(n_steps=300, t_begin=157, grad_mode=mode, replicas=16)
    assert np.array_equal(a.fields(), d.fields())


def test_gradient_mode_and_replica_count_switches_on_one_problem(fem):
    """One problem annealed in paper mode, then exact mode (its exact-mode buffers are
    allocated on first use), then exact mode with more replicas (every buffer
    reallocated), then paper mode again: each result equals a fresh problem's."""
    q = 4
    g = I.rgg(900, 9.0, seed=40)
    runs = [("paper", 16), ("exact", 16), ("exact", 32), ("paper", 32)]
    p = fem.Problem("bmincut", graph=g, q=q)
    for mode, R in runs:
        h0 = I.initial_fields(900, R, seed=41 + R, q=q)
        p.anneal(h_init=h0, n_steps=120, grad_mode=mode)
        fresh = fem.Problem("bmincut", graph=g, q=q).anneal(h_init=h0, n_steps=120, grad_mode=mode)
        assert np.array_equal(p.fields(), fresh.fields()), (mode, R)
        assert np.array_equal(p.best()["energy_i64"], fresh.best()["energy_i64"]), (mode, R)


def test_bmincut_reaches_bruteforce_optimum(fem):
    g = I.rgg(9, 4.0, seed=45)
    q, lam = 3, 1.0
    best = O.bmincut_bruteforce(g.n, g.ei, g.ej, g.w, q, lam)
    h0 = I.initial_fields(9, 32, seed=145, q=q)
    P = fem.Problem("bmincut", graph=g, q=q).anneal(h_init=h0, n_steps=1000, grad_mode="paper",
                                                     lambda_max=lam)
    assert P.best()["energy_i64"].min() == best


def test_bmincut_argument_errors(fem):
    g = I.rgg(100, 6.0, seed=32)
    P = fem.Problem("bmincut", graph=g, q=4)
    with pytest.raises(fem.FemError) as e:
        P.anneal(h_init=I.initial_fields(100, 8, seed=1, q=4), n_steps=10)
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    with pytest.raises(fem.FemError) as e:
        P.anneal(h_init=I.initial_fields(100, 16, seed=1, q=4), n_steps=10, lambda_max=-1.0)
    assert e.value.status == fem.FEM_ERR_INVALID_ARG



# ---- node-weighted bMinCut (SM, the FPGA task's community graphs)

def _node_weights(n, seed):
    return np.random.Generator(np.random.PCG64(seed)).integers(1, 6, size=n).astype(np.float64)


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_weighted_marginals_first_50_steps(fem, mode):
    g = I.rgg(800, 10.0, seed=81)
    V = _node_weights(800, 82)
    h0 = I.initial_fields(800, 16, seed=83, q=4)
    P, got, ref, cd, st = _traces(fem, g, h0, 4, CHECK, 1000, mode, V=V, lr=0.1, lambda_max=0.05)
    agree = _agree(got, ref, CHECK) if mode == "paper" else None
    if agree is not None:
        assert agree.sum() >= 12, agree.sum()
    parity.compare_trajectory(got, ref, cd, CHECK, mode, marg=parity.softmax, agree=agree, state=st,
                              forced=_forced(P, g, 1000, mode, V=V, lr=0.1, lambda_max=0.05))


def test_weighted_objectives_bit_exact_and_unit_weights_change_nothing(fem):
    g = I.rgg(900, 10.0, seed=84)
    V = _node_weights(900, 85)
    h0 = I.initial_fields(900, 16, seed=86, q=4)
    P = fem.Problem("bmincut", graph=g, q=4, node_weight=V).anneal(h_init=h0, n_steps=200, lambda_max=0.01)
    st = P.states()
    E, cut, sizes = O.bmincut_objective(g.ei, g.ej, g.w, st, 4, 0.01, V=V.astype(np.int64))
    res = P.best()
    assert np.allclose(res["energy_f64"], E, rtol=0, atol=1e-9 * np.abs(E).max())
    assert res["best_replica"] == int(np.argmin(E))
    # an integer lambda_max gives exact int64 energies
    P1 = fem.Problem("bmincut", graph=g, q=4, node_weight=V).anneal(h_init=h0, n_steps=50, lambda_max=1.0)
    E1, _, _ = O.bmincut_objective(g.ei, g.ej, g.w, P1.states(), 4, 1.0, V=V.astype(np.int64))
    assert np.array_equal(P1.best()["energy_i64"], E1)
    # V = 1 is the unweighted problem, bit for bit
    a = fem.Problem("bmincut", graph=g, q=4, node_weight=np.ones(900)).anneal(h_init=h0, n_steps=60).state()
    b = fem.Problem("bmincut", graph=g, q=4).anneal(h_init=h0, n_steps=60).state()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_weighted_member_in_a_batch_equals_alone(fem):
    gs = [I.rgg(700, 10.0, seed=87 + k) for k in range(3)]
    Vs = [_node_weights(700, 90 + k) if k != 1 else None for k in range(3)]
    h0 = [I.initial_fields(700, 16, seed=93 + k, q=4) for k in range(3)]
    alone = [fem.Problem("bmincut", graph=g, q=4, node_weight=V).anneal(h_init=h, n_steps=80).state()
             for g, V, h in zip(gs, Vs, h0)]
    probs = [fem.Problem("bmincut", graph=g, q=4, node_weight=V) for g, V in zip(gs, Vs)]
    fem.Batch(probs).anneal(h_inits=h0, replicas=16, n_steps=80)
    for p, ref in zip(probs, alone):
        for x, y in zip(p.state(), ref):
            assert np.array_equal(x, y)


def test_node_weight_validation(fem):
    g = I.rgg(50, 6.0, seed=96)
    for bad in (np.zeros(50), np.full(50, 1.5), np.full(50, 2.0 ** 21)):
        with pytest.raises(fem.FemError) as e:
            fem.Problem("bmincut", graph=g, q=4, node_weight=bad)
        assert e.value.status == fem.FEM_ERR_INVALID_ARG
    with pytest.raises(fem.FemError):
        fem.Problem("maxcut", graph=g, node_weight=np.ones(50))
