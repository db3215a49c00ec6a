"""GPU vs oracle parity for Max-k-SAT (single field, clause products), through the C ABI.

Marginals sigmoid(h) within 1e-4 max-abs over the first 50 fp32 steps (Adam,
lr 0.1; well-conditioned elements), teacher-forced windows for RMSprop/SGD, and
bit-exact unsatisfied-clause counts for the GPU's own assignments.
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


def _check(got, ref, cond, where, forced=None, prev=None, prev_state=None):
    return parity.compare(got, ref, cond, where, forced=forced, prev=prev, prev_state=prev_state)


def _forced(P, groups, n_steps, **kw):
    """One step on both sides from a given fp32 state (parity.one_step)."""
    run = {k: v for k, v in kw.items() if k != "optimizer"}
    return parity.one_step(P, ("sat", groups), n_steps, optimizer=kw.get("optimizer", "adam"),
                           opt_kw=_okw(kw), sched=_sched(kw), **run)


def _okw(kw):
    return {k: kw[k] for k in ("lr", "beta1", "beta2", "eps", "weight_decay", "momentum", "alpha",
                               "dampening") if k in kw} or dict(lr=0.1)


def _sched(kw):
    return dict(schedule=kw.get("schedule", "exponential"), beta_min=kw.get("beta_min", 0.05),
                beta_max=kw.get("beta_max", 5.0), gamma=kw.get("gamma_grad", 1.0))


def _mixed_clauses(n, m, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    ptr, lits = [0], []
    for _ in range(m):
        k = int(rng.integers(1, 6))
        vs = rng.choice(n, size=k, replace=False) + 1
        sg = rng.integers(0, 2, size=k) * 2 - 1
        lits += list(vs * sg)
        ptr.append(len(lits))
    return I.Clauses(n, np.array(ptr), np.array(lits))


@pytest.mark.parametrize("kind", ["3sat", "mixed"])
def test_marginals_first_50_steps(fem, kind):
    cl = I.random_ksat(2000, 8400, 3, seed=51) if kind == "3sat" else _mixed_clauses(1500, 5000, 52)
    groups = O.sat_arrays(cl.ptr, cl.lits)
    h0 = I.initial_fields(cl.n, 16, seed=53)
    P = fem.Problem("sat", clauses=cl)
    got, st = parity.gpu_windows(P, h0, CHECK, 1000)
    tr = {t: None for t in CHECK}
    cd = {t: None for t in CHECK}
    O.anneal(("sat", groups), h0.astype(np.float64), 1000, t_end=50, opt_kw=dict(lr=0.1), trace=tr,
             cond=cd)
    parity.compare_trajectory(got, tr, cd, CHECK, kind, state=st, forced=_forced(P, groups, 1000, lr=0.1))


@pytest.mark.parametrize("opt,kw", [
    ("rmsprop", dict(lr=0.03, alpha=0.7, momentum=0.5, weight_decay=0.01)),
    ("sgd", dict(lr=0.8, momentum=0.7, dampening=0.1, schedule="inverse_proportional",
                 beta_min=0.1, beta_max=30.0, gamma_grad=4.0)),
    ("adam", dict(lr=0.1)),
])
def test_teacher_forced_windows(fem, opt, kw):
    cl = I.random_ksat(1500, 6300, 3, seed=54)
    groups = O.sat_arrays(cl.ptr, cl.lits)
    h0 = I.initial_fields(cl.n, 32, seed=55)
    n_steps = 1000
    P = fem.Problem("sat", clauses=cl)
    P.anneal(h_init=h0, n_steps=n_steps, t_end=0, optimizer=opt, **kw)
    h, o = O.anneal(("sat", groups), h0.astype(np.float64), n_steps, t_end=0, optimizer=opt,
                    opt_kw=_okw(kw), **_sched(kw))
    t = 0
    for t0 in (0, 11, 60, 400, 900):
        if t0 > t:
            h, o = O.anneal(("sat", groups), h, n_steps, t_begin=t, t_end=t0, optimizer=opt, opt=o,
                            **_sched(kw))
        m, v = parity.opt_state(o)
        h32, m32, v32 = (x.astype(np.float32) for x in (h, m, v))
        h = h32.astype(np.float64)
        parity.set_opt_state(o, m32.astype(np.float64), v32.astype(np.float64))
        cd = {t0 + 3: None}
        h, o = O.anneal(("sat", groups), h, n_steps, t_begin=t0, t_end=t0 + 3, optimizer=opt, opt=o,
                        cond=cd, **_sched(kw))
        if t0 == 0:
            P.anneal(h_init=h32, n_steps=n_steps, t_end=3, optimizer=opt, **kw)
        else:
            P.set_state(h32, m32, v32, steps_done=t0)
            P.anneal(n_steps=n_steps, t_begin=t0, t_end=t0 + 3, optimizer=opt, replicas=32, **kw)
        _check(P.fields(), h, cd[t0 + 3], (opt, t0), forced=_forced(P, groups, n_steps, optimizer=opt, **kw),
               prev=t0, prev_state=(h32, m32, v32))
        t = t0 + 3


@pytest.mark.parametrize("kind,R", [("3sat", 16), ("mixed", 32), ("4sat", 48)])
def test_unsat_counts_bit_exact(fem, kind, R):
    if kind == "3sat":
        cl = I.random_ksat(3000, 12600, 3, seed=56)
    elif kind == "4sat":
        cl = I.random_ksat(800, 7000, 4, seed=57)
    else:
        cl = _mixed_clauses(900, 4000, 58)
    h0 = I.initial_fields(cl.n, R, seed=59)
    P = fem.Problem("sat", clauses=cl).anneal(h_init=h0, n_steps=800)
    st = P.states()
    assert np.array_equal(st, (P.fields() >= 0).astype(np.int32))
    unsat = O.sat_unsat(cl.ptr, cl.lits, st.astype(np.int8))
    res = P.best()
    assert np.array_equal(res["energy_i64"], unsat)
    b = O.best_replica(unsat)
    assert res["best_replica"] == b and np.array_equal(res["states"], st[:, b])
    if kind != "mixed":   # the mixed instance has conflicting unit clauses
        assert unsat.min() < 0.02 * cl.n_clauses  # far below a random assignment's M/2^k


def test_empty_clause_and_unused_variables(fem):
    cl = I.Clauses(6, np.array([0, 2, 2, 5, 6]), np.array([1, -2, 2, 3, -4, -1]))
    h0 = I.initial_fields(6, 16, seed=60)
    P = fem.Problem("sat", clauses=cl).anneal(h_init=h0, n_steps=200)
    unsat = O.sat_unsat(cl.ptr, cl.lits, P.states().astype(np.int8))
    assert np.array_equal(P.best()["energy_i64"], unsat)
    assert unsat.min() == 1                       # the empty clause is never satisfied


@pytest.mark.parametrize("seed", [43, 44])
def test_reaches_bruteforce_optimum(fem, seed):
    cl = I.random_ksat(16, 67, 3, seed=seed)
    best = O.sat_bruteforce(cl.n, cl.ptr, cl.lits)
    h0 = I.initial_fields(16, 32, seed=seed + 100)
    P = fem.Problem("sat", clauses=cl).anneal(h_init=h0, n_steps=1000)
    assert P.best()["energy_i64"].min() == best


def test_resume_and_checkpoint_bit_identical(fem):
    cl = I.random_ksat(1000, 4200, 3, seed=61)
    h0 = I.initial_fields(1000, 16, seed=62)
    a = fem.Problem("sat", clauses=cl).anneal(h_init=h0, n_steps=300)
    c = fem.Problem("sat", clauses=cl)
    c.anneal(h_init=h0, n_steps=300, t_end=133)
    ck = c.state()
    d = fem.Problem("sat", clauses=cl)
    d.anneal(h_init=h0, n_steps=300, t_end=0)
    d.set_state(*ck, steps_done=133)
    d.anneal(n_steps=300, t_begin=133, replicas=16)
    assert np.array_equal(a.fields(), d.fields())


@pytest.mark.parametrize("ptr,lits", [
    ([0, 3], [1, -1, 2]),          # repeated variable
    ([0, 2], [1, 9]),              # literal out of range
    ([0, 2], [1, 0]),              # zero literal
    ([0, 2, 1], [1, 2]),           # clause_ptr decreasing
    ([1, 2], [1, 2]),              # clause_ptr[0] != 0
])
def test_malformed_clauses_rejected(fem, ptr, lits):
    with pytest.raises(fem.FemError) as e:
        fem.Problem("sat", clauses=I.Clauses(4, np.array(ptr), np.array(lits)))
    assert e.value.status == fem.FEM_ERR_INVALID_ARG


def test_wide_clause_unsupported(fem):
    with pytest.raises(fem.FemError) as e:
        fem.Problem("sat", clauses=I.Clauses(12, np.array([0, 9]), np.arange(1, 10)))
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED


@pytest.mark.parametrize("opt", ["adam", "rmsprop"])
def test_three_sat_four_replica_path_matches_general_path(fem, opt):
    """Uniform 3-SAT with R % 4 == 0 runs the four-replicas-per-thread kernel (other-
    literal table, float4 gathers, occurrences a few at a time); R = 50 runs the
    general per-thread kernel.  Replicas are independent, so the first 4 / 16 / 32 / 48
    replicas of the R = 50 run must equal the narrow runs bit for bit."""
    c = I.random_ksat(3000, 12600, 3, seed=51)
    wide = I.initial_fields(c.n, 50, seed=52)
    kw = dict(optimizer=opt, lr=0.1 if opt == "adam" else 0.01)
    ref = fem.Problem("sat", clauses=c).anneal(h_init=wide, n_steps=200, **kw).state()
    for R in (4, 16, 32, 48):
        got = fem.Problem("sat", clauses=c).anneal(h_init=np.ascontiguousarray(wide[:, :R]), n_steps=200,
                                                    **kw).state()
        for a, b, name in zip(got, ref, "hmv"):
            assert np.array_equal(a, b[:, :R]), (R, name, int(np.sum(a != b[:, :R])))
