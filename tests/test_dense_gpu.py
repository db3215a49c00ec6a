"""Dense MaxCut (complete graphs, J = +-1) on the tensor cores vs the FP64 oracle.

Paper mode: the contraction of +-1 marginals with integer couplings is exact in
every precision (fp32 CUDA cores, bf16 and e4m3 tensor cores with fp32
accumulation), so marginals must match to 1e-4 over the first 50 steps on every
replica whose discrete trajectory agrees, exactly as for the sparse kernels.
Exact mode carries each precision's rounding of m: fp32 is held to 1e-4; the
bf16 hi+lo split keeps ~16 bits of m and bf16 alone ~8 bits - their measured
errors against the oracle are printed and bounded by the tolerances below.
Objectives are bit-exact int64 for the GPU's own states.
"""
import numpy as np
import pytest

import oracle as O
from paper_2412_09285_b300 import instances as I

pytestmark = pytest.mark.gpu

TOL_P = 1e-4
D_COND = 1e-6
MAX_ILL = 5e-3
# exact-mode error bounds per precision (max-abs in the marginals after one step from
# the oracle's state): fp32 rounding only; m split into two bf16 parts (~16 bits of m);
# m in one bf16 (8 bits), whose error in a sum of n ~ 1 terms is ~sqrt(n) * 2^-9
TOL_EXACT = {"fp32": 1e-4, "bf16x2": 1e-3, "bf16": 1e-1}
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


def _traces(fem, g, h0, checkpoints, mode, prec, n_steps=1000):
    P = fem.Problem("maxcut", dense=g.dense)
    got, t = {}, 0
    for T in checkpoints:
        P.anneal(h_init=h0 if t == 0 else None, replicas=h0.shape[1], n_steps=n_steps, t_begin=t, t_end=T,
                 grad_mode=mode, precision=prec)
        got[T] = P.fields()
        t = T
    W = g.dense.astype(np.float64)
    tr = {t: None for t in checkpoints}
    cd = {t: None for t in checkpoints}
    O.anneal(("maxcut", W), h0.astype(np.float64), n_steps, t_end=max(checkpoints), mode=mode, trace=tr,
             cond=cd)
    return P, got, tr, cd


@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp32"])
def test_paper_mode_marginals_first_50_steps(fem, prec):
    g = I.sk_dense(300, seed=81)
    h0 = I.initial_fields(300, 128, seed=82)
    _, got, ref, cd = _traces(fem, g, h0, CHECK, "paper", prec)
    agree = np.ones(128, bool)
    for t in CHECK:
        agree &= np.all((got[t] >= 0) == (ref[t] >= 0), axis=0)
    assert agree.sum() >= 120, agree.sum()
    for t in CHECK:
        err = np.abs(O.sigmoid(got[t][:, agree].astype(np.float64)) - O.sigmoid(ref[t][:, agree]))
        ok = cd[t][:, agree] >= D_COND
        assert (~ok).mean() <= MAX_ILL
        assert err[ok].max() <= TOL_P, (prec, t, float(err[ok].max()))


@pytest.mark.parametrize("prec", ["fp32", "bf16x2", "bf16"])
def test_exact_mode_error_per_precision(fem, prec):
    """One step from the oracle's own state (teacher forcing) at several points of the
    anneal.  Whole exact-mode trajectories are not compared here: on the all-to-all SK
    coupling one ill-conditioned element's rounding reaches every row through J at the
    next step, so fp32 and fp64 trajectories drift apart by ~1e-4 within a few steps in
    any fp32 implementation (an fp32 emulation of the update on the CPU does the same)."""
    g = I.sk_dense(256, seed=83)
    W = g.dense.astype(np.float64)
    h0 = I.initial_fields(256, 128, seed=84)
    n_steps = 1000
    P = fem.Problem("maxcut", dense=g.dense)
    P.anneal(h_init=h0, n_steps=n_steps, t_end=0, grad_mode="exact", precision=prec)
    h, o = O.anneal(("maxcut", W), h0.astype(np.float64), n_steps, t_end=0, mode="exact")
    worst, t = 0.0, 0
    for t0 in (0, 5, 20, 100, 400):
        if t0 > t:
            h, o = O.anneal(("maxcut", W), h, n_steps, t_begin=t, t_end=t0, mode="exact", opt=o)
        h32, m32, v32 = (x.astype(np.float32) for x in (h, o.m, o.v))
        h = h32.astype(np.float64)
        o.m, o.v = m32.astype(np.float64), v32.astype(np.float64)
        cd = {t0 + 1: None}
        h, o = O.anneal(("maxcut", W), h, n_steps, t_begin=t0, t_end=t0 + 1, mode="exact", opt=o, cond=cd)
        if t0 == 0:
            P.anneal(h_init=h32, n_steps=n_steps, t_end=1, grad_mode="exact", precision=prec)
        else:
            P.set_state(h32, m32, v32, steps_done=t0)
            P.anneal(n_steps=n_steps, t_begin=t0, t_end=t0 + 1, grad_mode="exact", precision=prec,
                     replicas=128)
        err = np.abs(O.sigmoid(P.fields().astype(np.float64)) - O.sigmoid(h))
        ok = cd[t0 + 1] >= D_COND
        assert (~ok).mean() <= MAX_ILL
        worst = max(worst, float(err[ok].max()))
        t = t0 + 1
    print(f"exact-mode one-step max marginal error vs fp64 oracle, {prec}: {worst:.2e}")
    assert worst <= TOL_EXACT[prec], (prec, worst)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "bf16x2", "fp32"])
def test_objectives_bit_exact(fem, prec):
    g = I.sk_dense(500, seed=85)
    h0 = I.initial_fields(500, 256, seed=86)
    mode = "exact" if prec == "bf16x2" else "paper"
    P = fem.Problem("maxcut", dense=g.dense).anneal(h_init=h0, n_steps=300, grad_mode=mode, precision=prec)
    st = P.states()
    assert np.array_equal(st, np.where(P.fields() >= 0, 1, -1))
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, st.astype(np.int8))
    res = P.best()
    assert np.array_equal(-res["energy_i64"], cut)
    b = O.best_replica(-cut)
    assert res["best_replica"] == b and np.array_equal(res["states"], st[:, b])
    assert cut.max() > 0  # an SK instance with a positive best cut after annealing


def test_full_size_dense_steps(fem):
    """n = 2000, R = 1024 (the dense SK workload): the first 3 paper-mode steps in bf16
    and fp8 against the oracle on every element of agreeing replicas."""
    g = I.sk_dense(2000, seed=87)
    h0 = I.initial_fields(2000, 1024, seed=88)
    W = g.dense.astype(np.float64)
    tr = {1: None, 2: None, 3: None}
    cd = {1: None, 2: None, 3: None}
    O.anneal(("maxcut", W), h0.astype(np.float64), 1000, t_end=3, mode="paper", trace=tr, cond=cd)
    for prec in ("bf16", "fp8"):
        P = fem.Problem("maxcut", dense=g.dense)
        got, t = {}, 0
        for T in (1, 2, 3):
            P.anneal(h_init=h0 if t == 0 else None, replicas=1024, n_steps=1000, t_begin=t, t_end=T,
                     grad_mode="paper", precision=prec)
            got[T] = P.fields()
            t = T
        agree = np.ones(1024, bool)
        for T in (1, 2, 3):
            agree &= np.all((got[T] >= 0) == (tr[T] >= 0), axis=0)
        assert agree.sum() >= 1000
        for T in (1, 2, 3):
            ok = cd[T][:, agree] >= D_COND
            err = np.abs(O.sigmoid(got[T][:, agree].astype(np.float64)) - O.sigmoid(tr[T][:, agree]))
            assert err[ok].max() <= TOL_P, (prec, T, float(err[ok].max()))


def test_dense_resume_and_checkpoint(fem):
    g = I.sk_dense(400, seed=89)
    h0 = I.initial_fields(400, 128, seed=90)
    a = fem.Problem("maxcut", dense=g.dense).anneal(h_init=h0, n_steps=200, precision="bf16")
    c = fem.Problem("maxcut", dense=g.dense)
    c.anneal(h_init=h0, n_steps=200, t_end=77, precision="bf16")
    ck = c.state()
    d = fem.Problem("maxcut", dense=g.dense)
    d.anneal(h_init=h0, n_steps=200, t_end=0, precision="bf16")
    d.set_state(*ck, steps_done=77)
    d.anneal(n_steps=200, t_begin=77, replicas=128, precision="bf16")
    assert np.array_equal(a.fields(), d.fields())


def test_dense_argument_errors(fem):
    g = I.sk_dense(64, seed=91)
    with pytest.raises(fem.FemError) as e:
        fem.Problem("maxcut", dense=g.dense).anneal(h_init=I.initial_fields(64, 96, seed=1), n_steps=10)
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    with pytest.raises(fem.FemError) as e:
        fem.Problem("maxcut", dense=g.dense).anneal(h_init=I.initial_fields(64, 128, seed=1), n_steps=10,
                                                    grad_mode="exact", precision="fp8")
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    bad = g.dense.astype(np.float32).copy()
    bad[0, 1] = 3.0
    with pytest.raises(fem.FemError) as e:
        fem.Problem("maxcut", dense=bad)
    assert e.value.status == fem.FEM_ERR_INVALID_ARG


def _run(fem, g, h0, launch, n_steps, windows, **kw):
    P = fem.Problem("maxcut", dense=g.dense)
    P.set_dense_launch(launch)
    t = 0
    for T in windows:
        P.anneal(h_init=h0 if t == 0 else None, replicas=h0.shape[1], n_steps=n_steps, t_begin=t, t_end=T, **kw)
        t = T
    return P


@pytest.mark.parametrize("n,launch,kind", [(300, "persistent", "persistent_single"),
                                           (500, "persistent", "persistent"),
                                           (500, "persistent_single", "persistent_single")])
@pytest.mark.parametrize("prec,mode,opt", [
    ("bf16", "paper", "adam"), ("fp8", "paper", "adam"), ("bf16x2", "exact", "adam"), ("bf16", "exact", "adam"),
    ("bf16", "paper", "rmsprop"), ("fp8", "paper", "sgd")])
def test_persistent_matches_per_step(fem, prec, mode, opt, n, launch, kind):
    """The persistent launch (state in tensor memory for the whole window, a barrier
    per step between the CTAs of a replica block) gives the per-step kernel's h, m, v
    bit for bit, in exact mode too (all kernels accumulate the K chunks in order): n = 300 (three row tiles, the last one ragged: one CTA per tile), n = 500
    (four row tiles: CTA pairs issuing 256-row MMAs, or single CTAs when asked), two
    replica blocks, and the window split [0, 37) + [37, 120) for the persistent run."""
    g = I.sk_dense(n, seed=92)
    h0 = I.initial_fields(n, 256, seed=93)
    kw = dict(precision=prec, grad_mode=mode, optimizer=opt)
    if opt == "rmsprop":
        kw.update(lr=0.01)
    if opt == "sgd":
        kw.update(lr=0.05, momentum=0.9)
    ref = _run(fem, g, h0, "per_step", 120, [120], **kw)
    assert ref.dense_last_launch() == "per_step"
    got = _run(fem, g, h0, launch, 120, [37, 120], **kw)
    assert got.dense_last_launch() == kind
    for a, b, name in zip(got.state(), ref.state(), "hmv"):
        assert np.array_equal(a, b), (name, int(np.sum(a != b)))


def test_persistent_full_size(fem):
    """n = 2000, R = 1024 (the dense SK workload, 128 co-resident CTAs in 64 pairs): 60
    persistent steps equal 60 per-step launches bit for bit, in bf16 and e4m3."""
    g = I.sk_dense(2000, seed=94)
    h0 = I.initial_fields(2000, 1024, seed=95)
    for prec in ("bf16", "fp8"):
        ref = _run(fem, g, h0, "per_step", 1000, [60], precision=prec).state()
        P = _run(fem, g, h0, "persistent", 1000, [60], precision=prec)
        assert P.dense_last_launch() == "persistent"
        for a, b, name in zip(P.state(), ref, "hmv"):
            assert np.array_equal(a, b), (prec, name, int(np.sum(a != b)))


def test_persistent_unsupported(fem):
    g = I.sk_dense(200, seed=96)
    h0 = I.initial_fields(200, 128, seed=97)
    with pytest.raises(fem.FemError) as e:
        _run(fem, g, h0, "persistent", 10, [10], precision="fp32")
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    with pytest.raises(fem.FemError):
        fem.Problem("maxcut", graph=I.er_gnm(50, 100, seed=1)).set_dense_launch("persistent")


def test_precision_and_replica_count_switches_on_one_problem(fem):
    """One dense problem annealed at bf16 with 128 replicas, then fp8 with 256, then
    bf16 hi+lo exact mode with 128 (each switch frees and reallocates the state):
    every result equals a fresh problem's bit for bit."""
    g = I.sk_dense(300, seed=61)
    runs = [("bf16", 128, "paper"), ("fp8", 256, "paper"), ("bf16x2", 128, "exact")]
    p = fem.Problem("maxcut", dense=g.dense)
    for prec, R, mode in runs:
        h0 = I.initial_fields(300, R, seed=62 + R)
        p.anneal(h_init=h0, n_steps=100, grad_mode=mode, precision=prec)
        fresh = fem.Problem("maxcut", dense=g.dense).anneal(h_init=h0, n_steps=100, grad_mode=mode,
                                                             precision=prec)
        assert np.array_equal(p.fields(), fresh.fields()), (prec, R)
        assert np.array_equal(p.best()["energy_i64"], fresh.best()["energy_i64"]), (prec, R)
