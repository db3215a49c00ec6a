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
import parity
from paper_2412_09285_b300 import instances as I

pytestmark = pytest.mark.gpu

TOL_P = parity.TOL_P
# exact-mode error bounds per precision (max-abs in the marginals after one step from
# the oracle's state): fp32 rounding only; m split into two bf16 parts (~16 bits of m);
# m in one bf16 (8 bits), whose error in a sum of n ~ 1 terms is ~sqrt(n) * 2^-9.  The
# sharper gate is on the applied gradient (test_exact_mode_error_per_precision).
TOL_EXACT = {"fp32": 1e-4, "bf16x2": 1e-3, "bf16": 5e-2}
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
    got, st = parity.gpu_windows(P, h0, checkpoints, n_steps, grad_mode=mode, precision=prec)
    W = g.dense.astype(np.float64)
    tr = {t: None for t in checkpoints}
    cd = {t: None for t in checkpoints}
    O.anneal(("maxcut", W), h0.astype(np.float64), n_steps, t_end=max(checkpoints), mode=mode, trace=tr,
             cond=cd)
    forced = parity.one_step(P, ("maxcut", W), n_steps, mode=mode, grad_mode=mode, precision=prec)
    return P, got, tr, cd, st, forced


def _agree(got, ref, checkpoints):
    agree = np.ones(got[checkpoints[0]].shape[1], bool)
    for t in checkpoints:
        agree &= np.all((got[t] >= 0) == (ref[t] >= 0), axis=0)
    return agree


@pytest.mark.parametrize("prec", ["bf16", "fp8", "fp32"])
def test_paper_mode_marginals_first_50_steps(fem, prec):
    g = I.sk_dense(300, seed=81)
    h0 = I.initial_fields(300, 128, seed=82)
    _, got, ref, cd, st, forced = _traces(fem, g, h0, CHECK, "paper", prec)
    agree = _agree(got, ref, CHECK)
    assert agree.sum() >= 120, agree.sum()
    parity.compare_trajectory(got, ref, cd, CHECK, prec, agree=agree, state=st, forced=forced)


# Relative rounding of each m_j in the contraction operand: bf16 keeps 8 significant bits
# (|m - bf16(m)| <= 2^-9 |m|); the hi + lo split leaves |m - hi - lo| <= 2^-9 |m - hi|
# <= 2^-18 |m|; fp32 operands are exact.
OPERAND_U = {"fp32": 0.0, "bf16x2": 2.0 ** -18, "bf16": 2.0 ** -9}


@pytest.mark.parametrize("prec", ["fp32", "bf16x2", "bf16"])
def test_exact_mode_error_per_precision(fem, prec):
    """One step from the oracle's own state (teacher forcing) at several points of the
    anneal.  Whole exact-mode trajectories are not compared here: on the all-to-all SK
    coupling one ill-conditioned element's rounding reaches every row through J at the
    next step, so fp32 and fp64 trajectories drift apart by ~1e-4 within a few steps in
    any fp32 implementation (an fp32 emulation of the update on the CPU does the same).

    Two gates per element.  (1) The gradient the kernel applied, read back from its
    first moment (g = (m' - beta1 m) / (1 - beta1)), is within the error bound of the
    precision: the field S_i = sum_j J_ij m_j is off by at most
    (u + n 2^-24) sum_j |J_ij m_j| (u: the operand's rounding, OPERAND_U; n 2^-24: fp32
    accumulation of n terms in any order), so g = (gamma/4)(2 S_i + h_i/beta)(1 - m_i^2)
    is off by (gamma/2)(1 - m_i^2) times that, plus 1e-8 + 1e-5 |g| for the fp32
    evaluation of the rest and the fp32 rounding of the moments it is read back from.  (2) The marginals after the step are within TOL_EXACT of
    the oracle's, except on elements whose optimizer denominator is below D_COND in
    this very step (there the update's slope in g is up to lr / eps): those are capped
    in number, and the oracle's optimizer fed with the applied gradient reproduces the
    kernel's fields within 1e-4."""
    g = I.sk_dense(256, seed=83)
    W = g.dense.astype(np.float64)
    absW = np.abs(W)
    n = W.shape[0]
    h0 = I.initial_fields(256, 128, seed=84)
    n_steps = 1000
    betas = O.beta_schedule("exponential", 0.05, 5.0, n_steps)
    P = fem.Problem("maxcut", dense=g.dense)
    P.anneal(h_init=h0, n_steps=n_steps, t_end=0, grad_mode="exact", precision=prec)
    h, o = O.anneal(("maxcut", W), h0.astype(np.float64), n_steps, t_end=0, mode="exact")
    worst, worst_g, t = 0.0, 0.0, 0
    for t0 in (0, 5, 20, 100, 400):
        if t0 > t:
            h, o = O.anneal(("maxcut", W), h, n_steps, t_begin=t, t_end=t0, mode="exact", opt=o)
        h32, m32, v32 = (x.astype(np.float32) for x in (h, o.m, o.v))
        h = h32.astype(np.float64)
        o.m, o.v = m32.astype(np.float64), v32.astype(np.float64)
        h_in, m_in, v_in = h.copy(), o.m.copy(), o.v.copy()
        cd = {t0 + 1: None}
        h, o = O.anneal(("maxcut", W), h, n_steps, t_begin=t0, t_end=t0 + 1, mode="exact", opt=o, cond=cd)
        if t0 == 0:
            P.anneal(h_init=h32, n_steps=n_steps, t_end=1, grad_mode="exact", precision=prec)
        else:
            P.set_state(h32, m32, v32, steps_done=t0)
            P.anneal(n_steps=n_steps, t_begin=t0, t_end=t0 + 1, grad_mode="exact", precision=prec,
                     replicas=128)
        h_got, m_got, _ = (x.astype(np.float64) for x in P.state())
        # (1) the applied gradient against the precision's bound
        b1 = o.b1
        g_got = (m_got - b1 * m_in) / (1.0 - b1)
        g_ref = (o.m - b1 * m_in) / (1.0 - b1)
        mm = np.tanh(0.5 * h_in)
        bound = (0.5 * (1.0 - mm * mm) * (OPERAND_U[prec] + n * 2.0 ** -24) * (absW @ np.abs(mm))
                 + 1e-8 + 1e-5 * np.abs(g_ref)
                 + 2.0 ** -23 * (b1 * np.abs(m_in) + np.abs(m_got)) / (1.0 - b1))  # fp32 moment read-back
        dg = np.abs(g_got - g_ref)
        worst_g = max(worst_g, float((dg / bound).max()))
        assert (dg <= bound).all(), (prec, t0, float((dg / bound).max()))
        # (2) marginals; ill-conditioned elements of this step by the optimizer replay
        err = np.abs(O.sigmoid(h_got) - O.sigmoid(h))
        ill = cd[t0 + 1] < parity.D_COND
        e_rep = 0.0
        if ill.any():
            o2 = O.Adam(h_in.shape, lr=0.1)
            o2.m, o2.v = m_in.copy(), v_in.copy()
            hh = h_in.copy()
            o2.step(hh, g_got, t0 + 1)
            e_rep = float(np.abs(O.sigmoid(hh) - O.sigmoid(h_got))[ill].max())
        print(f"PARITY exact-mode one step from t={t0}, {prec}: {err.size} compared, applied gradient within "
              f"{float((dg / bound).max()):.2f} of its bound | {int(ill.sum())} with denominator < "
              f"{parity.D_COND:g} (replayed update err {e_rep:.1e}) | max err {float(err[~ill].max()):.2e}")
        assert ill.mean() <= parity.MAX_ILL, (prec, t0, ill.mean())
        assert e_rep <= parity.TOL_P, (prec, t0, e_rep)
        worst = max(worst, float(err[~ill].max()))
        t = t0 + 1
    print(f"exact-mode one-step max marginal error vs fp64 oracle, {prec}: {worst:.2e}; applied gradient at "
          f"{worst_g:.2f} of its bound")
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
        got, st = parity.gpu_windows(P, h0, (1, 2, 3), 1000, grad_mode="paper", precision=prec)
        agree = _agree(got, tr, (1, 2, 3))
        assert agree.sum() >= 1000
        forced = parity.one_step(P, ("maxcut", W), 1000, mode="paper", grad_mode="paper", precision=prec)
        parity.compare_trajectory(got, tr, cd, (1, 2, 3), prec, agree=agree, state=st, forced=forced)


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


@pytest.mark.parametrize("defect,msg", [
    ("fraction", "dense_J[3][7] must be an integer with |J| <= 127"),
    ("too_large", "dense_J[3][7] must be an integer with |J| <= 127"),
    ("nan", "dense_J[3][7] must be an integer with |J| <= 127"),
    ("diagonal", "dense_J must have a zero diagonal"),
    ("asymmetric", "dense_J must be symmetric"),
])
def test_dense_validation_on_the_device(fem, defect, msg):
    """The couplings are validated on the device after one copy; the lowest offending
    entry in row-major order is reported (a second defect is planted further on), and
    the device stays usable."""
    n = 300
    g = I.sk_dense(n, seed=93)
    J = g.dense.astype(np.float32)
    J[200, 250] = J[250, 200] = 0.5          # the later defect
    if defect == "fraction":
        J[3, 7] = J[7, 3] = 1.5
    elif defect == "too_large":
        J[3, 7] = J[7, 3] = 128.0
    elif defect == "nan":
        J[3, 7] = J[7, 3] = np.nan
    elif defect == "diagonal":
        J[3, 3] = 1.0
    else:
        J[3, 7] = -J[7, 3]
    with pytest.raises(fem.FemError) as e:
        fem.Problem("maxcut", dense=J)
    assert e.value.status == fem.FEM_ERR_INVALID_ARG
    assert str(e.value).endswith(msg), str(e.value)
    P = fem.Problem("maxcut", dense=g.dense)
    P.anneal(h_init=I.initial_fields(n, 128, seed=2), n_steps=20)
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, P.states().astype(np.int8))
    assert np.array_equal(-P.best()["energy_i64"], cut)


def test_dense_fp8_needs_small_couplings(fem):
    """|J_ij| <= 16 is exact in e4m3; a coupling of 17 makes the fp8 path refuse the
    problem while bf16 runs it, with exact objectives."""
    n = 256
    g = I.sk_dense(n, seed=95)
    J = g.dense.astype(np.float32)
    J[10, 20] = J[20, 10] = 17.0
    P = fem.Problem("maxcut", dense=J)
    h0 = I.initial_fields(n, 128, seed=3)
    with pytest.raises(fem.FemError) as e:
        P.anneal(h_init=h0, n_steps=20, precision="fp8")
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    P.anneal(h_init=h0, n_steps=20, precision="bf16")
    iu, ju = np.triu_indices(n, k=1)
    cut = O.maxcut_cut_edges(iu, ju, J[iu, ju].astype(np.float64), P.states().astype(np.int8))
    assert np.array_equal(-P.best()["energy_i64"], cut)


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


def test_switches_on_a_side_stream(fem):
    """The same switches on a non-blocking torch side stream: the zeroed K padding of the
    reallocated operands is ordered before the first contraction on that stream."""
    import torch
    g = I.sk_dense(300, seed=63)
    side = torch.cuda.Stream()
    p = fem.Problem("maxcut", dense=g.dense, stream=side)
    for prec, R, mode in [("bf16", 128, "paper"), ("fp8", 256, "paper"), ("bf16x2", 128, "exact")]:
        h0 = I.initial_fields(300, R, seed=64 + R)
        p.anneal(h_init=h0, n_steps=60, grad_mode=mode, precision=prec)
        fresh = fem.Problem("maxcut", dense=g.dense).anneal(h_init=h0, n_steps=60, grad_mode=mode,
                                                             precision=prec)
        assert np.array_equal(p.fields(), fresh.fields()), (prec, R)
