"""GPU vs oracle parity for sparse MaxCut, through the C ABI.

Fields: sigmoid(h) within 1e-4 max-abs over the first 50 fp32 steps (exact
mode; paper mode on every replica whose discrete trajectory agrees with the
oracle's).  Objectives: bit-exact (int64) for the GPU's own discrete states.
"""
import numpy as np
import pytest

import oracle as O
from paper_2412_09285_b300 import instances as I

pytestmark = pytest.mark.gpu

TOL_P = 1e-4   # marginals, max-abs, first 50 fp32 steps


@pytest.fixture(scope="module")
def fem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2412_09285_b300 import build
    build.build()
    from paper_2412_09285_b300 import fem as F
    return F


def _gpu_trace(fem, graph, h0, checkpoints, n_steps, **kw):
    P = fem.Problem("maxcut", graph=graph)
    out, t = {}, 0
    for T in checkpoints:
        P.anneal(h_init=h0 if t == 0 else None, replicas=h0.shape[1], n_steps=n_steps,
                 t_begin=t, t_end=T, **kw)
        out[T] = P.fields()
        t = T
    return P, out


def _oracle_trace(graph, h0, checkpoints, n_steps, mode, **kw):
    W = O.coupling_matrix(graph.n, graph.ei, graph.ej, graph.w)
    tr = {t: None for t in checkpoints}
    okw = {k: kw[k] for k in ("lr", "beta1", "beta2", "eps", "weight_decay", "momentum", "alpha",
                              "dampening") if k in kw}
    O.anneal(("maxcut", W), h0.astype(np.float64), n_steps, t_end=max(checkpoints),
             schedule=kw.get("schedule", "exponential"), beta_min=kw.get("beta_min", 0.05),
             beta_max=kw.get("beta_max", 5.0), optimizer=kw.get("optimizer", "adam"),
             opt_kw=okw or dict(lr=0.1), mode=mode, gamma=kw.get("gamma_grad", 1.0), trace=tr)
    return tr


CHECK = [1, 2, 5, 10, 20, 35, 50]


@pytest.mark.parametrize("weights", ["unit", "pm1", "real"])
def test_exact_mode_marginals_first_50_steps(fem, weights):
    g = I.er_gnp(800, 0.06, seed=1, weights=weights)
    h0 = I.initial_fields(800, 32, seed=2)
    _, got = _gpu_trace(fem, g, h0, CHECK, 1000, grad_mode="exact", lr=0.1)
    ref = _oracle_trace(g, h0, CHECK, 1000, "exact", lr=0.1)
    for t in CHECK:
        err = np.abs(O.sigmoid(got[t].astype(np.float64)) - O.sigmoid(ref[t])).max()
        assert err <= TOL_P, (t, err)


def _paper_compare(got, ref, checkpoints):
    agree = np.ones(got[checkpoints[0]].shape[1], bool)
    for t in checkpoints:
        agree &= np.all((got[t] >= 0) == (ref[t] >= 0), axis=0)
    errs = [np.abs(O.sigmoid(got[t][:, agree].astype(np.float64)) - O.sigmoid(ref[t][:, agree])).max()
            for t in checkpoints] if agree.any() else [0.0]
    return agree, max(errs)


@pytest.mark.parametrize("weights", ["unit", "pm1", "real"])
def test_paper_mode_marginals_first_50_steps(fem, weights):
    g = I.er_gnp(800, 0.06, seed=3, weights=weights)
    h0 = I.initial_fields(800, 32, seed=4)
    _, got = _gpu_trace(fem, g, h0, CHECK, 1000, grad_mode="paper", lr=0.1)
    ref = _oracle_trace(g, h0, CHECK, 1000, "paper", lr=0.1)
    agree, err = _paper_compare(got, ref, CHECK)
    assert agree.sum() >= 30, agree.sum()      # sign disagreements are rare near-ties
    assert err <= TOL_P, err


@pytest.mark.parametrize("opt,kw", [
    ("rmsprop", dict(lr=0.03, alpha=0.56, momentum=0.63, weight_decay=0.013,
                     schedule="inverse_proportional", beta_min=1 / 1.16, beta_max=1 / 6e-5)),
    ("rmsprop", dict(lr=0.01, alpha=0.99, momentum=0.0)),
    ("sgd", dict(lr=0.5, momentum=0.71, dampening=0.11, weight_decay=0.018, gamma_grad=6.0,
                 schedule="inverse_proportional", beta_min=1 / 0.63, beta_max=1e5)),
    ("adam", dict(lr=0.05, beta1=0.8, beta2=0.99, eps=1e-6, weight_decay=0.01, gamma_grad=2.0)),
])
def test_other_optimizers_and_schedules(fem, opt, kw):
    g = I.er_gnp(500, 0.05, seed=5, weights="pm1")
    h0 = I.initial_fields(500, 64, seed=6)
    _, got = _gpu_trace(fem, g, h0, CHECK, 1000, grad_mode="exact", optimizer=opt, **kw)
    ref = _oracle_trace(g, h0, CHECK, 1000, "exact", optimizer=opt, **kw)
    for t in CHECK:
        err = np.abs(O.sigmoid(got[t].astype(np.float64)) - O.sigmoid(ref[t])).max()
        assert err <= TOL_P, (t, err)


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


def test_resume_is_bit_identical(fem):
    g = I.er_gnp(600, 0.05, seed=10, weights="pm1")
    h0 = I.initial_fields(600, 32, seed=11)
    a = fem.Problem("maxcut", graph=g).anneal(h_init=h0, n_steps=400, grad_mode="paper")
    b = fem.Problem("maxcut", graph=g)
    b.anneal(h_init=h0, n_steps=400, t_end=123, grad_mode="paper")
    b.anneal(n_steps=400, t_begin=123, t_end=400, grad_mode="paper", replicas=32)
    assert np.array_equal(a.fields(), b.fields())
    for mode in ("exact",):
        a = fem.Problem("maxcut", graph=g).anneal(h_init=h0, n_steps=100, grad_mode=mode)
        b = fem.Problem("maxcut", graph=g)
        b.anneal(h_init=h0, n_steps=100, t_end=37, grad_mode=mode)
        b.anneal(n_steps=100, t_begin=37, grad_mode=mode, replicas=32)
        assert np.array_equal(a.fields(), b.fields())


@pytest.mark.parametrize("n,p,R", [(1, 0.0, 32), (37, 0.0, 32), (300, 0.004, 64), (257, 0.03, 96)])
def test_edge_cases_isolated_empty_multiword(fem, n, p, R):
    g = I.er_gnp(n, p, seed=12, weights="pm1")
    h0 = I.initial_fields(n, R, seed=13)
    _, got = _gpu_trace(fem, g, h0, [1, 10, 50], 200, grad_mode="exact")
    ref = _oracle_trace(g, h0, [1, 10, 50], 200, "exact", lr=0.1)
    for t in (1, 10, 50):
        assert np.abs(O.sigmoid(got[t].astype(np.float64)) - O.sigmoid(ref[t])).max() <= TOL_P
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
        P.anneal(h_init=I.initial_fields(100, 48, seed=1), n_steps=10)
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    P.anneal(h_init=I.initial_fields(100, 32, seed=1), n_steps=10, t_end=5)
    with pytest.raises(fem.FemError) as e:
        P.anneal(n_steps=10, t_begin=4, replicas=32)
    assert e.value.status == fem.FEM_ERR_STATE
    P.sync()


def test_full_size_sparse_steps_match_oracle(fem):
    """N = 2^20, mean degree 6, +-1 weights, R = 32 (the sparse-at-scale
    workload) in the launch configuration the benchmark times: every element
    of the first 3 steps against the oracle, then exact objectives after 30."""
    n = 1 << 20
    g = I.er_gnm(n, 3 * n, seed=2024, weights="pm1")
    h0 = I.initial_fields(n, 32, seed=2025)
    for mode in ("paper", "exact"):
        _, got = _gpu_trace(fem, g, h0, [1, 2, 3], 2000, grad_mode=mode)
        ref = _oracle_trace(g, h0, [1, 2, 3], 2000, mode, lr=0.1)
        for t in (1, 2, 3):
            diff = np.abs(O.sigmoid(got[t].astype(np.float64)) - O.sigmoid(ref[t]))
            if mode == "paper":
                agree = np.all((got[t] >= 0) == (ref[t] >= 0), axis=0)
                diff = diff[:, agree]
                assert agree.sum() >= 28
            assert diff.max() <= TOL_P, (mode, t, diff.max())
    P = fem.Problem("maxcut", graph=g).anneal(h_init=h0, n_steps=2000, t_end=30)
    st = P.states()
    res = P.best()
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, st.astype(np.int8))
    assert np.array_equal(-res["energy_i64"], cut)
