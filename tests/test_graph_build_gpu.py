"""The device builders (fem_create_problem for large edge and clause lists) against the
host builders: the same graph built both ways must anneal to the same fields and
energies bit for bit (the CSR order and every row sum agree), in paper and exact mode,
for unit, +-1, integer and real weights, MaxCut, QUBO and bMinCut, with hub rows that
take the block sort (degree 33 .. 4096) and the host fallback (degree > 4096); a
duplicate edge is rejected by the device builder as by the host one.  Clause lists
(Max-3-SAT, mixed widths, 3-spin and mixed p-spin terms) likewise: the same occurrence
order, so the same fields and energies bit for bit.  Invalid edges, clauses and terms
are reported by the device validation with the host builder's message, naming the
lowest offending one."""
import numpy as np
import pytest

import oracle as O
from paper_2412_09285_b300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2412_09285_b300 import build
    build.build()
    from paper_2412_09285_b300 import fem as F
    yield F
    F.fem_set_device_graph_build(1 << 16)


def _with_hubs(g, spec, seed):
    """g plus, for each (count, width) in spec, `count` hubs joined to `width` random nodes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    have = {(a, b): x for a, b, x in zip(g.ei.tolist(), g.ej.tolist(), g.w.tolist())}
    for count, width in spec:
        for h in rng.choice(g.n, count, replace=False).tolist():
            for j in rng.choice(g.n, width, replace=False).tolist():
                if j != h:
                    have.setdefault((min(h, j), max(h, j)), float(rng.choice([-1.0, 1.0])))
    e = list(have)
    rng.shuffle(e)
    return I.Graph(g.n, [a for a, _ in e], [b for _, b in e], [have[k] for k in e])


def _both(fem, make):
    out = []
    for thr in (0, -1):   # device build, host build
        fem.fem_set_device_graph_build(thr)
        out.append(make())
    fem.fem_set_device_graph_build(1 << 16)
    return out


def _same_run(fem, kind, g, R, modes, q=2, **pk):
    for mode in modes:
        h0 = I.initial_fields(g.n, R, seed=5, q=q)
        dev, host = _both(fem, lambda: fem.Problem(kind, graph=g, q=q, **pk))
        for P in (dev, host):
            P.anneal(h_init=h0, n_steps=200, t_end=60, grad_mode=mode)
        for a, b, name in zip(dev.state(), host.state(), "hmv"):
            assert np.array_equal(a, b), (kind, mode, name)
        rd, rh = dev.best(), host.best()
        assert np.array_equal(rd["energy_i64"], rh["energy_i64"]) and np.array_equal(rd["energy_f64"], rh["energy_f64"])


@pytest.mark.parametrize("weights", ["pm1", "unit", "int", "real"])
def test_maxcut_device_build_equals_host_build(fem, weights):
    g = I.er_gnm(50000, 150000, seed=11, weights="real" if weights == "real" else
                 ("unit" if weights in ("unit", "int") else "pm1"))
    if weights == "int":
        g.w = np.random.Generator(np.random.PCG64(12)).integers(1, 5, g.n_edges).astype(np.float64)
    _same_run(fem, "maxcut", g, 32, ["paper", "exact"])


def test_hub_rows_block_sort_and_host_fallback(fem):
    g = _with_hubs(I.er_gnm(20000, 60000, seed=13, weights="pm1"), [(20, 200), (2, 5000)], seed=14)
    _same_run(fem, "maxcut", g, 32, ["paper", "exact"])


def test_qubo_and_bmincut_device_build(fem):
    g = I.er_gnm(30000, 90000, seed=15, weights="pm1")
    d = np.random.Generator(np.random.PCG64(16)).integers(-2, 3, 30000).astype(np.float64)
    _same_run(fem, "qubo", g, 32, ["exact"], linear=d)
    r = I.rgg(30000, 10.0, seed=17)
    _same_run(fem, "bmincut", r, 16, ["paper", "exact"], q=4)
    rw = I.Graph(r.n, r.ei, r.ej, np.random.Generator(np.random.PCG64(18)).uniform(0.5, 2.0, r.n_edges))
    _same_run(fem, "bmincut", rw, 16, ["paper"], q=3)


def test_device_build_rejects_duplicates_and_empty_rows_work(fem):
    g = I.er_gnm(40000, 120000, seed=19, weights="pm1")
    ei = np.concatenate([g.ei, [g.ej[77]]])
    ej = np.concatenate([g.ej, [g.ei[77]]])   # edge 77 again, reversed
    w = np.concatenate([g.w, [1.0]])
    fem.fem_set_device_graph_build(0)
    try:
        with pytest.raises(fem.FemError) as e:
            fem.Problem("maxcut", graph=I.Graph(g.n, ei, ej, w))
        assert e.value.status == fem.FEM_ERR_INVALID_ARG
        # many isolated nodes (n much larger than the edges touch)
        sparse = I.Graph(1 << 18, g.ei, g.ej, g.w)
    finally:
        fem.fem_set_device_graph_build(1 << 16)
    _same_run(fem, "maxcut", sparse, 32, ["paper"])


@pytest.mark.parametrize("defect", ["out_of_range", "self_loop", "nan_weight", "zero_weight", "negative_bmincut"])
def test_device_validation_names_the_first_invalid_edge(fem, defect):
    """Large edge lists are validated on the device: two invalid edges are planted and
    the error names the lower one, with the host builder's message."""
    n = 40000
    g = I.er_gnm(n, 120000, seed=21, weights="pm1")
    ei, ej, w = g.ei.copy(), g.ej.copy(), g.w.copy()
    kind, q = "maxcut", 2
    if defect == "negative_bmincut":
        kind, q = "bmincut", 4
        w = np.abs(w)
    for b in (99999, 70001):
        if defect == "out_of_range":
            ej[b] = n
        elif defect == "self_loop":
            ej[b] = ei[b]
        elif defect == "nan_weight":
            w[b] = np.nan
        elif defect == "zero_weight":
            w[b] = 0.0
        else:
            w[b] = -1.0
    msgs = []
    try:
        for thr in (0, -1):   # device validation, host validation
            fem.fem_set_device_graph_build(thr)
            with pytest.raises(fem.FemError) as e:
                fem.Problem(kind, graph=I.Graph(n, ei, ej, w), q=q)
            assert e.value.status == fem.FEM_ERR_INVALID_ARG
            msgs.append(str(e.value))
    finally:
        fem.fem_set_device_graph_build(1 << 16)
    assert "edge 70001:" in msgs[0], msgs[0]
    assert msgs[0] == msgs[1]
    # the device is still usable: a valid problem of the same size builds and anneals
    P = fem.Problem("maxcut", graph=g)
    P.anneal(h_init=I.initial_fields(n, 32, seed=22), n_steps=20)
    assert P.best()["energy_i64"].shape == (32,)


def _clauses_from(n, clauses):
    ptr = np.concatenate([[0], np.cumsum([len(c) for c in clauses])]).astype(np.int64)
    return I.Clauses(n, ptr, np.concatenate(clauses).astype(np.int32))


def _mixed(n, m, k_lo, k_hi, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [((rng.choice(n, size=int(k), replace=False) + 1) * (rng.integers(0, 2, size=int(k)) * 2 - 1))
            for k in rng.integers(k_lo, k_hi + 1, size=m)]


def _same_clause_run(fem, make, n, R=16, seed=41):
    h0 = I.initial_fields(n, R, seed=seed)
    dev, host = _both(fem, make)
    for P in (dev, host):
        P.anneal(h_init=h0, n_steps=200, t_end=60)
    for a, b, name in zip(dev.state(), host.state(), "hmv"):
        assert np.array_equal(a, b), name
    rd, rh = dev.best(), host.best()
    assert np.array_equal(rd["energy_i64"], rh["energy_i64"]) and np.array_equal(rd["energy_f64"], rh["energy_f64"])
    assert rd["best_replica"] == rh["best_replica"]


def test_clause_lists_device_build_equals_host_build(fem):
    n = 30000
    sat3 = I.random_ksat(n, 126000, 3, seed=31)
    _same_clause_run(fem, lambda: fem.Problem("sat", clauses=sat3), n)
    mixed = _clauses_from(n, _mixed(n, 60000, 1, 8, seed=32))
    _same_clause_run(fem, lambda: fem.Problem("sat", clauses=mixed), n)
    rng = np.random.Generator(np.random.PCG64(33))
    J3, b3 = rng.normal(size=sat3.n_clauses), 0.3 * rng.normal(size=n)
    _same_clause_run(fem, lambda: fem.Problem("pspin", clauses=sat3, term_weight=J3, linear=b3), n)
    terms = _clauses_from(n, _mixed(n, 50000, 2, 5, seed=34))
    Ji, bi = np.round(3 * rng.normal(size=terms.n_clauses)), np.round(2 * rng.normal(size=n))
    _same_clause_run(fem, lambda: fem.Problem("pspin", clauses=terms, term_weight=Ji, linear=bi), n)


@pytest.mark.parametrize("defect", ["zero_literal", "out_of_range", "repeated_variable", "too_wide",
                                    "decreasing_ptr", "nan_term"])
def test_device_clause_validation_names_the_first_invalid_clause(fem, defect):
    n, m = 30000, 126000
    cl = [c for c in _mixed(n, m, 3, 3, seed=35)]
    ptr_fix = None
    for c in (99999, 70001):
        x = cl[c].copy()
        if defect == "zero_literal":
            x[0] = 0
        elif defect == "out_of_range":
            x[1] = n + 1
        elif defect == "repeated_variable":
            x[2] = -x[0]
        elif defect == "too_wide":
            x = np.concatenate([x, (np.arange(6) + (x.max() % 1000) + 20000) % n + 1])
        cl[c] = x
    clauses = _clauses_from(n, cl)
    if defect == "decreasing_ptr":
        ptr_fix = clauses.ptr.copy()
        ptr_fix[70002] = ptr_fix[70001] - 1
        ptr_fix[100000] = ptr_fix[99999] - 1
        clauses = I.Clauses(n, ptr_fix, clauses.lits)
    tw = np.ones(m)
    if defect == "nan_term":
        tw[70001] = tw[99999] = np.nan
    msgs = []
    try:
        for thr in (0, -1):   # device validation, host validation
            fem.fem_set_device_graph_build(thr)
            with pytest.raises(fem.FemError) as e:
                if defect == "nan_term":
                    fem.Problem("pspin", clauses=clauses, term_weight=tw)
                else:
                    fem.Problem("sat", clauses=clauses)
            msgs.append((e.value.status, str(e.value)))
    finally:
        fem.fem_set_device_graph_build(1 << 16)
    assert msgs[0] == msgs[1], msgs
    expect = {"too_wide": fem.FEM_ERR_UNSUPPORTED}.get(defect, fem.FEM_ERR_INVALID_ARG)
    assert msgs[0][0] == expect
    if defect != "decreasing_ptr":
        assert "70001" in msgs[0][1], msgs[0][1]
    # the device is still usable
    ok = I.random_ksat(n, m, 3, seed=36)
    P = fem.Problem("sat", clauses=ok)
    P.anneal(h_init=I.initial_fields(n, 16, seed=37), n_steps=20)
    assert np.array_equal(P.best()["energy_i64"], O.sat_unsat(ok.ptr, ok.lits, P.states().astype(np.int8)))
