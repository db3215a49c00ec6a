"""The device CSR builder (fem_create_problem for large edge lists) against the host
builder: the same graph built both ways must anneal to the same fields and energies bit
for bit (the CSR order and every row sum agree), in paper and exact mode, for unit,
+-1, integer and real weights, MaxCut, QUBO and bMinCut, with hub rows that take the
block sort (degree 33 .. 4096) and the host fallback (degree > 4096); a duplicate edge
is rejected by the device builder as by the host one."""
import numpy as np
import pytest

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
