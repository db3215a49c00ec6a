"""The sparse MaxCut / QUBO steps on their two kernels each: the tile kernels that stage
their operands in shared memory (the defaults: exact mode with TMA gather4 copies of
the neighbours' lines, paper mode with bulk copies of the state and producer-gathered
sign words) and the kernels that load everything directly.  Both sum the neighbours in
CSR order with the same fp32 update, so every field, moment and energy must agree bit
for bit: unit, +-1 and real weights; hub rows longer than a tile's staged capacity
(the direct remainder); isolated nodes and n not a multiple of the tile; R = 32 and 64
(two replica blocks); QUBO offsets; Adam, RMSprop and SGD; both gradient modes.  The
oracle parity of both modes runs in tests/test_maxcut_gpu.py and tests/test_qubo_gpu.py
on the default kernels."""
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
    F.fem_set_tma_gather(True)


def _with_hubs(g, spec, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    have = {(a, b): x for a, b, x in zip(g.ei.tolist(), g.ej.tolist(), g.w.tolist())}
    for count, width in spec:
        for h in rng.choice(g.n, count, replace=False).tolist():
            for j in rng.choice(g.n, width, replace=False).tolist():
                if j != h:
                    have.setdefault((min(h, j), max(h, j)), float(rng.choice([-1.0, 1.0])))
    e = list(have)
    return I.Graph(g.n, [a for a, _ in e], [b for _, b in e], [have[k] for k in e])


def _both(fem, make, R, n_steps=120, t_end=60, mode="exact", **kw):
    out = []
    for on in (True, False):
        fem.fem_set_tma_gather(on)
        P = make()
        P.anneal(h_init=I.initial_fields(P.n, R, seed=7), n_steps=n_steps, t_end=t_end, grad_mode=mode, **kw)
        out.append((P.state(), P.best()))
    fem.fem_set_tma_gather(True)
    (sa, ra), (sb, rb) = out
    for x, y, name in zip(sa, sb, "hmv"):
        assert np.array_equal(x, y), name
    assert np.array_equal(ra["energy_i64"], rb["energy_i64"]) and np.array_equal(ra["energy_f64"], rb["energy_f64"])
    assert ra["best_replica"] == rb["best_replica"]


@pytest.mark.parametrize("mode", ["exact", "paper"])
@pytest.mark.parametrize("weights", ["unit", "pm1", "real"])
@pytest.mark.parametrize("R", [32, 64])
def test_tile_kernel_equals_direct_kernel(fem, weights, R, mode):
    g = I.er_gnm(20011, 60000, seed=3, weights=weights)   # n not a multiple of the tile
    _both(fem, lambda: fem.Problem("maxcut", graph=g), R, mode=mode)


@pytest.mark.parametrize("mode", ["exact", "paper"])
@pytest.mark.parametrize("weights", ["pm1", "real"])
def test_hub_rows_and_isolated_nodes(fem, mode, weights):
    g = _with_hubs(I.er_gnm(20000, 30000, seed=4, weights="pm1"), [(3, 300), (1, 6000)], seed=5)
    w = g.w if weights == "pm1" else np.random.Generator(np.random.PCG64(55)).uniform(0.5, 2.0, g.n_edges)
    sparse = I.Graph(1 << 16, g.ei, g.ej, w)   # many isolated nodes
    _both(fem, lambda: fem.Problem("maxcut", graph=sparse), 32, mode=mode)


@pytest.mark.parametrize("mode", ["exact", "paper"])
@pytest.mark.parametrize("opt,kw", [("rmsprop", dict(lr=0.02, alpha=0.9, momentum=0.5)),
                                    ("sgd", dict(lr=0.5, momentum=0.6, dampening=0.1))])
def test_other_optimizers(fem, opt, kw, mode):
    g = I.er_gnm(9000, 27000, seed=6, weights="pm1")
    _both(fem, lambda: fem.Problem("maxcut", graph=g), 32, mode=mode, optimizer=opt, **kw)


def test_qubo_offsets(fem):
    g = I.er_gnm(15000, 45000, seed=8, weights="pm1")
    d = np.random.Generator(np.random.PCG64(9)).integers(-2, 3, 15000).astype(np.float64)
    _both(fem, lambda: fem.Problem("qubo", graph=g, linear=d), 32)


@pytest.mark.parametrize("mode", ["exact", "paper"])
def test_full_size_one_window(fem, mode):
    g = I.er_gnm(1 << 20, 3 << 20, seed=2024, weights="pm1")
    _both(fem, lambda: fem.Problem("maxcut", graph=g), 32, n_steps=2000, t_end=5, mode=mode)
