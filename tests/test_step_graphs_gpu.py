"""Short-step windows of small problems run as cached CUDA graphs: the fields after a
graph-replayed window must equal those of the same steps launched one by one."""
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
    return F


CASES = [
    ("maxcut", dict(graph=I.er_gnm(300, 1500, seed=61, weights="pm1")), 32, 2, dict(grad_mode="paper")),
    ("maxcut", dict(graph=I.er_gnm(300, 1500, seed=62, weights="unit")), 64, 2, dict(grad_mode="exact")),
    ("bmincut", dict(graph=I.rgg(400, 8.0, seed=63)), 16, 4, dict(grad_mode="paper")),
    ("sat", dict(clauses=I.random_ksat(300, 1260, 3, seed=64)), 16, 2, dict(optimizer="rmsprop", lr=0.01)),
]


@pytest.mark.parametrize("kind,inst,R,q,kw", CASES)
def test_graph_windows_equal_direct_steps(fem, kind, inst, R, q, kw):
    n = (inst.get("graph") or inst.get("clauses")).n
    h0 = I.initial_fields(n, R, seed=65, q=q) if kind == "bmincut" else I.initial_fields(n, R, seed=65)
    extra = dict(q=q) if kind == "bmincut" else {}
    # direct: the whole anneal is the problem's first window
    ref = fem.Problem(kind, **inst, **extra).anneal(h_init=h0, n_steps=120, **kw).state()
    P = fem.Problem(kind, **inst, **extra)
    for rep in range(2):   # first: capture, second: the cached graph
        P.anneal(h_init=h0, n_steps=120, t_end=1, **kw)
        P.anneal(n_steps=120, t_begin=1, replicas=R, **kw)
        got = P.state()
        for a, b, name in zip(got, ref, "hmv"):
            assert np.array_equal(a, b), (kind, rep, name, int(np.sum(a != b)))
