"""Failure detection without a GPU fault: a device allocation that fails (injected
on the host) and the persistent dense kernel's step barrier running out of time (a
row tile whose CTAs never arrive, injected on the host).  Both surface as status
codes, and the device stays usable."""
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


def test_injected_allocation_failure(fem):
    g = I.er_gnm(500, 2000, seed=71, weights="pm1")
    h0 = I.initial_fields(500, 32, seed=72)
    failed = 0
    try:
        for after in range(0, 24, 2):
            fem.fem_inject_allocation_failure(after)
            try:
                fem.Problem("maxcut", graph=g).anneal(h_init=h0, n_steps=20).best()
            except fem.FemError as e:
                assert e.status == fem.FEM_ERR_OOM, e
                failed += 1
    finally:
        fem.fem_inject_allocation_failure(-1)
    assert failed >= 3
    ref = fem.Problem("maxcut", graph=g).anneal(h_init=h0, n_steps=20).best()
    assert ref["energy_i64"].min() < 0


@pytest.mark.parametrize("n,kind,tile", [(300, "persistent_single", 1), (500, "persistent", 0),
                                         (500, "persistent", 3)])
def test_step_barrier_timeout_is_reported(fem, n, kind, tile):
    """The CTAs of one row tile never arrive at the step barrier (a counter that never
    reaches its target, injected on the host); the CTAs waiting at it give up after
    1 ms.  n = 300: three row tiles, one CTA each; n = 500: four, in CTA pairs (the
    stalled CTA the even or the odd one of its pair)."""
    g = I.sk_dense(n, seed=73)
    h0 = I.initial_fields(n, 256, seed=74)
    P = fem.Problem("maxcut", dense=g.dense)
    P.set_dense_launch("persistent")
    fem.fem_set_step_barrier_timeout(P.handle, 1_000_000)
    fem.fem_inject_step_stall(P.handle, tile)
    P.anneal(h_init=h0, n_steps=50, precision="bf16")
    assert P.dense_last_launch() == kind
    with pytest.raises(fem.FemError) as e:
        P.best()
    assert e.value.status == fem.FEM_ERR_TIMEOUT
    # a fresh start without the stall clears the error and gives the normal result
    fem.fem_inject_step_stall(P.handle, -1)
    fem.fem_set_step_barrier_timeout(P.handle, 2_000_000_000)
    got = P.anneal(h_init=h0, n_steps=50, precision="bf16").state()
    Q = fem.Problem("maxcut", dense=g.dense)
    Q.set_dense_launch("per_step")
    ref = Q.anneal(h_init=h0, n_steps=50, precision="bf16").state()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    with pytest.raises(fem.FemError):
        fem.fem_set_step_barrier_timeout(P.handle, -1)
    with pytest.raises(fem.FemError):
        fem.fem_inject_step_stall(P.handle, -2)
