"""Batched anneal (bMinCut + Max-k-SAT members, two launches per step, CUDA-graph
step loop, autotuned work items) against the same members annealed one by one.

Every member's arithmetic is the single-problem kernel's and the shared counts are
integers / fixed point, so each member's fields must be bit-identical to the
member annealed alone (which the other test files tie to the FP64 oracle).
"""
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
    return F


def _members(fem, seed):
    sizes = I.loguniform_sizes(5, 300, 4000, seed=seed)
    graphs = [I.rgg(int(n), 10.0, seed=seed + 10 + k) for k, n in enumerate(sizes)]
    sats = [I.random_ksat(int(n), int(4.2 * n), 3, seed=seed + 30 + k)
            for k, n in enumerate(I.loguniform_sizes(3, 500, 5000, seed=seed + 1))]
    return graphs, sats


def _make(fem, graphs, sats, q=4):
    return ([fem.Problem("bmincut", graph=g, q=q) for g in graphs]
            + [fem.Problem("sat", clauses=c) for c in sats])


@pytest.mark.parametrize("mode,q", [("paper", 4), ("exact", 4), ("paper", 8), ("exact", 8)])
def test_batch_bit_identical_to_members_alone(fem, mode, q):
    graphs, sats = _members(fem, 100)
    R = 16
    h0 = ([I.initial_fields(g.n, R, seed=200 + k, q=q) for k, g in enumerate(graphs)]
          + [I.initial_fields(c.n, R, seed=300 + k) for k, c in enumerate(sats)])
    solo = _make(fem, graphs, sats, q)
    for p, h in zip(solo, h0):
        p.anneal(h_init=h, n_steps=300, grad_mode=mode)
    probs = _make(fem, graphs, sats, q)
    b = fem.Batch(probs)
    b.anneal(h_inits=h0, replicas=R, n_steps=300, grad_mode=mode)
    for a, s in zip(probs, solo):
        assert np.array_equal(a.fields(), s.fields())
        ra, rs = a.best(), s.best()
        assert np.array_equal(ra["energy_i64"], rs["energy_i64"]) and ra["best_replica"] == rs["best_replica"]
    # and the batched read-out is the oracle's objective for the batched states
    for a, g in zip(probs[:len(graphs)], graphs):
        E, _, _ = O.bmincut_objective(g.ei, g.ej, g.w, a.states(), q, 1.0)
        assert np.array_equal(a.best()["energy_i64"], E)
    for a, c in zip(probs[len(graphs):], sats):
        assert np.array_equal(a.best()["energy_i64"], O.sat_unsat(c.ptr, c.lits, a.states().astype(np.int8)))


def test_batch_resume_and_repeat(fem):
    graphs, sats = _members(fem, 110)
    R = 16
    h0 = ([I.initial_fields(g.n, R, seed=400 + k, q=4) for k, g in enumerate(graphs)]
          + [I.initial_fields(c.n, R, seed=500 + k) for k, c in enumerate(sats)])
    full = _make(fem, graphs, sats)
    fem.Batch(full).anneal(h_inits=h0, replicas=R, n_steps=200)
    split = _make(fem, graphs, sats)
    b = fem.Batch(split)
    b.anneal(h_inits=h0, replicas=R, n_steps=200, t_end=71)
    b.anneal(replicas=R, n_steps=200, t_begin=71)
    for x, y in zip(full, split):
        assert np.array_equal(x.fields(), y.fields())
    # a second full anneal of the same batch (cached tuning and graph) repeats exactly
    b.anneal(h_inits=h0, replicas=R, n_steps=200)
    for x, y in zip(full, split):
        assert np.array_equal(x.fields(), y.fields())


def test_batch_rejects_unsupported_members(fem):
    g = I.er_gnp(100, 0.05, seed=1, weights="pm1")
    with pytest.raises(fem.FemError) as e:
        fem.Batch([fem.Problem("maxcut", graph=g)])
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    rg = I.rgg(200, 8.0, seed=2)
    with pytest.raises(fem.FemError) as e:
        fem.Batch([fem.Problem("bmincut", graph=rg, q=4), fem.Problem("bmincut", graph=rg, q=3)])
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED


def test_one_shot_batch_call_equals_batch_object(fem):
    """fem_anneal_batch (the batch built for one call and released after it) gives the
    batch object's results bit for bit, in two windows as in one."""
    graphs, sats = _members(fem, 140)
    R = 16
    h0 = ([I.initial_fields(g.n, R, seed=240 + k, q=4) for k, g in enumerate(graphs)]
          + [I.initial_fields(c.n, R, seed=340 + k) for k, c in enumerate(sats)])
    ref = _make(fem, graphs, sats)
    fem.Batch(ref).anneal(h_inits=h0, replicas=R, n_steps=200)
    got = _make(fem, graphs, sats)
    fem.anneal_batch(got, h0, replicas=R, n_steps=200, t_end=70)
    fem.anneal_batch(got, None, replicas=R, n_steps=200, t_begin=70)
    for a, b in zip(got, ref):
        assert np.array_equal(a.fields(), b.fields())
