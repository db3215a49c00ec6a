"""The allocation-free MaxCut energy entry point against the library's own read-out.

fem_maxcut_energies_noalloc serves callers that cannot allocate device memory
(memory owned by a pool manager, or loops where an allocation could synchronise
the device): they pass every buffer in, and the entry point's only scratch is a
fixed array in the library's device image.  This test calls it through the C ABI
twice in a row, on two different problems, and checks both results against
fem_read_best (integer energies: bit-exact) and against the oracle's cut of the same
states.  Further cases: the largest replica count (1024, every scratch row and every
thread of the final argmin), a graph of a few hundred nodes (fewer blocks than scratch
rows), a malformed CSR (reported as best replica -1, nothing read out of bounds, the
next call clean again), and oversized requests refused before anything runs.  It is
collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
from paper_2412_09285_b300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2412_09285_b300 import build
    build.build()
    from paper_2412_09285_b300 import fem
    return fem, torch


def _library_csr(g):
    """Both directions of every edge, rows sorted by column, the +-1 weight in bit 31."""
    src = np.concatenate([g.ei, g.ej]).astype(np.int64)
    dst = np.concatenate([g.ej, g.ei]).astype(np.int64)
    w = np.concatenate([g.w, g.w])
    order = np.lexsort((dst, src))
    src, dst, w = src[order], dst[order], w[order]
    row_ptr = np.zeros(g.n + 1, np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    col = (dst.astype(np.uint32) | np.where(w < 0, np.uint32(1 << 31), np.uint32(0))).astype(np.uint32)
    return row_ptr, col


def _sign_words(states):
    n, R = states.shape
    bits = (states == -1).reshape(n, R // 32, 32)
    return np.packbits(bits, axis=2, bitorder="little").view(np.uint32).reshape(n, R // 32)


def _call(fem, torch, row_ptr, col, n, words, R):
    dev = torch.device("cuda")
    d_row = torch.from_numpy(row_ptr).to(dev)
    d_col = torch.from_numpy(col.view(np.int32)).to(dev)
    d_words = torch.from_numpy(words.view(np.int32)).to(dev)
    energy = torch.full((R,), 7, dtype=torch.int64, device=dev)
    best = torch.full((1,), -2, dtype=torch.int32, device=dev)
    fem.fem_maxcut_energies_noalloc(d_row, d_col, n, d_words, R, energy, best)
    torch.cuda.synchronize()
    return energy.cpu().numpy(), int(best.cpu().item())


def _run_case(fem, torch, n, m, R, seed):
    g = I.er_gnm(n, m, seed=seed, weights="pm1")
    P = fem.Problem("maxcut", graph=g)
    P.anneal(h_init=I.initial_fields(n, R, seed=seed + 1), n_steps=300)
    ref = P.best()
    states = P.states()
    row_ptr, col = _library_csr(g)
    energy, best = _call(fem, torch, row_ptr, col, n, _sign_words(states), R)
    assert np.array_equal(energy, ref["energy_i64"])
    assert best == ref["best_replica"]
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, states.astype(np.int8))
    assert np.array_equal(energy, -cut)
    assert best == O.best_replica(-cut)
    return g, states


def test_noalloc_energies_match_read_best_two_calls(env):
    fem, torch = env
    _run_case(fem, torch, 4000, 12000, 32, seed=71)     # first call (sets the scratch address up)
    _run_case(fem, torch, 2500, 9000, 64, seed=73)      # second call reuses the scratch


def test_noalloc_largest_replica_count_and_small_graph(env):
    fem, torch = env
    _run_case(fem, torch, 3000, 9000, 1024, seed=75)    # every scratch row, 1024-thread argmin
    _run_case(fem, torch, 300, 900, 96, seed=77)        # 38 blocks of the first kernel


def test_noalloc_malformed_csr_reported(env):
    """A column index >= n and a row range beyond row_ptr[n] are skipped by the kernel
    and reported as best replica -1; the next call on valid input is clean again."""
    fem, torch = env
    g = I.er_gnm(500, 1500, seed=79, weights="pm1")
    row_ptr, col = _library_csr(g)
    states = np.where(I.initial_fields(500, 32, seed=80) >= 0, 1, -1)
    words = _sign_words(states)
    bad_col = col.copy()
    bad_col[7] = (bad_col[7] & np.uint32(1 << 31)) | np.uint32(500)
    _, best = _call(fem, torch, row_ptr, bad_col, 500, words, 32)
    assert best == -1
    bad_row = row_ptr.copy()
    bad_row[250] = bad_row[-1] + 5
    _, best = _call(fem, torch, bad_row, col, 500, words, 32)
    assert best == -1
    energy, best = _call(fem, torch, row_ptr, col, 500, words, 32)
    cut = O.maxcut_cut_edges(g.ei, g.ej, g.w, states.astype(np.int8))
    assert np.array_equal(energy, -cut) and best == O.best_replica(-cut)


def test_noalloc_rejects_oversized_requests(env):
    fem, torch = env
    dev = torch.device("cuda")
    dummy = torch.zeros(16, dtype=torch.int32, device=dev)
    energy = torch.zeros(2048, dtype=torch.int64, device=dev)
    with pytest.raises(fem.FemError) as e:
        fem.fem_maxcut_energies_noalloc(dummy, dummy, 4, dummy, 2048, energy, dummy)
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    with pytest.raises(fem.FemError) as e:
        fem.fem_maxcut_energies_noalloc(dummy, dummy, 4, dummy, 48, energy, dummy)
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
