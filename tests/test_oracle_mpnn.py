"""Pins of the warm-start network's FP64 oracle (backward vs finite differences,
the spin-flip symmetry, the bf16 rounding)."""
import numpy as np
import pytest

import oracle as O
from paper_2412_09285_b300 import instances as I


def _setup(n=60, R=3, seed=0):
    g = I.er_gnm(n, 4 * n, seed=seed, weights="pm1")
    P, deg, W = O.mpnn_propagation(g.n, g.ei, g.ej, g.w)
    feats = O.mpnn_features(deg, W)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    z = rng.standard_normal((n, R))
    m_t = np.tanh(rng.standard_normal((n, R)))
    params = I.mpnn_init(seed + 2)
    params["C"] = rng.standard_normal((64, 4)) * 0.3        # non-trivial taps for the test
    params["c"] = rng.standard_normal(4) * 0.3
    for l in (1, 2, 3):
        params[f"b{l}"] = rng.standard_normal(64) * 0.1
    return P, feats, z, m_t, params


def test_backward_matches_finite_differences():
    P, feats, z, m_t, params = _setup()
    y, cache = O.mpnn_forward(params, P, feats, z, round_weights=False)
    grads = O.mpnn_backward(cache, y, m_t)
    rng = np.random.Generator(np.random.PCG64(9))
    eps = 1e-6
    for name in O.PARAM_ORDER:
        flat = params[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = O.mpnn_loss(O.mpnn_forward(params, P, feats, z, round_weights=False)[0], m_t)
            flat[idx] = old - eps
            lm = O.mpnn_loss(O.mpnn_forward(params, P, feats, z, round_weights=False)[0], m_t)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = grads[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 + 1e-6 * abs(fd), (name, idx, fd, an)


def test_prediction_is_odd_in_the_replica_fields():
    P, feats, z, _, params = _setup()
    y1, _ = O.mpnn_forward(params, P, feats, z)
    y2, _ = O.mpnn_forward(params, P, feats, -z)
    assert np.allclose(y1, -y2, rtol=0, atol=1e-13)


def test_initial_taps_reproduce_the_input_fields():
    P, feats, z, _, _ = _setup()
    params = I.mpnn_init(5)
    params["C"][:] = 0.0                                      # theta = c = (1, 0, 0, 0)
    y, _ = O.mpnn_forward(params, P, feats, z)
    assert np.allclose(y, z, rtol=0, atol=1e-15)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.14159265, 0.0])
    r = O.bf16_round(x)
    assert r[0] == 1.0 and r[5] == 0.0
    # ties go to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> 1; 1 + 3*2^-8 -> 1 + 2^-6
    assert O.bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert O.bf16_round(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert O.bf16_round(np.array([-3.14159265]))[0] == -3.140625
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-300)


def test_normalize_sets_the_column_rms_and_keeps_directions():
    rng = np.random.Generator(np.random.PCG64(4))
    y = rng.standard_normal((500, 6)) * np.array([1e-4, 0.3, 1.0, 7.0, 1e3, 1.0])
    y[:, 5] = 0.0
    out = O.mpnn_normalize(y, 0.1)
    rms = np.sqrt((out ** 2).mean(axis=0))
    assert np.allclose(rms[:5], 0.1, rtol=1e-12) and rms[5] == 0.0
    # a positive multiple of the input column: the cosine with it is 1
    for r in range(5):
        c = out[:, r] @ y[:, r] / (np.linalg.norm(out[:, r]) * np.linalg.norm(y[:, r]))
        assert abs(c - 1.0) < 1e-12
