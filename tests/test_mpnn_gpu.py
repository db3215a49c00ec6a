"""The warm-start network on the GPU against its FP64 oracle (forward, gradients,
rescaled prediction), and what the trained network gains over plain random-initialised
FEM and over the shortened schedule without it."""
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
    from paper_2412_09285_b300 import fem, warmstart
    return fem, warmstart, torch


def _params(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    p = I.mpnn_init(seed)
    p["C"] = rng.standard_normal((64, 4)) * 0.3
    p["c"] = rng.standard_normal(4) * 0.3
    for l in (1, 2, 3):
        p[f"b{l}"] = rng.standard_normal(64) * 0.1
    return p


def _case(fem, torch, n=500, m=2000, R=32, seed=3):
    g = I.er_gnm(n, m, seed=seed, weights="pm1")
    prob = fem.Problem("maxcut", graph=g)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    z = rng.standard_normal((n, R)).astype(np.float32)
    ht = (2.0 * rng.standard_normal((n, R))).astype(np.float32)
    P, deg, W = O.mpnn_propagation(g.n, g.ei, g.ej, g.w)
    feats = O.mpnn_features(deg, W)
    dev = torch.device("cuda")
    return g, prob, z, ht, P, feats, torch.from_numpy(z).to(dev), torch.from_numpy(ht).to(dev)


def test_forward_matches_oracle(env):
    fem, ws, torch = env
    g, prob, z, ht, P, feats, zd, _ = _case(fem, torch)
    params = _params(11)
    net = ws.Mpnn(params)
    y = torch.empty_like(zd)
    net.predict(prob, zd, z.shape[1], y)
    torch.cuda.synchronize()
    y_ref, _ = O.mpnn_forward(params, P, feats, z.astype(np.float64))
    err = np.abs(y.cpu().numpy() - y_ref).max() / np.abs(y_ref).max()
    assert err <= 1e-4, err


def test_gradients_match_oracle(env):
    fem, ws, torch = env
    g, prob, z, ht, P, feats, zd, htd = _case(fem, torch)
    params = _params(12)
    net = ws.Mpnn(params)
    grads, loss = net.grad(prob, zd, htd, z.shape[1])
    y_ref, cache = O.mpnn_forward(params, P, feats, z.astype(np.float64))
    m_t = np.tanh(0.5 * ht.astype(np.float64))
    ref = O.mpnn_backward(cache, y_ref, m_t)
    assert loss == pytest.approx(O.mpnn_loss(y_ref, m_t), rel=1e-5)
    for name in O.PARAM_ORDER:
        scale = np.abs(ref[name]).max()
        err = np.abs(grads[name] - ref[name]).max()
        assert err <= 1e-3 * scale + 1e-9, (name, err, scale)


def test_predict_rms_matches_oracle(env):
    fem, ws, torch = env
    g, prob, z, ht, P, feats, zd, _ = _case(fem, torch)
    params = _params(13)
    net = ws.Mpnn(params)
    y = torch.empty_like(zd)
    net.predict(prob, zd, z.shape[1], y, rms=0.1)
    torch.cuda.synchronize()
    y_ref = O.mpnn_normalize(O.mpnn_forward(params, P, feats, z.astype(np.float64))[0], 0.1)
    err = np.abs(y.cpu().numpy() - y_ref).max() / np.abs(y_ref).max()
    assert err <= 1e-4, err
    with pytest.raises(fem.FemError):
        net.predict(prob, zd, z.shape[1], y, rms=-1.0)


def test_training_and_warm_start_gain(env):
    """Train on FEM's converged fields of small ER graphs (+-1 weights, mean degree 8),
    then on held-out graphs compare best cuts (32 replicas) of
      * the warm start: the prediction rescaled to rms 0.1, then a quarter-length
        schedule from beta(N/4) of the full one,
      * the same schedule from random fields of the same rms (the control: what the
        shortened schedule gives without the network),
      * plain FEM with the same budget and with the full budget N.
    The numbers are printed; the test requires the training loss to fall and the warm
    start to beat the control on average over the held-out graphs."""
    fem, ws, torch = env
    dev = torch.device("cuda")
    R, N = 32, 400
    train = ws.make_graphs(32, 1500, 4000, 8.0, seed=7)
    held = ws.make_graphs(8, 1500, 4000, 8.0, seed=8)
    net = ws.Mpnn(seed=1)
    losses = ws.train(net, train, 8, R, N, lr=3e-3, seed=11)
    assert losses[-1] < losses[0], losses
    cut = lambda r: -int(r["energy_i64"].min())
    res = {}
    for k, g in enumerate(held):
        z = torch.from_numpy(I.initial_fields(g.n, R, seed=777 + k) * np.float32(1000.0)).to(dev)
        pf = fem.Problem("maxcut", graph=g).anneal(h_init=z * 0.001, replicas=R, n_steps=N)
        full = cut(pf.best())
        y = torch.empty_like(z)
        net.predict(pf, z, R, y, rms=0.1)
        zn = torch.empty_like(z)
        ws.Mpnn(I.mpnn_init(0) | {"C": np.zeros((64, 4)), "c": np.array([1.0, 0.0, 0.0, 0.0])}).predict(
            pf, z, R, zn, rms=0.1)  # taps (1, 0, 0, 0): the noise itself, rescaled by the same kernels
        b = N // 4
        for name, h in (("warm", y), ("control", zn)):
            p = fem.Problem("maxcut", graph=g)
            ws.warm_anneal(p, h, b, N, N // 4)
            res.setdefault(name, []).append(cut(p.best()) - full)
        plain = fem.Problem("maxcut", graph=g).anneal(h_init=z * 0.001, replicas=R, n_steps=b)
        res.setdefault("plain", []).append(cut(plain.best()) - full)
    print(f"\ntraining loss by epoch: {[round(x, 4) for x in losses]}")
    for name, v in res.items():
        print(f"{name:8s} ({N // 4} steps): best cut minus plain FEM's at {N} steps, mean {np.mean(v):+.1f}, "
              f"per graph {v}")
    assert np.mean(res["warm"]) > np.mean(res["control"])
