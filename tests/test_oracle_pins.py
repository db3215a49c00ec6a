"""Pins of the FP64 oracle against things other than itself.

Each test ties an oracle function to a definition, a closed form, an invariant, a
library routine or a brute-force result, chosen so that a dropped term, a wrong
sign, a factor 2 or a transposed operand fails at least one of them.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_09285_b300 import instances as I


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------- schedules

def test_beta_schedules_endpoints_and_shape():
    n = 1000
    b = O.beta_schedule("exponential", 0.05, 5.0, n)
    assert b[0] == pytest.approx(0.05, rel=1e-15) and b[-1] == pytest.approx(5.0, rel=1e-14)
    r = b[1:] / b[:-1]                                      # geometric: constant ratio
    assert np.allclose(r, (5.0 / 0.05) ** (1.0 / (n - 1)), rtol=1e-12)
    b2 = O.beta_schedule("inverse_proportional", 1 / 1.16, 1 / 6e-5, 1100)
    T = 1.0 / b2                                            # linear cooling in T
    assert T[0] == pytest.approx(1.16) and T[-1] == pytest.approx(6e-5)
    assert np.allclose(np.diff(T), (6e-5 - 1.16) / 1099, rtol=1e-9)
    lam = O.lambda_ramp(2.0, 11)
    assert lam[0] == 0.0 and lam[-1] == 2.0 and np.allclose(np.diff(lam), 0.2)
    assert O.beta_schedule("exponential", 0.05, 5.0, 1)[0] == 0.05


# ---------------------------------------------------- free energies by Eq. FP

def _small_graph(n, p, seed, weights):
    g = I.er_gnp(n, p, seed, weights)
    return g, O.coupling_matrix(g.n, g.ei, g.ej, g.w)


def test_maxcut_free_energy_matches_enumeration():
    g, W = _small_graph(7, 0.6, 1, "real")
    h = _rng(2).normal(size=(7, 2))
    beta = 0.7
    F = O.maxcut_free_energy(W, h, beta)
    for r in range(2):
        P = O.sigmoid(h[:, r])
        marg = np.stack([P, 1 - P], axis=1)                 # state 0 = sigma +1
        # ordered-pair energy: each edge counted twice, E2 = -2 sum_E W [x_i != x_j]
        E = lambda X: -2.0 * (g.w[None, :] * (X[:, g.ei] != X[:, g.ej])).sum(axis=1)
        ref = O.mf_free_energy_by_enumeration(marg, E, beta)
        assert F[r] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_bmincut_free_energy_matches_enumeration():
    g, W = _small_graph(5, 0.7, 3, "real")
    q, beta, lam = 3, 1.3, 0.4
    h = _rng(4).normal(size=(5, 2, q))
    F = O.bmincut_free_energy(W, h, beta, lam)
    for r in range(2):
        z = np.exp(h[:, r] - h[:, r].max(axis=1, keepdims=True))
        marg = z / z.sum(axis=1, keepdims=True)

        def E(X):
            cut = (g.w[None, :] * (X[:, g.ei] != X[:, g.ej])).sum(axis=1)
            sizes = np.stack([(X == s).sum(axis=1) for s in range(q)], axis=1)
            return 2.0 * cut + lam * (sizes * (sizes - 1)).sum(axis=1)

        ref = O.mf_free_energy_by_enumeration(marg, E, beta)
        assert F[r] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_sat_free_energy_matches_enumeration():
    cl = I.random_ksat(6, 11, 3, seed=5)
    groups = O.sat_arrays(cl.ptr, cl.lits)
    h = _rng(6).normal(size=(6, 2))
    beta = 0.9
    F = O.sat_free_energy(groups, h, beta)
    for r in range(2):
        p = O.sigmoid(h[:, r])
        marg = np.stack([1 - p, p], axis=1)                 # state index = sigma value

        def E(X):
            out = np.zeros(X.shape[0])
            for m in range(cl.n_clauses):
                sat = np.zeros(X.shape[0], bool)
                for l in cl.lits[cl.ptr[m]:cl.ptr[m + 1]]:
                    sat |= (X[:, abs(l) - 1] == (1 if l > 0 else 0))
                out += ~sat
            return out

        ref = O.mf_free_energy_by_enumeration(marg, E, beta)
        assert F[r] == pytest.approx(ref, rel=1e-12, abs=1e-12)


# ------------------------------------------- exact gradients = FD of the energy

def _fd(Ffun, h, eps=1e-6):
    g = np.zeros_like(h)
    flat = h.reshape(h.shape[0], h.shape[1], -1)
    gflat = g.reshape(flat.shape)
    for i in range(flat.shape[0]):
        for s in range(flat.shape[2]):
            hp = flat.copy(); hp[i, :, s] += eps
            hm = flat.copy(); hm[i, :, s] -= eps
            gflat[i, :, s] = (Ffun(hp.reshape(h.shape)) - Ffun(hm.reshape(h.shape))) / (2 * eps)
    return g


@pytest.mark.parametrize("weights", ["unit", "pm1", "real"])
def test_maxcut_exact_gradient_is_fd_of_F(weights):
    g, W = _small_graph(12, 0.4, 7, weights)
    h = _rng(8).normal(size=(12, 3)) * 1.5
    beta = 0.8
    ana = O.maxcut_grad(W, h, beta, mode="exact")
    fd = _fd(lambda x: O.maxcut_free_energy(W, x, beta), h)
    assert np.max(np.abs(ana - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_bmincut_exact_gradient_is_fd_of_F():
    g, W = _small_graph(8, 0.5, 9, "real")
    h = _rng(10).normal(size=(8, 2, 4))
    beta, lam = 0.6, 0.3
    ana = O.bmincut_grad(W, h, beta, lam, mode="exact")
    fd = _fd(lambda x: O.bmincut_free_energy(W, x, beta, lam), h)
    assert np.max(np.abs(ana - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))
    # softmax invariance: the field gradient sums to zero over the states
    assert np.allclose(ana.sum(axis=2), 0.0, atol=1e-13)


def test_sat_gradient_is_fd_of_F():
    cl = I.random_ksat(10, 30, 3, seed=11)
    groups = O.sat_arrays(cl.ptr, cl.lits)
    h = _rng(12).normal(size=(10, 2))
    beta = 1.1
    ana = O.sat_grad(groups, h, beta)
    fd = _fd(lambda x: O.sat_free_energy(groups, x, beta), h)
    assert np.max(np.abs(ana - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_sat_gradient_mixed_widths_is_fd_of_F():
    ptr = np.array([0, 2, 5, 9, 10])
    lits = np.array([1, -2, 2, 3, -4, -1, 4, 5, -3, 5])
    groups = O.sat_arrays(ptr, lits)
    h = _rng(13).normal(size=(5, 2))
    ana = O.sat_grad(groups, h, 0.5)
    fd = _fd(lambda x: O.sat_free_energy(groups, x, 0.5), h)
    assert np.max(np.abs(ana - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


# ------------------------------------------------- paper-mode reduction identities

def test_maxcut_paper_mode_reduces_to_exact():
    g, W = _small_graph(20, 0.3, 14, "pm1")
    h = _rng(15).normal(size=(20, 4))
    exact = O.maxcut_grad(W, h, 0.7, mode="exact")
    red = O.maxcut_grad(W, h, 0.7, mode="paper", c=np.full(20, 2.0), discretise=False)
    assert np.allclose(red, exact, rtol=1e-13, atol=1e-15)


def test_maxcut_paper_mode_formula_and_ties():
    # a 3-node path 0-1-2 with weights 1 and -2; h_1 = 0 must count as sgn = +1
    W = O.coupling_matrix(3, [0, 1], [1, 2], [1.0, -2.0])
    h = np.array([[0.3], [0.0], [-0.2]])
    g = O.maxcut_grad(W, h, 2.0, gamma=1.0, mode="paper")
    m = np.tanh(h[:, 0] / 2)
    # node 0: c = 1, neighbour 1 has sgn +1;  node 1: c = 1/3, sum = 1*(+1) - 2*(-1) = 3
    # node 2: c = 1/2, neighbour 1 sgn +1, weight -2
    s = np.array([1.0, 3.0 / 3.0, -2.0 / 2.0])
    expect = 0.25 * (s + h[:, 0] / 2.0) * (1 - m * m)
    assert np.allclose(g[:, 0], expect, rtol=1e-14)
    assert O.maxcut_states(np.array([[0.0], [-0.0], [-1e-300]]))[:, 0].tolist() == [1, 1, -1]


def test_bmincut_paper_mode_reduces_to_exact():
    g, W = _small_graph(10, 0.5, 16, "real")
    h = _rng(17).normal(size=(10, 3, 4))
    exact = O.bmincut_grad(W, h, 0.9, 0.25, mode="exact")
    red = O.bmincut_grad(W, h, 0.9, 0.25, mode="paper", cf=np.full(10, 2.0),
                         ca=np.full(10, 2.0), discretise=False)
    assert np.allclose(red, exact, rtol=1e-12, atol=1e-14)


def test_bmincut_argmax_ties_lowest_index():
    h = np.array([[[0.5, 0.5, 0.1, 0.5]]])
    assert O.bmincut_states(h)[0, 0] == 0


# --------------------------------------------------- mean-field fixed point

def test_exact_mode_fixed_point_is_mean_field_equation():
    """At a fixed beta, the exact-gradient stationary point satisfies the
    mean-field equation m = tanh(-beta W m) (SM, 'mean field equations for the
    Ising problem', with W -> -W for the antiferromagnetic MaxCut coupling)."""
    g, W = _small_graph(24, 0.3, 18, "pm1")
    h0 = _rng(19).normal(size=(24, 3))
    beta = 0.35
    h, _ = O.anneal(("maxcut", W), h0, 6000, schedule="exponential", beta_min=beta,
                    beta_max=beta, optimizer="sgd", opt_kw=dict(lr=1.0), mode="exact")
    m = np.tanh(h / 2)
    resid = np.abs(m - np.tanh(-beta * (W @ m)))
    assert resid.max() < 1e-9
    # and the fixed point is not the trivial one for this beta (the test has teeth)
    assert np.abs(m).max() > 0.1


# -------------------------------------------------------------- optimizers

def _torch_run(opt_cls, kw, gs, h0):
    p = torch.tensor(h0, dtype=torch.float64, requires_grad=True)
    opt = opt_cls([p], **kw)
    for g in gs:
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    return p.detach().numpy()


@pytest.mark.parametrize("name,kw", [
    ("adam", dict(lr=0.1, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.0)),
    ("adam", dict(lr=0.03, betas=(0.8, 0.99), eps=1e-6, weight_decay=0.01)),
    ("rmsprop", dict(lr=0.03, alpha=0.56, eps=1e-8, weight_decay=0.013, momentum=0.63)),
    ("rmsprop", dict(lr=0.01, alpha=0.99, eps=1e-8, weight_decay=0.0, momentum=0.0)),
    ("sgd", dict(lr=1.27, momentum=0.71, dampening=0.11, weight_decay=0.018)),
    ("sgd", dict(lr=0.2, momentum=0.0, dampening=0.0, weight_decay=0.0)),
])
def test_optimizers_match_torch(name, kw):
    rng = _rng(20)
    h0 = rng.normal(size=(5, 3))
    gs = [rng.normal(size=(5, 3)) for _ in range(25)]
    cls = {"adam": torch.optim.Adam, "rmsprop": torch.optim.RMSprop, "sgd": torch.optim.SGD}[name]
    ref = _torch_run(cls, kw, gs, h0)
    okw = dict(kw)
    if "betas" in okw:
        okw["beta1"], okw["beta2"] = okw.pop("betas")
    opt = O.make_optimizer(name, h0.shape, **okw)
    h = h0.copy()
    for t, g in enumerate(gs, start=1):
        opt.step(h, g, t)
    assert np.allclose(h, ref, rtol=1e-12, atol=1e-14)


def test_adam_first_step_closed_form():
    g = np.array([[3.0, -1e-3, 0.0]])
    h = np.zeros_like(g)
    O.Adam(g.shape, lr=0.1).step(h, g, 1)
    assert np.allclose(h, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-15)


# ------------------------------- full exact-mode trajectories vs autograd + torch.optim

def _torch_maxcut_F(Wt, h, beta):
    P = torch.sigmoid(h)
    cut = 0
    for Ps in (P, 1 - P):
        cut = cut + ((Wt @ Ps) * (1 - Ps)).sum(0)
    S = -(P * P.log() + (1 - P) * (1 - P).log()).sum(0)
    return -cut - S / beta


def test_maxcut_exact_trajectory_matches_autograd_adam():
    g, W = _small_graph(15, 0.4, 21, "pm1")
    h0 = I.initial_fields(15, 4, seed=22).astype(np.float64)
    n_step = 40
    h, _ = O.anneal(("maxcut", W), h0, n_step, mode="exact", optimizer="adam",
                    opt_kw=dict(lr=0.1))
    Wt = torch.tensor(W.toarray())
    ht = torch.tensor(h0, requires_grad=True)
    opt = torch.optim.Adam([ht], lr=0.1)
    for beta in O.beta_schedule("exponential", 0.05, 5.0, n_step):
        F = _torch_maxcut_F(Wt, ht, float(beta))
        opt.zero_grad()
        F.backward(gradient=torch.ones_like(F))
        opt.step()
    assert np.allclose(h, ht.detach().numpy(), rtol=1e-9, atol=1e-11)


def test_bmincut_exact_trajectory_matches_autograd_adam():
    g, W = _small_graph(12, 0.4, 23, "unit")
    q, n_step, lam_max = 3, 30, 0.5
    h0 = I.initial_fields(12, 3, seed=24, q=q).astype(np.float64)
    h, _ = O.anneal(("bmincut", W), h0, n_step, mode="exact", optimizer="adam",
                    opt_kw=dict(lr=0.05), lambda_max=lam_max)
    Wt = torch.tensor(W.toarray())
    ht = torch.tensor(h0.transpose(1, 0, 2).copy(), requires_grad=True)   # [R, N, q] like the listing
    opt = torch.optim.Adam([ht], lr=0.05)
    betas = O.beta_schedule("exponential", 0.05, 5.0, n_step)
    lams = O.lambda_ramp(lam_max, n_step)
    for beta, lam in zip(betas, lams):
        p = torch.softmax(ht, dim=2)
        cut = ((Wt @ p) * (1 - p)).sum((1, 2))
        bal = (p.sum(1) ** 2).sum(1) - (p ** 2).sum(2).sum(1)
        S = -(p * p.log()).sum(2).sum(1)
        F = cut + float(lam) * bal - S / float(beta)
        opt.zero_grad()
        F.backward(gradient=torch.ones_like(F))
        opt.step()
    assert np.allclose(h, ht.detach().numpy().transpose(1, 0, 2), rtol=1e-9, atol=1e-11)


def test_sat_trajectory_matches_autograd_adam():
    cl = I.random_ksat(12, 50, 3, seed=25)
    groups = O.sat_arrays(cl.ptr, cl.lits)
    h0 = I.initial_fields(12, 3, seed=26).astype(np.float64)
    n_step = 30
    h, _ = O.anneal(("sat", groups), h0, n_step, optimizer="adam", opt_kw=dict(lr=0.1))
    var = torch.tensor(np.abs(cl.lits.reshape(-1, 3)) - 1)
    pos = torch.tensor(cl.lits.reshape(-1, 3) > 0)
    ht = torch.tensor(h0, requires_grad=True)
    opt = torch.optim.Adam([ht], lr=0.1)
    for beta in O.beta_schedule("exponential", 0.05, 5.0, n_step):
        p = torch.sigmoid(ht)
        pv = p[var]                                          # [M, 3, R]
        u = torch.where(pos[..., None], 1 - pv, pv)
        S = -(p * p.log() + (1 - p) * (1 - p).log()).sum(0)
        F = u.prod(1).sum(0) - S / float(beta)
        opt.zero_grad()
        F.backward(gradient=torch.ones_like(F))
        opt.step()
    assert np.allclose(h, ht.detach().numpy(), rtol=1e-9, atol=1e-11)


# ------------------------------------------------------------- objectives

@pytest.mark.parametrize("weights", ["unit", "pm1", "real"])
def test_cut_three_recomputations_agree(weights):
    g, W = _small_graph(60, 0.1, 27, weights)
    sigma = np.where(_rng(28).random((60, 8)) < 0.5, 1, -1).astype(np.int8)
    a = O.maxcut_cut_edges(g.ei, g.ej, g.w, sigma)
    b = O.maxcut_cut_spin(g.ei, g.ej, g.w, sigma)
    c = O.maxcut_cut_matrix(W, sigma)
    if weights == "real":
        assert np.allclose(a, b, rtol=1e-12) and np.allclose(a, c, rtol=1e-12)
    else:
        assert a.dtype == np.int64 and np.array_equal(a, b) and np.array_equal(a, np.rint(c))
    # brute force on a single replica by a plain loop
    for r in range(2):
        ref = sum(w for i, j, w in zip(g.ei, g.ej, g.w) if sigma[i, r] != sigma[j, r])
        assert a[r] == pytest.approx(ref)


def test_sat_unsat_direct_scan():
    cl = I.random_ksat(20, 80, 3, seed=29)
    st = (_rng(30).random((20, 5)) < 0.5).astype(np.int8)
    got = O.sat_unsat(cl.ptr, cl.lits, st)
    for r in range(5):
        cnt = 0
        for m in range(cl.n_clauses):
            lits = cl.lits[cl.ptr[m]:cl.ptr[m + 1]]
            if not any((st[abs(l) - 1, r] == 1) == (l > 0) for l in lits):
                cnt += 1
        assert got[r] == cnt


def test_bmincut_objective_sizes_and_energy():
    g = I.rgg(200, 8, seed=31)
    st = _rng(32).integers(0, 4, size=(200, 3)).astype(np.int32)
    E, cut, sizes = O.bmincut_objective(g.ei, g.ej, g.w, st, 4, 1.0)
    assert np.all(sizes.sum(axis=1) == 200)
    for r in range(3):
        c = sum(1 for i, j in zip(g.ei, g.ej) if st[i, r] != st[j, r])
        n = np.bincount(st[:, r], minlength=4)
        assert cut[r] == c and E[r] == c + int((n * (n - 1)).sum())


# ------------------------------------------- end to end: FEM reaches brute-force optima

@pytest.mark.parametrize("seed,weights", [(40, "unit"), (41, "pm1"), (42, "pm1")])
def test_oracle_maxcut_reaches_bruteforce_optimum(seed, weights):
    g, W = _small_graph(16, 0.3, seed, weights)
    best = O.maxcut_bruteforce(g.n, g.ei, g.ej, g.w)
    h0 = I.initial_fields(16, 32, seed=seed + 100).astype(np.float64)
    h, _ = O.anneal(("maxcut", W), h0, 1000, mode="paper", optimizer="adam",
                    opt_kw=dict(lr=0.1))
    cuts = O.maxcut_cut_edges(g.ei, g.ej, g.w, O.maxcut_states(h))
    assert cuts.max() == best


@pytest.mark.parametrize("seed", [43, 44])
def test_oracle_sat_reaches_bruteforce_optimum(seed):
    cl = I.random_ksat(16, 67, 3, seed=seed)
    best = O.sat_bruteforce(cl.n, cl.ptr, cl.lits)
    groups = O.sat_arrays(cl.ptr, cl.lits)
    h0 = I.initial_fields(16, 32, seed=seed + 100).astype(np.float64)
    h, _ = O.anneal(("sat", groups), h0, 1000, optimizer="adam", opt_kw=dict(lr=0.1))
    unsat = O.sat_unsat(cl.ptr, cl.lits, O.sat_states(h))
    assert unsat.min() == best


@pytest.mark.parametrize("seed", [45, 46])
def test_oracle_bmincut_reaches_bruteforce_optimum(seed):
    g = I.rgg(9, 4.0, seed=seed)
    W = O.coupling_matrix(g.n, g.ei, g.ej, g.w)
    q, lam = 3, 1.0
    best = O.bmincut_bruteforce(g.n, g.ei, g.ej, g.w, q, lam)
    h0 = I.initial_fields(9, 32, seed=seed + 100, q=q).astype(np.float64)
    h, _ = O.anneal(("bmincut", W), h0, 1000, mode="paper", optimizer="adam",
                    opt_kw=dict(lr=0.1), lambda_max=lam)
    E, _, _ = O.bmincut_objective(g.ei, g.ej, g.w, O.bmincut_states(h), q, lam)
    assert E.min() == best


# ---- node-weighted bMinCut (SM, partitioning community graphs of the FPGA task)

def _weights(n, seed):
    return _rng(seed).integers(1, 6, size=n).astype(np.float64)


def test_weighted_bmincut_free_energy_matches_enumeration():
    g, W = _small_graph(5, 0.7, 31, "real")
    q, beta, lam = 3, 1.1, 0.35
    V = _weights(5, 32)
    h = _rng(33).normal(size=(5, 2, q))
    F = O.bmincut_free_energy(W, h, beta, lam, V=V)
    for r in range(2):
        z = np.exp(h[:, r] - h[:, r].max(axis=1, keepdims=True))
        marg = z / z.sum(axis=1, keepdims=True)

        def E(X):
            cut = (g.w[None, :] * (X[:, g.ei] != X[:, g.ej])).sum(axis=1)
            n_s = np.stack([((X == s) * V[None]).sum(axis=1) for s in range(q)], axis=1)
            sq_s = np.stack([((X == s) * V[None] ** 2).sum(axis=1) for s in range(q)], axis=1)
            return 2.0 * cut + lam * (n_s ** 2 - sq_s).sum(axis=1)

        ref = O.mf_free_energy_by_enumeration(marg, E, beta)
        assert F[r] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_weighted_bmincut_exact_gradient_is_fd_of_F():
    g, W = _small_graph(8, 0.5, 34, "real")
    V = _weights(8, 35)
    h = _rng(36).normal(size=(8, 2, 4))
    beta, lam = 0.7, 0.2
    ana = O.bmincut_grad(W, h, beta, lam, mode="exact", V=V)
    fd = _fd(lambda x: O.bmincut_free_energy(W, x, beta, lam, V=V), h)
    assert np.max(np.abs(ana - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_unit_node_weights_reduce_to_the_unweighted_forms():
    g, W = _small_graph(9, 0.5, 37, "unit")
    h = _rng(38).normal(size=(9, 3, 3))
    one = np.ones(9)
    for mode in ("exact", "paper"):
        assert np.array_equal(O.bmincut_grad(W, h, 0.8, 0.3, mode=mode, V=one),
                              O.bmincut_grad(W, h, 0.8, 0.3, mode=mode))
    st = O.bmincut_states(h)
    a = O.bmincut_objective(g.ei, g.ej, g.w, st, 3, 1.0, V=one.astype(np.int64))
    b = O.bmincut_objective(g.ei, g.ej, g.w, st, 3, 1.0)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_weighted_objective_is_the_coarsened_graph_of_tied_nodes():
    """Coarsening (SM, FPGA task): nodes of a community always share a group; the
    community graph has node weight = community size and edge weight = the sum of the
    edges between communities.  For every assignment of the community graph, the
    weighted energy plus lam * sum_i V_i (V_i - 1) (the pairs inside communities, which
    never leave a group) equals the unweighted energy of the lifted fine assignment."""
    rng = _rng(39)
    fine_n, q, lam = 9, 3, 2.0
    comm = np.array([0, 0, 1, 1, 1, 2, 3, 3, 4])           # 5 communities
    fg = I.er_gnp(fine_n, 0.6, seed=40, weights="unit")
    V = np.bincount(comm).astype(np.int64)
    acc = {}
    for i, j, w in zip(fg.ei, fg.ej, fg.w):
        a, b = comm[i], comm[j]
        if a != b:
            key = (min(a, b), max(a, b))
            acc[key] = acc.get(key, 0) + int(w)
    cei = np.array([k[0] for k in acc]); cej = np.array([k[1] for k in acc])
    cw = np.array([acc[k] for k in acc], dtype=np.int64)
    states = O.all_qary(5, q).T.astype(np.int32)                      # [community, assignment]
    states = states[:, rng.choice(states.shape[1], size=60, replace=False)]
    Ec, _, _ = O.bmincut_objective(cei, cej, cw, states, q, lam, V=V)
    Ef, _, _ = O.bmincut_objective(fg.ei, fg.ej, fg.w, states[comm], q, lam)
    assert np.array_equal(Ec + int(lam) * int((V * (V - 1)).sum()), Ef)


# ---- graph colouring (q-state Potts; SM, problems of multi-valued variables)

def test_coloring_free_energy_matches_enumeration():
    g, W = _small_graph(5, 0.7, 41, "real")
    q, beta = 3, 0.9
    h = _rng(42).normal(size=(5, 2, q))
    F = O.coloring_free_energy(W, h, beta)
    for r in range(2):
        z = np.exp(h[:, r] - h[:, r].max(axis=1, keepdims=True))
        marg = z / z.sum(axis=1, keepdims=True)

        def E(X):
            return (g.w[None, :] * (X[:, g.ei] == X[:, g.ej])).sum(axis=1)

        ref = O.mf_free_energy_by_enumeration(marg, E, beta)
        assert F[r] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_coloring_exact_gradient_is_fd_of_F():
    g, W = _small_graph(8, 0.5, 43, "real")
    h = _rng(44).normal(size=(8, 2, 4))
    ana = O.coloring_grad(W, h, 0.8, mode="exact")
    fd = _fd(lambda x: O.coloring_free_energy(W, x, 0.8), h)
    assert np.max(np.abs(ana - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_coloring_paper_mode_reduces_to_exact():
    g, W = _small_graph(10, 0.5, 45, "real")
    h = _rng(46).normal(size=(10, 3, 3))
    exact = O.coloring_grad(W, h, 1.1, mode="exact")
    red = O.coloring_grad(W, h, 1.1, mode="paper", cf=np.ones(10), discretise=False)
    assert np.allclose(red, exact, rtol=1e-12, atol=1e-14)


def test_coloring_oracle_reaches_a_proper_colouring():
    """A 3-colourable graph (a random graph on three planted colour classes, no edge
    inside a class): brute force finds 0 violations, and so does the oracle's best
    replica (exact mode, Adam, 1000 steps, beta 0.05 -> 20: a violation costs 1, so the
    end temperature must be well below 1)."""
    rng = _rng(47)
    n = 12
    cls = np.arange(n) % 3
    ei, ej = [], []
    for i in range(n):
        for j in range(i + 1, n):
            if cls[i] != cls[j] and rng.random() < 0.55:
                ei.append(i); ej.append(j)
    ei, ej = np.array(ei), np.array(ej)
    w = np.ones(len(ei))
    assert O.coloring_bruteforce(n, ei, ej, w, 3) == 0
    W = O.coupling_matrix(n, ei, ej, w)
    h0 = 0.001 * rng.normal(size=(n, 16, 3))
    h, _ = O.anneal(("coloring", W), h0, 1000, mode="exact", beta_max=20.0)
    E = O.coloring_energy(ei, ej, w, O.bmincut_states(h))
    assert E.min() == 0


# ---- QUBO (SM, COPs that translate into QUBO formulations)

def _qubo(n, p, seed):
    g = I.er_gnp(n, p, seed, "real")
    Q = O.coupling_matrix(g.n, g.ei, g.ej, g.w)
    d = _rng(seed + 1).normal(size=n)
    return g, Q, d


def test_qubo_free_energy_matches_enumeration():
    g, Q, d = _qubo(6, 0.6, 51)
    beta = 0.8
    h = _rng(53).normal(size=(6, 2))
    F = O.qubo_free_energy(Q, d, h, beta)
    for r in range(2):
        p = O.sigmoid(h[:, r])
        marg = np.stack([1.0 - p, p], axis=1)           # states 0, 1

        def E(X):
            Xf = X.astype(np.float64)
            return (2.0 * g.w[None, :] * Xf[:, g.ei] * Xf[:, g.ej]).sum(axis=1) + Xf @ d

        ref = O.mf_free_energy_by_enumeration(marg, E, beta)
        assert F[r] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_qubo_gradient_is_fd_of_F():
    g, Q, d = _qubo(9, 0.5, 54)
    h = _rng(56).normal(size=(9, 3))
    ana = O.qubo_grad(Q, d, h, 0.7)
    fd = _fd(lambda x: O.qubo_free_energy(Q, d, x, 0.7), h)
    assert np.max(np.abs(ana - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_maxcut_as_qubo_free_energy_identity():
    """MaxCut as a QUBO: -cut = sum_E 2 w s_i s_j - sum_i (sum_j w_ij) s_i with s in {0, 1},
    i.e. Q = W, d_i = -sum_j W_ij.  Then U_QUBO = -cut_MF (each edge once) while the
    MaxCut free energy counts ordered pairs, so F_maxcut(h, beta) = 2 F_QUBO(h, 2 beta);
    the sigmoid fields agree (p_i = P(sigma_i = +1) = P(s_i = 1))."""
    g, W = _small_graph(10, 0.5, 57, "real")
    d = -np.asarray(W.sum(axis=1)).ravel()
    h = _rng(58).normal(size=(10, 3))
    assert np.allclose(O.maxcut_free_energy(W, h, 0.9), 2.0 * O.qubo_free_energy(W, d, h, 1.8),
                       rtol=1e-12, atol=1e-12)


def test_qubo_oracle_reaches_the_maximum_independent_set():
    """Maximum independent set as a QUBO (a prominent example listed in the SM):
    E = -sum_i s_i + 2 sum_E s_i s_j (penalty 2 per violated edge); its minimum is minus
    the largest independent set.  Brute force over 2^14 states and the oracle's best
    replica (Adam, 1000 steps, beta 0.05 -> 20) agree."""
    g = I.er_gnp(14, 0.3, 59, "unit")
    w = np.ones(g.ei.size)                      # 2 w s_i s_j with w = 1: penalty 2 per edge
    d = -np.ones(14)
    best = O.qubo_bruteforce(14, g.ei, g.ej, w, d)
    Q = O.coupling_matrix(14, g.ei, g.ej, w)
    h0 = 0.001 * _rng(60).normal(size=(14, 32))
    h, _ = O.anneal(("qubo", (Q, d)), h0, 1000, mode="exact", beta_max=20.0)
    E = O.qubo_energy(g.ei, g.ej, w, d, O.qubo_states(h))
    assert E.min() == best


# ---- higher-order interactions (SM, p-spin / quantum error correction Hamiltonians)

def _pspin(n, m, k_max, seed):
    rng = _rng(seed)
    ks = rng.integers(1, k_max + 1, size=m)
    ptr = np.concatenate([[0], np.cumsum(ks)])
    var = np.concatenate([rng.choice(n, size=k, replace=False) for k in ks])
    J = rng.normal(size=m)
    b = rng.normal(size=n)
    return ptr, var, J, b


def test_pspin_free_energy_matches_enumeration():
    ptr, var, J, b = _pspin(6, 7, 4, 61)
    beta = 0.9
    h = _rng(62).normal(size=(6, 2))
    F = O.pspin_free_energy(ptr, var, J, b, h, beta)
    for r in range(2):
        p = O.sigmoid(h[:, r])
        marg = np.stack([1.0 - p, p], axis=1)            # state 0 <-> sigma = -1, 1 <-> +1

        def E(X):
            S = 2.0 * X.astype(np.float64) - 1.0
            out = S @ b
            for t in range(len(J)):
                out = out + J[t] * S[:, var[ptr[t]:ptr[t + 1]]].prod(axis=1)
            return out

        ref = O.mf_free_energy_by_enumeration(marg, E, beta)
        assert F[r] == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_pspin_gradient_is_fd_of_F():
    ptr, var, J, b = _pspin(9, 12, 5, 63)
    h = _rng(64).normal(size=(9, 3))
    ana = O.pspin_grad(ptr, var, J, b, h, 0.6)
    fd = _fd(lambda x: O.pspin_free_energy(ptr, var, J, b, x, 0.6), h)
    assert np.max(np.abs(ana - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_two_body_pspin_is_maxcut():
    """Pair terms J_ij = W_ij / 2 and no field: E = sum_E (W/2) s_i s_j = W_tot/2 - cut, so
    F_maxcut(h, beta) = 2 F_pspin(h, 2 beta) - W_tot (the MaxCut free energy counts
    ordered pairs; both use p_i = P(s_i = +1) = sigmoid(h_i))."""
    g, W = _small_graph(10, 0.5, 65, "real")
    ptr = np.arange(0, 2 * g.ei.size + 1, 2)
    var = np.stack([g.ei, g.ej], axis=1).ravel()
    h = _rng(66).normal(size=(10, 3))
    lhs = O.maxcut_free_energy(W, h, 0.7)
    rhs = 2.0 * O.pspin_free_energy(ptr, var, g.w / 2.0, np.zeros(10), h, 1.4) - g.w.sum()
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_pspin_oracle_against_brute_force():
    """Ten seeded field-free instances with 2-, 3- and 4-spin terms (the QEC shape): no
    replica's energy is below the brute-force minimum over all 2^12 states (the energy
    and the brute force agree), and mean-field annealing (1000 steps, beta 0.05 -> 20)
    reaches the exact ground state on at least four of them.  The method is a heuristic
    on such instances; its mathematics is pinned exactly by the tests above."""
    reached = 0
    for seed in range(67, 77):
        r = _rng(seed)
        ks = r.integers(2, 5, size=30)
        ptr = np.concatenate([[0], np.cumsum(ks)])
        var = np.concatenate([r.choice(12, size=k, replace=False) for k in ks])
        J = np.round(3 * r.normal(size=30))
        b = np.zeros(12)
        best = O.pspin_bruteforce(12, ptr, var, J, b)
        h0 = 0.001 * _rng(68).normal(size=(12, 32))
        h, _ = O.anneal(("pspin", (ptr, var, J, b)), h0, 1000, mode="exact", beta_max=20.0)
        E = O.pspin_energy(ptr, var, J, b, O.maxcut_states(h))
        assert E.min() >= best
        reached += int(E.min() == best)
    assert reached >= 4, reached


# ---- the paper's example CNF (Results, "The MaxSAT problem"), a golden fixture
def _golden_cnf():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "maxsat_methods_cnf.txt")
    clauses, table = [], []
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("clause"):
            clauses.append([int(x) for x in line.split()[1:]])
        else:
            table.append([int(x) for x in line.split()])
    return clauses, np.array(table, np.int64)


def test_paper_cnf_unsatisfied_counts():
    """The oracle's clause scan reproduces the hand-derived count of unsatisfied clauses
    of the paper's example formula for all 16 assignments (6 satisfy it)."""
    clauses, table = _golden_cnf()
    ptr = np.concatenate([[0], np.cumsum([len(c) for c in clauses])])
    lits = np.concatenate(clauses)
    states = table[:, :4].T.astype(np.int8)  # [n, R]: one assignment per replica
    assert np.array_equal(O.sat_unsat(ptr, lits, states), table[:, 4])
    assert int((table[:, 4] == 0).sum()) == 6


def test_paper_cnf_repeated_variable_reading():
    """The printed C1 repeats ~s2.  The library reads clauses as sets of distinct
    variables and rejects the repeat; the set form (s1 v ~s2) has the same count table."""
    from paper_2412_09285_b300 import fem
    clauses, table = _golden_cnf()
    mk = lambda cl: I.Clauses(4, np.concatenate([[0], np.cumsum([len(c) for c in cl])]), np.concatenate(cl))
    with pytest.raises(fem.FemError) as e:
        fem.Problem("sat", clauses=mk(clauses))
    assert e.value.status == fem.FEM_ERR_INVALID_ARG
    sets = [list(dict.fromkeys(c)) for c in clauses]
    c = mk(sets)
    states = table[:, :4].T.astype(np.int8)
    assert np.array_equal(O.sat_unsat(c.ptr, c.lits, states), table[:, 4])


def test_single_field_is_the_two_state_softmax():
    """The single-field form (P_i(+1) = sigmoid(h_i)) is the two-state softmax with
    fields (h_i, 0) (Eq. gradients_wrt_h for q = 2; MaxCut's energy is bMinCut's cut term
    with W -> -W and no balance term): equal free energies, and the single-field
    gradient equals dF/dh(+1) = -dF/dh(-1) of the softmax form."""
    g, W = _small_graph(9, 0.5, 21, "real")
    h = _rng(22).normal(size=(9, 3))
    H = np.stack([h, np.zeros_like(h)], axis=2)
    beta = 0.8
    assert np.allclose(O.maxcut_free_energy(W, h, beta), O.bmincut_free_energy(-W, H, beta, 0.0),
                       rtol=1e-12, atol=1e-12)
    gm = O.maxcut_grad(W, h, beta, mode="exact")
    gb = O.bmincut_grad(-W, H, beta, 0.0, mode="exact")
    assert np.allclose(gm, gb[:, :, 0], rtol=1e-10, atol=1e-13)
    assert np.allclose(gm, -gb[:, :, 1], rtol=1e-10, atol=1e-13)


def test_pure_entropy_fields_relax_to_zero():
    """With no couplings the free energy is -S/beta, minimised by P = 1/2 (h = 0): the
    gradient has the sign of h and vanishes at h = 0, and small gradient-descent steps
    at fixed beta shrink every |h| monotonically."""
    g, W = _small_graph(6, 0.5, 23, "unit")
    W = 0.0 * W
    h = _rng(24).normal(size=(6, 4))
    gr = O.maxcut_grad(W, h, 1.0, mode="exact")
    assert np.all(np.sign(gr) == np.sign(h))
    assert np.all(O.maxcut_grad(W, np.zeros_like(h), 1.0, mode="exact") == 0.0)
    tr = {t: None for t in range(1, 41)}
    O.anneal(("maxcut", W), h, 40, beta_min=1.0, beta_max=1.0, optimizer="sgd", opt_kw=dict(lr=0.5),
             mode="exact", trace=tr)
    mags = np.stack([np.abs(h)] + [np.abs(tr[t]) for t in range(1, 41)])
    assert np.all(np.diff(mags, axis=0) <= 0.0) and np.all(mags[-1] < mags[0])
