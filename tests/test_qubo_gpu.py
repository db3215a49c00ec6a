"""QUBO (binary variables, one sigmoid field each) on the MaxCut data path against the
FP64 oracle: marginals within 1e-4 over the first 50 steps, energies bit-exact (int64)
for the GPU's own states with integer coefficients, and the argument checks."""
import numpy as np
import pytest

import oracle as O
import parity
from paper_2412_09285_b300 import instances as I

pytestmark = pytest.mark.gpu

CHECK = [1, 2, 5, 10, 20, 35, 50]


@pytest.fixture(scope="module")
def fem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2412_09285_b300 import build
    build.build()
    from paper_2412_09285_b300 import fem as F
    return F


def test_qubo_marginals_first_50_steps(fem):
    g = I.er_gnm(600, 2400, seed=111, weights="real")
    d = np.random.Generator(np.random.PCG64(112)).normal(size=600)
    Q = O.coupling_matrix(g.n, g.ei, g.ej, g.w)
    h0 = I.initial_fields(600, 32, seed=113)
    P = fem.Problem("qubo", graph=g, linear=d)
    got, st = parity.gpu_windows(P, h0, CHECK, 1000, grad_mode="exact")
    tr = {t: None for t in CHECK}
    cd = {t: None for t in CHECK}
    O.anneal(("qubo", (Q, d)), h0.astype(np.float64), 1000, t_end=50, mode="exact", trace=tr, cond=cd)
    parity.compare_trajectory(got, tr, cd, CHECK, "qubo", state=st,
                              forced=parity.one_step(P, ("qubo", (Q, d)), 1000, grad_mode="exact"))


def test_mis_qubo_energies_bit_exact(fem):
    """Maximum independent set, E = -sum_i s_i + 2 sum_E s_i s_j (integer coefficients)."""
    g = I.er_gnm(3000, 9000, seed=114, weights="unit")
    d = -np.ones(3000)
    h0 = I.initial_fields(3000, 64, seed=115)
    P = fem.Problem("qubo", graph=g, linear=d).anneal(h_init=h0, n_steps=1000, grad_mode="exact", beta_max=20.0)
    st = P.states()
    assert set(np.unique(st)) <= {0, 1}
    E = O.qubo_energy(g.ei, g.ej, g.w, d, st)
    res = P.best()
    assert np.array_equal(res["energy_i64"], E)
    assert res["best_replica"] == int(np.argmin(E))
    s = st[:, res["best_replica"]]
    viol = int((s[g.ei] * s[g.ej]).sum())
    print(f"\nMIS QUBO, ER n = 3000, mean degree 6: best replica E = {int(E.min())}, "
          f"{int(s.sum())} nodes chosen, {viol} violated edges")
    assert E.min() < -0.3 * 3000


def test_qubo_arguments(fem):
    g = I.er_gnm(100, 300, seed=116, weights="unit")
    with pytest.raises(fem.FemError) as e:
        fem.Problem("qubo", graph=g).anneal(h_init=I.initial_fields(100, 32, seed=1), n_steps=10,
                                             grad_mode="paper")
    assert e.value.status == fem.FEM_ERR_UNSUPPORTED
    with pytest.raises(fem.FemError) as e:
        fem.Problem("maxcut", graph=g, linear=np.ones(100))
    assert e.value.status == fem.FEM_ERR_INVALID_ARG
    with pytest.raises(fem.FemError):
        fem.Problem("qubo", graph=g, linear=np.full(100, np.inf))
