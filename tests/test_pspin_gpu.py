"""Higher-order interactions (p-spin / QEC Hamiltonian) on the Max-k-SAT data path,
against the FP64 oracle: marginals within 1e-4 over the first 50 steps, energies
bit-exact (int64) for the GPU's own states with integer coefficients, negated literals
equal to negated coefficients, and a p-spin member of a batch equal to annealing it
alone."""
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


def _instance(n, m, k_lo, k_hi, seed, integer=False):
    """m terms of k_lo..k_hi distinct spins (positive literals), coefficients J, fields b."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = rng.integers(k_lo, k_hi + 1, size=m)
    ptr = np.concatenate([[0], np.cumsum(ks)])
    var = np.concatenate([rng.choice(n, size=k, replace=False) for k in ks])
    J = rng.normal(size=m)
    b = 0.3 * rng.normal(size=n)
    if integer:
        J, b = np.round(3 * J), np.round(2 * b)
    return I.Clauses(n, ptr, var + 1), ptr, var, J, b


def test_pspin_marginals_first_50_steps(fem):
    cl, ptr, var, J, b = _instance(2000, 6000, 1, 4, seed=121)
    h0 = I.initial_fields(2000, 32, seed=122)
    P = fem.Problem("pspin", clauses=cl, term_weight=J, linear=b)
    got, st = parity.gpu_windows(P, h0, CHECK, 1000)
    tr = {t: None for t in CHECK}
    cd = {t: None for t in CHECK}
    O.anneal(("pspin", (ptr, var, J, b)), h0.astype(np.float64), 1000, t_end=50, mode="exact", trace=tr, cond=cd)
    parity.compare_trajectory(got, tr, cd, CHECK, "pspin", state=st,
                              forced=parity.one_step(P, ("pspin", (ptr, var, J, b)), 1000))


def test_pspin_energies_bit_exact_and_negation_folding(fem):
    cl, ptr, var, J, b = _instance(3000, 9000, 2, 4, seed=123, integer=True)
    h0 = I.initial_fields(3000, 32, seed=124)
    P = fem.Problem("pspin", clauses=cl, term_weight=J, linear=b).anneal(h_init=h0, n_steps=600, beta_max=20.0)
    st = P.states()
    assert set(np.unique(st)) <= {-1, 1}
    E = O.pspin_energy(ptr, var, J, b, st)
    res = P.best()
    assert np.array_equal(res["energy_i64"], E)
    assert res["best_replica"] == int(np.argmin(E))
    # negate the first literal of every other term and the term's coefficient with it
    lits = cl.lits.copy()
    flip = np.arange(len(J)) % 2 == 1
    lits[ptr[:-1][flip]] *= -1
    Q = fem.Problem("pspin", clauses=I.Clauses(3000, ptr, lits), term_weight=np.where(flip, -J, J), linear=b)
    Q.anneal(h_init=h0, n_steps=600, beta_max=20.0)
    for x, y in zip(Q.state(), P.state()):
        assert np.array_equal(x, y)


def test_pspin_member_in_a_batch_equals_alone(fem):
    cl, _, _, J, b = _instance(1500, 4000, 2, 4, seed=125)
    sat = I.random_ksat(1200, 5040, 3, seed=126)
    h0 = [I.initial_fields(1500, 16, seed=127), I.initial_fields(1200, 16, seed=128)]
    mk = lambda: [fem.Problem("pspin", clauses=cl, term_weight=J, linear=b), fem.Problem("sat", clauses=sat)]
    alone = [p.anneal(h_init=h, n_steps=80).state() for p, h in zip(mk(), h0)]
    probs = mk()
    fem.Batch(probs).anneal(h_inits=h0, replicas=16, n_steps=80)
    for p, ref in zip(probs, alone):
        for x, y in zip(p.state(), ref):
            assert np.array_equal(x, y)


def test_pspin_arguments(fem):
    cl, _, _, J, b = _instance(50, 60, 2, 3, seed=129)
    with pytest.raises(fem.FemError) as e:
        fem.Problem("pspin", clauses=cl)
    assert e.value.status == fem.FEM_ERR_INVALID_ARG
    with pytest.raises(fem.FemError) as e:
        fem.Problem("sat", clauses=cl, term_weight=J)
    assert e.value.status == fem.FEM_ERR_INVALID_ARG


def test_three_spin_four_replica_path_matches_general_path(fem):
    """3-spin terms with R % 4 == 0 take the four-replicas-per-thread kernel (other-spin
    table, each occurrence carrying its term's coupling, negations folded in); R = 50
    takes the per-element kernel.  Replicas are independent, so the first 4 / 16 / 48
    replicas of the R = 50 run must equal the narrow runs bit for bit."""
    cl, ptr, var, J, b = _instance(3000, 9000, 3, 3, seed=131)
    lits = cl.lits.copy()
    lits[::5] *= -1  # some negated spins (their sign goes into the term's coupling)
    mk = lambda: fem.Problem("pspin", clauses=I.Clauses(3000, ptr, lits), term_weight=J, linear=b)
    wide = I.initial_fields(3000, 50, seed=132)
    ref = mk().anneal(h_init=wide, n_steps=200).state()
    for R in (4, 16, 48):
        got = mk().anneal(h_init=np.ascontiguousarray(wide[:, :R]), n_steps=200).state()
        for x, y, name in zip(got, ref, "hmv"):
            assert np.array_equal(x, y[:, :R]), (R, name, int(np.sum(x != y[:, :R])))
