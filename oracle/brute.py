"""Brute-force optima and mean-field sums by full enumeration - TEST INFRASTRUCTURE ONLY.

These enumerate every configuration of tiny instances (N <= 20 binary, q^N <= 2^20
for q states) and are the ground truth the FEM oracle must reach at large beta.
They also evaluate the variational free energy straight from its definition
(Results Eq. FP: sum over all configurations of P_MF(sigma) E(sigma) plus the
entropy of the product distribution), which pins the closed forms in ``fem.py``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "all_binary", "all_qary", "maxcut_bruteforce", "bmincut_bruteforce", "coloring_bruteforce", "qubo_bruteforce",
    "pspin_bruteforce",
    "sat_bruteforce", "mf_free_energy_by_enumeration",
]


def all_binary(n):
    """All 2^n configurations as a [2^n, n] array of 0/1."""
    idx = np.arange(1 << n, dtype=np.int64)
    return ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int8)


def all_qary(n, q):
    """All q^n configurations as a [q^n, n] array of states 0..q-1."""
    idx = np.arange(q ** n, dtype=np.int64)
    out = np.empty((idx.shape[0], n), dtype=np.int8)
    for i in range(n):
        out[:, i] = idx % q
        idx = idx // q
    return out


def maxcut_bruteforce(n, ei, ej, w):
    """Maximum cut sum_{(i,j) in E} W_ij [sigma_i != sigma_j] over all 2^n states."""
    X = all_binary(n)
    cut = (np.asarray(w)[None, :] * (X[:, ei] != X[:, ej])).sum(axis=1)
    return cut.max()


def bmincut_bruteforce(n, ei, ej, w, q, lam):
    """Minimum of E = cut + lam * sum_s n_s (n_s - 1) (Eq. bmincut) over all q^n states."""
    X = all_qary(n, q)
    cut = (np.asarray(w)[None, :] * (X[:, ei] != X[:, ej])).sum(axis=1)
    sizes = np.stack([(X == s).sum(axis=1) for s in range(q)], axis=1)
    return (cut + lam * (sizes * (sizes - 1)).sum(axis=1)).min()


def coloring_bruteforce(n, ei, ej, w, q):
    """Minimum violated edge weight sum_E W_ij [sigma_i == sigma_j] over all q^n colourings."""
    X = all_qary(n, q)
    return (np.asarray(w)[None, :] * (X[:, ei] == X[:, ej])).sum(axis=1).min()


def qubo_bruteforce(n, ei, ej, w, d):
    """Minimum of sum_E 2 w sigma_i sigma_j + sum_i d_i sigma_i over all 2^n binary states."""
    X = all_binary(n).astype(np.float64)
    E = (2.0 * np.asarray(w)[None, :] * X[:, ei] * X[:, ej]).sum(axis=1) + X @ np.asarray(d, np.float64)
    return E.min()


def pspin_bruteforce(n, ptr, var, J, b):
    """Minimum of sum_v J_v prod_{i in v} s_i + sum_i b_i s_i over all 2^n spin states."""
    S = 2.0 * all_binary(n).astype(np.float64) - 1.0
    E = S @ np.asarray(b, np.float64)
    ptr = np.asarray(ptr)
    var = np.asarray(var)
    for t in range(ptr.shape[0] - 1):
        E = E + J[t] * S[:, var[ptr[t]:ptr[t + 1]]].prod(axis=1)
    return E.min()


def sat_bruteforce(n, ptr, lits):
    """Minimum number of unsatisfied clauses over all 2^n assignments (sigma in {0,1})."""
    X = all_binary(n)
    ptr = np.asarray(ptr)
    lits = np.asarray(lits)
    unsat = np.zeros(X.shape[0], dtype=np.int64)
    for m in range(ptr.shape[0] - 1):
        L = lits[ptr[m]:ptr[m + 1]]
        sat = np.zeros(X.shape[0], dtype=bool)
        for l in L:
            v = X[:, abs(l) - 1]
            sat |= (v == 1) if l > 0 else (v == 0)
        unsat += ~sat
    return unsat.min()


def mf_free_energy_by_enumeration(marginals, energy_of, beta):
    """F = sum_sigma P_MF(sigma) E(sigma) + (1/beta) sum_sigma P_MF ln P_MF (Eq. FP),
    by enumerating every configuration of the product distribution.

    marginals: [n, q] array of P_i(s) (rows sum to 1); energy_of(X) maps a
    [K, n] array of states to K energies."""
    n, q = marginals.shape
    X = all_qary(n, q) if q > 2 else all_binary(n)
    PX = np.ones(X.shape[0])
    for i in range(n):
        PX = PX * marginals[i, X[:, i]]
    E = energy_of(X)
    nz = PX > 0
    return (PX * E).sum() + (PX[nz] * np.log(PX[nz])).sum() / beta
