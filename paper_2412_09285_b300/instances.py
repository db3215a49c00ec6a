"""Seeded synthetic instances for the Free-Energy Machine (FEM) workloads.

This module holds input generation only: graphs, clause lists and initial
fields.  It contains none of the method's arithmetic, so both the CUDA path and
the CPU oracle can take their inputs from it without sharing any computation.

The paper's data sets (G-set, K2000, Walshaw graphs, MaxSAT-2016) are not used;
the generators below produce instances with the same shapes:

* Erdos-Renyi G(n, p) and G(n, m) graphs with unit or +-1 weights
  (G-set random graphs, Results section "Applications to the Maximum-Cut problem").
* Dense Sherrington-Kirkpatrick couplings J_ij = +-1 (the K2000 shape).
* Random geometric graphs in the unit square with unit weights (the sparse,
  spatially local graphs of the bMinCut benchmarks).
* Random Max-k-SAT with k distinct variables per clause and Bernoulli(1/2) signs.
* Initial fields h = 0.001 * N(0, 1) (SM, "numerical experiment of the MaxCut
  problem on the G-set": the fields are initialised with 0.001*randn).

Every generator takes an integer seed and uses numpy's PCG64 stream, so the same
seed always gives the same instance.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Graph", "Clauses", "er_gnp", "er_gnm", "sk_dense", "rgg", "random_ksat",
    "initial_fields", "loguniform_sizes",
]


class Graph:
    """Undirected graph as an edge list: each edge once, i != j, no duplicates.

    ``ei``, ``ej`` are int32 endpoint arrays of length |E| and ``w`` the float64
    weights.  ``dense`` optionally carries the full n x n symmetric matrix (for the
    complete-graph instances) as int8 with a zero diagonal.
    """

    def __init__(self, n, ei, ej, w, dense=None, name=""):
        self.n = int(n)
        self.ei = np.ascontiguousarray(ei, dtype=np.int32)
        self.ej = np.ascontiguousarray(ej, dtype=np.int32)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.dense = dense
        self.name = name

    @property
    def n_edges(self) -> int:
        return int(self.ei.shape[0])

    def __repr__(self):
        return f"Graph({self.name}, n={self.n}, |E|={self.n_edges})"


class Clauses:
    """CNF clause list in DIMACS style: ``lits`` holds signed, 1-based variable
    indices (+v for the literal v, -v for its negation); clause m owns
    ``lits[ptr[m]:ptr[m+1]]``."""

    def __init__(self, n, ptr, lits, name=""):
        self.n = int(n)
        self.ptr = np.ascontiguousarray(ptr, dtype=np.int64)
        self.lits = np.ascontiguousarray(lits, dtype=np.int32)
        self.name = name

    @property
    def n_clauses(self) -> int:
        return int(self.ptr.shape[0] - 1)

    def __repr__(self):
        return f"Clauses({self.name}, n={self.n}, M={self.n_clauses})"


def _weights(rng, m, weights):
    if weights == "unit":
        return np.ones(m, dtype=np.float64)
    if weights == "pm1":
        return rng.integers(0, 2, size=m).astype(np.float64) * 2.0 - 1.0
    if weights == "real":
        return rng.uniform(0.5, 2.0, size=m)
    raise ValueError(f"unknown weight kind {weights!r}")


def er_gnp(n: int, p: float, seed: int, weights: str = "unit") -> Graph:
    """G(n, p): every unordered pair i < j is an edge with probability p."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < p
    ei, ej = iu[keep], ju[keep]
    return Graph(n, ei, ej, _weights(rng, ei.shape[0], weights), name=f"gnp{n}_{p}")


def er_gnm(n: int, m: int, seed: int, weights: str = "unit") -> Graph:
    """G(n, m): m distinct edges drawn uniformly, no self-loops, no multi-edges."""
    rng = np.random.Generator(np.random.PCG64(seed))
    keys = np.empty(0, dtype=np.int64)
    while keys.shape[0] < m:
        need = int((m - keys.shape[0]) * 1.05) + 16
        a = rng.integers(0, n, size=need, dtype=np.int64)
        b = rng.integers(0, n, size=need, dtype=np.int64)
        ok = a != b
        lo, hi = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        s = np.sort(np.concatenate([keys, lo * n + hi]))   # sorted distinct keys (== np.unique)
        keys = s[np.concatenate(([True], s[1:] != s[:-1]))] if s.size else s
    # keep a uniform subset of exactly m distinct pairs, then sort by (i, j)
    keys = np.sort(rng.permutation(keys)[:m])
    ei, ej = (keys // n).astype(np.int32), (keys % n).astype(np.int32)
    return Graph(n, ei, ej, _weights(rng, m, weights), name=f"gnm{n}_{m}")


def sk_dense(n: int, seed: int) -> Graph:
    """Complete graph with J_ij = +-1 uniform, symmetric, zero diagonal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    iu, ju = np.triu_indices(n, k=1)
    w = rng.integers(0, 2, size=iu.shape[0]).astype(np.int8) * 2 - 1
    dense = np.zeros((n, n), dtype=np.int8)
    dense[iu, ju] = w
    dense[ju, iu] = w
    return Graph(n, iu, ju, w.astype(np.float64), dense=dense, name=f"sk{n}")


def rgg(n: int, mean_degree: float, seed: int) -> Graph:
    """Random geometric graph: n points uniform in the unit square, an edge for
    every pair closer than r, with n*pi*r^2 = mean_degree; unit weights."""
    from scipy.spatial import cKDTree

    rng = np.random.Generator(np.random.PCG64(seed))
    pts = rng.random((n, 2))
    r = float(np.sqrt(mean_degree / (np.pi * n)))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray").astype(np.int64)
    if pairs.shape[0]:
        pairs = np.sort(pairs, axis=1)
        order = np.lexsort((pairs[:, 1], pairs[:, 0]))
        pairs = pairs[order]
    ei = pairs[:, 0].astype(np.int32) if pairs.shape[0] else np.zeros(0, np.int32)
    ej = pairs[:, 1].astype(np.int32) if pairs.shape[0] else np.zeros(0, np.int32)
    return Graph(n, ei, ej, np.ones(ei.shape[0]), name=f"rgg{n}")


def random_ksat(n: int, m: int, k: int, seed: int) -> Clauses:
    """Random k-SAT: each clause draws k distinct variables uniformly and a
    Bernoulli(1/2) sign for each literal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    # k distinct variables per clause: argsort of random keys over a small pool is
    # too slow for large n, so draw with rejection of clauses that repeat a variable.
    var = rng.integers(0, n, size=(m, k), dtype=np.int64)
    while True:
        s = np.sort(var, axis=1)
        bad = np.any(s[:, 1:] == s[:, :-1], axis=1) if k > 1 else np.zeros(m, bool)
        if not bad.any():
            break
        var[bad] = rng.integers(0, n, size=(int(bad.sum()), k), dtype=np.int64)
    sign = rng.integers(0, 2, size=(m, k)) * 2 - 1
    lits = ((var + 1) * sign).astype(np.int32).reshape(-1)
    ptr = np.arange(0, m * k + 1, k, dtype=np.int64)
    return Clauses(n, ptr, lits, name=f"{k}sat{n}_{m}")


def initial_fields(n: int, replicas: int, seed: int, q: int = 1) -> np.ndarray:
    """Initial local fields 0.001 * N(0, 1), rounded to float32.

    Layout: ``[n, replicas]`` for the single-field (q = 2) problems (q=1 here means
    one field per variable) and ``[n, replicas, q]`` for q-state softmax fields.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (n, replicas) if q == 1 else (n, replicas, q)
    return (0.001 * rng.standard_normal(shape)).astype(np.float32)


MPNN_SHAPES = [("A1", (4, 64)), ("B1", (4, 64)), ("b1", (64,)), ("A2", (64, 64)), ("B2", (64, 64)),
               ("b2", (64,)), ("A3", (64, 64)), ("B3", (64, 64)), ("b3", (64,)), ("C", (64, 4)), ("c", (4,))]


def mpnn_init(seed: int) -> dict:
    """Initial weights of the warm-start network: Glorot-uniform matrices, zero biases,
    filter taps starting at (1, 0, 0, 0) (prediction = the replica's own fields)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for name, shape in MPNN_SHAPES:
        if len(shape) == 2:
            lim = np.sqrt(6.0 / (shape[0] + shape[1]))
            out[name] = rng.uniform(-lim, lim, size=shape) * (0.1 if name == "C" else 1.0)
        else:
            out[name] = np.zeros(shape)
    out["c"][0] = 1.0
    return out


def mpnn_flatten(params: dict) -> np.ndarray:
    """Parameters as one float32 vector in the library's order (row-major blocks)."""
    return np.concatenate([np.asarray(params[k], np.float64).ravel() for k, _ in MPNN_SHAPES]).astype(np.float32)


def mpnn_unflatten(vec) -> dict:
    out, off = {}, 0
    for k, shape in MPNN_SHAPES:
        size = int(np.prod(shape))
        out[k] = np.asarray(vec[off:off + size], np.float64).reshape(shape)
        off += size
    return out


def loguniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``count`` integers drawn log-uniformly from [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)
