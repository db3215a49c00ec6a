"""FEM oracle: schedules, free energies, gradients, optimizers, anneal, readout.

TEST INFRASTRUCTURE ONLY (see the package header).  Everything is float64 numpy;
a scipy sparse or numpy dense matrix product serves as the library primitive for
sums of the form sum_j W_ij x_j.  No blocking, fusion or reordering beyond what
the equations state.

Conventions (readings of the paper where it is silent or inconsistent):

* Ordered pairs.  The free energies and gradients use the convention of the
  paper's PyTorch listing (``cut(W, p) = ((W @ p) * (1 - p)).sum()``, Methods and
  SM "PyTorch implementation"): sums run over ordered pairs (i, j), so each edge
  counts twice.  The explicit gradients of the SM (Eq. S-maxcut_gradient and the
  bMinCut gradient, both with the factor 2) are the derivatives of that form.
  Discrete objectives (the cut, the number of unsatisfied clauses) count each
  edge or clause once, as in Eqs. (maxcut1), (bmincut), (maxksat_E).
* Single field for the two-state problems (SM "Simplification of FEM for solving
  the MaxCut problem"): P_i = sigmoid(h_i) is the marginal of the state
  sigma_i = +1 (MaxCut) or sigma_i = 1 (SAT); m_i = 2 P_i - 1 = tanh(h_i / 2).
* Discretisation and argmax ties: a single-field variable takes the state of
  P_i when h_i >= 0 (so sgn(0) = +1); a q-state variable takes the lowest index
  among the maximal fields.  Argmax of softmax(h) equals argmax of h.
* Isolated nodes: the normalisers c_i, c^f_i, c^a_i are set to 0.
* Step t (0-based) uses beta(t) and lambda(t) and is Adam step number t + 1.
* N_step = 1: beta(0) = beta_min and lambda(0) = 0.

Pins (tests that tie this module to something other than itself) are listed in
tests/test_oracle_*.py; full multi-step trajectories are pinned only for the
exact-gradient modes (against autograd of the paper's free energy with the
PyTorch optimizers).  Paper-mode trajectories are pinned by the exact-mode
reduction identities and by end-to-end brute-force optima, not step by step.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

__all__ = [
    "beta_schedule", "lambda_ramp", "coupling_matrix", "sigmoid",
    "maxcut_free_energy", "maxcut_grad", "maxcut_normaliser",
    "bmincut_free_energy", "bmincut_grad", "bmincut_normalisers",
    "coloring_free_energy", "coloring_grad", "coloring_energy",
    "qubo_free_energy", "qubo_grad", "qubo_states", "qubo_energy",
    "pspin_free_energy", "pspin_grad", "pspin_energy",
    "sat_arrays", "sat_free_energy", "sat_grad",
    "Adam", "RMSprop", "SGD", "make_optimizer", "anneal",
    "maxcut_states", "maxcut_cut_edges", "maxcut_cut_spin", "maxcut_cut_matrix",
    "bmincut_states", "bmincut_objective", "sat_states", "sat_unsat",
    "best_replica",
]


# ----------------------------------------------------------------------------
# Annealing schedules (Methods, "Different annealing schedules for the inverse
# temperature"); the lambda ramp of bMinCut (SM, "Demonstration of FEM solving
# the bMinCut problem": lambda rises linearly from 0 to lambda_max).
# ----------------------------------------------------------------------------

def beta_schedule(kind: str, beta_min: float, beta_max: float, n_step: int) -> np.ndarray:
    """beta(t_s) for t_s = 0 .. n_step-1.

    exponential:          beta = exp(ln beta_min + t (ln beta_max - ln beta_min)/(N-1))
    inverse_proportional: 1/beta = 1/beta_min + t (1/beta_max - 1/beta_min)/(N-1)
    """
    t = np.arange(n_step, dtype=np.float64)
    if n_step == 1:
        return np.array([beta_min], dtype=np.float64)
    if kind == "exponential":
        return np.exp((math.log(beta_max) - math.log(beta_min)) / (n_step - 1) * t
                      + math.log(beta_min))
    if kind == "inverse_proportional":
        return 1.0 / ((1.0 / beta_max - 1.0 / beta_min) / (n_step - 1) * t + 1.0 / beta_min)
    raise ValueError(kind)


def lambda_ramp(lambda_max: float, n_step: int) -> np.ndarray:
    """lambda(t) = lambda_max * t / (N_step - 1)."""
    if n_step == 1:
        return np.zeros(1)
    return lambda_max * np.arange(n_step, dtype=np.float64) / (n_step - 1)


# ----------------------------------------------------------------------------
# Couplings
# ----------------------------------------------------------------------------

def coupling_matrix(n, ei, ej, w):
    """Symmetric sparse W with W_ij = W_ji = w for each undirected edge."""
    W = sp.coo_matrix((np.asarray(w, np.float64), (np.asarray(ei), np.asarray(ej))),
                      shape=(n, n))
    return (W + W.T).tocsr()


def _row_sums(W, absolute=False):
    if sp.issparse(W):
        A = abs(W) if absolute else W
        return np.asarray(A.sum(axis=1)).ravel()
    A = np.abs(W) if absolute else W
    return np.asarray(A, np.float64).sum(axis=1)


def sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def _xlogx(p):
    out = np.zeros_like(p)
    nz = p > 0
    out[nz] = p[nz] * np.log(p[nz])
    return out


# ----------------------------------------------------------------------------
# MaxCut, single field (SM "Simplification of FEM for solving the MaxCut problem")
# ----------------------------------------------------------------------------

def maxcut_free_energy(W, h, beta):
    """F per replica for P_i(+1) = sigmoid(h_i), in the listing's ordered-pair form:
    F = -sum_{i,j} W_ij sum_s P_i(s)(1 - P_j(s)) + (1/beta) sum_i sum_s P_i(s) ln P_i(s)
    (Methods, the MaxCut free energy; SM listing ``F = -cut(W,p) - S(p)/beta``).
    h: [N, R].  Returns [R]."""
    P = sigmoid(h)
    cut = np.zeros(h.shape[1])
    for Ps in (P, 1.0 - P):            # the two states s = +1, -1
        cut += ((W @ Ps) * (1.0 - Ps)).sum(axis=0)
    ent = (_xlogx(P) + _xlogx(1.0 - P)).sum(axis=0)
    return -cut + ent / beta


def maxcut_normaliser(W):
    """c_i = 1 / sum_j |W_ij| (SM, after Eq. maxcut_modified_gradient); 0 when isolated."""
    s = _row_sums(W, absolute=True)
    c = np.zeros_like(s)
    c[s > 0] = 1.0 / s[s > 0]
    return c


def maxcut_grad(W, h, beta, gamma=1.0, mode="paper", c=None, discretise=True):
    """g^h_i for the single-field MaxCut (SM Eq. grad_m_h):

    exact: g_i = (gamma/4) [ 2 sum_j W_ij m_j + h_i / beta ] (1 - m_i^2)
           (the true dF/dh_i of ``maxcut_free_energy`` when gamma = 1;
            from Eq. S-maxcut_gradient through the chain rule Eq. gradients_wrt_h)
    paper: g_i = (gamma/4) [ c_i sum_j W_ij sgn(m_j) + h_i / beta ] (1 - m_i^2)
           with c_i = 1/sum_j |W_ij| (Eq. maxcut_modified_gradient reduced to one field).

    ``c`` and ``discretise`` override the normaliser and the discretisation
    (used only by the reduction-identity tests)."""
    m = np.tanh(0.5 * h)
    if mode == "exact":
        field = 2.0 * (W @ m)
    elif mode == "paper":
        if c is None:
            c = maxcut_normaliser(W)
        s = np.where(h >= 0, 1.0, -1.0) if discretise else m
        field = np.asarray(c, np.float64)[:, None] * (W @ s)
    else:
        raise ValueError(mode)
    return gamma / 4.0 * (field + h / beta) * (1.0 - m * m)


# ----------------------------------------------------------------------------
# Balanced MinCut, q-state softmax fields (Methods Eq. loss:bmincut; SM bMinCut
# gradient and manipulated gradient; chain rule Eq. gradients_wrt_h)
# ----------------------------------------------------------------------------

def _softmax(h):
    z = h - h.max(axis=-1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=-1, keepdims=True)


def _log_softmax(h):
    z = h - h.max(axis=-1, keepdims=True)
    return z - np.log(np.exp(z).sum(axis=-1, keepdims=True))


def _apply(W, X):
    """sum_j W_ij X_j for X of shape [N, ...]."""
    n = X.shape[0]
    return np.asarray(W @ X.reshape(n, -1)).reshape(X.shape)


def bmincut_free_energy(W, h, beta, lam, V=None):
    """F per replica, listing form ``cut + penalty*balance - S/beta``:
    F = sum_{i,j} W_ij sum_s P_i(s)(1-P_j(s)) + lam sum_s[(sum_i V_i P_i(s))^2 - sum_i V_i^2 P_i(s)^2]
        + (1/beta) sum P ln P.      h: [N, R, q] -> [R].
    V: node weights (SM, FPGA partitioning of community graphs: a coarsened node weighs
    the number of nodes it groups); None means every V_i = 1."""
    P = _softmax(h)
    Vn = np.ones(h.shape[0]) if V is None else np.asarray(V, np.float64)
    cut = (_apply(W, P) * (1.0 - P)).sum(axis=(0, 2))
    col = (Vn[:, None, None] * P).sum(axis=0)             # [R, q]
    balance = (col ** 2).sum(axis=1) - ((Vn[:, None, None] * P) ** 2).sum(axis=(0, 2))
    ent = _xlogx(P).sum(axis=(0, 2))
    return cut + lam * balance + ent / beta


def bmincut_normalisers(W, q):
    """c^f_i = q / sum_j W_ij and c^a_i = q / sqrt(sum_j W_ij) (SM bMinCut); 0 when isolated."""
    s = _row_sums(W)
    cf = np.zeros_like(s)
    ca = np.zeros_like(s)
    cf[s > 0] = q / s[s > 0]
    ca[s > 0] = q / np.sqrt(s[s > 0])
    return cf, ca


def bmincut_grad(W, h, beta, lam, gamma=1.0, mode="paper", cf=None, ca=None, discretise=True, V=None):
    """g^h_i(s) = gamma [ghat_i(s) - sum_s' P_i(s') ghat_i(s')] P_i(s)  (Eq. gradients_wrt_h)

    exact: ghat = -2 sum_j W_ij P_j(s) + 2 lam V_i [sum_j V_j P_j(s) - V_i P_i(s)] + (ln P_i(s) + 1)/beta
    paper: ghat = -c^f_i sum_j W_ij e_j(s) + lam c^a_i V_i [sum_j V_j e_j(s) - V_i e_i(s)] + (ln P_i(s) + 1)/beta
    with e_j the one-hot argmax of P_j and node weights V (SM, node-weighted balance
    term; None: every V_i = 1).  h: [N, R, q]."""
    q = h.shape[2]
    P = _softmax(h)
    logP = _log_softmax(h)
    Vn = (np.ones(h.shape[0]) if V is None else np.asarray(V, np.float64))[:, None, None]
    if mode == "exact":
        VP = Vn * P
        ghat = -2.0 * _apply(W, P) + 2.0 * lam * Vn * (VP.sum(axis=0)[None] - VP) + (logP + 1.0) / beta
    elif mode == "paper":
        if cf is None or ca is None:
            cf0, ca0 = bmincut_normalisers(W, q)
            cf = cf0 if cf is None else cf
            ca = ca0 if ca is None else ca
        if discretise:
            e = np.zeros_like(P)
            idx = np.argmax(h, axis=2)                       # first maximum wins ties
            np.put_along_axis(e, idx[..., None], 1.0, axis=2)
        else:
            e = P
        cf = np.asarray(cf, np.float64)[:, None, None]
        ca = np.asarray(ca, np.float64)[:, None, None]
        Ve = Vn * e
        ghat = -cf * _apply(W, e) + lam * ca * Vn * (Ve.sum(axis=0)[None] - Ve) + (logP + 1.0) / beta
    else:
        raise ValueError(mode)
    return gamma * (ghat - (P * ghat).sum(axis=2, keepdims=True)) * P


# ----------------------------------------------------------------------------
# QUBO (SM, COPs that translate into QUBO formulations): binary sigma_i in {0, 1},
#   E(sigma) = sum_{i != j} Q_ij sigma_i sigma_j + sum_i d_i sigma_i,
# Q symmetric with zero diagonal and d the diagonal of the paper's Q (sigma_i^2 =
# sigma_i for binary variables, so the diagonal is linear).  Single field
# p_i = P(sigma_i = 1) = sigmoid(h_i).
# ----------------------------------------------------------------------------

def qubo_free_energy(Q, d, h, beta):
    """F = sum_{i != j} Q_ij p_i p_j + sum_i d_i p_i + (1/beta) sum_i [p ln p + (1-p) ln(1-p)]
    (U_MF is the exact expectation of E under the product distribution).  h: [N, R] -> [R]."""
    p = sigmoid(h)
    U = (p * np.asarray(Q @ p)).sum(axis=0) + (np.asarray(d, np.float64)[:, None] * p).sum(axis=0)
    return U + (_xlogx(p) + _xlogx(1.0 - p)).sum(axis=0) / beta


def qubo_grad(Q, d, h, beta, gamma=1.0):
    """dF/dh_i = gamma p_i (1 - p_i) [2 sum_j Q_ij p_j + d_i + h_i / beta]
    (Eq. gradients_wrt_h for one field: ln(p / (1 - p)) = h)."""
    p = sigmoid(h)
    return gamma * p * (1.0 - p) * (2.0 * np.asarray(Q @ p) + np.asarray(d, np.float64)[:, None] + h / beta)


def qubo_states(h):
    """sigma_i = 1 where h_i >= 0 (p >= 1/2) else 0.  h: [N, R] -> int8 [N, R]."""
    return (np.asarray(h) >= 0).astype(np.int8)


def qubo_energy(ei, ej, w, d, sigma):
    """E = sum_{(i,j) in E} 2 Q_ij sigma_i sigma_j + sum_i d_i sigma_i per replica (each
    off-diagonal pair listed once in (ei, ej, w))."""
    w = _as_exact(w)
    d = _as_exact(d)
    s = sigma.astype(np.int64)
    return (2 * w[:, None] * s[ei] * s[ej]).sum(axis=0) + (d[:, None] * s).sum(axis=0)


# ----------------------------------------------------------------------------
# Graph colouring (q-state Potts; SM, problems of multi-valued variables):
#   E(sigma) = sum_{(i,j) in E} W_ij delta(sigma_i, sigma_j)   (violated edges)
#   U_MF = sum_{(i,j) in E} W_ij sum_s P_i(s) P_j(s)
# ----------------------------------------------------------------------------

def coloring_free_energy(W, h, beta):
    """F = sum_{(i,j) in E} W_ij sum_s P_i(s) P_j(s) + (1/beta) sum P ln P  (each edge once:
    half the ordered-pair sum of the symmetric W).  h: [N, R, q] -> [R]."""
    P = _softmax(h)
    U = 0.5 * (_apply(W, P) * P).sum(axis=(0, 2))
    return U + _xlogx(P).sum(axis=(0, 2)) / beta


def coloring_grad(W, h, beta, gamma=1.0, mode="exact", cf=None, discretise=True):
    """g^h_i(s) = gamma [ghat_i(s) - sum_s' P_i(s') ghat_i(s')] P_i(s)  (Eq. gradients_wrt_h)
    exact: ghat = sum_j W_ij P_j(s) + (ln P_i(s) + 1)/beta  (the derivative of F)
    paper: ghat = c^f_i sum_j W_ij e_j(s) + (ln P_i(s) + 1)/beta, e_j the one-hot argmax
           (the bMinCut manipulation with the coupling's sign: same colours cost)."""
    q = h.shape[2]
    P = _softmax(h)
    logP = _log_softmax(h)
    if mode == "exact":
        ghat = _apply(W, P) + (logP + 1.0) / beta
    elif mode == "paper":
        if cf is None:
            cf, _ = bmincut_normalisers(W, q)
        if discretise:
            e = np.zeros_like(P)
            np.put_along_axis(e, np.argmax(h, axis=2)[..., None], 1.0, axis=2)
        else:
            e = P
        ghat = np.asarray(cf, np.float64)[:, None, None] * _apply(W, e) + (logP + 1.0) / beta
    else:
        raise ValueError(mode)
    return gamma * (ghat - (P * ghat).sum(axis=2, keepdims=True)) * P


def coloring_energy(ei, ej, w, states):
    """Violated edge weight sum_{(i,j) in E} W_ij [sigma_i == sigma_j] per replica."""
    w = _as_exact(w)
    return (w[:, None] * (states[ei] == states[ej])).sum(axis=0)


# ----------------------------------------------------------------------------
# Max-k-SAT, single field P_i = P(sigma_i = 1) = sigmoid(h_i)
# (Methods Eq. maxksat_F; SM "The MaxSAT problem" explicit gradient)
# ----------------------------------------------------------------------------

def sat_arrays(ptr, lits):
    """Group clauses by width: list of (var[M_k, k] 0-based, sign[M_k, k] = +1 for a
    positive literal (W_mi = 1), -1 for a negated one (W_mi = 0))."""
    ptr = np.asarray(ptr, np.int64)
    lits = np.asarray(lits, np.int64)
    widths = np.diff(ptr)
    groups = []
    for k in np.unique(widths):
        ms = np.nonzero(widths == k)[0]
        idx = ptr[ms][:, None] + np.arange(k)[None, :]
        L = lits[idx]
        groups.append((np.abs(L) - 1, np.sign(L).astype(np.float64)))
    return groups


def _sat_u(groups_entry, p):
    var, sgn = groups_entry
    pv = p[var]                                            # [M, k, R]
    # u_mi = 1 - P_i(W_mi): positive literal -> 1 - p_i, negated -> p_i
    return np.where(sgn[..., None] > 0, 1.0 - pv, pv)


def sat_free_energy(groups, h, beta):
    """F = sum_m prod_{i in dm} [1 - P_i(W_mi)] + (1/beta) sum P ln P.  h: [N, R]."""
    p = sigmoid(h)
    U = np.zeros(h.shape[1])
    for g in groups:
        U += _sat_u(g, p).prod(axis=1).sum(axis=0)
    ent = (_xlogx(p) + _xlogx(1.0 - p)).sum(axis=0)
    return U + ent / beta


def sat_grad(groups, h, beta, gamma=1.0):
    """g_i = gamma p_i (1 - p_i) [ -sum_{m in di} s_mi prod_{k in dm, k != i} u_mk + h_i/beta ]

    from the SM gradient (-sum_m delta(sigma_i, W_mi) prod_{k != i}[1 - P_k(W_mk)]
    + (ln P + 1)/beta) taken through Eq. gradients_wrt_h for the two states of
    sigma_i; s_mi = +1 for a positive and -1 for a negated literal.  The SAT
    gradient is not manipulated, so exact and paper modes coincide."""
    p = sigmoid(h)
    G = np.zeros_like(h)
    for var, sgn in groups:
        u = _sat_u((var, sgn), p)                         # [M, k, R]
        k = var.shape[1]
        for a in range(k):
            others = np.ones_like(u[:, 0])
            for b in range(k):
                if b != a:
                    others = others * u[:, b]
            np.add.at(G, var[:, a], sgn[:, a, None] * others)
    return gamma * p * (1.0 - p) * (-G + h / beta)


# ----------------------------------------------------------------------------
# Optimizers: PyTorch's Adam, RMSprop and SGD (Methods, "Hyperparameter tunning";
# the paper uses the PyTorch implementations with their defaults).
# ----------------------------------------------------------------------------

class Adam:
    """Kingma & Ba's Adam with PyTorch's placement of eps and L2 weight decay:
    g += wd h; m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
    h -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, shape, lr=0.1, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, **_):
        self.lr, self.b1, self.b2, self.eps, self.wd = lr, beta1, beta2, eps, weight_decay
        self.m = np.zeros(shape)
        self.v = np.zeros(shape)

    def step(self, h, g, t):
        if self.wd:
            g = g + self.wd * h
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mhat = self.m / (1.0 - self.b1 ** t)
        vhat = self.v / (1.0 - self.b2 ** t)
        h -= self.lr * mhat / (np.sqrt(vhat) + self.eps)

    def denominator(self, t):
        return np.sqrt(self.v / (1.0 - self.b2 ** t)) + self.eps


class RMSprop:
    """PyTorch RMSprop (not centred): g += wd h; v = a v + (1-a) g^2;
    with momentum mu > 0: buf = mu buf + g/(sqrt(v)+eps), h -= lr buf; else h -= lr g/(sqrt(v)+eps)."""

    def __init__(self, shape, lr=0.01, alpha=0.99, eps=1e-8, weight_decay=0.0, momentum=0.0, **_):
        self.lr, self.alpha, self.eps, self.wd, self.mu = lr, alpha, eps, weight_decay, momentum
        self.v = np.zeros(shape)
        self.buf = np.zeros(shape)

    def step(self, h, g, t):
        if self.wd:
            g = g + self.wd * h
        self.v = self.alpha * self.v + (1.0 - self.alpha) * g * g
        avg = np.sqrt(self.v) + self.eps
        if self.mu > 0:
            self.buf = self.mu * self.buf + g / avg
            h -= self.lr * self.buf
        else:
            h -= self.lr * g / avg

    def denominator(self, t):
        return np.sqrt(self.v) + self.eps


class SGD:
    """PyTorch SGD (no Nesterov): g += wd h; with momentum mu != 0:
    buf = g at the first step, else buf = mu buf + (1 - dampening) g; g = buf; h -= lr g."""

    def __init__(self, shape, lr=0.01, momentum=0.0, dampening=0.0, weight_decay=0.0, **_):
        self.lr, self.mu, self.damp, self.wd = lr, momentum, dampening, weight_decay
        self.buf = np.zeros(shape)

    def step(self, h, g, t):
        if self.wd:
            g = g + self.wd * h
        if self.mu != 0:
            if t == 1:
                self.buf = g.copy()
            else:
                self.buf = self.mu * self.buf + (1.0 - self.damp) * g
            g = self.buf
        h -= self.lr * g

    def denominator(self, t):
        return np.full(self.buf.shape, np.inf)


def make_optimizer(name, shape, **kw):
    return {"adam": Adam, "rmsprop": RMSprop, "sgd": SGD}[name](shape, **kw)


# ----------------------------------------------------------------------------
# The FEM outer loop (Results "Free-Energy Machine": fields -> marginals ->
# gradient -> optimizer step, while beta is annealed; then argmax per replica
# and the replica of minimum energy).
# ----------------------------------------------------------------------------

def anneal(problem, h0, n_step, *, t_begin=0, t_end=None, schedule="exponential",
           beta_min=0.05, beta_max=5.0, optimizer="adam", opt_kw=None, mode="paper",
           gamma=1.0, lambda_max=1.0, opt=None, trace=None, cond=None):
    """Run anneal steps t_begin .. t_end-1 from fields h0 (copied, float64).

    problem: ("maxcut", W) | ("bmincut", W) | ("bmincut", W, V) | ("coloring", W) | ("qubo", (Q, d))
             | ("pspin", (ptr, var, J, b)) | ("sat", groups)
    Returns (h, opt); pass ``opt`` back in to resume.  ``trace``, if a dict
    {t: None}, is filled with copies of h after step t (1-based count of steps done).
    ``cond``, if a dict {t: None}, is filled with the elementwise minimum over the
    steps up to t of the optimizer's denominator (a conditioning record for
    comparisons in fp32: the update divides by it, so gradient rounding is
    amplified where it is small)."""
    kind, data = problem[0], problem[1]
    node_w = problem[2] if len(problem) > 2 else None
    t_end = n_step if t_end is None else t_end
    h = np.array(h0, dtype=np.float64, copy=True)
    betas = beta_schedule(schedule, beta_min, beta_max, n_step)
    lams = lambda_ramp(lambda_max, n_step)
    if opt is None:
        opt = make_optimizer(optimizer, h.shape, **(opt_kw or {}))
    gm = np.full(h.shape, np.inf) if cond is not None else None
    for t in range(t_begin, t_end):
        beta = betas[t]
        if kind == "maxcut":
            g = maxcut_grad(data, h, beta, gamma=gamma, mode=mode)
        elif kind == "bmincut":
            g = bmincut_grad(data, h, beta, lams[t], gamma=gamma, mode=mode, V=node_w)
        elif kind == "coloring":
            g = coloring_grad(data, h, beta, gamma=gamma, mode=mode)
        elif kind == "qubo":
            g = qubo_grad(data[0], data[1], h, beta, gamma=gamma)
        elif kind == "pspin":
            g = pspin_grad(*data, h, beta, gamma=gamma)
        elif kind == "sat":
            g = sat_grad(data, h, beta, gamma=gamma)
        else:
            raise ValueError(kind)
        opt.step(h, g, t + 1)
        if gm is not None:
            np.minimum(gm, opt.denominator(t + 1), out=gm)
            if (t + 1) in cond:
                cond[t + 1] = gm.copy()
        if trace is not None and (t + 1) in trace:
            trace[t + 1] = h.copy()
    return h, opt


# ----------------------------------------------------------------------------
# Higher-order interactions (SM, problems with multi-variable interactions: p-spin
# glasses and the quantum error-correction Hamiltonian): spins sigma_i in {-1, +1},
#   E(sigma) = sum_v J_v prod_{i in v} sigma_i + sum_i b_i sigma_i,
# <E> = sum_v J_v prod_{i in v} m_i + sum_i b_i m_i with m_i = tanh(h_i / 2) =
# P_i(+1) - P_i(-1).  Terms are given as (ptr, var) lists of 0-based variables.
# ----------------------------------------------------------------------------

def _pspin_terms(ptr, var):
    ptr = np.asarray(ptr, np.int64)
    var = np.asarray(var, np.int64)
    return [var[ptr[t]:ptr[t + 1]] for t in range(ptr.shape[0] - 1)]


def pspin_free_energy(ptr, var, J, b, h, beta):
    """F = <E> + (1/beta) sum_i [p ln p + (1-p) ln(1-p)], p = sigmoid(h).  h: [N, R] -> [R]."""
    m = np.tanh(0.5 * np.asarray(h, np.float64))
    U = (np.asarray(b, np.float64)[:, None] * m).sum(axis=0)
    for Jt, vs in zip(np.asarray(J, np.float64), _pspin_terms(ptr, var)):
        U = U + Jt * m[vs].prod(axis=0)
    p = sigmoid(h)
    return U + (_xlogx(p) + _xlogx(1.0 - p)).sum(axis=0) / beta


def pspin_grad(ptr, var, J, b, h, beta, gamma=1.0):
    """dF/dh_i = gamma (1 - m_i^2) / 4 [2 (sum_{v ni i} J_v prod_{k in v, k != i} m_k + b_i) + h_i / beta]
    (dm/dh = (1 - m^2)/2 and the entropy term h/beta p(1-p) = h/beta (1 - m^2)/4)."""
    m = np.tanh(0.5 * np.asarray(h, np.float64))
    dE = np.repeat(np.asarray(b, np.float64)[:, None], h.shape[1], axis=1)
    for Jt, vs in zip(np.asarray(J, np.float64), _pspin_terms(ptr, var)):
        for a, i in enumerate(vs):
            others = np.delete(vs, a)
            dE[i] += Jt * (m[others].prod(axis=0) if others.size else 1.0)
    return gamma * 0.25 * (1.0 - m * m) * (2.0 * dE + h / beta)


def pspin_energy(ptr, var, J, b, sigma):
    """E = sum_v J_v prod_{i in v} sigma_i + sum_i b_i sigma_i per replica, sigma in {-1, +1}."""
    J = _as_exact(J)
    b = _as_exact(b)
    s = sigma.astype(np.int64)
    E = (b[:, None] * s).sum(axis=0)
    for Jt, vs in zip(J, _pspin_terms(ptr, var)):
        E = E + Jt * s[vs].prod(axis=0)
    return E


# ----------------------------------------------------------------------------
# Readout (Results Eqs. for sigma~ = argmax P and sigma^ = argmin E) and the
# exact integer objectives (Eqs. maxcut1, bmincut, maxksat_E).
# ----------------------------------------------------------------------------

def maxcut_states(h):
    """sigma_i = +1 where h_i >= 0 else -1.  h: [N, R] -> int8 [N, R]."""
    return np.where(np.asarray(h) >= 0, 1, -1).astype(np.int8)


def _as_exact(w):
    w = np.asarray(w, np.float64)
    if np.all(w == np.round(w)):
        return w.astype(np.int64)
    return w


def maxcut_cut_edges(ei, ej, w, sigma):
    """C = sum_{(i,j) in E} W_ij [sigma_i != sigma_j], per replica (edge-list scan)."""
    w = _as_exact(w)
    diff = (sigma[ei] != sigma[ej])                        # [E, R]
    return (w[:, None] * diff).sum(axis=0)


def maxcut_cut_spin(ei, ej, w, sigma):
    """Spin form C = (W_tot - sum_E W_ij s_i s_j) / 2, an independent recomputation."""
    w = _as_exact(w)
    s = sigma.astype(np.int64)
    tot = w.sum()
    corr = (w[:, None] * s[ei] * s[ej]).sum(axis=0)
    return (tot - corr) // 2 if w.dtype == np.int64 else (tot - corr) / 2


def maxcut_cut_matrix(W, sigma):
    """Matrix form C = (1/2) sum_{i,j} W_ij [sigma_i != sigma_j] over ordered pairs."""
    s = sigma.astype(np.float64)
    tot = _row_sums(W).sum()
    return 0.25 * (tot - (s * (W @ s)).sum(axis=0))


def bmincut_states(h):
    """argmax_s h_i(s), lowest index on ties.  h: [N, R, q] -> int32 [N, R]."""
    return np.argmax(np.asarray(h), axis=2).astype(np.int32)


def bmincut_objective(ei, ej, w, states, q, lam, V=None):
    """(E, cut, sizes) per replica with E = cut + lam * sum_s [n_s^2 - sum_{i in s} V_i^2],
    n_s = sum_{i in s} V_i (Eq. bmincut with the node-weighted balance term; for V = 1 it
    is lam * sum_i sum_{j != i} delta(sigma_i, sigma_j) = lam * sum_s n_s(n_s - 1))."""
    w = _as_exact(w)
    cut = (w[:, None] * (states[ei] != states[ej])).sum(axis=0)
    R = states.shape[1]
    Vn = np.ones(states.shape[0], dtype=np.int64) if V is None else np.asarray(V, np.int64)
    sizes = np.zeros((R, q), dtype=np.int64)
    for s in range(q):
        sizes[:, s] = (Vn[:, None] * (states == s)).sum(axis=0)
    bal = (sizes * sizes).sum(axis=1) - (Vn * Vn).sum()
    lam_exact = int(lam) if float(lam).is_integer() and w.dtype == np.int64 else lam
    return cut + lam_exact * bal, cut, sizes


def sat_states(h):
    """sigma_i = 1 where h_i >= 0 else 0.  h: [N, R] -> int8 [N, R]."""
    return (np.asarray(h) >= 0).astype(np.int8)


def sat_unsat(ptr, lits, states):
    """Number of unsatisfied clauses per replica (direct clause scan)."""
    ptr = np.asarray(ptr, np.int64)
    lits = np.asarray(lits, np.int64)
    R = states.shape[1]
    sat = np.zeros((ptr.shape[0] - 1, R), dtype=bool)
    widths = np.diff(ptr)
    for a in range(int(widths.max()) if widths.size else 0):
        has = widths > a
        L = lits[ptr[:-1][has] + a]
        val = states[np.abs(L) - 1]                        # [M', R]
        true_lit = np.where(L[:, None] > 0, val == 1, val == 0)
        sat[has] |= true_lit
    return (~sat).sum(axis=0).astype(np.int64)


def best_replica(energy):
    """argmin over replicas; the lowest replica index wins ties."""
    energy = np.asarray(energy)
    return int(np.argmin(energy))
