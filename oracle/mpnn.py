"""FP64 reference of the warm-start message-passing network - TEST INFRASTRUCTURE ONLY.

The network predicts initial local fields for MaxCut FEM from the graph and each
replica's random initial fields z (in units of the 0.001 scale of the paper's
0.001*randn initialisation).  It is not part of the paper; its design:

  P = D^-1 W (row-normalised signed couplings, zero rows for isolated nodes)
  s_i = [1, deg_i / mean deg, (sum_j W_ij)/deg_i, 1/sqrt(deg_i + 1)]     (4 features)
  x^0 = s;  for l = 1..3:  a^l = P x^(l-1),  x^l = tanh(x^(l-1) A_l + a^l B_l + b_l)   (width 64)
  theta = x^3 C + c                                   (K = 4 filter taps per node)
  u_0 = z,  u_k = P u_(k-1);   y_ir = sum_k theta_ik u_k,ir       (predicted fields)
  loss L = mean_ir (tanh(y_ir / 2) - m_ir)^2,  m = FEM's marginals tanh(h/2) at the target step

y is linear in z, so the prediction is odd under z -> -z, which is MaxCut's global
spin-flip symmetry.  Weights are used rounded to bf16 in the forward pass (both here
and on the GPU); gradients are the exact derivatives with respect to those weights.
Pinned by central finite differences of ``loss`` (tests/test_oracle_mpnn.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["mpnn_propagation", "mpnn_features", "bf16_round", "mpnn_forward", "mpnn_loss",
           "mpnn_backward", "mpnn_normalize", "PARAM_ORDER"]

PARAM_ORDER = ["A1", "B1", "b1", "A2", "B2", "b2", "A3", "B3", "b3", "C", "c"]


def mpnn_propagation(n, ei, ej, w):
    """(P, deg): P = D^-1 W as a CSR matrix, deg = number of neighbours."""
    W = sp.coo_matrix((np.asarray(w, np.float64), (np.asarray(ei), np.asarray(ej))), shape=(n, n))
    W = (W + W.T).tocsr()
    deg = np.diff(W.indptr).astype(np.float64)
    inv = np.zeros(n)
    inv[deg > 0] = 1.0 / deg[deg > 0]
    return sp.diags(inv) @ W, deg, W


def mpnn_features(deg, W):
    n = deg.shape[0]
    rowsum = np.asarray(W.sum(axis=1)).ravel()
    f = np.zeros((n, 4))
    f[:, 0] = 1.0
    f[:, 1] = deg / max(deg.mean(), 1e-12)
    f[deg > 0, 2] = rowsum[deg > 0] / deg[deg > 0]
    f[:, 3] = 1.0 / np.sqrt(deg + 1.0)
    return f


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    x32 = np.asarray(x, np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def mpnn_forward(params, P, feats, z, taps=4, round_weights=True):
    """Returns (y [n, R], cache).  params: dict of float64 arrays, rounded to bf16 here
    (round_weights=False keeps them exact, for finite-difference checks)."""
    p = {k: (bf16_round(v) if round_weights else np.asarray(v, np.float64)) for k, v in params.items()}
    xs, As = [feats], []
    x = feats
    for l in (1, 2, 3):
        a = P @ x
        x = np.tanh(x @ p[f"A{l}"] + a @ p[f"B{l}"] + p[f"b{l}"])
        As.append(a)
        xs.append(x)
    theta = x @ p["C"] + p["c"]
    us = [z]
    for _ in range(1, taps):
        us.append(P @ us[-1])
    y = sum(theta[:, k:k + 1] * us[k] for k in range(taps))
    return y, dict(p=p, xs=xs, As=As, theta=theta, us=us, P=P)


def mpnn_loss(y, m_target):
    return float(np.mean((np.tanh(0.5 * y) - m_target) ** 2))


def mpnn_backward(cache, y, m_target):
    """Gradients of mpnn_loss with respect to every parameter (dict, float64)."""
    p, xs, As, us, P = cache["p"], cache["xs"], cache["As"], cache["us"], cache["P"]
    t = np.tanh(0.5 * y)
    dy = 2.0 * (t - m_target) * 0.5 * (1.0 - t * t) / y.size
    g = {}
    dtheta = np.stack([(dy * us[k]).sum(axis=1) for k in range(len(us))], axis=1)
    g["C"] = xs[3].T @ dtheta
    g["c"] = dtheta.sum(axis=0)
    dx = dtheta @ p["C"].T
    PT = P.T.tocsr()
    for l in (3, 2, 1):
        x_in, a, x_out = xs[l - 1], As[l - 1], xs[l]
        dpre = dx * (1.0 - x_out * x_out)
        g[f"A{l}"] = x_in.T @ dpre
        g[f"B{l}"] = a.T @ dpre
        g[f"b{l}"] = dpre.sum(axis=0)
        dx = dpre @ p[f"A{l}"].T + PT @ (dpre @ p[f"B{l}"].T)
    return g


def mpnn_normalize(y, rms):
    """Every replica's column rescaled to root-mean-square rms (the magnitude of the warm
    start; the network gives its direction).  An all-zero column stays zero."""
    y = np.asarray(y, np.float64)
    cur = np.sqrt(np.mean(y * y, axis=0))
    scale = np.where(cur > 0, rms / np.where(cur > 0, cur, 1.0), 0.0)
    return y * scale
