"""FP64 oracle of the learned adaptation proposer (TEST INFRASTRUCTURE).

The paper has no learned part; this is the proposer the library adds on
top of the method's own criterion (Sec. 3.4): a small MLP that, from local
macroscopic features, predicts which cells can decide a split/merge, so that
the criterion is evaluated only on that check set.  Everything here is plain
numpy in float64 and written from these definitions:

features (8 per cell i; rho, U, T from the moments of f, R = 1/2, T_ref = 1)
  0  log rho_i
  1  U_x / sqrt(R T_ref)
  2  U_y / sqrt(R T_ref)
  3  U_z / sqrt(R T_ref) in 3D; |q_i| / (rho_i (R T_i)^(3/2)) in 2D
  4  log T_i
  5  log(lambda_i / dx_i), lambda from Eq. (4) with the VHS viscosity of Eq. (3),
     dx_i = |V_i|^(1/D)
  6  max over face neighbours |rho_j - rho_i| / rho_i
  7  max over face neighbours |T_j - T_i| / T_i
labels (4 per cell) from m_ik = s max(M1_ik, M2_ik) and M_k = max_i m_ik
  0  split witness:   some node k below the level cap has m_ik > C1
  1  dominant:        some node k with M_k >= C2 has m_ik == M_k
  2  near-dominant:   some node k with M_k >= C2 has m_ik >= M_k / 2
  3  merge blocker:   some node k of level >= 1 has m_ik >= C2
network  x (8) -> 64 ReLU -> 64 ReLU -> 4 logits; loss = mean BCE with logits.
"""
from __future__ import annotations

import math

import numpy as np

H = 64
NF = 8
NO = 4


def features(D, Wc, q, vol, faceL, faceR, R=0.5, mu_ref=1.0, omega=0.81, T_ref=1.0):
    """Per-cell features (see module docstring) from conserved W and heat flux q."""
    rho = Wc[:, 0]
    U = Wc[:, 1:1 + D] / rho[:, None]
    RT = (Wc[:, D + 1] - 0.5 * (Wc[:, 1:1 + D] ** 2).sum(1) / rho) / (1.5 * rho)
    T = RT / R
    mu = mu_ref * (T / T_ref) ** omega
    lam = 2.0 * mu * (5 - 2 * omega) * (7 - 2 * omega) / (15.0 * rho * np.sqrt(2 * math.pi * RT))
    dx = vol ** (1.0 / D)
    X = np.zeros((len(rho), NF))
    X[:, 0] = np.log(rho)
    su = math.sqrt(R * T_ref)
    X[:, 1] = U[:, 0] / su
    X[:, 2] = U[:, 1] / su
    X[:, 3] = U[:, 2] / su if D == 3 else np.sqrt((q * q).sum(1)) / (rho * RT ** 1.5)
    X[:, 4] = np.log(T)
    X[:, 5] = np.log(lam / dx)
    inner = faceR >= 0
    L, Rr = faceL[inner], faceR[inner]
    for a, b in ((L, Rr), (Rr, L)):
        np.maximum.at(X[:, 6], a, np.abs(rho[b] - rho[a]) / rho[a])
        np.maximum.at(X[:, 7], a, np.abs(T[b] - T[a]) / T[a])
    return X


def criterion_values(D, xi, w, f, Wc, s):
    """Scaled criterion values m[i, k] = s * max(M1_ik, M2_ik) (Eqs.
    criterion_rho, criterion_e) in the oracle's operation order."""
    rho = Wc[:, 0]
    U = Wc[:, 1:1 + D] / rho[:, None]
    mm = np.zeros_like(rho)
    for d in range(D):
        mm = mm + Wc[:, 1 + d] * Wc[:, 1 + d]
    eint = Wc[:, D + 1] - 0.5 * mm / rho
    wg = w[None, :] * f[:, 0, :]
    m1 = wg / rho[:, None]
    c2 = np.zeros_like(wg)
    for d in range(D):
        c = xi[None, :, d] - U[:, d:d + 1]
        c2 = c2 + c * c
    m2 = ((0.5 * wg) * c2) / eint[:, None]
    return s * np.maximum(m1, m2)


def labels(m, M, level, C1, C2, max_refine):
    """Per-cell labels from the scaled criterion values m[i, k] and their max M[k].
    max_refine: the level cap, one value or one per node (refinement zones)."""
    act = M >= C2
    y = np.zeros((m.shape[0], NO))
    y[:, 0] = ((m > C1) & (level < max_refine)[None, :]).any(1)
    y[:, 1] = ((m == M[None, :]) & act[None, :]).any(1)
    y[:, 2] = ((m >= 0.5 * M[None, :]) & act[None, :]).any(1)
    y[:, 3] = ((m >= C2) & (level >= 1)[None, :]).any(1)
    return y


def init_params(seed=2212):
    """He-uniform initial weights from a seeded generator (shared input)."""
    rng = np.random.default_rng(seed)
    def lin(n_out, n_in):
        b = math.sqrt(6.0 / n_in)
        return rng.uniform(-b, b, size=(n_out, n_in)), np.zeros(n_out)
    W1, b1 = lin(H, NF)
    W2, b2 = lin(H, H)
    W3, b3 = lin(NO, H)
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3)


def forward(p, X):
    Z1 = X @ p["W1"].T + p["b1"]
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ p["W2"].T + p["b2"]
    A2 = np.maximum(Z2, 0.0)
    Z3 = A2 @ p["W3"].T + p["b3"]
    return Z3, (X, Z1, A1, Z2, A2)


def loss(p, X, Y):
    Z3, _ = forward(p, X)
    # mean binary cross-entropy with logits, numerically stable form
    return float(np.mean(np.maximum(Z3, 0) - Z3 * Y + np.log1p(np.exp(-np.abs(Z3)))))


def backward(p, X, Y):
    """Gradients of `loss` with respect to every parameter."""
    Z3, (X, Z1, A1, Z2, A2) = forward(p, X)
    n = X.shape[0] * NO
    S = 1.0 / (1.0 + np.exp(-Z3))
    dZ3 = (S - Y) / n
    g = {}
    g["W3"] = dZ3.T @ A2
    g["b3"] = dZ3.sum(0)
    dA2 = dZ3 @ p["W3"]
    dZ2 = dA2 * (Z2 > 0)
    g["W2"] = dZ2.T @ A1
    g["b2"] = dZ2.sum(0)
    dA1 = dZ2 @ p["W2"]
    dZ1 = dA1 * (Z1 > 0)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(0)
    return g


def sgd(p, g, lr):
    return {k: p[k] - lr * g[k] for k in p}
