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
For the diatomic (Rykov) gas of Sec. 2.1, T is the translational temperature
T_t, (3/2) rho R T_t = rho E - rho U^2 / 2 - rho E_rot: the temperature of the
velocity distribution G the velocity mesh resolves, and the one the model's
viscosity and relaxation time take; q is the total heat flux q_t + q_r.
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


def features(D, Wc, q, vol, faceL, faceR, R=0.5, mu_ref=1.0, omega=0.81, T_ref=1.0, rykov=False):
    """Per-cell features (see module docstring) from conserved W and heat flux q.
    rykov: W carries rho E_rot in column D+2 and T is the translational T_t."""
    rho = Wc[:, 0]
    U = Wc[:, 1:1 + D] / rho[:, None]
    eint = Wc[:, D + 1] - 0.5 * (Wc[:, 1:1 + D] ** 2).sum(1) / rho
    if rykov:
        eint = eint - Wc[:, D + 2]
    RT = eint / (1.5 * rho)
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


def bf16_round(x):
    """Nearest BF16 value (ties to even) of float32(x), as float64."""
    a = np.ascontiguousarray(x, np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gradient_error_bound(p, X, Y, u=2.0 ** -8, u32=2.0 ** -24):
    """First-order elementwise bound on |g' - g| for every parameter gradient
    g of `loss`, where g' is computed with BF16 operands in every product.

    Model of g': the weights in p and the inputs X are already BF16 values
    (the same in both); the activations A1, A2 are rounded to BF16 before the
    next layer's product, and so are the backward signals dZ3, dZ2, dZ1 before
    their products (unit roundoff u each); the products accumulate in FP32 (a
    K-term sum errs by at most K u32 times the sum of the absolute terms); the
    bias gradients sum the unrounded FP32 signals; the sigmoid is evaluated to
    a few FP32 ulp.  Each error is carried through the layers with absolute
    values (ReLU and the sum are 1-Lipschitz, the sigmoid 1/4-Lipschitz).  A
    ReLU whose input lies within its own error bound of zero may switch, which
    adds the whole derivative at that element.  Returns (bounds per parameter
    like `backward`, bound on the logits)."""
    Z3, (X, Z1, A1, Z2, A2) = forward(p, X)
    n = X.shape[0]
    nn = n * NO
    aW1, aW2, aW3 = np.abs(p["W1"]), np.abs(p["W2"]), np.abs(p["W3"])
    aX, aA1, aA2 = np.abs(X), np.abs(A1), np.abs(A2)
    g8, g64, gn = NF * u32, H * u32, n * u32
    # forward
    eZ1 = g8 * (aX @ aW1.T + np.abs(p["b1"]))
    eA1b = eZ1 + u * (aA1 + eZ1)
    eZ2 = eA1b @ aW2.T + g64 * (aA1 @ aW2.T + np.abs(p["b2"]))
    eA2b = eZ2 + u * (aA2 + eZ2)
    eZ3 = eA2b @ aW3.T + g64 * (aA2 @ aW3.T + np.abs(p["b3"]))
    # backward
    S = 1.0 / (1.0 + np.exp(-Z3))
    dZ3 = (S - Y) / nn
    aD3 = np.abs(dZ3)
    e3 = (0.25 * eZ3 + 2.0 ** -20 * S) / nn
    e3b = e3 + u * (aD3 + e3)
    dA2 = dZ3 @ p["W3"]
    edA2 = e3b @ aW3 + NO * u32 * (aD3 @ aW3)
    amb2 = np.abs(Z2) <= eZ2
    dZ2 = dA2 * (Z2 > 0)
    e2 = np.where(amb2, np.abs(dA2) + edA2, edA2 * (Z2 > 0))
    aD2 = np.abs(dZ2)
    e2b = e2 + u * (aD2 + e2)
    dA1 = dZ2 @ p["W2"]
    edA1 = e2b @ aW2 + g64 * (aD2 @ aW2)
    amb1 = np.abs(Z1) <= eZ1
    dZ1 = dA1 * (Z1 > 0)
    e1 = np.where(amb1, np.abs(dA1) + edA1, edA1 * (Z1 > 0))
    aD1 = np.abs(dZ1)
    e1b = e1 + u * (aD1 + e1)
    b = {}
    b["W3"] = e3b.T @ aA2 + aD3.T @ eA2b + e3b.T @ eA2b + gn * (aD3.T @ aA2)
    b["b3"] = e3.sum(0) + gn * aD3.sum(0)
    b["W2"] = e2b.T @ aA1 + aD2.T @ eA1b + e2b.T @ eA1b + gn * (aD2.T @ aA1)
    b["b2"] = e2.sum(0) + gn * aD2.sum(0)
    b["W1"] = e1b.T @ aX + gn * (aD1.T @ aX)
    b["b1"] = e1.sum(0) + gn * aD1.sum(0)
    return b, eZ3


def backward_bf16_emulated(p, X, Y):
    """The gradients as a BF16-operand pipeline computes them (the model of
    gradient_error_bound), emulated in numpy: float32 arithmetic, BF16
    rounding of A1, A2, dZ3, dZ2, dZ1 before each product.  Used only to
    check that the bound holds; the GPU kernels are checked against the bound
    directly."""
    f32 = np.float32
    W1, W2, W3 = (p[k].astype(f32) for k in ("W1", "W2", "W3"))
    b1, b2, b3 = (p[k].astype(f32) for k in ("b1", "b2", "b3"))
    Xf = X.astype(f32)
    Z1 = Xf @ W1.T + b1
    A1 = np.maximum(Z1, f32(0))
    A1b = bf16_round(A1).astype(f32)
    Z2 = A1b @ W2.T + b2
    A2 = np.maximum(Z2, f32(0))
    A2b = bf16_round(A2).astype(f32)
    Z3 = A2b @ W3.T + b3
    nn = f32(X.shape[0] * NO)
    dZ3 = ((f32(1) / (f32(1) + np.exp(-Z3))) - Y.astype(f32)) / nn
    d3b = bf16_round(dZ3).astype(f32)
    g = {}
    g["W3"] = d3b.T @ A2b
    g["b3"] = dZ3.sum(0)
    dZ2 = (d3b @ W3) * (Z2 > 0)
    d2b = bf16_round(dZ2).astype(f32)
    g["W2"] = d2b.T @ A1b
    g["b2"] = dZ2.sum(0)
    dZ1 = (d2b @ W2) * (Z1 > 0)
    d1b = bf16_round(dZ1).astype(f32)
    g["W1"] = d1b.T @ Xf
    g["b1"] = dZ1.sum(0)
    return {k: v.astype(np.float64) for k, v in g.items()}, Z3.astype(np.float64)
