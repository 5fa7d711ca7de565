"""Pins of the FP64 MLP oracle: central finite differences of the loss pin
every gradient; the BCE form matches its definition -[y log s + (1-y) log(1-s)];
features of a uniform state take their closed-form values."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp
from paper_2212_05645_gb300 import workloads as wl


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(3)
    X = rng.standard_normal((37, mlp.NF))
    Y = (rng.random((37, mlp.NO)) > 0.6).astype(float)
    g = mlp.backward(p, X, Y)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            q = {k: v.copy() for k, v in p.items()}
            q[name].reshape(-1)[idx] += h
            lp = mlp.loss(q, X, Y)
            q[name].reshape(-1)[idx] -= 2 * h
            lm = mlp.loss(q, X, Y)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[idx]) < 1e-7 + 1e-5 * abs(fd), (name, idx)


def test_bce_definition_and_sgd_descends():
    rng = np.random.default_rng(1)
    p = mlp.init_params(4)
    X = rng.standard_normal((50, mlp.NF))
    Y = (rng.random((50, mlp.NO)) > 0.5).astype(float)
    Z, _ = mlp.forward(p, X)
    s = 1 / (1 + np.exp(-Z))
    ref = -np.mean(Y * np.log(s) + (1 - Y) * np.log(1 - s))
    assert math.isclose(mlp.loss(p, X, Y), ref, rel_tol=1e-12)
    l0 = mlp.loss(p, X, Y)
    for _ in range(20):
        p = mlp.sgd(p, mlp.backward(p, X, Y), 0.5)
    assert mlp.loss(p, X, Y) < l0


def test_features_uniform_state_closed_form():
    """A uniform state at rest: log rho, zero velocity, log T, log(Kn / dx)
    (the reference mean free path equals Kn), zero neighbour jumps."""
    w = wl.sweep_box((4, 4))
    m = w.mesh
    rho, T = 1.0, 1.0
    Wc = np.tile([rho, 0.0, 0.0, 1.5 * rho * 0.5 * T], (m.Nc, 1))
    q = np.zeros((m.Nc, 2))
    Kn = 0.05
    mu = O.mu_ref_from_Kn(Kn, 0.81)
    X = mlp.features(2, Wc, q, m.vol, m.faceL, m.faceR, mu_ref=mu)
    assert np.allclose(X[:, :5], 0.0)
    assert np.allclose(X[:, 5], math.log(Kn / 0.25), rtol=1e-13)
    assert np.all(X[:, 6:] == 0.0)


@pytest.mark.parametrize("D", [2, 3])
def test_features_rykov_take_the_translational_temperature(D):
    """Diatomic gas (Sec. 2.1): the temperature features are those of T_t,
    whatever the rotational temperature.  W written by hand for rho = 2,
    U = (0.3, -0.2[, 0.1]), T_t = 1.2 and a T_r that differs from cell to cell:
    rho E_rot = rho R T_r, rho E = rho U^2/2 + (3/2) rho R T_t + rho E_rot.
    The mean free path of Eq. 4 scales as T^(omega - 1/2) / rho from its
    reference value Kn at rho = T = 1."""
    w = wl.sweep_box((4, 4)) if D == 2 else wl.sphere(n_r=2, n_theta=3, n_phi=4, max_refine=1)
    m = w.mesh
    R, rho, Tt, Kn, omega = 0.5, 2.0, 1.2, 0.05, 0.81
    U = np.array([0.3, -0.2, 0.1][:D])
    Tr = 0.4 + 0.05 * np.arange(m.Nc)
    Wc = np.zeros((m.Nc, D + 3))
    Wc[:, 0] = rho
    Wc[:, 1:1 + D] = rho * U
    Wc[:, D + 2] = rho * R * Tr
    Wc[:, D + 1] = 0.5 * rho * (U * U).sum() + 1.5 * rho * R * Tt + Wc[:, D + 2]
    q = np.zeros((m.Nc, D))
    mu = O.mu_ref_from_Kn(Kn, omega)
    X = mlp.features(D, Wc, q, m.vol, m.faceL, m.faceR, mu_ref=mu, omega=omega, rykov=True)
    su = math.sqrt(R)
    assert np.allclose(X[:, 0], math.log(rho), rtol=1e-14)
    for d in range(D):
        assert np.allclose(X[:, 1 + d], U[d] / su, rtol=1e-14)
    assert np.allclose(X[:, 4], math.log(Tt), rtol=1e-12)
    lam = Kn * Tt ** (omega - 0.5) / rho
    assert np.allclose(X[:, 5], np.log(lam / m.vol ** (1.0 / D)), rtol=1e-12, atol=1e-13)
    assert np.all(np.abs(X[:, 7]) < 1e-13)            # T_r varies, T_t does not
    assert np.all(X[:, 6] == 0.0)


def test_labels_small_case_by_hand():
    m = np.array([[5.0, 0.1, 0.0], [1.0, 0.2, 3e-4], [1.0, 0.05, 1e-5]])
    M = m.max(0)
    level = np.array([0, 1, 1])
    y = mlp.labels(m, M, level, C1=2.0, C2=1e-3, max_refine=2)
    assert y[:, 0].tolist() == [1, 0, 0]          # only cell 0 exceeds C1
    assert y[:, 1].tolist() == [1, 1, 0]          # argmax of node 0 and node 1 (node 2 inactive)
    assert y[:, 2].tolist() == [1, 1, 0]          # 0.1 >= 0.2/2, 0.2; 0.05 < 0.1
    assert y[:, 3].tolist() == [1, 1, 1]          # level-1 nodes with m >= C2


def _bf16_case(seed, n=301):
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    p["b1"] = 0.1 * rng.standard_normal(mlp.H)
    for k in ("W1", "W2", "W3"):
        p[k] = mlp.bf16_round(p[k])
    X = mlp.bf16_round(rng.standard_normal((n, mlp.NF)))
    Y = (rng.random((n, mlp.NO)) > 0.6).astype(np.float64)
    return p, X, Y


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_bf16_gradient_bound_holds(seed):
    """The elementwise bound of a BF16-operand forward/backward pass (the
    tolerance of the GPU gradient test) contains the deviation of an emulated
    BF16 pipeline from the FP64 gradients on every element.  It is a
    worst-case bound (absolute values through the layers, no cancellation):
    on the elements that matter (|g| above 1 % of the layer's largest) its
    median stays below |g| for the last two layers and below 10 |g| for the
    first, where two products of absolute values stack up; the GPU test
    therefore also compares with the emulated pipeline."""
    p, X, Y = _bf16_case(seed)
    ref = mlp.backward(p, X, Y)
    bound, ez3 = mlp.gradient_error_bound(p, X, Y)
    emu, z3 = mlp.backward_bf16_emulated(p, X, Y)
    z_ref, _ = mlp.forward(p, X)
    assert np.all(np.abs(z3 - z_ref) <= ez3)
    for k in ref:
        d = np.abs(emu[k] - ref[k])
        assert np.all(d <= bound[k]), (k, float((d / np.maximum(bound[k], 1e-300)).max()))
        big = np.abs(ref[k]) > 0.01 * np.abs(ref[k]).max()
        med = np.median(bound[k][big] / np.abs(ref[k][big]))
        assert med < (10.0 if k in ("W1", "b1") else 1.0), (k, med)


def test_bf16_emulation_matches_definition_without_rounding():
    """The emulated pipeline with its BF16 roundings replaced by the identity
    reproduces backward() to float32 accuracy: the emulation differs from the
    definition only by those roundings."""
    p, X, Y = _bf16_case(5, n=40)
    saved = mlp.bf16_round
    try:
        mlp.bf16_round = lambda x: np.asarray(x, np.float64)
        emu, z3 = mlp.backward_bf16_emulated(p, X, Y)
    finally:
        mlp.bf16_round = saved
    ref = mlp.backward(p, X, Y)
    for k in ref:
        assert np.allclose(emu[k], ref[k], rtol=1e-5, atol=1e-7 * np.abs(ref[k]).max()), k
