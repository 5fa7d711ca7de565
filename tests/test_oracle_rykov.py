"""Pins of the oracle's Rykov model (diatomic gas; Sec. 2.1, Eqs. updat_W, 8,
GHR_equ, 11-13) against closed-form moments of its equilibrium, its reduction
to the Shakhov model, conservation laws, the closed-form relaxation of the
rotational energy in a uniform gas, and the free-transport and continuum
limits of the step."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl

R = 0.5
Z = O.RYKOV_ZROT
DELTA, W0_, W1_ = O.RYKOV_DELTA, O.RYKOV_OMEGA0, O.RYKOV_OMEGA1


def uniform_forest(D, n, lo, hi):
    nb = np.array([n] * D, np.int32)
    level, base, key = O.forest_base(D, nb)
    return O.forest_geom(D, nb, [lo] * D, [hi] * D, level, base, key)


def _state(D):
    rho = 1.1
    U = np.array([0.3, -0.2, 0.1])[:D]
    RTt, RTr = R * 1.5, R * 0.9
    qt = np.array([0.04, -0.03, 0.02])[:D]
    qr = np.array([-0.02, 0.05, 0.01])[:D]
    return rho, U, RTt, RTr, qt, qr


@pytest.mark.parametrize("D", [2, 3])
def test_rykov_equilibrium_moments(D):
    """On a fine uniform mesh: mass, momentum and total energy of W; the
    rotational energy (1 - 1/Z) rho R T_r + (1/Z) rho R T; the translational
    heat flux [(1 - 1/Z) + omega0/Z] q_t / 3; the rotational heat flux
    (1 - delta)[(1 - 1/Z) T_r/T_t + omega1/Z] q_r."""
    rho, U, RTt, RTr, qt, qr = _state(D)
    RT = (3 * RTt + 2 * RTr) / 5
    sig = math.sqrt(max(RTt, RT))
    n, span = (120, 11) if D == 2 else (44, 8)
    xi, w = uniform_forest(D, n, -span * sig, span * sig)
    g = O.gas(Kn=0.1, model="rykov")
    f = O.rykov_field(D, xi, g, rho, U, RTt, RTr, qt, qr)[None]
    Wc, qt_g, qr_g = O.moments_rykov(D, xi, w, f)
    tol = 1e-10 if D == 2 else 2e-7
    E = 0.5 * rho * U @ U + 1.5 * rho * RTt + rho * RTr
    assert Wc[0, 0] == pytest.approx(rho, rel=tol)
    assert np.allclose(Wc[0, 1:1 + D], rho * U, rtol=0, atol=tol * rho * sig)
    assert Wc[0, D + 1] == pytest.approx(E, rel=tol)
    assert Wc[0, D + 2] == pytest.approx((1 - 1 / Z) * rho * RTr + rho * RT / Z, rel=tol)
    lam_t = ((1 - 1 / Z) + W0_ / Z) / 3
    lam_r = (1 - DELTA) * ((1 - 1 / Z) * RTr / RTt + W1_ / Z)
    assert np.allclose(qt_g[0], lam_t * qt, rtol=0, atol=50 * tol * rho * sig ** 3)
    assert np.allclose(qr_g[0], lam_r * qr, rtol=0, atol=50 * tol * rho * sig ** 3)


def test_rykov_reduces_to_shakhov_without_rotational_exchange():
    """1/Z = 0: (g^G, g^H) is the Shakhov equilibrium at T_t with q_t and
    Pr = 2/3 (Eqs. 14-17), and g^R = R T_r (g^G + (1 - delta) c.q_r g_t / (p_t R T_t))."""
    D = 2
    rho, U, RTt, RTr, qt, qr = _state(D)
    xi, w = uniform_forest(D, 24, -4.0, 4.0)
    g = O.gas(Kn=0.1, model="rykov", Zrot=1e300)
    out = O.rykov_field(D, xi, g, rho, U, RTt, RTr, qt, qr)
    gG, gH = O.shakhov_field(D, xi, 2.0 / 3.0, rho, U, RTt, qt)
    assert np.allclose(out[0], gG, rtol=1e-14, atol=1e-16)
    assert np.allclose(out[1], gH, rtol=1e-14, atol=1e-16)
    gt = O.maxwell_init(D, xi, np.concatenate([[rho], U, [RTt / R]])[None])[0, 0]
    cqr = (xi - U) @ qr
    ref = RTr * (gG + (1 - DELTA) * cqr / (rho * RTt * RTt) * gt)
    assert np.allclose(out[2], ref, rtol=1e-13, atol=1e-16)


def _box(n, D=2):
    return wl.cartesian_mesh((n,) * D, (1.0,) * D, periodic=(True,) * D)


def test_uniform_gas_rotational_relaxation_closed_form():
    """Uniform gas at rest on a periodic box with T_r != T_t: no net transport,
    the total energy stays, and per step the rotational energy follows
    E_rot^{n+1} = (E_rot^n + a rho R T)/(1 + a), a = dt/(Z tau(T_t)) (Eq. S_rot
    taken implicitly, R28); the moments of f^{n+1} equal the new W."""
    m = _box(3)
    mh = O.MeshHandle(m)
    g = O.gas(Kn=0.05, model="rykov")
    sig = math.sqrt(R * 1.6)
    xi, w = uniform_forest(2, 48, -10 * sig, 10 * sig)
    Wp = np.tile([1.0, 0.0, 0.0, 1.6, 0.6], (m.Nc, 1))
    f = O.maxwell_init_rykov(2, xi, Wp)
    Wc = O.moments_rykov(2, xi, w, f)[0]
    dt = 0.4 * O.dt_unit(mh, xi)
    E0 = Wc[0, 3]
    for _ in range(4):
        rho = Wc[0, 0]
        RTr = Wc[0, 4] / rho
        RTt = (Wc[0, 3] - Wc[0, 4]) / (1.5 * rho)
        RT = (3 * RTt + 2 * RTr) / 5
        mu = g.mu_ref * (RTt / R) ** g.omega
        tau = mu / (rho * RTt)
        a = dt / (Z * tau)
        Er = (Wc[0, 4] + a * rho * RT) / (1 + a)
        f = O.step(mh, g, xi, w, dt, f, Wc)
        assert np.allclose(Wc[:, 4], Er, rtol=1e-12)
        assert np.allclose(Wc[:, 3], E0, rtol=1e-13)
        Wf = O.moments_rykov(2, xi, w, f)[0]
        assert np.allclose(Wf, Wc, rtol=1e-10, atol=1e-12)
    assert abs(Wc[0, 4] / Wc[0, 0] - RT) < abs(0.6 * R - RT)     # moved toward equilibrium


def test_conservation_periodic():
    w = wl.sweep_box((6, 6), base=(10, 10), max_refine=1)
    w.model = "rykov"
    r = O.Run(w)
    r.init_field(amp=1e-3)
    assert r.f.shape[1] == 3 and r.Wc.shape[1] == 5
    tot0 = (r.Wc * w.mesh.vol[:, None]).sum(0)
    dt = r.dt()
    for _ in range(3):
        r.step(dt)
    tot = (r.Wc * w.mesh.vol[:, None]).sum(0)
    assert np.allclose(tot[:4], tot0[:4], rtol=1e-14, atol=1e-14)


def test_free_transport_limit_carries_R_like_G():
    """tau -> infinity, first order: every array, R included, takes the
    first-order upwind update of free transport."""
    n = 4
    m = _box(n)
    mh = O.MeshHandle(m)
    g = O.gas(Kn=1e14, limiter=0, model="rykov")
    xi, w = uniform_forest(2, 2, -1.0, 1.0)
    rng = np.random.default_rng(4)
    Wp = np.column_stack([1 + 0.2 * rng.random(n * n), 0.1 * rng.standard_normal((n * n, 2)),
                          1 + 0.2 * rng.random(n * n), 0.8 + 0.2 * rng.random(n * n)])
    f = O.maxwell_init_rykov(2, xi, Wp) * (1 + 0.3 * rng.random((n * n, 3, 4)))
    Wc = O.moments_rykov(2, xi, w, f)[0]
    dt = 0.05
    fo = O.step(mh, g, xi, w, dt, f, Wc)
    F = f.reshape(n, n, 3, 4)
    exp = np.empty_like(F)
    dx = 1.0 / n
    for k, (ux, uy) in enumerate(xi):
        for a in range(3):
            u = F[:, :, a, k]
            Wn = np.roll(u, 1, axis=1); En = np.roll(u, -1, axis=1)
            Sn = np.roll(u, 1, axis=0); Nn = np.roll(u, -1, axis=0)
            exp[:, :, a, k] = u - dt / dx * (max(ux, 0) * (u - Wn) + min(ux, 0) * (En - u)
                                             + max(uy, 0) * (u - Sn) + min(uy, 0) * (Nn - u))
    assert np.allclose(fo.reshape(n, n, 3, 4), exp, rtol=1e-13, atol=1e-15)


def test_continuum_limit_is_equilibrated_rykov():
    """tau -> 0: the rotational energy is fully exchanged (T_r = T_t = T) and
    f^{n+1} is the Rykov equilibrium of the predicted W with the lagged heat
    fluxes of f^n."""
    n = 4
    m = _box(n)
    mh = O.MeshHandle(m)
    g = O.gas(Kn=1e-10, model="rykov")
    xi, w = uniform_forest(2, 12, -3.0, 3.0)
    W = wl.sweep_W(m)
    Wp = np.column_stack([W, 0.8 * W[:, 3]])
    f = O.maxwell_init_rykov(2, xi, Wp, amp=1e-2, seed=5)
    Wc, qt, qr = O.moments_rykov(2, xi, w, f)
    dt = 0.5 * O.dt_unit(mh, xi)
    fo = O.step(mh, g, xi, w, dt, f, Wc)
    for i in range(m.Nc):
        rho = Wc[i, 0]; U = Wc[i, 1:3] / rho
        RT = (Wc[i, 3] - 0.5 * rho * U @ U) / (2.5 * rho)
        assert Wc[i, 4] / rho == pytest.approx(RT, rel=1e-8)
        ref = O.rykov_field(2, xi, g, rho, U, RT, RT, qt[i], qr[i])
        assert np.allclose(fo[i], ref, rtol=0, atol=1e-7 * ref.max())


def test_criterion_energy_includes_rotation():
    """Same G and U: M2 scales with the inverse internal energy, which for the
    Rykov W includes rho E_rot (R30); M1 is unchanged."""
    D = 2
    xi, w = uniform_forest(D, 16, -4.0, 4.0)
    Wp = np.array([[1.0, 0.3, 0.0, 1.2, 1.2]])
    f_r = O.maxwell_init_rykov(D, xi, Wp)
    f_s = f_r[:, :2].copy()
    Wr = O.moments_rykov(D, xi, w, f_r)[0]
    Ws, _ = O.moments(D, xi, w, f_s)
    Mr = O.criterion(D, xi, w, f_r, Wr)
    Ms = O.criterion(D, xi, w, f_s, Ws)
    rho = Ws[0, 0]
    e_s = Ws[0, 3] - 0.5 * Ws[0, 1] ** 2 / rho
    e_r = Wr[0, 3] - 0.5 * Wr[0, 1] ** 2 / rho
    assert e_r == pytest.approx(e_s + Wr[0, 4], rel=1e-14)       # rho E adds int R
    assert e_r / e_s == pytest.approx(5.0 / 3.0, rel=1e-4)        # T_r = T_t: 5/2 over 3/2 (coarse mesh)
    m1 = w * f_s[0, 0] / rho
    m2s = 0.5 * w * f_s[0, 0] * ((xi - Ws[0, 1:3] / rho) ** 2).sum(1) / e_s
    assert np.allclose(Ms, np.maximum(m1, m2s), rtol=1e-14)
    assert np.allclose(Mr, np.maximum(m1, m2s * e_s / e_r), rtol=1e-13)


def test_correction_restores_rykov_moments():
    """Sec. 3.3 with the equilibrium set (g^eq(T_t), (3-D) R T_t g, R T_r g):
    after a remap the correction restores all five moments, the gap shrinking
    every pass."""
    D = 2
    xi, w = uniform_forest(D, 8, -4.0, 4.0)
    Wp = np.array([[1.0, 0.4, -0.2, 1.1, 0.7], [0.9, -0.1, 0.3, 0.9, 1.0]])
    f = O.maxwell_init_rykov(D, xi, Wp, amp=0.05, seed=2)
    W = O.moments_rykov(D, xi, w, f)[0]
    nb = np.array([8, 8], np.int32)
    level, base, key = O.forest_base(D, nb)
    M = np.zeros(len(level)); M[27] = M[36] = 10.0
    nl, nbb, nk, src, kind = O.adapt_tree(D, level, base, key, M, 1.0, 1.0, 1e-9, 3)
    xi2, w2 = O.forest_geom(D, nb, [-4.0] * D, [4.0] * D, nl, nbb, nk)
    f2 = O.remap(D, f, src, kind)
    gaps = []
    for it in (1, 2, 4, 8, 16):
        g2 = f2.copy()
        gaps.append(O.correct_rykov(D, xi2, w2, W, g2, iters=it))
    assert all(b < a for a, b in zip(gaps, gaps[1:]))
    assert gaps[-1] < 1e-13


# ---------------------------------------------------------------- implicit step (Eqs. SGS_w, SGS_wrot, SGS_phi)
def test_implicit_uniform_gas_rotational_relaxation_fixed_point():
    """Uniform gas at rest, T_r != T_t, periodic box: no net transport, so the
    converged macroscopic sweeps solve the backward-Euler rotational exchange
    E_rot^{n+1} = E_rot^n + dt (rho R T - E_rot^{n+1}) / (Z tau(T_t^{n+1}))
    of Eq. (SGS_wrot) with rho R T fixed by the total energy; mass, momentum
    and total energy stay."""
    m = _box(3)
    mh = O.MeshHandle(m)
    g = O.gas(Kn=0.05, model="rykov")
    sig = math.sqrt(R * 1.6)
    xi, w = uniform_forest(2, 40, -10 * sig, 10 * sig)
    Wp = np.tile([1.0, 0.0, 0.0, 1.6, 0.6], (m.Nc, 1))
    f = O.maxwell_init_rykov(2, xi, Wp)
    Wc = O.moments_rykov(2, xi, w, f)[0]
    W0 = Wc.copy()
    col, nc = O.colors(mh)
    dt = 2.0 * O.dt_unit(mh, xi)
    O.step_implicit(mh, g, xi, w, dt, f, Wc, col, nc, k_macro=60, k_micro=2)
    rho = W0[0, 0]
    RT = W0[0, 3] / (2.5 * rho)
    E = Wc[:, 4]
    RTt = (W0[0, 3] - E) / (1.5 * rho)
    tau = g.mu_ref * (RTt / R) ** g.omega / (rho * RTt)
    resid = E - W0[:, 4] - dt * (rho * RT - E) / (Z * tau)
    assert np.abs(resid).max() < 1e-12 * W0[0, 4]
    assert np.allclose(Wc[:, :4], W0[:, :4], rtol=1e-13, atol=1e-15)
    assert (E > W0[:, 4]).all() and (E < rho * RT).all()        # toward equilibrium, not past it


def test_implicit_rykov_sweeps_converge_independent_of_order_and_conserve():
    from test_oracle_pins import _other_coloring
    w = wl.sweep_box((6, 5), base=(10, 10), max_refine=1)
    w.model = "rykov"
    vol = w.mesh.vol[:, None]
    outs = []
    for col in (None, _other_coloring(w.mesh)):
        r = O.Run(w)
        Wp = np.column_stack([w.W_init, 0.8 * w.W_init[:, 3]])
        r.init_field(Wp, amp=1e-2, seed=8)
        dt = r.dt(1.5)
        tot0 = (r.Wc * vol).sum(0)
        r.step_implicit(dt, k_macro=300, k_micro=300, color=col)
        tot = (r.Wc * vol).sum(0)
        assert np.allclose(tot[:4], tot0[:4], rtol=1e-12, atol=1e-13)
        outs.append((r.f.copy(), r.Wc.copy()))
    assert np.abs(outs[0][0] - outs[1][0]).max() <= 1e-11 * np.abs(outs[0][0]).max()
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 1e-11 * np.abs(outs[0][1]).max()


def test_implicit_rykov_matches_explicit_to_first_order_in_dt():
    w = wl.sweep_box((6, 5), base=(10, 10), max_refine=1)
    w.model = "rykov"
    ratio = []
    for cfl in (0.4, 0.2):
        re, ri = O.Run(w), O.Run(w)
        Wp = np.column_stack([w.W_init, 0.8 * w.W_init[:, 3]])
        for r in (re, ri):
            r.init_field(Wp, amp=1e-2, seed=9)
        f0 = re.f.copy()
        dt = re.dt(cfl)
        re.step(dt)
        ri.step_implicit(dt, k_macro=200, k_micro=200)
        ratio.append(np.abs(ri.f - re.f).max() / np.abs(re.f - f0).max())
    assert 0.35 < ratio[1] / ratio[0] < 0.65, ratio
