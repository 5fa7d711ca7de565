"""Pins of the oracle's boundary faces and of its limiter.

Boundary faces (reading R8: diffuse isothermal wall with zero net mass flux,
far field imposing the free-stream Maxwellian on incoming nodes) are pinned by
what diffuse reflection means, not by the oracle's own formula:

* a single cell between two boundary faces, with collisions switched off
  (tau -> infinity) and first-order reconstruction, so that the step is
  f^{n+1} = f - dt/|V| sum_faces A (xi . n) phi_face.  Solving that for the
  incoming phi of each boundary face recovers what the boundary emitted, node
  by node.  It must be a Maxwellian at the wall's velocity and temperature
  (R = 1/2, T in units of T_inf) scaled to zero net mass flux, with
  H = (3 - D) R T_w G; a far-field face must emit the free-stream Maxwellian
  itself, density included;
* gas in equilibrium with its walls (a closed box at rest at the wall
  temperature, a channel between walls sliding at the gas velocity) is left
  unchanged by a collisional second-order step.

The diatomic gas (Rykov model, reading R29) is pinned by the same solve: the
incoming R distribution of a boundary face is the rotational equilibrium at
the boundary temperature, R T_b times the emitted G.

The limiter (Sec. 2.3.3, reading R6) is pinned by Venkatakrishnan's function
in its ratio form phi(y) = (y^2 + 2y)/(y^2 + y + 2), y = d+/d-, by its limits,
and by a limited gradient worked out by hand on a ring of three cells.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl

R = 0.5


def maxwellian(xi, rho, U, T):
    """rho / (2 pi R T)^(D/2) exp(-|xi - U|^2 / (2 R T)), written out here."""
    D = xi.shape[1]
    c2 = ((xi - np.asarray(U, float)[None, :D]) ** 2).sum(1)
    return rho / (2.0 * math.pi * R * T) ** (D / 2.0) * np.exp(-c2 / (2.0 * R * T))


def _forest(nb, vlo, vhi):
    D = len(nb)
    nb = np.array(nb, np.int32)
    level, base, key = O.forest_base(D, nb)
    return O.forest_geom(D, nb, vlo, vhi, level, base, key)


def _one_cell_step(D, lo_bc, hi_bc, nb, vlo, vhi, seed=11):
    """One collisionless first-order step of a unit cell whose x faces are the
    given boundaries (periodic in the other directions).  Returns xi, w, f,
    f^{n+1}, dt."""
    bcs = [(lo_bc, hi_bc)] + [((), ())] * (D - 1)
    m = wl.cartesian_mesh((1,) * D, (1.0,) * D, bcs=bcs, periodic=(False,) + (True,) * (D - 1))
    mh = O.MeshHandle(m)
    g = O.gas(Kn=1e14, limiter=0)
    xi, w = _forest(nb, vlo, vhi)
    assert np.all(np.abs(xi[:, 0]) > 1e-3)            # no node tangential to the boundary faces
    rng = np.random.default_rng(seed)
    nA = O.n_arrays(D)
    f = maxwellian(xi, 1.0, [0.2, -0.1, 0.05], 1.1)[None, None, :] * rng.uniform(0.5, 1.5, size=(1, nA, len(w)))
    Wc, _ = O.moments(D, xi, w, f)
    dt = 0.2 * O.dt_unit(mh, xi)
    fo = O.step(mh, g, xi, w, dt, f, Wc)
    return xi, w, f[0], fo[0], dt


def _emitted(xi, f, fo, dt, side):
    """Incoming phi of the high (side=+1) or low (side=-1) x face on its
    incoming nodes, from f^{n+1} = f - dt (xi_x phi_hi - xi_x phi_lo) (unit
    cell, unit faces); the other face's outgoing phi is f itself."""
    x = xi[:, 0]
    if side > 0:
        sel = x < 0.0                         # incoming at the high face, outgoing at the low face
        phi = f[:, sel] - (fo[:, sel] - f[:, sel]) / (dt * x[sel])
    else:
        sel = x > 0.0
        phi = f[:, sel] + (fo[:, sel] - f[:, sel]) / (dt * x[sel])
    return sel, phi


@pytest.mark.parametrize("D", [2, 3])
def test_wall_emits_maxwellian_at_wall_state_with_zero_net_mass_flux(D):
    """R8 diffuse wall: what the wall sends into the cell is rho_w M(U_w, T_w)
    node by node (the shape fixed by the wall's own velocity and temperature
    with R = 1/2, H = (3 - D) R T_w G), and rho_w makes the net mass flux
    through the wall zero.  Catches R T_w -> T_w, a dropped or sign-flipped
    wall velocity, a wrong H factor and a wrong density balance."""
    Uw = (0.0, 0.3, -0.2)[:D]
    Tw = 1.4
    wall = wl._bc_row(wl.BC_WALL, T=Tw, U=Uw)
    far = wl._bc_row(wl.BC_FARFIELD, rho=0.7, U=(0.4, -0.2, 0.1)[:D], T=1.6)
    nb = (6, 5, 4)[:D]
    vlo = (-2.4, -2.0, -2.1)[:D]
    vhi = (2.6, 2.2, 1.9)[:D]
    xi, w, f, fo, dt = _one_cell_step(D, far, wall, nb, vlo, vhi)
    sel, phi = _emitted(xi, f, fo, dt, +1)
    M = maxwellian(xi[sel], 1.0, Uw, Tw)
    rho_w = phi[0] / M
    # one density scales the wall Maxwellian on every incoming node
    assert np.ptp(rho_w) <= 1e-10 * rho_w.mean(), rho_w
    # zero net mass flux: incoming = outgoing through the wall
    x = xi[:, 0]
    out = (w[~sel] * x[~sel] * f[0, ~sel]).sum()
    inc = (w[sel] * (-x[sel]) * phi[0]).sum()
    assert inc == pytest.approx(out, rel=1e-11)
    if D == 2:
        assert np.allclose(phi[1], (3 - D) * R * Tw * phi[0], rtol=1e-10, atol=0)


@pytest.mark.parametrize("D", [2, 3])
def test_far_field_emits_free_stream_maxwellian(D):
    """R8 far field: incoming nodes get g^eq(W_inf) itself: its density,
    velocity and temperature, with H = (3 - D) R T_inf G."""
    rho, U, T = 0.7, (0.4, -0.2, 0.1)[:D], 1.6
    far = wl._bc_row(wl.BC_FARFIELD, rho=rho, U=U, T=T)
    wall = wl._bc_row(wl.BC_WALL, T=0.9)
    nb = (6, 5, 4)[:D]
    vlo = (-2.4, -2.0, -2.1)[:D]
    vhi = (2.6, 2.2, 1.9)[:D]
    xi, w, f, fo, dt = _one_cell_step(D, far, wall, nb, vlo, vhi, seed=12)
    sel, phi = _emitted(xi, f, fo, dt, -1)
    M = maxwellian(xi[sel], rho, U, T)
    assert np.allclose(phi[0], M, rtol=1e-10, atol=0)
    if D == 2:
        assert np.allclose(phi[1], R * T * M, rtol=1e-10, atol=0)


def _one_cell_step_rykov(D, lo_bc, hi_bc, nb, vlo, vhi, seed=11):
    """_one_cell_step for the diatomic gas: f holds G, [H,] R (the last array
    the rotational energy distribution), each a perturbed Maxwellian."""
    bcs = [(lo_bc, hi_bc)] + [((), ())] * (D - 1)
    m = wl.cartesian_mesh((1,) * D, (1.0,) * D, bcs=bcs, periodic=(False,) + (True,) * (D - 1))
    mh = O.MeshHandle(m)
    g = O.gas(Kn=1e14, limiter=0, model="rykov")
    xi, w = _forest(nb, vlo, vhi)
    assert np.all(np.abs(xi[:, 0]) > 1e-3)
    rng = np.random.default_rng(seed)
    nA = 3 if D == 2 else 2
    f = maxwellian(xi, 1.0, [0.2, -0.1, 0.05], 1.1)[None, None, :] * rng.uniform(0.5, 1.5, size=(1, nA, len(w)))
    Wc = O.moments_rykov(D, xi, w, f)[0]
    dt = 0.2 * O.dt_unit(mh, xi)
    fo = O.step(mh, g, xi, w, dt, f, Wc)
    return xi, w, f[0], fo[0], dt


@pytest.mark.parametrize("D", [2, 3])
def test_rykov_wall_emits_rotational_equilibrium_at_wall_temperature(D):
    """R29: a diffuse wall in the diatomic gas sends rho_w M(U_w, T_w) in G,
    (3 - D) R T_w times it in H and R T_w times it in R (rotational
    equilibrium at the wall temperature), with zero net mass flux.  Catches
    R T_w -> T_w in R, R at the gas's own rotational temperature, and R left
    as the cell's outgoing values."""
    Uw = (0.0, 0.3, -0.2)[:D]
    Tw = 1.4
    wall = wl._bc_row(wl.BC_WALL, T=Tw, U=Uw)
    far = wl._bc_row(wl.BC_FARFIELD, rho=0.7, U=(0.4, -0.2, 0.1)[:D], T=1.6)
    nb = (6, 5, 4)[:D]
    vlo = (-2.4, -2.0, -2.1)[:D]
    vhi = (2.6, 2.2, 1.9)[:D]
    xi, w, f, fo, dt = _one_cell_step_rykov(D, far, wall, nb, vlo, vhi)
    sel, phi = _emitted(xi, f, fo, dt, +1)
    M = maxwellian(xi[sel], 1.0, Uw, Tw)
    rho_w = phi[0] / M
    assert np.ptp(rho_w) <= 1e-10 * rho_w.mean(), rho_w
    x = xi[:, 0]
    out = (w[~sel] * x[~sel] * f[0, ~sel]).sum()
    inc = (w[sel] * (-x[sel]) * phi[0]).sum()
    assert inc == pytest.approx(out, rel=1e-11)
    assert np.allclose(phi[-1], R * Tw * phi[0], rtol=1e-10, atol=0)
    if D == 2:
        assert np.allclose(phi[1], (3 - D) * R * Tw * phi[0], rtol=1e-10, atol=0)


@pytest.mark.parametrize("D", [2, 3])
def test_rykov_far_field_emits_free_stream_equilibrium(D):
    """R29 far field in the diatomic gas: G = g^eq(W_inf) with its density,
    velocity and temperature, R = R T_inf G (rotational temperature equal to
    the free stream's), H = (3 - D) R T_inf G."""
    rho, U, T = 0.7, (0.4, -0.2, 0.1)[:D], 1.6
    far = wl._bc_row(wl.BC_FARFIELD, rho=rho, U=U, T=T)
    wall = wl._bc_row(wl.BC_WALL, T=0.9)
    nb = (6, 5, 4)[:D]
    vlo = (-2.4, -2.0, -2.1)[:D]
    vhi = (2.6, 2.2, 1.9)[:D]
    xi, w, f, fo, dt = _one_cell_step_rykov(D, far, wall, nb, vlo, vhi, seed=12)
    sel, phi = _emitted(xi, f, fo, dt, -1)
    M = maxwellian(xi[sel], rho, U, T)
    assert np.allclose(phi[0], M, rtol=1e-10, atol=0)
    assert np.allclose(phi[-1], R * T * M, rtol=1e-10, atol=0)
    if D == 2:
        assert np.allclose(phi[1], R * T * M, rtol=1e-10, atol=0)


def _equilibrium_run(mesh, xi, w, rho, U, T, Kn=0.05):
    mh = O.MeshHandle(mesh)
    g = O.gas(Kn=Kn, limiter=1)
    D = mesh.D
    Wp = np.tile([rho, *U[:D], T], (mesh.Nc, 1))
    f = O.maxwell_init(D, xi, Wp)
    Wc, _ = O.moments(D, xi, w, f)
    dt = 0.8 * O.dt_unit(mh, xi)
    fo = O.step(mh, g, xi, w, dt, f, Wc)
    return f, fo


def test_gas_at_rest_in_equilibrium_with_walls_stays_put():
    """A closed box, every wall at T_w, holding gas at rest in equilibrium at
    T_w (a discrete Maxwellian on a velocity mesh symmetric about 0): one
    collisional step leaves f unchanged to round-off.  Catches a wall that
    emits at the wrong temperature (R T_w -> T_w) or with the wrong H."""
    Tw = 1.3
    wall = wl._bc_row(wl.BC_WALL, T=Tw)
    m = wl.cartesian_mesh((4, 4), (1.0, 1.0), bcs=[(wall, wall), (wall, wall)])
    s = 8.0 * math.sqrt(R * Tw)
    xi, w = _forest((32, 32), (-s, -s), (s, s))
    f, fo = _equilibrium_run(m, xi, w, 1.0, (0.0, 0.0), Tw)
    assert np.abs(fo - f).max() <= 1e-13 * f.max()


def test_gas_sliding_with_its_walls_stays_put():
    """A channel (periodic in x) between two walls that slide at U_w along x,
    at T_w, holding gas that moves with them in equilibrium at (U_w, T_w):
    one collisional step leaves f unchanged to round-off.  Catches a dropped,
    sign-flipped or transposed wall velocity and a wrong wall temperature."""
    Tw, Uw = 1.3, (0.4, 0.0)
    wall = wl._bc_row(wl.BC_WALL, T=Tw, U=Uw)
    m = wl.cartesian_mesh((3, 4), (1.0, 1.0), bcs=[((), ()), (wall, wall)], periodic=(True, False))
    s = 8.0 * math.sqrt(R * Tw)
    xi, w = _forest((32, 32), (Uw[0] - s, -s), (Uw[0] + s, s))
    f, fo = _equilibrium_run(m, xi, w, 1.0, Uw, Tw)
    assert np.abs(fo - f).max() <= 1e-13 * f.max()


def test_uniform_stream_between_far_fields_stays_uniform():
    """A box with far-field faces on every side, holding the free stream
    itself: one step leaves f unchanged up to the velocity quadrature of the
    Maxwellian's heat flux.  Catches a far field that emits the wrong density,
    velocity or temperature."""
    rho, U, T = 0.8, (0.6, -0.3), 1.2
    far = wl._bc_row(wl.BC_FARFIELD, rho=rho, U=U, T=T)
    m = wl.cartesian_mesh((4, 4), (1.0, 1.0), bcs=[(far, far), (far, far)])
    s = 8.0 * math.sqrt(R * T)
    xi, w = _forest((32, 32), (U[0] - s, U[1] - s), (U[0] + s, U[1] + s))
    f, fo = _equilibrium_run(m, xi, w, rho, U, T)
    assert np.abs(fo - f).max() <= 1e-13 * f.max()


# ---------------------------------------------------------------- limiter
def _venkat_ratio_form(dp, dm):
    """Venkatakrishnan's function with epsilon = 0 in terms of y = d+/d-,
    capped at 1: (y^2 + 2y) / (y^2 + y + 2)."""
    y = dp / dm
    return min(1.0, (y * y + 2.0 * y) / (y * y + y + 2.0))


@pytest.mark.parametrize("dp,dm,exact", [
    (1.0, 1.0, 3.0 / 4.0),          # y = 1
    (0.5, 1.0, 5.0 / 11.0),         # y = 1/2
    (4.0, 3.0, 20.0 / 23.0),        # y = 4/3
    (2.0, 1.0, 1.0),                # y = 2: the function reaches 1 exactly
    (-1.0, -0.75, 20.0 / 23.0),     # the negative side (d- < 0 uses the smallest difference)
    (0.0, 0.3, 0.0),                # the cell is a local extremum: first order
])
def test_venkatakrishnan_function_values(dp, dm, exact):
    """Closed-form values of Venkatakrishnan's function at epsilon = 0.
    Catches swapped arguments (y -> 1/y changes every y != 1 row), a dropped
    factor 2, a minmod or Barth-Jespersen limiter in its place."""
    assert O.venkat(dp, dm, 0.0) == pytest.approx(exact, rel=1e-15, abs=1e-300)
    assert O.venkat(dp, dm, 0.0) == pytest.approx(_venkat_ratio_form(dp, dm), rel=1e-15, abs=1e-300)


def test_venkatakrishnan_function_limits():
    """Limits: large y -> 1 (capped); y -> 0+ -> 0; monotone in y on [0, 2];
    differences small against epsilon leave the gradient unlimited (-> 1),
    differences large against it give the epsilon = 0 value.  A worked value
    with epsilon: d+ = 1, d- = 2, eps^2 = 1 gives 6/12."""
    assert O.venkat(100.0, 1.0, 0.0) == 1.0
    assert O.venkat(1e-9, 1.0, 0.0) == pytest.approx(1e-9, rel=1e-6)
    ys = np.linspace(0.0, 2.0, 41)
    vals = [O.venkat(y, 1.0, 0.0) for y in ys]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    assert O.venkat(1e-6, 1e-6, 1e-6) == pytest.approx(1.0, abs=1e-5)
    assert O.venkat(1e-6, 1e-6, 1e-6) < 1.0
    assert O.venkat(1.0, 1.0, 1e-14) == pytest.approx(0.75, abs=1e-13)
    assert O.venkat(1.0, 2.0, 1.0) == pytest.approx(0.5, rel=1e-15)


def test_limited_gradient_three_cell_ring_by_hand():
    """LSQ gradient with weights 1/|d|^2 and the Venkatakrishnan factor on a
    ring of three cells of width h = 1/3 (periodic in x, one cell in y), with
    phi = (0, 1, 3):
      middle cell: central difference (3 - 0)/(2h) = 4.5; face changes +-0.75;
        largest / smallest neighbour differences 2 and -1; the + side gives
        y = 8/3 (capped at 1), the - side y = 4/3, so L = 20/23 at epsilon = 0;
        with epsilon^2 = (K dx)^3 phi_C^2, K = 0.3, dx = |V|^(1/2) = (1/3)^(1/2),
        phi_C = 1: L = (2.5 + eps^2) / (2.875 + eps^2);
      end cells: local minimum and maximum, L = 0.
    The H array holds 2 phi: the same factor (epsilon scales with the value).
    Catches a wrong LSQ weight, a limiter over the wrong neighbour difference
    or face offset, and a different epsilon (K, power, length or value scale)."""
    m = wl.cartesian_mesh((3, 1), (1.0, 1.0), periodic=(True, True))
    mh = O.MeshHandle(m)
    phi = np.array([0.0, 1.0, 3.0])
    f = np.stack([phi, 2.0 * phi], axis=1)[:, :, None].copy()     # G and H = 2 G, one velocity node
    g0 = O.gas(Kn=1.0, limiter=1, lim_K=1e-9)
    grad, lim = O.limited_gradients(mh, g0, f)
    assert grad[1, 0, 0] == pytest.approx([4.5, 0.0], abs=1e-14)
    assert grad[1, 1, 0] == pytest.approx([9.0, 0.0], abs=1e-14)
    assert grad[0, 0, 0, 0] == pytest.approx(-3.0, rel=1e-14)
    assert grad[2, 0, 0, 0] == pytest.approx(-1.5, rel=1e-14)
    assert lim[1, 0, 0] == pytest.approx(20.0 / 23.0, rel=1e-12)
    assert lim[1, 1, 0] == pytest.approx(20.0 / 23.0, rel=1e-12)       # scale-free at epsilon = 0
    assert lim[0, 0, 0] == pytest.approx(0.0, abs=1e-20) and lim[2, 0, 0] == pytest.approx(0.0, abs=1e-20)

    g = O.gas(Kn=1.0, limiter=1)                                       # the paper's reading: K = 0.3
    _, lim = O.limited_gradients(mh, g, f)
    e2 = (0.3 * math.sqrt(1.0 / 3.0)) ** 3
    assert lim[1, 0, 0] == pytest.approx((2.5 + e2) / (2.875 + e2), rel=1e-14)
    # H = 2 G: differences of 4 and -2, face changes +-1.5, phi_C = 2: epsilon^2 4 e2
    assert lim[1, 1, 0] == pytest.approx((10.0 + 4.0 * e2) / (11.5 + 4.0 * e2), rel=1e-14)
    assert lim[1, 1, 0] == pytest.approx(lim[1, 0, 0], rel=1e-14)

    g2 = O.gas(Kn=1.0, limiter=2)                                      # unlimited
    _, lim = O.limited_gradients(mh, g2, f)
    assert np.all(lim == 1.0)


def test_limiter_factor_is_scale_free():
    """Reading R6: epsilon^2 = (K dx)^3 phi_C^2 scales with the limited value,
    so the limiter factor of c f equals that of f at every cell and node, for
    c over twelve orders of magnitude (f spans as many over the velocity
    nodes); with the unscaled epsilon^2 = (K dx)^3 the factor of a small
    multiple of f would be 1 (no limiting in the tails of the distribution)."""
    m = wl.cartesian_mesh((6, 5), (1.0, 1.0), periodic=(True, True))
    mh = O.MeshHandle(m)
    rng = np.random.default_rng(17)
    f = rng.uniform(0.2, 1.0, size=(m.Nc, 2, 7))
    g = O.gas(Kn=1.0, limiter=1)
    _, lim = O.limited_gradients(mh, g, f)
    assert (lim < 1.0).mean() > 0.3                     # the limiter acts on this field
    for c in (1e-9, 1e-3, 1e3):
        _, lc = O.limited_gradients(mh, g, c * f)
        assert np.allclose(lc, lim, rtol=1e-12, atol=0), c
