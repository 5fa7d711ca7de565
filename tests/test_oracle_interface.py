"""Pin of the oracle's interface flux (Eq. equ28 with reading R4) in the
continuum limit, against the Euler flux written out here.

When the collision time is far below the time step, the interface
distribution tau/(tau+h) phi_bar + h/(tau+h) g(W_ij, q_ij) is the Maxwellian of
the interface state W_ij (the moments of the foot distribution phi_bar, Eq.
w_interface), whose flux moments are the Euler flux of W_ij: mass flux rho u,
momentum flux rho u U + p e_x, energy flux (rho E + p) u with p = rho R T and
rho E = rho |U|^2 / 2 + (3/2) rho R T (the 2D reduced distributions carry the
third translational degree in H).  Two cells side by side, first-order
reconstruction (so phi_bar is the upwind cell's f), far-field faces outside:
the interior face's flux is read back from the oracle's conservative update of
cell 0 and compared with the Euler flux of W_ij summed here from the two
cells' f.  A swapped blend (the free-molecular flux of phi_bar), W_ij from one
cell only, or a wrong energy-flux weight fails it."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl

R = 0.5


def maxwellian(xi, rho, U, T):
    D = xi.shape[1]
    c2 = ((xi - np.asarray(U, float)[None, :D]) ** 2).sum(1)
    return rho / (2.0 * math.pi * R * T) ** (D / 2.0) * np.exp(-c2 / (2.0 * R * T))


def moments(xi, w, G, H):
    """rho, rho U (D), rho E of reduced distributions (plain sums; H = 0 in 3D)."""
    x2 = (xi ** 2).sum(1)
    return np.array([(w * G).sum(), *[(w * xi[:, d] * G).sum() for d in range(xi.shape[1])],
                     0.5 * (w * (x2 * G + H)).sum()])


def flux(xi, w, G, H, n):
    """Discrete flux moments sum w (xi . n) psi phi."""
    sn = xi @ n
    x2 = (xi ** 2).sum(1)
    return np.array([(w * sn * G).sum(), *[(w * sn * xi[:, d] * G).sum() for d in range(xi.shape[1])],
                     0.5 * (w * sn * (x2 * G + H)).sum()])


def euler_flux_x(W):
    """Euler flux through a face of normal e_x: rho u, rho u U + p e_x, (rho E + p) u."""
    D = len(W) - 2
    rho, m, E = W[0], np.asarray(W[1:1 + D]), W[D + 1]
    U = m / rho
    p = (E - 0.5 * rho * U @ U) / 1.5                     # rho R T from rho E = rho|U|^2/2 + 3/2 rho R T
    mom = m * U[0]
    mom[0] += p
    return np.array([m[0], *mom, (E + p) * U[0]])


def _interior_face_flux(Kn, D=2):
    """The interior face's flux read back from the oracle's update of cell 0,
    the Euler flux of the interface state and the free-molecular flux of the
    foot distribution, both summed here."""
    st = [(1.0, (0.3, 0.1, -0.05), 1.0), (0.6, (-0.2, 0.05, 0.1), 1.4)]
    st = [(r, U[:D], T) for r, U, T in st]
    far = [wl._bc_row(wl.BC_FARFIELD, rho=r, U=(*U, 0.0)[:3], T=T) for r, U, T in st]
    m = wl.cartesian_mesh((2,) + (1,) * (D - 1), (2.0,) + (1.0,) * (D - 1),
                          bcs=[(far[0], far[1])] + [((), ())] * (D - 1), periodic=(False,) + (True,) * (D - 1))
    assert list(m.faceL[:3]) == [0, 0, 1] and list(m.faceR[:3]) == [-1, 1, -2]
    mh = O.MeshHandle(m)
    g = O.gas(Kn=Kn, limiter=0)
    n = 48 if D == 2 else 24
    nb = np.array([n] * D, np.int32)
    level, base, key = O.forest_base(D, nb)
    xi, w = O.forest_geom(D, nb, (-7.0,) * D, (7.0,) * D, level, base, key)
    nA = O.n_arrays(D)
    f = np.zeros((2, nA, len(w)))
    for i, (r, U, T) in enumerate(st):
        f[i, 0] = maxwellian(xi, r, U, T)
        if D == 2:
            f[i, 1] = R * T * f[i, 0]
    Hof = (lambda a: a[1]) if D == 2 else (lambda a: np.zeros_like(a[0]))
    W0 = np.stack([moments(xi, w, f[i, 0], Hof(f[i])) for i in range(2)])
    Wc = W0.copy()
    dt = 0.5 * O.dt_unit(mh, xi)
    O.step(mh, g, xi, w, dt, f, Wc)                         # Wc <- W~ = W - dt/|V| sum A F
    # cell 0: W~ = W - dt (F_left + F_int), unit areas and volume
    x = xi[:, 0]
    inc = x > 0.0                                           # incoming at the left far-field face (normal -x)
    Mf = maxwellian(xi, *st[0])
    ex = np.zeros(D)
    ex[0] = 1.0
    HL = np.where(inc, R * st[0][2] * Mf, f[0, 1]) if D == 2 else np.zeros_like(Mf)
    F_left = flux(xi, w, np.where(inc, Mf, f[0, 0]), HL, -ex)
    F_int = (W0[0] - Wc[0]) / dt - F_left
    # the foot distribution (upwind cell's f) and the interface state, its moments
    up = x >= 0.0
    Gb = np.where(up, f[0, 0], f[1, 0])
    Hb = np.where(up, f[0, 1], f[1, 1]) if D == 2 else np.zeros_like(Gb)
    FE = euler_flux_x(moments(xi, w, Gb, Hb))
    Fk = flux(xi, w, Gb, Hb, ex)
    return F_int, FE, Fk


@pytest.mark.parametrize("D", [2, 3])
def test_interface_flux_continuum_limit_is_the_euler_flux_of_the_interface_state(D):
    F_int, FE, Fk = _interior_face_flux(1e-10, D)
    scale = np.abs(FE).max()
    assert np.all(np.abs(F_int - FE) <= 1e-6 * scale), (F_int, FE)
    assert np.abs(Fk - FE).max() > 1e-2 * scale          # the two limits differ by far more


@pytest.mark.parametrize("D", [2, 3])
def test_interface_flux_free_molecular_limit_is_the_flux_of_the_foot_distribution(D):
    """tau >> h: the interface distribution is phi_bar itself."""
    F_int, FE, Fk = _interior_face_flux(1e14, D)
    assert np.all(np.abs(F_int - Fk) <= 1e-12 * np.abs(Fk).max()), (F_int, Fk)


# ---- the diatomic gas (Rykov model; reading R27 of its interface state)

def rk_moments(xi, w, G, H, Rr):
    """rho, rho u, rho v, rho E (total: translational and rotational), rho E_rot."""
    x2 = (xi ** 2).sum(1)
    return np.array([(w * G).sum(), (w * xi[:, 0] * G).sum(), (w * xi[:, 1] * G).sum(),
                     0.5 * (w * (x2 * G + H)).sum() + (w * Rr).sum(), (w * Rr).sum()])


def rk_flux(xi, w, G, H, Rr, n):
    sn = xi @ n
    x2 = (xi ** 2).sum(1)
    return np.array([(w * sn * G).sum(), (w * sn * xi[:, 0] * G).sum(), (w * sn * xi[:, 1] * G).sum(),
                     (w * sn * (0.5 * (x2 * G + H) + Rr)).sum(), (w * sn * Rr).sum()])


def rk_euler_flux_x(W):
    """Euler flux of a diatomic gas in rotational equilibrium: rho E = rho |U|^2/2
    + (5/2) rho R T, p = rho R T; the rotational energy rho R T moves with u."""
    rho, mu, mv, E, _ = W
    u, v = mu / rho, mv / rho
    p = (E - 0.5 * rho * (u * u + v * v)) / 2.5
    return np.array([mu, mu * u + p, mv * u, (E + p) * u, p * u])


def _interior_face_flux_rykov(Kn):
    """As _interior_face_flux for the diatomic gas; each cell's f is G, H, R of
    a Maxwellian at T_t with a rotational temperature T_r = 0.7 T_t."""
    st = [(1.0, (0.3, 0.1), 1.0), (0.6, (-0.2, 0.05), 1.4)]
    far = [wl._bc_row(wl.BC_FARFIELD, rho=r, U=(*U, 0.0), T=T) for r, U, T in st]
    m = wl.cartesian_mesh((2, 1), (2.0, 1.0), bcs=[(far[0], far[1]), ((), ())], periodic=(False, True))
    mh = O.MeshHandle(m)
    g = O.gas(Kn=Kn, limiter=0, model="rykov")
    nb = np.array([48, 48], np.int32)
    level, base, key = O.forest_base(2, nb)
    xi, w = O.forest_geom(2, nb, (-7.0, -7.0), (7.0, 7.0), level, base, key)
    f = np.zeros((2, 3, len(w)))
    for i, (r, U, T) in enumerate(st):
        f[i, 0] = maxwellian(xi, r, U, T)
        f[i, 1] = R * T * f[i, 0]
        f[i, 2] = R * 0.7 * T * f[i, 0]
    W0 = np.stack([rk_moments(xi, w, *f[i]) for i in range(2)])
    Wc = W0.copy()
    dt = 0.5 * O.dt_unit(mh, xi)
    O.step(mh, g, xi, w, dt, f, Wc)
    x = xi[:, 0]
    inc = x > 0.0
    Mf = maxwellian(xi, *st[0])
    Tf = st[0][2]
    F_left = rk_flux(xi, w, np.where(inc, Mf, f[0, 0]), np.where(inc, R * Tf * Mf, f[0, 1]),
                     np.where(inc, R * Tf * Mf, f[0, 2]), np.array([-1.0, 0.0]))
    F_int = (W0[0] - Wc[0]) / dt - F_left
    up = x >= 0.0
    feet = [np.where(up, f[0, a], f[1, a]) for a in range(3)]
    FE = rk_euler_flux_x(rk_moments(xi, w, *feet))
    Fk = rk_flux(xi, w, *feet, np.array([1.0, 0.0]))
    return F_int, FE, Fk


def test_rykov_interface_flux_continuum_limit_is_the_diatomic_euler_flux():
    """tau << h: the interface relaxes the rotational energy fully and carries
    the Euler flux of a diatomic gas in equilibrium (mass, momentum and total
    energy: the cell's own rotational source then relaxes E_rot as well, so
    its flux cannot be read back)."""
    F_int, FE, Fk = _interior_face_flux_rykov(1e-10)
    scale = np.abs(FE).max()
    assert np.all(np.abs(F_int[:4] - FE[:4]) <= 1e-6 * scale), (F_int, FE)
    assert np.abs(Fk[:4] - FE[:4]).max() > 1e-2 * scale


def test_rykov_interface_flux_free_molecular_limit_is_the_flux_of_the_feet():
    """tau >> h: no relaxation anywhere; every component, E_rot included, is
    the flux of the feet."""
    F_int, FE, Fk = _interior_face_flux_rykov(1e14)
    assert np.all(np.abs(F_int - Fk) <= 1e-12 * np.abs(Fk).max()), (F_int, Fk)
