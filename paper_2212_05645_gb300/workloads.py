"""Seeded, synthetic inputs shared by the CUDA path and its CPU oracle.

This module holds input synthesis only: physical meshes (geometry), the flow
conditions of each workload, the velocity-forest bounds and a counter-based
normal generator.  It contains none of the method's arithmetic (no
equilibrium, moment, flux, criterion or adaptation formula): both the oracle
and the CUDA library receive these arrays and compute everything else on
their own.

Mesh format (face list, used by both sides)
-------------------------------------------
* ``D``        physical (= velocity) dimension, 2 or 3
* ``Nc, Nf``   number of cells / faces
* ``faceL``    int32[Nf]  left cell of each face (always an interior cell)
* ``faceR``    int32[Nf]  right cell, or ``-1 - b`` for boundary condition ``b``
* ``An``       float64[Nf, D] face area times unit normal, pointing L -> R
               (outward from the domain for boundary faces)
* ``rL, rR``   float64[Nf, D] face centre minus cell centre of L / R.  For a
               periodic face ``rR`` uses the periodic image of R.  Zero for
               boundary faces.
* ``vol``      float64[Nc] cell volume (area in 2D)
* ``xc``       float64[Nc, D] cell centre (diagnostics only)
* ``bc``       float64[nbc, 6]: type (1 = isothermal diffuse wall,
               2 = far field), rho, U0, U1, U2, T
* ``dims``     structured sizes (fastest index first)

Units follow the paper's non-dimensionalisation (Table of dimensionless
quantities, Sec. 4.5): rho_inf = T_inf = 1, length unit L_ref and velocity
unit sqrt(2 R T_inf), so the gas constant is R = 1/2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

R_GAS = 0.5          # velocity unit sqrt(2 R T_inf) with T_inf = 1
GAMMA_MONO = 5.0 / 3.0

BC_WALL = 1
BC_FARFIELD = 2

# --------------------------------------------------------------------------
# counter-based normal numbers (SplitMix64, Steele, Lea & Flood 2014;
# Box-Muller 1958).  The CUDA library and the C oracle implement the same
# published definition independently; this copy is used by tests.
# --------------------------------------------------------------------------
_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_SM_M1 = np.uint64(0xBF58476D1CE4E5B9)
_SM_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to state ``x + gamma``."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + _SM_GAMMA).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _SM_M1
        z = (z ^ (z >> np.uint64(27))) * _SM_M2
        return z ^ (z >> np.uint64(31))


def normal_field(seed: int, n_cells: int, n_nodes: int) -> np.ndarray:
    """Standard normals z[i, k] for cell i, node k.

    key = (i << 32) | k;  u1 = splitmix64(seed ^ splitmix64(2 key)),
    u2 = splitmix64(seed ^ splitmix64(2 key + 1));  U1 = ((u1 >> 11) + 1) 2^-53,
    U2 = (u2 >> 11) 2^-53;  z = sqrt(-2 ln U1) cos(2 pi U2).
    """
    i = np.arange(n_cells, dtype=np.uint64)[:, None]
    k = np.arange(n_nodes, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        key = (i << np.uint64(32)) | k
        s = np.uint64(seed)
        u1 = splitmix64(s ^ splitmix64(key * np.uint64(2)))
        u2 = splitmix64(s ^ splitmix64(key * np.uint64(2) + np.uint64(1)))
    U1 = ((u1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    U2 = (u2 >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.sqrt(-2.0 * np.log(U1)) * np.cos(2.0 * math.pi * U2)


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
@dataclass
class Mesh:
    D: int
    faceL: np.ndarray
    faceR: np.ndarray
    An: np.ndarray
    rL: np.ndarray
    rR: np.ndarray
    vol: np.ndarray
    xc: np.ndarray
    bc: np.ndarray
    dims: tuple = ()
    name: str = ""

    @property
    def Nc(self) -> int:
        return int(self.vol.shape[0])

    @property
    def Nf(self) -> int:
        return int(self.faceL.shape[0])

    def contiguous(self) -> "Mesh":
        for k in ("faceL", "faceR"):
            setattr(self, k, np.ascontiguousarray(getattr(self, k), dtype=np.int32))
        for k in ("An", "rL", "rR", "vol", "xc", "bc"):
            setattr(self, k, np.ascontiguousarray(getattr(self, k), dtype=np.float64))
        return self


def _bc_row(kind: int, rho=1.0, U=(0.0, 0.0, 0.0), T=1.0):
    U = tuple(U) + (0.0,) * (3 - len(U))
    return [float(kind), float(rho), float(U[0]), float(U[1]), float(U[2]), float(T)]


def cartesian_mesh(n, length, bcs=None, periodic=None) -> Mesh:
    """Uniform Cartesian mesh in 2D or 3D.

    ``n``, ``length``: cells and box size per axis.  ``bcs``: for every axis a
    pair (low, high) of rows as built by ``_bc_row`` (ignored on periodic
    axes).  Cell index = a0 + n0 (a1 + n1 a2).  Faces are listed axis by axis;
    within an axis in index order, so each cell sees its low face before its
    high face.
    """
    D = len(n)
    n = tuple(int(v) for v in n)
    h = [float(length[d]) / n[d] for d in range(D)]
    periodic = tuple(periodic) if periodic is not None else (False,) * D
    Nc = int(np.prod(n))
    vol = np.full(Nc, float(np.prod(h)))
    grids = np.meshgrid(*[(np.arange(n[d]) + 0.5) * h[d] for d in range(D)], indexing="ij")
    # flatten with axis 0 fastest
    xc = np.stack([g.transpose(*reversed(range(D))).reshape(-1) for g in grids], axis=1)

    bc_rows = []
    faceL, faceR, An, rL, rR = [], [], [], [], []

    def cid(idx):
        c = 0
        s = 1
        for d in range(D):
            c += idx[d] * s
            s *= n[d]
        return c

    for d in range(D):
        area = float(np.prod([h[e] for e in range(D) if e != d]))
        others = [range(n[e]) for e in range(D) if e != d]
        if not periodic[d]:
            lo_id = len(bc_rows)
            bc_rows.append(list(bcs[d][0]))
            hi_id = len(bc_rows)
            bc_rows.append(list(bcs[d][1]))
        npos = n[d] if periodic[d] else n[d] + 1
        # iterate: outer over the other axes (highest first), inner over position
        import itertools
        for rest in itertools.product(*reversed(others)):
            rest = tuple(reversed(rest))
            for a in range(npos):
                def full(pos):
                    idx = list(rest)
                    idx.insert(d, pos)
                    return idx
                e = np.zeros(D)
                e[d] = 1.0
                off = np.zeros(D)
                off[d] = 0.5 * h[d]
                if periodic[d]:
                    L = cid(full((a - 1) % n[d]))
                    R = cid(full(a))
                    faceL.append(L); faceR.append(R)
                    An.append(e * area); rL.append(off.copy()); rR.append(-off)
                elif a == 0:
                    faceL.append(cid(full(0))); faceR.append(-1 - lo_id)
                    An.append(-e * area); rL.append(-off); rR.append(np.zeros(D))
                elif a == n[d]:
                    faceL.append(cid(full(n[d] - 1))); faceR.append(-1 - hi_id)
                    An.append(e * area); rL.append(off.copy()); rR.append(np.zeros(D))
                else:
                    faceL.append(cid(full(a - 1))); faceR.append(cid(full(a)))
                    An.append(e * area); rL.append(off.copy()); rR.append(-off)
    bc = np.array(bc_rows, dtype=np.float64).reshape(-1, 6)
    return Mesh(D, np.array(faceL), np.array(faceR), np.array(An), np.array(rL),
                np.array(rR), vol, xc, bc, dims=n, name="cartesian").contiguous()


def _polygon_area_centroid(P):
    """Area and centroid of a simple polygon with vertices P[m, 2] (CCW)."""
    x, y = P[:, 0], P[:, 1]
    x1, y1 = np.roll(x, -1), np.roll(y, -1)
    cr = x * y1 - x1 * y
    A = 0.5 * cr.sum()
    cx = ((x + x1) * cr).sum() / (6.0 * A)
    cy = ((y + y1) * cr).sum() / (6.0 * A)
    return A, np.array([cx, cy])


def quad_ring_mesh(P, bc_inner, bc_outer, name="quad-ring") -> Mesh:
    """Body-fitted 2D O-type mesh from vertices P[m, j, 2].

    m = 0..nr runs from the body (inner ring) outward, j = 0..nt-1 around the
    body (periodic).  Cell (j, m) has index j + nt m.  Faces: first the edges
    of constant j (between circumferential neighbours, periodic), then the
    edges of constant m (m = 0: body, m = nr: outer boundary).
    """
    nr = P.shape[0] - 1
    nt = P.shape[1]
    Nc = nr * nt
    vol = np.zeros(Nc)
    xc = np.zeros((Nc, 2))
    for m in range(nr):
        for j in range(nt):
            jp = (j + 1) % nt
            poly = np.array([P[m, j], P[m, jp], P[m + 1, jp], P[m + 1, j]])
            A, c = _polygon_area_centroid(poly)
            if A < 0:
                A, c = _polygon_area_centroid(poly[::-1])
            vol[j + nt * m] = A
            xc[j + nt * m] = c
    faceL, faceR, An, rL, rR = [], [], [], [], []

    def add(L, R, a, b, outward_from_L):
        mid = 0.5 * (a + b)
        t = b - a
        nvec = np.array([t[1], -t[0]])
        if np.dot(nvec, mid - xc[L]) < 0:
            nvec = -nvec
        faceL.append(L)
        faceR.append(R)
        An.append(nvec)
        rL.append(mid - xc[L])
        rR.append(mid - xc[R] if R >= 0 else np.zeros(2))

    for m in range(nr):                       # constant-j edges
        for j in range(nt):
            L = (j - 1) % nt + nt * m
            R = j + nt * m
            add(L, R, P[m, j], P[m + 1, j], True)
    for m in range(nr + 1):                   # constant-m edges
        for j in range(nt):
            jp = (j + 1) % nt
            if m == 0:
                add(j, -1, P[0, j], P[0, jp], True)
            elif m == nr:
                add(j + nt * (nr - 1), -2, P[nr, j], P[nr, jp], True)
            else:
                add(j + nt * (m - 1), j + nt * m, P[m, j], P[m, jp], True)
    bc = np.array([bc_inner, bc_outer], dtype=np.float64)
    return Mesh(2, np.array(faceL), np.array(faceR), np.array(An), np.array(rL),
                np.array(rR), vol, xc, bc, dims=(nt, nr), name=name).contiguous()


def geometric_spacing(r0, r1, n, first):
    """n+1 radii from r0 to r1 whose first interval is ``first`` and whose
    intervals grow geometrically (ratio found by bisection)."""
    L = r1 - r0
    if abs(first * n - L) < 1e-14 * L:
        q = 1.0
    else:
        lo, hi = 1.0 + 1e-12, 2.0
        while first * (hi ** n - 1) / (hi - 1) < L:
            hi *= 2
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if first * (mid ** n - 1) / (mid - 1) < L:
                lo = mid
            else:
                hi = mid
        q = 0.5 * (lo + hi)
    d = first * q ** np.arange(n)
    r = r0 + np.concatenate([[0.0], np.cumsum(d)])
    r[-1] = r1
    return r


def cylinder_omesh(n_theta=96, n_r=128, r_body=1.0, r_out=15.0, first=0.01,
                   bc_wall=None, bc_far=None) -> Mesh:
    """O-mesh around a circular cylinder (paper Sec. 4.1: radius 1, outer
    radius 15, first layer 0.01)."""
    r = geometric_spacing(r_body, r_out, n_r, first)
    th = 2.0 * math.pi * np.arange(n_theta) / n_theta
    P = np.stack([r[:, None] * np.cos(th)[None, :], r[:, None] * np.sin(th)[None, :]], axis=2)
    return quad_ring_mesh(P, bc_wall, bc_far, name="cylinder-omesh")


def _blunt_wedge_outline(R=1.0, half_angle_deg=10.0, length=6.0, n=2000):
    """Closed CCW outline of a blunt wedge: nose arc of radius R centred at
    the origin, flanks tangent to it at +-half_angle, flat base at x = length
    (lengths in units of the nose radius; paper Sec. 4.3 gives R = 20 mm,
    L = 120 mm, theta = 10 deg)."""
    a = math.radians(half_angle_deg)
    # tangent points on the arc: normal direction (-sin a ... ) -> point at angle pi/2 + a
    tp = math.pi / 2 + a
    arc = np.linspace(tp, 2 * math.pi - tp, n)
    pts = [np.stack([R * np.cos(arc), R * np.sin(arc)], axis=1)]
    # lower flank from the lower tangent point to the base
    p_lo = np.array([R * math.cos(2 * math.pi - tp), R * math.sin(2 * math.pi - tp)])
    y_base = p_lo[1] - (length - p_lo[0]) * math.tan(a)
    pts.append(np.array([[length, y_base], [length, -y_base]]))
    return np.concatenate(pts, axis=0)


def _ray_polygon(c, d, poly):
    """Smallest positive t with c + t d on the closed polygon."""
    best = np.inf
    q = np.roll(poly, -1, axis=0)
    for p0, p1 in zip(poly, q):
        e = p1 - p0
        M = np.array([[d[0], -e[0]], [d[1], -e[1]]])
        det = np.linalg.det(M)
        if abs(det) < 1e-14:
            continue
        t, s = np.linalg.solve(M, p0 - c)
        if t > 0 and -1e-12 <= s <= 1 + 1e-12:
            best = min(best, t)
    return best


def blunt_body_mesh(n_theta=240, n_r=160, r_out=30.0, first=1e-3 * 6.0,
                    bc_wall=None, bc_far=None) -> Mesh:
    """Body-fitted O-type mesh around a synthetic blunt wedge, clustered to
    the wall (geometric growth from a first cell of 1e-3 of the body length).
    Rays start at an interior point on the axis."""
    outline = _blunt_wedge_outline()
    c = np.array([2.0, 0.0])
    th = 2.0 * math.pi * np.arange(n_theta) / n_theta
    P = np.zeros((n_r + 1, n_theta, 2))
    for j, t in enumerate(th):
        d = np.array([math.cos(t), math.sin(t)])
        rb = _ray_polygon(c, d, outline)
        r = geometric_spacing(rb, r_out, n_r, first)
        P[:, j, :] = c[None, :] + r[:, None] * d[None, :]
    return quad_ring_mesh(P, bc_wall, bc_far, name="blunt-wedge")


def sphere_shell_mesh(n_r=64, n_theta=48, n_phi=48, r_body=1.0, r_out=10.0, first=0.01,
                      bc_wall=None, bc_far=None) -> Mesh:
    """Spherical-shell mesh around a sphere of radius 1 (paper Sec. 4.6 uses
    the diameter as reference length; here the radius is 1).  Cell
    (p, t, m) has index p + n_phi (t + n_theta m).  Area vectors are the exact
    surface integrals of the unit normal over each face, so every cell's
    faces sum to zero.  The faces on the polar axis have zero area and are
    left out of the face list."""
    r = geometric_spacing(r_body, r_out, n_r, first)
    th = np.linspace(0.0, math.pi, n_theta + 1)
    ph = 2.0 * math.pi * np.arange(n_phi + 1) / n_phi
    Nc = n_r * n_theta * n_phi

    def cid(p, t, m):
        return (p % n_phi) + n_phi * (t + n_theta * m)

    vol = np.zeros(Nc)
    xc = np.zeros((Nc, 3))
    for m in range(n_r):
        for t in range(n_theta):
            for p in range(n_phi):
                i = cid(p, t, m)
                vol[i] = (r[m + 1] ** 3 - r[m] ** 3) / 3.0 * (math.cos(th[t]) - math.cos(th[t + 1])) * (ph[p + 1] - ph[p])
                rm = 0.5 * (r[m] + r[m + 1]); tm = 0.5 * (th[t] + th[t + 1]); pm = 0.5 * (ph[p] + ph[p + 1])
                xc[i] = [rm * math.sin(tm) * math.cos(pm), rm * math.sin(tm) * math.sin(pm), rm * math.cos(tm)]

    def sph(rr, tt, pp):
        return np.array([rr * math.sin(tt) * math.cos(pp), rr * math.sin(tt) * math.sin(pp), rr * math.cos(tt)])

    faceL, faceR, An, rL, rR = [], [], [], [], []

    def add(L, R, a, xf):
        faceL.append(L); faceR.append(R); An.append(a)
        rL.append(xf - xc[L]); rR.append(xf - xc[R] if R >= 0 else np.zeros(3))

    # phi-faces (planar), between (p-1) and p, periodic
    for m in range(n_r):
        for t in range(n_theta):
            for p in range(n_phi):
                area = 0.5 * (r[m + 1] ** 2 - r[m] ** 2) * (th[t + 1] - th[t])
                nphi = np.array([-math.sin(ph[p]), math.cos(ph[p]), 0.0])
                xf = sph(0.5 * (r[m] + r[m + 1]), 0.5 * (th[t] + th[t + 1]), ph[p])
                add(cid(p - 1, t, m), cid(p, t, m), area * nphi, xf)
    # theta-faces (cones) between (t-1) and t; t = 0 and t = n_theta are the axis
    for m in range(n_r):
        for t in range(1, n_theta):
            for p in range(n_phi):
                s = math.sin(th[t]); co = math.cos(th[t])
                k = 0.5 * (r[m + 1] ** 2 - r[m] ** 2) * s
                a = k * np.array([co * (math.sin(ph[p + 1]) - math.sin(ph[p])),
                                  co * (math.cos(ph[p]) - math.cos(ph[p + 1])),
                                  -s * (ph[p + 1] - ph[p])])
                xf = sph(0.5 * (r[m] + r[m + 1]), th[t], 0.5 * (ph[p] + ph[p + 1]))
                add(cid(p, t - 1, m), cid(p, t, m), a, xf)
    # r-faces (sphere patches) between (m-1) and m; m = 0 body, m = n_r outer

    def rpatch(rr, t, p):
        i_s2 = (th[t + 1] / 2 - math.sin(2 * th[t + 1]) / 4) - (th[t] / 2 - math.sin(2 * th[t]) / 4)
        i_sc = 0.5 * (math.sin(th[t + 1]) ** 2 - math.sin(th[t]) ** 2)
        return rr * rr * np.array([i_s2 * (math.sin(ph[p + 1]) - math.sin(ph[p])),
                                   i_s2 * (math.cos(ph[p]) - math.cos(ph[p + 1])),
                                   i_sc * (ph[p + 1] - ph[p])])

    for m in range(n_r + 1):
        for t in range(n_theta):
            for p in range(n_phi):
                a = rpatch(r[m], t, p)
                xf = sph(r[m], 0.5 * (th[t] + th[t + 1]), 0.5 * (ph[p] + ph[p + 1]))
                if m == 0:
                    add(cid(p, t, 0), -1, -a, xf)
                elif m == n_r:
                    add(cid(p, t, n_r - 1), -2, a, xf)
                else:
                    add(cid(p, t, m - 1), cid(p, t, m), a, xf)
    bc = np.array([bc_wall, bc_far], dtype=np.float64)
    return Mesh(3, np.array(faceL), np.array(faceR), np.array(An), np.array(rL),
                np.array(rR), vol, xc, bc, dims=(n_phi, n_theta, n_r), name="sphere-shell").contiguous()


# --------------------------------------------------------------------------
# flow conditions and velocity forests of the workloads
# --------------------------------------------------------------------------
@dataclass
class FlowSpec:
    """Flow data of a workload whose velocity space each side derives by the
    adaptive-parameter rules of Sec. 3.5 (inputs only; the rules themselves
    live in the library and, separately, in the oracle)."""
    Ma: float
    gamma: float = GAMMA_MONO
    T_inf: float = 1.0
    T_w: float = 1.0
    dir: tuple = (1.0, 0.0, 0.0)
    h_std: float = 0.6
    rdv_sigma: float = 4.0
    separated: bool = False


@dataclass
class Workload:
    """Everything needed to set up one run (inputs only)."""
    name: str
    mesh: Mesh
    D: int
    base: tuple            # base-forest cells per velocity axis
    vlo: tuple
    vhi: tuple
    max_refine: int
    Kn: float
    omega: float
    Pr: float
    C1: float
    C2: float
    W_inf: tuple           # rho, U (D), T  of the free stream (or lid)
    W_init: np.ndarray     # Nc x (D+2): rho, U..., T
    precision: str = "fp64"    # "fp64" | "mixed"
    learned: bool = False
    limiter: int = 1
    cfl: float = 0.8
    steps: int = 200
    adapt_first_n: int = 3
    adapt_every: int = 50
    extra: dict = field(default_factory=dict)
    flow: FlowSpec = None      # set: base, vlo, vhi, max_refine, C1, C2 come from the Sec. 3.5 rules
    model: str = "shakhov"     # "shakhov" (monatomic) or "rykov" (diatomic, K = 2)
    Zrot: float = 3.5          # rotational collision number of the Rykov model


def mach_speed(Ma, gamma=GAMMA_MONO, T=1.0):
    """Free-stream speed for a Mach number, in units of sqrt(2 R T_inf)."""
    return Ma * math.sqrt(gamma * R_GAS * T)


def sqrt_RT(T=1.0):
    """sqrt(R T) in units of sqrt(2 R T_inf): converts velocity bounds quoted
    in sqrt(R T) units into the solver's units."""
    return math.sqrt(R_GAS * T)


K_SIGMA = 3.3546e-4      # printed ratio of the merge to the split threshold (Eq. c2c1)


def _uniform_W(Nc, D, rho, U, T):
    W = np.zeros((Nc, D + 2))
    W[:, 0] = rho
    W[:, 1:1 + D] = np.asarray(U)[:D]
    W[:, D + 1] = T
    return W


def cavity(n=32, C1=6.0, max_refine=1, precision="fp64") -> Workload:
    """Lid-driven cavity (paper Sec. 4.2): 32x32 uniform cells on the unit
    square, isothermal walls at T0 = 1, lid speed 0.16 sqrt(2 R T0), Kn 0.075,
    forest 16x16 over [-4, 4]^2 sqrt(R T0), at most one refinement level."""
    wall = _bc_row(BC_WALL, T=1.0)
    lid = _bc_row(BC_WALL, U=(0.16, 0.0), T=1.0)
    mesh = cartesian_mesh((n, n), (1.0, 1.0), bcs=[(wall, wall), (wall, lid)])
    v = 4.0 * sqrt_RT(1.0)
    return Workload("cavity-32x32", mesh, 2, (16, 16), (-v, -v), (v, v), max_refine,
                    Kn=0.075, omega=0.81, Pr=2.0 / 3.0, C1=C1, C2=K_SIGMA * C1,
                    W_inf=(1.0, 0.16, 0.0, 1.0), W_init=_uniform_W(mesh.Nc, 2, 1.0, (0, 0), 1.0),
                    precision=precision, steps=200)


def cylinder(n_theta=96, n_r=128, Ma=5.0, Kn=0.1, C1=1.0, max_refine=4, precision="mixed") -> Workload:
    """Supersonic cylinder (paper Sec. 4.1 shape): O-mesh 128 radial x 96
    circumferential, r in [1, 15], first layer 0.01, Ma 5, Kn 0.1, isothermal
    wall at T_inf, forest 24x24 over [-15, 15]^2 sqrt(R T_inf), up to 4 levels.
    The gas starts at rest and the Ma 5 stream enters through the far field
    (an impulsive start empties the first wake cell within a few steps)."""
    U = mach_speed(Ma)
    wall = _bc_row(BC_WALL, T=1.0)
    far = _bc_row(BC_FARFIELD, rho=1.0, U=(U, 0.0), T=1.0)
    mesh = cylinder_omesh(n_theta, n_r, bc_wall=wall, bc_far=far)
    v = 15.0 * sqrt_RT(1.0)
    return Workload(f"cylinder-omesh-{n_r}x{n_theta}", mesh, 2, (24, 24), (-v, -v), (v, v), max_refine,
                    Kn=Kn, omega=0.81, Pr=2.0 / 3.0, C1=C1, C2=K_SIGMA * C1,
                    W_inf=(1.0, U, 0.0, 1.0), W_init=_uniform_W(mesh.Nc, 2, 1.0, (0.0, 0.0), 1.0),
                    precision=precision, steps=200)


def cylinder_zones(n_theta=96, n_r=128, Ma=5.0, Kn=0.1, separated=False, rdv_sigma=4.0, precision="mixed",
                   learned=False) -> Workload:
    """The cylinder O-mesh with the velocity space of Sec. 3.5: domain,
    levels, refinement zones and thresholds from Ma, T_w = T_inf and the
    paper's h_std = 0.6, R_dv = 4 sigma_0 (the paper's setting for this case)."""
    U = mach_speed(Ma)
    wall = _bc_row(BC_WALL, T=1.0)
    far = _bc_row(BC_FARFIELD, rho=1.0, U=(U, 0.0), T=1.0)
    mesh = cylinder_omesh(n_theta, n_r, bc_wall=wall, bc_far=far)
    return Workload(f"cylinder-zones-{n_r}x{n_theta}", mesh, 2, None, None, None, None,
                    Kn=Kn, omega=0.81, Pr=2.0 / 3.0, C1=None, C2=None,
                    W_inf=(1.0, U, 0.0, 1.0), W_init=_uniform_W(mesh.Nc, 2, 1.0, (0.0, 0.0), 1.0),
                    precision=precision, learned=learned,
                    flow=FlowSpec(Ma=Ma, T_w=1.0, rdv_sigma=rdv_sigma, separated=separated))


def sphere_zones(n_r=64, n_theta=48, n_phi=48, Ma=4.25, Kn=0.031, rdv_sigma=4.0, precision="mixed",
                 learned=False) -> Workload:
    """The sphere shell with the velocity space of Sec. 3.5 (octree)."""
    U = mach_speed(Ma)
    wall = _bc_row(BC_WALL, T=1.0)
    far = _bc_row(BC_FARFIELD, rho=1.0, U=(U, 0.0, 0.0), T=1.0)
    mesh = sphere_shell_mesh(n_r, n_theta, n_phi, bc_wall=wall, bc_far=far)
    return Workload(f"sphere-zones-{n_r}x{n_theta}x{n_phi}", mesh, 3, None, None, None, None,
                    Kn=Kn, omega=0.81, Pr=2.0 / 3.0, C1=None, C2=None,
                    W_inf=(1.0, U, 0.0, 0.0, 1.0), W_init=_uniform_W(mesh.Nc, 3, 1.0, (0.0, 0.0, 0.0), 1.0),
                    precision=precision, learned=learned,
                    flow=FlowSpec(Ma=Ma, T_w=1.0, rdv_sigma=rdv_sigma))


def blunt_wedge(n_theta=240, n_r=160, Ma=8.0, Kn=0.01, C1=0.5, max_refine=5, precision="mixed",
                learned=True) -> Workload:
    """Blunt wedge (paper Sec. 4.3 shape): 240x160 body-fitted cells clustered
    to the wall, Ma 8, Kn 0.01, forest 32x32 over [-20, 20]^2 (read as
    sqrt(R T_inf) units), up to 5 levels, learned proposer."""
    U = mach_speed(Ma)
    wall = _bc_row(BC_WALL, T=1.0)
    far = _bc_row(BC_FARFIELD, rho=1.0, U=(U, 0.0), T=1.0)
    mesh = blunt_body_mesh(n_theta, n_r, bc_wall=wall, bc_far=far)
    v = 20.0 * sqrt_RT(1.0)
    return Workload(f"blunt-wedge-{n_theta}x{n_r}", mesh, 2, (32, 32), (-v, -v), (v, v), max_refine,
                    Kn=Kn, omega=0.81, Pr=2.0 / 3.0, C1=C1, C2=K_SIGMA * C1,
                    W_inf=(1.0, U, 0.0, 1.0), W_init=_uniform_W(mesh.Nc, 2, 1.0, (0.0, 0.0), 1.0),
                    precision=precision, learned=learned)


def sphere(n_r=64, n_theta=48, n_phi=48, Ma=4.25, Kn=0.031, C1=2.0, max_refine=3,
           precision="mixed", learned=True) -> Workload:
    """Sphere (paper Sec. 4.6 shape): spherical shell 64 r x 48 theta x 48 phi,
    r in [1, 10], Ma 4.25, Kn 0.031, octree 16^3 over [-12, 12]^3 (read as
    sqrt(R T_inf) units), up to 3 levels."""
    U = mach_speed(Ma)
    wall = _bc_row(BC_WALL, T=1.0)
    far = _bc_row(BC_FARFIELD, rho=1.0, U=(U, 0.0, 0.0), T=1.0)
    mesh = sphere_shell_mesh(n_r, n_theta, n_phi, bc_wall=wall, bc_far=far)
    v = 12.0 * sqrt_RT(1.0)
    return Workload(f"sphere-shell-{n_r}x{n_theta}x{n_phi}", mesh, 3, (16, 16, 16), (-v,) * 3, (v,) * 3,
                    max_refine, Kn=Kn, omega=0.81, Pr=2.0 / 3.0, C1=C1, C2=K_SIGMA * C1,
                    W_inf=(1.0, U, 0.0, 0.0, 1.0), W_init=_uniform_W(mesh.Nc, 3, 1.0, (0.0, 0.0, 0.0), 1.0),
                    precision=precision, learned=learned)


def triangle_mesh(n_points=120, seed=5, bc_wall=None) -> Mesh:
    """Unstructured mesh of triangles on the unit square: Delaunay
    triangulation of seeded random interior points plus points along the
    sides; every boundary edge is a face to the given boundary condition.
    Faces are edges, oriented from the lower-numbered triangle outwards."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    m = max(3, int(round(math.sqrt(n_points) / 1.5)))
    side = np.linspace(0.0, 1.0, m + 1)[:-1]
    edge = np.concatenate([np.stack([side, np.zeros(m)], 1), np.stack([np.ones(m), side], 1),
                           np.stack([1.0 - side, np.ones(m)], 1), np.stack([np.zeros(m), 1.0 - side], 1)])
    P = np.concatenate([edge, 0.05 + 0.9 * rng.random((n_points, 2))])
    tri = Delaunay(P).simplices
    a, b, c = P[tri[:, 0]], P[tri[:, 1]], P[tri[:, 2]]
    area = 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    tri[area < 0] = tri[area < 0][:, [0, 2, 1]]
    xc = P[tri].mean(1)
    owner = {}
    faceL, faceR, An, rL, rR = [], [], [], [], []
    for t, (i, j, k) in enumerate(tri):
        for p0, p1 in ((i, j), (j, k), (k, i)):
            key = (min(p0, p1), max(p0, p1))
            if key in owner:
                L, q0, q1 = owner.pop(key)
                mid = 0.5 * (P[q0] + P[q1])
                e = P[q1] - P[q0]
                faceL.append(L); faceR.append(t)
                An.append(np.array([e[1], -e[0]]))          # outward of L (counter-clockwise L)
                rL.append(mid - xc[L]); rR.append(mid - xc[t])
            else:
                owner[key] = (t, p0, p1)
    for (_, _), (L, q0, q1) in sorted(owner.items()):
        mid = 0.5 * (P[q0] + P[q1])
        e = P[q1] - P[q0]
        faceL.append(L); faceR.append(-1)
        An.append(np.array([e[1], -e[0]]))
        rL.append(mid - xc[L]); rR.append(np.zeros(2))
    vol = np.abs(0.5 * ((P[tri[:, 1], 0] - P[tri[:, 0], 0]) * (P[tri[:, 2], 1] - P[tri[:, 0], 1])
                        - (P[tri[:, 1], 1] - P[tri[:, 0], 1]) * (P[tri[:, 2], 0] - P[tri[:, 0], 0])))
    bc = np.array([bc_wall if bc_wall is not None else _bc_row(BC_WALL, T=1.0)])
    return Mesh(2, np.array(faceL), np.array(faceR), np.array(An), np.array(rL), np.array(rR), vol, xc, bc,
                name="triangles").contiguous()


def triangle_box(n_points=120, seed=5, Kn=0.05, C1=2.0, base=(10, 10), max_refine=1, precision="fp64") -> Workload:
    """Unstructured-mesh case: triangles on the unit square with isothermal
    walls, the smooth field of the kernel sweep as initial state."""
    mesh = triangle_mesh(n_points, seed)
    v = 4.0 * sqrt_RT(1.0)
    return Workload(f"triangles-{mesh.Nc}", mesh, 2, tuple(base), (-v, -v), (v, v), max_refine, Kn=Kn,
                    omega=0.81, Pr=2.0 / 3.0, C1=C1, C2=K_SIGMA * C1, W_inf=(1.0, 0.0, 0.0, 1.0),
                    W_init=sweep_W(mesh), precision=precision)


def sweep_W(mesh: Mesh) -> np.ndarray:
    """Smooth synthetic macroscopic field of the kernel sweep:
    rho = 1 + 0.1 sin(2 pi x) sin(2 pi y), U = 0.3 (sin 2 pi y, cos 2 pi x[, 0]),
    T = 1 + 0.1 cos(2 pi x).  Returned as rho, U..., T per cell."""
    x = mesh.xc[:, 0]
    y = mesh.xc[:, 1]
    D = mesh.D
    W = np.zeros((mesh.Nc, D + 2))
    W[:, 0] = 1.0 + 0.1 * np.sin(2 * math.pi * x) * np.sin(2 * math.pi * y)
    W[:, 1] = 0.3 * np.sin(2 * math.pi * y)
    W[:, 2] = 0.3 * np.cos(2 * math.pi * x)
    W[:, D + 1] = 1.0 + 0.1 * np.cos(2 * math.pi * x)
    return W


def sweep_box(n, Kn=0.05, C1=4.0, base=None, max_refine=2, precision="fp64", vbound=4.0) -> Workload:
    """Kernel-sweep case: periodic unit box with the smooth field of
    ``sweep_W``; near-Maxwellian f with a 1e-3 seeded perturbation is formed
    by each side from these W and ``normal_field``."""
    D = len(n)
    mesh = cartesian_mesh(n, (1.0,) * D, periodic=(True,) * D)
    base = base or (8,) * D
    v = vbound * sqrt_RT(1.0)
    return Workload(f"sweep-box-{'x'.join(map(str, n))}", mesh, D, tuple(base), (-v,) * D, (v,) * D,
                    max_refine, Kn=Kn, omega=0.81, Pr=2.0 / 3.0, C1=C1, C2=K_SIGMA * C1,
                    W_inf=(1.0,) + (0.0,) * D + (1.0,), W_init=sweep_W(mesh), precision=precision)
