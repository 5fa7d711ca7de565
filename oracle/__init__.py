"""CPU oracle of the UGKS + adaptive-velocity-space hot path (arXiv 2212.05645).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It is
a plain FP64 C implementation (``avs_oracle.c``, built with gcc and
``-ffp-contract=off``) wrapped with ctypes, plus :mod:`oracle.mlp` (numpy
FP64).  It shares no code with the CUDA library; the only common module is
the input generator :mod:`paper_2212_05645_gb300.workloads`.

Parity status of each routine (what pins it) is listed in the tests under
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libavs_oracle.so")
_lock = threading.Lock()
_lib = None

OM_COPY, OM_MERGE = 0, 1


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over cells, no FMA contraction)."""
    src = os.path.join(_HERE, "avs_oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "avs_oracle.h"))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            up = C.POINTER(C.c_uint)
            L.om_mu_ref_from_Kn.restype = C.c_double
            L.om_mu_ref_from_Kn.argtypes = [C.c_double, C.c_double, C.c_double]
            L.om_shakhov_field.restype = None
            L.om_shakhov_field.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_double, dp, C.c_double,
                                           dp, dp, dp]
            L.om_forest_base.restype = C.c_int
            L.om_forest_base.argtypes = [C.c_int, ip, ip, ip, up]
            L.om_forest_geom.restype = None
            L.om_forest_geom.argtypes = [C.c_int, ip, dp, dp, C.c_int, ip, ip, up, dp, dp]
            L.om_maxwell_init.restype = None
            L.om_maxwell_init.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, C.c_double, C.c_double,
                                          C.c_ulonglong, dp]
            L.om_normal_field.restype = None
            L.om_normal_field.argtypes = [C.c_ulonglong, C.c_int, C.c_int, dp]
            L.om_moments.restype = None
            L.om_moments.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp]
            L.om_dt_unit.restype = C.c_double
            L.om_dt_unit.argtypes = [C.c_void_p, C.c_int, dp]
            L.om_limited_gradients.restype = None
            L.om_limited_gradients.argtypes = [C.c_void_p, C.c_void_p, C.c_int, dp, dp, dp]
            L.om_venkat.restype = C.c_double
            L.om_venkat.argtypes = [C.c_double, C.c_double, C.c_double]
            L.om_step.restype = C.c_int
            L.om_step.argtypes = [C.c_void_p, C.c_void_p, C.c_int, dp, dp, C.c_double, dp, dp, dp]
            L.om_colors.restype = C.c_int
            L.om_colors.argtypes = [C.c_void_p, ip]
            L.om_step_implicit.restype = C.c_int
            L.om_step_implicit.argtypes = [C.c_void_p, C.c_void_p, C.c_int, dp, dp, C.c_double, dp, dp, dp, ip,
                                           C.c_int, C.c_int, C.c_int]
            L.om_criterion.restype = None
            L.om_criterion.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp]
            L.om_adapt_tree.restype = C.c_int
            L.om_adapt_tree.argtypes = [C.c_int, C.c_int, ip, ip, up, dp, C.c_double, C.c_double,
                                        C.c_double, C.c_int, ip, C.c_int, ip, ip, up, ip, ip]
            L.om_remap.restype = None
            L.om_remap.argtypes = [C.c_int, C.c_int, C.c_int, dp, C.c_int, ip, ip, dp]
            L.om_correct.restype = C.c_double
            L.om_correct.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, C.c_double, C.c_int, dp, dp]
            L.om_rykov_field.restype = None
            L.om_rykov_field.argtypes = [C.c_int, C.c_int, dp, C.c_void_p, C.c_double, dp, C.c_double,
                                         C.c_double, dp, dp, dp]
            L.om_maxwell_init_rykov.restype = None
            L.om_maxwell_init_rykov.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, C.c_double, C.c_double,
                                                C.c_ulonglong, dp]
            L.om_moments_rykov.restype = None
            L.om_moments_rykov.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp]
            L.om_criterion_nw.restype = None
            L.om_criterion_nw.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp]
            L.om_remap_n.restype = None
            L.om_remap_n.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, C.c_int, ip, ip, dp]
            L.om_correct_rykov.restype = C.c_double
            L.om_correct_rykov.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp, C.c_double, C.c_int, dp, dp]
            _lib = L
    return _lib


class _Mesh(C.Structure):
    _fields_ = [("D", C.c_int), ("Nc", C.c_int), ("Nf", C.c_int), ("nbc", C.c_int),
                ("faceL", C.POINTER(C.c_int)), ("faceR", C.POINTER(C.c_int)),
                ("An", C.POINTER(C.c_double)), ("rL", C.POINTER(C.c_double)),
                ("rR", C.POINTER(C.c_double)), ("vol", C.POINTER(C.c_double)),
                ("bc", C.POINTER(C.c_double))]


class _Gas(C.Structure):
    _fields_ = [("R", C.c_double), ("Pr", C.c_double), ("omega", C.c_double),
                ("mu_ref", C.c_double), ("T_ref", C.c_double), ("lim_K", C.c_double),
                ("limiter", C.c_int), ("model", C.c_int), ("Zrot", C.c_double), ("omega0", C.c_double),
                ("omega1", C.c_double), ("delta", C.c_double)]


# Rykov coefficients for nitrogen (Sec. 2.1, after Eq. 13); Z_rot is not given
# in the paper (reading R26)
RYKOV_DELTA = 1.0 / 1.55
RYKOV_OMEGA0 = 0.2354
RYKOV_OMEGA1 = 0.3049
RYKOV_ZROT = 3.5


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _up(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def n_arrays(D: int) -> int:
    """Reduced distributions per node: G and H in 2D, G alone in 3D (Eq. 6)."""
    return 2 if D == 2 else 1


# ---------------------------------------------------------------------------
# thin wrappers (numpy in, numpy out)
# ---------------------------------------------------------------------------
def mu_ref_from_Kn(Kn, omega, R=0.5):
    return lib().om_mu_ref_from_Kn(Kn, omega, R)


def shakhov_field(D, xi, Pr, rho, U, RT, q):
    """Shakhov equilibrium G (and H in 2D) of one state at the nodes (Eqs. 14-17)."""
    xi = _f64(xi); U = _f64(U); q = _f64(q)
    Nv = xi.shape[0]
    gG = np.zeros(Nv); gH = np.zeros(Nv)
    lib().om_shakhov_field(D, Nv, _dp(xi), Pr, rho, _dp(U), RT, _dp(q), _dp(gG), _dp(gH))
    return gG, gH


def forest_base(D, nb):
    nb = np.ascontiguousarray(nb, dtype=np.int32)
    n = int(np.prod(nb))
    level = np.zeros(n, np.int32)
    base = np.zeros(n, np.int32)
    key = np.zeros(n, np.uint32)
    lib().om_forest_base(D, _ip(nb), _ip(level), _ip(base), _up(key))
    return level, base, key


def forest_geom(D, nb, vlo, vhi, level, base, key):
    nb = np.ascontiguousarray(nb, dtype=np.int32)
    vlo = _f64(vlo); vhi = _f64(vhi)
    level = np.ascontiguousarray(level, np.int32)
    base = np.ascontiguousarray(base, np.int32)
    key = np.ascontiguousarray(key, np.uint32)
    Nv = len(level)
    xi = np.zeros((Nv, D)); w = np.zeros(Nv)
    lib().om_forest_geom(D, _ip(nb), _dp(vlo), _dp(vhi), Nv, _ip(level), _ip(base), _up(key), _dp(xi), _dp(w))
    return xi, w


def maxwell_init(D, xi, Wp, R=0.5, amp=0.0, seed=12345):
    xi = _f64(xi); Wp = _f64(Wp)
    Nc, Nv = Wp.shape[0], xi.shape[0]
    f = np.zeros((Nc, n_arrays(D), Nv))
    lib().om_maxwell_init(D, Nc, Nv, _dp(xi), _dp(Wp), R, amp, seed, _dp(f))
    return f


def normal_field(seed, Nc, Nv):
    z = np.zeros((Nc, Nv))
    lib().om_normal_field(seed, Nc, Nv, _dp(z))
    return z


def moments(D, xi, w, f):
    """Conserved W (rho, rho U, rho E) and heat flux q of every cell (Eqs. 7-8)."""
    xi = _f64(xi); w = _f64(w); f = _f64(f)
    Nc, Nv = f.shape[0], f.shape[-1]
    Wc = np.zeros((Nc, D + 2)); q = np.zeros((Nc, D))
    lib().om_moments(D, Nc, Nv, _dp(xi), _dp(w), _dp(f), _dp(Wc), _dp(q))
    return Wc, q


class MeshHandle:
    """Keeps the numpy arrays alive behind the C struct."""

    def __init__(self, mesh):
        self.mesh = mesh
        self._keep = [mesh.faceL, mesh.faceR, mesh.An, mesh.rL, mesh.rR, mesh.vol, mesh.bc]
        self.s = _Mesh(mesh.D, mesh.Nc, mesh.Nf, mesh.bc.shape[0], _ip(mesh.faceL), _ip(mesh.faceR),
                       _dp(mesh.An), _dp(mesh.rL), _dp(mesh.rR), _dp(mesh.vol), _dp(mesh.bc))

    @property
    def ptr(self):
        return C.byref(self.s)


def gas(R=0.5, Pr=2.0 / 3.0, omega=0.81, mu_ref=None, Kn=None, T_ref=1.0, lim_K=0.3, limiter=1,
        model="shakhov", Zrot=RYKOV_ZROT):
    if mu_ref is None:
        mu_ref = mu_ref_from_Kn(Kn, omega, R)
    return _Gas(R, Pr, omega, mu_ref, T_ref, lim_K, limiter, 1 if model == "rykov" else 0, Zrot,
                RYKOV_OMEGA0, RYKOV_OMEGA1, RYKOV_DELTA)


def rykov_field(D, xi, g, rho, U, RTt, RTr, qt, qr):
    """Rykov equilibrium (g^G, [g^H,] g^R) at every node, shape (nA, Nv)."""
    xi = _f64(xi)
    Nv = xi.shape[0]
    nA = 3 if D == 2 else 2
    out = np.zeros((nA, Nv))
    lib().om_rykov_field(D, Nv, _dp(xi), C.byref(g), float(rho), _dp(_f64(U)), float(RTt), float(RTr),
                         _dp(_f64(qt)), _dp(_f64(qr)), _dp(out))
    return out


def maxwell_init_rykov(D, xi, Wp, R=0.5, amp=0.0, seed=12345):
    """Initial f of the Rykov model; Wp per cell rho, U (D), T_t[, T_r] (T_r = T_t if absent)."""
    xi = _f64(xi); Wp = _f64(Wp)
    if Wp.shape[1] == D + 2:
        Wp = np.concatenate([Wp, Wp[:, D + 1:D + 2]], axis=1)
    Wp = _f64(Wp)
    Nc, Nv = Wp.shape[0], xi.shape[0]
    f = np.zeros((Nc, 3 if D == 2 else 2, Nv))
    lib().om_maxwell_init_rykov(D, Nc, Nv, _dp(xi), _dp(Wp), R, amp, seed, _dp(f))
    return f


def moments_rykov(D, xi, w, f):
    """W = (rho, rho U, rho E, rho E_rot), q_t and q_r of every cell."""
    xi = _f64(xi); w = _f64(w); f = _f64(f)
    Nc, Nv = f.shape[0], f.shape[-1]
    Wc = np.zeros((Nc, D + 3)); qt = np.zeros((Nc, D)); qr = np.zeros((Nc, D))
    lib().om_moments_rykov(D, Nc, Nv, _dp(xi), _dp(w), _dp(f), _dp(Wc), _dp(qt), _dp(qr))
    return Wc, qt, qr


def correct_rykov(D, xi, w, Wc_target, f, iters=3, R=0.5):
    xi = _f64(xi); w = _f64(w); Wc_target = _f64(Wc_target)
    assert f.dtype == np.float64 and f.flags.c_contiguous
    Nc, Nv = f.shape[0], f.shape[-1]
    return lib().om_correct_rykov(D, Nc, Nv, _dp(xi), _dp(w), R, iters, _dp(Wc_target), _dp(f))


def conserved_rykov(D, Wp, R=0.5):
    """(rho, rho U, rho E, rho E_rot) from rho, U, T_t[, T_r] with K = 2:
    rho E = rho U^2/2 + (3/2) rho R T_t + rho R T_r, rho E_rot = rho R T_r."""
    Wp = _f64(Wp)
    if Wp.shape[-1] == D + 2:
        Wp = np.concatenate([Wp, Wp[..., D + 1:D + 2]], axis=-1)
    Wc = np.zeros(Wp.shape[:-1] + (D + 3,))
    rho = Wp[..., 0]
    U = Wp[..., 1:1 + D]
    Wc[..., 0] = rho
    Wc[..., 1:1 + D] = rho[..., None] * U
    Wc[..., D + 2] = rho * R * Wp[..., D + 2]
    Wc[..., D + 1] = 0.5 * rho * (U * U).sum(-1) + 1.5 * rho * R * Wp[..., D + 1] + Wc[..., D + 2]
    return Wc


def primitive_rykov(D, Wc, R=0.5):
    """rho, U, T_t, T_r from (rho, rho U, rho E, rho E_rot) (K = 2)."""
    Wc = _f64(Wc)
    Wp = np.zeros_like(Wc)
    rho = Wc[..., 0]
    Wp[..., 0] = rho
    Wp[..., 1:1 + D] = Wc[..., 1:1 + D] / rho[..., None]
    m2 = (Wc[..., 1:1 + D] ** 2).sum(-1)
    Wp[..., D + 2] = Wc[..., D + 2] / rho / R
    Wp[..., D + 1] = (Wc[..., D + 1] - 0.5 * m2 / rho - Wc[..., D + 2]) / (1.5 * rho * R)
    return Wp


def dt_unit(mh: MeshHandle, xi):
    xi = _f64(xi)
    return lib().om_dt_unit(mh.ptr, xi.shape[0], _dp(xi))


def limited_gradients(mh: MeshHandle, g: _Gas, f_in):
    """Step 1 of the step alone (Sec. 2.3.3): the unlimited least-squares
    gradient [Nc][nA][Nv][D] and the Venkatakrishnan factor [Nc][nA][Nv]."""
    f_in = _f64(f_in)
    Nc, nA, Nv = f_in.shape
    D = mh.mesh.D
    grad = np.zeros((Nc, nA, Nv, D))
    lim = np.zeros((Nc, nA, Nv))
    lib().om_limited_gradients(mh.ptr, C.byref(g), Nv, _dp(f_in), _dp(grad), _dp(lim))
    return grad, lim


def venkat(d1, d2, eps2):
    """Venkatakrishnan's function of (largest neighbour difference, unlimited
    change, epsilon^2), capped at 1."""
    return lib().om_venkat(float(d1), float(d2), float(eps2))


def step(mh: MeshHandle, g: _Gas, xi, w, dt, f_in, Wc):
    """One explicit step; returns f_out and updates Wc in place."""
    xi = _f64(xi); w = _f64(w); f_in = _f64(f_in)
    assert Wc.dtype == np.float64 and Wc.flags.c_contiguous
    f_out = np.empty_like(f_in)
    rc = lib().om_step(mh.ptr, C.byref(g), xi.shape[0], _dp(xi), _dp(w), float(dt), _dp(f_in), _dp(f_out), _dp(Wc))
    if rc != 0:
        raise FloatingPointError(f"oracle step: non-positive density or temperature (status {rc})")
    return f_out


def colors(mh: MeshHandle):
    """Greedy colouring of the cells in index order; returns (color, ncolor)."""
    c = np.zeros(mh.mesh.Nc, dtype=np.int32)
    n = lib().om_colors(mh.ptr, _ip(c))
    return c, n


def step_implicit(mh: MeshHandle, g: _Gas, xi, w, dt, f_in, Wc, color, ncolor, k_macro=60, k_micro=2):
    """One implicit (IUGKS) step; returns f_out and updates Wc in place."""
    xi = _f64(xi); w = _f64(w); f_in = _f64(f_in)
    color = np.ascontiguousarray(color, dtype=np.int32)
    assert Wc.dtype == np.float64 and Wc.flags.c_contiguous
    f_out = np.empty_like(f_in)
    rc = lib().om_step_implicit(mh.ptr, C.byref(g), xi.shape[0], _dp(xi), _dp(w), float(dt), _dp(f_in),
                                _dp(f_out), _dp(Wc), _ip(color), int(ncolor), int(k_macro), int(k_micro))
    if rc != 0:
        raise FloatingPointError(f"oracle implicit step: non-positive density or temperature (status {rc})")
    return f_out


def criterion(D, xi, w, f, Wc):
    xi = _f64(xi); w = _f64(w); f = _f64(f); Wc = _f64(Wc)
    Nc, nA, Nv = f.shape
    M = np.zeros(Nv)
    lib().om_criterion_nw(D, nA, Wc.shape[1], Nc, Nv, _dp(xi), _dp(w), _dp(f), _dp(Wc), _dp(M))
    return M


def adapt_tree(D, level, base, key, M, s, C1, C2, max_refine, cap=None, lcap=None):
    """Marks and the new tree; lcap: per-node refinement cap (zones), else max_refine."""
    level = np.ascontiguousarray(level, np.int32)
    base = np.ascontiguousarray(base, np.int32)
    key = np.ascontiguousarray(key, np.uint32)
    M = _f64(M)
    Nv = len(level)
    cap = cap or Nv * (1 << D)
    nl = np.zeros(cap, np.int32); nb = np.zeros(cap, np.int32); nk = np.zeros(cap, np.uint32)
    src = np.zeros(cap, np.int32); kind = np.zeros(cap, np.int32)
    lc = None if lcap is None else np.ascontiguousarray(lcap, np.int32)
    n = lib().om_adapt_tree(D, Nv, _ip(level), _ip(base), _up(key), _dp(M), float(s), float(C1), float(C2),
                            int(max_refine), None if lc is None else _ip(lc), int(cap), _ip(nl), _ip(nb),
                            _up(nk), _ip(src), _ip(kind))
    if n < 0:
        raise MemoryError("adapted tree exceeds the node capacity")
    return nl[:n].copy(), nb[:n].copy(), nk[:n].copy(), src[:n].copy(), kind[:n].copy()


def remap(D, f_old, src, kind):
    f_old = _f64(f_old)
    Nc, nA, Nv_old = f_old.shape
    src = np.ascontiguousarray(src, np.int32); kind = np.ascontiguousarray(kind, np.int32)
    f_new = np.zeros((Nc, nA, len(src)))
    lib().om_remap_n(D, nA, Nc, Nv_old, _dp(f_old), len(src), _ip(src), _ip(kind), _dp(f_new))
    return f_new


def correct(D, xi, w, Wc_target, f, iters=3, R=0.5):
    """Conservation correction in place; returns the remaining relative gap."""
    xi = _f64(xi); w = _f64(w); Wc_target = _f64(Wc_target)
    assert f.dtype == np.float64 and f.flags.c_contiguous
    Nc, Nv = f.shape[0], f.shape[-1]
    return lib().om_correct(D, Nc, Nv, _dp(xi), _dp(w), R, iters, _dp(Wc_target), _dp(f))


def paper_parameters(D, Ma, gamma, T_inf=1.0, T_w=1.0, direction=(1.0, 0.0, 0.0), h_std=0.6, rdv_sigma=4.0,
                     separated=False, R=0.5):
    """Adaptive parameters of Sec. 3.5 from the flow data, step by step:
    sigma = sqrt(R T) for T_inf, the total temperature T_0 (Eq.
    totaltemperature) and T_w; the velocity domain of radius R_dv = rdv_sigma
    sigma_0 about 0.4 U_inf; L_std the least level with 2^L >= 2 R_dv / h_std,
    L_max = L_std, h_inf = 2 R_dv / 2^L_max; L_w, L_min and L_sep by their
    case rules; the three zones; C1 from the fitted law (Eq. C1_Ma) and
    C2 = k_sigma C1 (Eq. c2c1).  The base forest is read as the level-L_min
    mesh of the root element, so levels in the returned tree fields count from
    L_min (reading R21)."""
    sig_inf = math.sqrt(R * T_inf)
    T0 = T_inf * (1.0 + 0.5 * (gamma - 1.0) * Ma * Ma)
    sig0 = math.sqrt(R * T0)
    sigw = math.sqrt(R * T_w)
    speed = Ma * math.sqrt(gamma * R * T_inf)
    norm = math.sqrt(sum(direction[d] * direction[d] for d in range(D)))
    U = [speed * (direction[d] / norm) for d in range(D)]
    R_dv = rdv_sigma * sig0
    L_max = 0
    while 2.0 ** L_max < 2.0 * R_dv / h_std:
        L_max += 1
    h_inf = 2.0 * R_dv / 2 ** L_max
    L_w = L_max if T_w / T_inf < 4.0 else L_max - 1
    L_min = min(4 if (D == 2 and Ma > 5.0) else 3, L_max)
    L_sep = max(L_min, L_w - 1)
    centre = [0.4 * U[d] for d in range(D)]
    zones = [(tuple(U), 0.0, 3.0 * sig_inf, L_max - L_min),
             (tuple([0.0] * D), 0.0, 3.0 * sigw, max(0, L_w - L_min))]
    if separated:
        zones.append((tuple([0.0] * D), 3.0 * sigw, 5.0 * sigw, L_sep - L_min))
    C1 = 13.749 * math.pow(Ma, -1.465)
    return dict(T0=T0, sigma_inf=sig_inf, sigma_0=sig0, sigma_w=sigw, U=tuple(U), R_dv=R_dv, L_max=L_max,
                h_inf=h_inf, L_w=L_w, L_min=L_min, L_sep=L_sep,
                base=tuple([2 ** L_min] * D), vlo=tuple(centre[d] - R_dv for d in range(D)),
                vhi=tuple(centre[d] + R_dv for d in range(D)), max_refine=L_max - L_min, zones=zones,
                outside=0, init_refine=max(0, L_w - 1 - L_min), C1=C1, C2=3.3546e-4 * C1)


def node_caps(D, xi, zones, outside, max_refine):
    """Largest level each node may split to: the largest level of the zones
    whose ring r_in^2 <= |xi - c|^2 < r_out^2 holds the node centre, else
    `outside`; max_refine for every node when there are no zones."""
    Nv = len(xi)
    if not zones:
        return np.full(Nv, max_refine, np.int32)
    cap = np.full(Nv, outside, np.int32)
    for c, r_in, r_out, level in zones:
        d2 = np.zeros(Nv)
        for d in range(D):
            t = xi[:, d] - c[d]
            d2 = d2 + t * t
        inside = (d2 >= r_in * r_in) & (d2 < r_out * r_out)
        cap[inside] = np.maximum(cap[inside], level)
    return cap


def conserved_from_primitive(D, Wp, R=0.5):
    """rho, rho U, rho E with rho E = rho U^2 / 2 + (3/2) rho R T (monatomic)."""
    Wp = _f64(Wp)
    Wc = np.zeros_like(Wp)
    rho = Wp[..., 0]
    U = Wp[..., 1:1 + D]
    Wc[..., 0] = rho
    Wc[..., 1:1 + D] = rho[..., None] * U
    Wc[..., D + 1] = 0.5 * rho * (U * U).sum(-1) + 1.5 * rho * R * Wp[..., D + 1]
    return Wc


def primitive_from_conserved(D, Wc, R=0.5):
    """rho, U, T from rho, rho U, rho E (monatomic, inverse of the above)."""
    Wc = _f64(Wc)
    Wp = np.zeros_like(Wc)
    rho = Wc[..., 0]
    Wp[..., 0] = rho
    Wp[..., 1:1 + D] = Wc[..., 1:1 + D] / rho[..., None]
    m2 = (Wc[..., 1:1 + D] ** 2).sum(-1)
    Wp[..., D + 1] = (Wc[..., D + 1] - 0.5 * m2 / rho) / (1.5 * rho * R)
    return Wp


# ---------------------------------------------------------------------------
# whole-run driver
# ---------------------------------------------------------------------------
class Run:
    """Oracle state for one workload: velocity forest, f, carried W."""

    def __init__(self, wl, limiter=None, corr_iters=3, build_tree=True):
        self.wl = wl
        self.D = wl.D
        self.mh = MeshHandle(wl.mesh)
        self.rykov = getattr(wl, "model", "shakhov") == "rykov"
        self.g = gas(R=0.5, Pr=wl.Pr, omega=wl.omega, Kn=wl.Kn,
                     limiter=wl.limiter if limiter is None else limiter,
                     model="rykov" if self.rykov else "shakhov", Zrot=getattr(wl, "Zrot", RYKOV_ZROT))
        self.corr_iters = corr_iters
        if getattr(wl, "flow", None) is not None:
            fl = wl.flow
            self.p = paper_parameters(self.D, fl.Ma, fl.gamma, fl.T_inf, fl.T_w, fl.dir, fl.h_std, fl.rdv_sigma,
                                      fl.separated)
        else:
            self.p = dict(base=tuple(wl.base), vlo=tuple(wl.vlo), vhi=tuple(wl.vhi), max_refine=wl.max_refine,
                          zones=[], outside=0, init_refine=0, C1=wl.C1, C2=wl.C2)
        self.nb = np.array(self.p["base"], np.int32)
        self.s = float(np.prod(self.p["base"]))     # uniform-share normalisation (R10)
        self.level, self.base, self.key = forest_base(self.D, self.nb)
        self._geom()
        if build_tree:
            self.initial_tree()
        self.f = None
        self.Wc = None

    def _geom(self):
        self.xi, self.w = forest_geom(self.D, self.nb, self.p["vlo"], self.p["vhi"], self.level, self.base, self.key)
        self.ncap = node_caps(self.D, self.xi, self.p["zones"], self.p["outside"], self.p["max_refine"])

    def _marks(self, M):
        p = self.p
        return adapt_tree(self.D, self.level, self.base, self.key, M, self.s, p["C1"], p["C2"], p["max_refine"],
                          lcap=self.ncap)

    @property
    def Nv(self):
        return len(self.level)

    # model-dependent pieces: Shakhov (G[, H]; W = rho, rho U, rho E) or
    # Rykov (G[, H], R; W adds rho E_rot)
    def _init_f(self, Wp, amp=0.0, seed=12345):
        if self.rykov:
            return maxwell_init_rykov(self.D, self.xi, Wp, amp=amp, seed=seed)
        return maxwell_init(self.D, self.xi, Wp, amp=amp, seed=seed)

    def _moments(self, f):
        if self.rykov:
            return moments_rykov(self.D, self.xi, self.w, f)[0]
        return moments(self.D, self.xi, self.w, f)[0]

    def _cons(self, Wp):
        return conserved_rykov(self.D, Wp) if self.rykov else conserved_from_primitive(self.D, Wp)

    def _prim(self, Wc):
        return primitive_rykov(self.D, Wc) if self.rykov else primitive_from_conserved(self.D, Wc)

    def initial_tree(self):
        """Step-0 AVS (Sec. 3.5, steps 1-3; reading R13): adapt on the two
        pseudo cells g^eq(W_inf) and g^eq(rho_inf, 0, T_inf) until stable."""
        D = self.D
        Winf = np.array(self.wl.W_inf, dtype=np.float64)
        W0 = Winf.copy(); W0[1:1 + D] = 0.0
        Wp = np.stack([Winf, W0])
        Wc = self._cons(Wp)
        for _ in range(self.p["init_refine"]):         # step 2: split every element
            nl, nb, nk, _, _ = adapt_tree(D, self.level, self.base, self.key, np.full(self.Nv, np.inf), self.s,
                                          0.0, -1.0, self.p["max_refine"])
            self.level, self.base, self.key = nl, nb, nk
            self._geom()
        for _ in range(max(1, self.p["max_refine"])):
            f = self._init_f(Wp)
            M = criterion(D, self.xi, self.w, f, Wc)
            nl, nb, nk, src, kind = self._marks(M)
            changed = len(nl) != self.Nv or np.any(nl != self.level) or np.any(nk != self.key)
            self.level, self.base, self.key = nl, nb, nk
            self._geom()
            if not changed:
                break

    def init_field(self, Wp=None, amp=0.0, seed=12345):
        Wp = self.wl.W_init if Wp is None else Wp
        self.f = self._init_f(Wp, amp=amp, seed=seed)
        self.Wc = self._moments(self.f)

    def dt(self, cfl=None):
        return (self.wl.cfl if cfl is None else cfl) * dt_unit(self.mh, self.xi)

    def step(self, dt):
        self.f = step(self.mh, self.g, self.xi, self.w, dt, self.f, self.Wc)

    def step_implicit(self, dt, k_macro=60, k_micro=2, color=None):
        """IUGKS step (Sec. 2.3.1): macro PRSGS then micro SGS sweeps."""
        if color is None:
            if not hasattr(self, "_colors"):
                self._colors = colors(self.mh)
            color, nc = self._colors
        else:
            nc = int(np.max(color)) + 1
        self.f = step_implicit(self.mh, self.g, self.xi, self.w, dt, self.f, self.Wc, color, nc, k_macro, k_micro)

    def adapt(self, Wc_override=None, correct_f=True, bypass=False):
        """One adaptation: criterion on the moments of f (Eq. 7), marks, new
        tree, consanguinity remap, conservation correction (Secs. 3.2-3.4).
        With bypass, f on the new mesh is g^eq of the carried W instead
        (the bypass for weakly non-equilibrium flows, end of Sec. 3.3)."""
        D = self.D
        Wf = self._moments(self.f)
        Wcrit = Wf if Wc_override is None else Wc_override
        M = criterion(D, self.xi, self.w, self.f, Wcrit)
        nl, nb, nk, src, kind = self._marks(M)
        f_new = None if bypass else remap(D, self.f, src, kind)
        self.level, self.base, self.key = nl, nb, nk
        self._geom()
        gap = 0.0
        if bypass:
            f_new = self._init_f(self._prim(self.Wc))
        elif correct_f:
            corr = correct_rykov if self.rykov else correct
            gap = corr(D, self.xi, self.w, Wf, f_new, iters=self.corr_iters)
        self.f = f_new
        return dict(M=M, src=src, kind=kind, gap=gap, Nv=self.Nv)
