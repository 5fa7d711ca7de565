"""Thin Python binding of the C ABI in ``include/avs.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA
library ``_build/libavs_gb300.so``.  Loading fails loudly when the library
has not been built; there is no CPU fallback.  Device buffers are torch CUDA
tensors (``data_ptr``), streams are torch streams (``cuda_stream``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as wlmod

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libavs_gb300.so")
_lib = None

AVS_OK = 0
STATUS = {0: "AVS_OK", -1: "AVS_EINVAL", -2: "AVS_ENOMEM", -3: "AVS_ECUDA", -4: "AVS_ETIMEOUT",
          -5: "AVS_ENUMERIC", -6: "AVS_ENOTCONV", -7: "AVS_ECAPACITY"}
FP64, MIXED = 0, 1

EXPORTED = ["avs_create", "avs_destroy", "avs_last_error", "avs_num_nodes", "avs_num_cells", "avs_init_field",
            "avs_dt", "ugks_step", "ugks_step_dt", "ugks_step_implicit", "avs_adapt", "avs_moments", "avs_f_moments", "avs_set_W",
            "avs_criterion", "avs_get_tree", "avs_get_f", "avs_get_f_cells", "avs_set_f", "avs_sync",
            "avs_kernel_launches",
            "avs_mlp_set_params", "avs_mlp_get_params", "avs_mlp_forward", "avs_mlp_grad", "avs_features",
            "avs_mlp_train", "avs_mlp_check_set", "avs_measure_fma_peak", "avs_grid_barrier_check", "avs_stage_wait_check",
            "avs_paper_parameters"]
MLP_NPARAM = 4996


class AVSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


MAX_ZONES = 4


class Zone(C.Structure):
    _fields_ = [("c", C.c_double * 3), ("r_in", C.c_double), ("r_out", C.c_double), ("level", C.c_int)]


class Config(C.Structure):
    _fields_ = [("dim", C.c_int), ("base", C.c_int * 3), ("max_refine", C.c_int),
                ("vlo", C.c_double * 3), ("vhi", C.c_double * 3), ("precision", C.c_int),
                ("learned", C.c_int), ("R", C.c_double), ("Pr", C.c_double), ("omega", C.c_double),
                ("Kn", C.c_double), ("T_ref", C.c_double), ("C1", C.c_double), ("C2", C.c_double),
                ("W_inf", C.c_double * 5), ("limiter", C.c_int), ("lim_K", C.c_double),
                ("corr_iters", C.c_int), ("max_nodes", C.c_int), ("learned_full_every", C.c_int),
                ("nzones", C.c_int), ("zone_outside_level", C.c_int), ("zones", Zone * MAX_ZONES),
                ("init_refine", C.c_int), ("model", C.c_int), ("Zrot", C.c_double)]


class FlowSpecS(C.Structure):
    _fields_ = [("dim", C.c_int), ("Ma", C.c_double), ("gamma", C.c_double), ("R", C.c_double),
                ("T_inf", C.c_double), ("T_w", C.c_double), ("dir", C.c_double * 3), ("h_std", C.c_double),
                ("rdv_sigma", C.c_double), ("separated", C.c_int)]


class MeshS(C.Structure):
    _fields_ = [("dim", C.c_int), ("Nc", C.c_int), ("Nf", C.c_int), ("nbc", C.c_int),
                ("faceL", C.POINTER(C.c_int)), ("faceR", C.POINTER(C.c_int)),
                ("An", C.POINTER(C.c_double)), ("rL", C.POINTER(C.c_double)),
                ("rR", C.POINTER(C.c_double)), ("vol", C.POINTER(C.c_double)),
                ("bc", C.POINTER(C.c_double))]


class AdaptStats(C.Structure):
    _fields_ = [("Nv_old", C.c_int), ("Nv", C.c_int), ("splits", C.c_int), ("merges", C.c_int),
                ("gap", C.c_double), ("checked_cells", C.c_int), ("missed_nodes", C.c_int), ("full", C.c_int)]


class AdaptOpts(C.Structure):
    _fields_ = [("W_override", C.c_void_p), ("W_is_device", C.c_int), ("skip_correction", C.c_int),
                ("force_full", C.c_int), ("bypass", C.c_int)]


def load():
    """Loads the CUDA library; raises if it is missing (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run paper_2212_05645_gb300.build.build())")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.c_void_p, C.c_void_p
    sig = {
        "avs_create": (C.c_int, [C.POINTER(Config), C.POINTER(MeshS), vp, C.POINTER(vp)]),
        "avs_destroy": (None, [vp]),
        "avs_last_error": (C.c_char_p, [vp]),
        "avs_num_nodes": (C.c_int, [vp]),
        "avs_num_cells": (C.c_int, [vp]),
        "avs_init_field": (C.c_int, [vp, dp, C.c_int, C.c_double, C.c_uint64]),
        "avs_dt": (C.c_int, [vp, C.c_double, C.POINTER(C.c_double)]),
        "ugks_step": (C.c_int, [vp, C.c_int, C.c_double, C.POINTER(C.c_double)]),
        "ugks_step_dt": (C.c_int, [vp, C.c_int, C.c_double]),
        "avs_adapt": (C.c_int, [vp, C.POINTER(AdaptOpts), C.POINTER(AdaptStats)]),
        "avs_moments": (C.c_int, [vp, dp, dp, C.c_int]),
        "avs_f_moments": (C.c_int, [vp, dp, C.c_int]),
        "avs_set_W": (C.c_int, [vp, dp, C.c_int]),
        "avs_criterion": (C.c_int, [vp, dp, C.c_int, dp, C.c_int]),
        "avs_get_tree": (C.c_int, [vp, ip, ip, ip, dp, dp]),
        "avs_get_f": (C.c_int, [vp, dp, C.c_int]),
        "ugks_step_implicit": (C.c_int, [vp, C.c_int, C.c_double, C.c_int, C.c_int]),
        "avs_get_f_cells": (C.c_int, [vp, C.POINTER(C.c_int), C.c_int, dp]),
        "avs_set_f": (C.c_int, [vp, dp, C.c_int]),
        "avs_sync": (C.c_int, [vp]),
        "avs_kernel_launches": (C.c_uint64, [vp]),
        "avs_mlp_set_params": (C.c_int, [vp, dp]),
        "avs_mlp_get_params": (C.c_int, [vp, dp]),
        "avs_mlp_forward": (C.c_int, [vp, dp, C.c_int, dp]),
        "avs_mlp_grad": (C.c_int, [vp, dp, dp, C.c_int, C.c_float, dp, C.POINTER(C.c_float)]),
        "avs_features": (C.c_int, [vp, dp, dp]),
        "avs_mlp_train": (C.c_int, [vp, C.c_int, C.c_float, C.POINTER(C.c_float)]),
        "avs_mlp_check_set": (C.c_int, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "avs_measure_fma_peak": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double)]),
        "avs_grid_barrier_check": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
        "avs_stage_wait_check": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int)]),
        "avs_paper_parameters": (C.c_int, [C.POINTER(FlowSpecS), C.POINTER(Config)]),
    }
    for name, (rt, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = rt
        fn.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """(pointer, is_device) of a numpy array or a torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data, 0
    # torch tensor
    return a.data_ptr(), int(a.is_cuda)


def _check_buf(a, n, name):
    """Reject a buffer that is not at least n contiguous float64 values (the
    library reads or writes n values through its pointer)."""
    if a is None:
        return
    if _is_torch(a):
        import torch
        ok = a.dtype == torch.float64 and a.is_contiguous() and a.numel() >= n
    else:
        ok = isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.size >= n
    if not ok:
        raise ValueError(f"{name}: need a contiguous float64 buffer of at least {n} values")


def _cur_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return None


class AVS:
    """One UGKS/AVS problem on the GPU (a context of the C library)."""

    def __init__(self, wl: "wlmod.Workload", precision=None, limiter=None, corr_iters=3, max_nodes=0,
                 stream=None, learned=None, full_every=4):
        L = load()
        self.wl = wl
        self.D = wl.D
        self.rykov = getattr(wl, "model", "shakhov") == "rykov"
        self.NA = (3 if wl.D == 2 else 2) if self.rykov else (2 if wl.D == 2 else 1)
        self.NW = wl.D + (3 if self.rykov else 2)
        m = wl.mesh
        self._mesh_keep = [m.faceL, m.faceR, m.An, m.rL, m.rR, m.vol, m.bc]
        dp = C.POINTER(C.c_double)
        ipt = C.POINTER(C.c_int)
        ms = MeshS(m.D, m.Nc, m.Nf, m.bc.shape[0], m.faceL.ctypes.data_as(ipt), m.faceR.ctypes.data_as(ipt),
                   m.An.ctypes.data_as(dp), m.rL.ctypes.data_as(dp), m.rR.ctypes.data_as(dp),
                   m.vol.ctypes.data_as(dp), m.bc.ctypes.data_as(dp))
        prec = wl.precision if precision is None else precision
        cfg = Config()
        cfg.dim = wl.D
        if wl.flow is None:
            for d in range(wl.D):
                cfg.base[d] = wl.base[d]
                cfg.vlo[d] = wl.vlo[d]
                cfg.vhi[d] = wl.vhi[d]
            cfg.max_refine = wl.max_refine
            cfg.C1 = wl.C1
            cfg.C2 = wl.C2
        cfg.precision = MIXED if prec in ("mixed", MIXED) else FP64
        cfg.learned = int(wl.learned if learned is None else learned)
        cfg.R = wlmod.R_GAS
        cfg.Pr = wl.Pr
        cfg.omega = wl.omega
        cfg.Kn = wl.Kn
        cfg.T_ref = 1.0
        for j, v in enumerate(wl.W_inf):
            cfg.W_inf[j] = v
        cfg.limiter = wl.limiter if limiter is None else limiter
        cfg.lim_K = 0.3
        cfg.corr_iters = corr_iters
        cfg.max_nodes = max_nodes
        cfg.learned_full_every = full_every
        cfg.model = 1 if self.rykov else 0
        cfg.Zrot = float(getattr(wl, "Zrot", 3.5))
        if wl.flow is not None:
            _fill_paper_parameters(L, wl.D, wl.flow, cfg)
        self.cfg = cfg
        self.stream = _cur_stream() if stream is None else stream
        h = C.c_void_p()
        st = L.avs_create(C.byref(cfg), C.byref(ms), self.stream, C.byref(h))
        if st != AVS_OK:
            raise AVSError(st, "avs_create failed (see stderr)")
        self.h = h
        self.L = L

    # ------------------------------------------------------------------ helpers
    def _ck(self, st):
        if st != AVS_OK:
            raise AVSError(st, self.L.avs_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.avs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def Nv(self):
        return self.L.avs_num_nodes(self.h)

    @property
    def Nc(self):
        return self.L.avs_num_cells(self.h)

    # ------------------------------------------------------------------ API
    def init_field(self, Wp=None, amp=0.0, seed=12345):
        """Maxwellian start from primitive W per cell (rho, U, T; the Rykov
        model also takes T_r as a last column, else T_r = T)."""
        Wp = np.ascontiguousarray(self.wl.W_init if Wp is None else Wp, dtype=np.float64) \
            if not _is_torch(Wp) else Wp
        if self.rykov and Wp.shape[1] == self.D + 2:
            if _is_torch(Wp):
                import torch
                Wp = torch.cat([Wp, Wp[:, self.D + 1:self.D + 2]], dim=1).contiguous()
            else:
                Wp = np.ascontiguousarray(np.concatenate([Wp, Wp[:, self.D + 1:self.D + 2]], axis=1))
        _check_buf(Wp, self.Nc * self.NW, "Wp")
        p, dev = _ptr(Wp)
        self._ck(self.L.avs_init_field(self.h, p, dev, float(amp), int(seed)))

    def dt(self, cfl=None):
        out = C.c_double()
        self._ck(self.L.avs_dt(self.h, float(self.wl.cfl if cfl is None else cfl), C.byref(out)))
        return out.value

    def step_implicit(self, nsteps=1, dt=None, cfl=None, k_macro=60, k_micro=2):
        """Implicit (IUGKS) steps; dt defaults to cfl (default the workload's) times the explicit bound."""
        if dt is None:
            dt = self.dt(cfl)
        self._ck(self.L.ugks_step_implicit(self.h, int(nsteps), float(dt), int(k_macro), int(k_micro)))
        return dt

    def grid_barrier_check(self, blocks, rounds, short_by=0):
        """Barriers passed (summed over blocks) by the bounded grid-barrier
        self-test; raises AVSError(AVS_ETIMEOUT) when short_by > 0."""
        out = C.c_int()
        self._ck(self.L.avs_grid_barrier_check(self.h, int(blocks), int(rounds), int(short_by), C.byref(out)))
        return out.value

    def stage_wait_check(self, arrive=True):
        """1 when a bulk copy completed the staged kernels' bounded mbarrier
        wait with the right bytes; raises AVSError(AVS_ETIMEOUT) when nothing
        arrives (arrive=False)."""
        out = C.c_int()
        self._ck(self.L.avs_stage_wait_check(self.h, int(bool(arrive)), C.byref(out)))
        return out.value

    def step(self, nsteps=1, dt=None, cfl=None):
        if dt is not None:
            self._ck(self.L.ugks_step_dt(self.h, int(nsteps), float(dt)))
            return dt
        out = C.c_double()
        self._ck(self.L.ugks_step(self.h, int(nsteps), float(self.wl.cfl if cfl is None else cfl), C.byref(out)))
        return out.value

    def adapt(self, W_override=None, skip_correction=False, force_full=False, bypass=False):
        o = AdaptOpts()
        keep = None
        if W_override is not None:
            keep = W_override if _is_torch(W_override) else np.ascontiguousarray(W_override, np.float64)
            _check_buf(keep, self.Nc * self.NW, "W_override")
            p, dev = _ptr(keep)
            o.W_override = p
            o.W_is_device = dev
        o.skip_correction = int(skip_correction)
        o.force_full = int(force_full)
        o.bypass = int(bypass)
        s = AdaptStats()
        self._ck(self.L.avs_adapt(self.h, C.byref(o), C.byref(s)))
        return {k: getattr(s, k) for k, _ in AdaptStats._fields_}

    def moments(self, out_W=None, out_q=None):
        """Carried conserved W and heat flux q of f (host numpy by default)."""
        if out_W is None and out_q is None:
            out_W = np.zeros((self.Nc, self.NW))
            out_q = np.zeros((self.Nc, self.D))
        _check_buf(out_W, self.Nc * self.NW, "out_W")
        _check_buf(out_q, self.Nc * self.D, "out_q")
        pW, dW = _ptr(out_W)
        pq, dq = _ptr(out_q)
        if out_W is not None and out_q is not None and dW != dq:
            raise ValueError("out_W and out_q: both on the host or both on the device")
        self._ck(self.L.avs_moments(self.h, pW, pq, dW or dq))
        return out_W, out_q

    def f_moments(self):
        out = np.zeros((self.Nc, self.NW))
        self._ck(self.L.avs_f_moments(self.h, out.ctypes.data, 0))
        return out

    def set_W(self, Wc):
        Wc = np.ascontiguousarray(Wc, np.float64)
        _check_buf(Wc, self.Nc * self.NW, "Wc")
        self._ck(self.L.avs_set_W(self.h, Wc.ctypes.data, 0))

    def criterion(self, Wc=None):
        M = np.zeros(self.Nv)
        if Wc is not None:
            Wc = np.ascontiguousarray(Wc, np.float64)
            _check_buf(Wc, self.Nc * self.NW, "Wc")
        self._ck(self.L.avs_criterion(self.h, None if Wc is None else Wc.ctypes.data, 0, M.ctypes.data, 0))
        return M

    def tree(self):
        n = self.Nv
        level = np.zeros(n, np.int32)
        base = np.zeros(n, np.int32)
        key = np.zeros(n, np.uint32)
        xi = np.zeros((n, self.D))
        w = np.zeros(n)
        self._ck(self.L.avs_get_tree(self.h, level.ctypes.data, base.ctypes.data, key.ctypes.data,
                                     xi.ctypes.data, w.ctypes.data))
        return dict(level=level, base=base, key=key, xi=xi, w=w)

    def get_f(self, out=None):
        if out is None:
            out = np.zeros((self.Nc, self.NA, self.Nv))
        _check_buf(out, self.Nc * self.NA * self.Nv, "out")
        p, dev = _ptr(out)
        self._ck(self.L.avs_get_f(self.h, p, dev))
        return out

    def get_f_cells(self, cells):
        """FP64 copy of f for the listed cells, [n][nA][Nv] (host)."""
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        out = np.zeros((len(cells), self.NA, self.Nv))
        self._ck(self.L.avs_get_f_cells(self.h, cells.ctypes.data_as(C.POINTER(C.c_int)), len(cells),
                                        out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def set_f(self, f):
        if not _is_torch(f):
            f = np.ascontiguousarray(f, np.float64)
            assert f.shape == (self.Nc, self.NA, self.Nv), f.shape
        _check_buf(f, self.Nc * self.NA * self.Nv, "f")
        p, dev = _ptr(f)
        self._ck(self.L.avs_set_f(self.h, p, dev))

    def sync(self):
        self._ck(self.L.avs_sync(self.h))

    @property
    def launches(self):
        return int(self.L.avs_kernel_launches(self.h))

    # ------------------------------------------------------------------ learned proposer
    def mlp_set_params(self, P):
        P = np.ascontiguousarray(P, np.float32).reshape(-1)
        assert P.size == MLP_NPARAM
        self._ck(self.L.avs_mlp_set_params(self.h, P.ctypes.data))

    def mlp_get_params(self):
        P = np.zeros(MLP_NPARAM, np.float32)
        self._ck(self.L.avs_mlp_get_params(self.h, P.ctypes.data))
        return P

    def mlp_forward(self, X):
        X = np.ascontiguousarray(X, np.float32)
        out = np.zeros((X.shape[0], 4), np.float32)
        self._ck(self.L.avs_mlp_forward(self.h, X.ctypes.data, X.shape[0], out.ctypes.data))
        return out

    def mlp_grad(self, X, Y, lr=0.0):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.float32)
        g = np.zeros(MLP_NPARAM, np.float32)
        loss = C.c_float()
        self._ck(self.L.avs_mlp_grad(self.h, X.ctypes.data, Y.ctypes.data, X.shape[0], float(lr), g.ctypes.data,
                                     C.byref(loss)))
        return g, loss.value

    def features(self):
        X = np.zeros((self.Nc, 8), np.float32)
        Y = np.zeros((self.Nc, 4), np.float32)
        self._ck(self.L.avs_features(self.h, X.ctypes.data, Y.ctypes.data))
        return X, Y

    def mlp_train(self, iters, lr=0.1):
        loss = C.c_float()
        self._ck(self.L.avs_mlp_train(self.h, int(iters), float(lr), C.byref(loss)))
        return loss.value

    def check_set(self):
        """Cells of the last learned adaptation's check set (sorted), or None
        when that call evaluated none."""
        n = C.c_int()
        self._ck(self.L.avs_mlp_check_set(self.h, None, C.byref(n)))
        if n.value < 0:
            return None
        cells = np.zeros(max(1, n.value), np.int32)
        self._ck(self.L.avs_mlp_check_set(self.h, cells.ctypes.data_as(C.POINTER(C.c_int)), C.byref(n)))
        return np.sort(cells[:n.value])


def _fill_paper_parameters(L, D, flow, cfg):
    sp = FlowSpecS()
    sp.dim = D
    sp.Ma = flow.Ma
    sp.gamma = flow.gamma
    sp.R = wlmod.R_GAS
    sp.T_inf = flow.T_inf
    sp.T_w = flow.T_w
    for d in range(3):
        sp.dir[d] = flow.dir[d] if d < len(flow.dir) else 0.0
    sp.h_std = flow.h_std
    sp.rdv_sigma = flow.rdv_sigma
    sp.separated = int(flow.separated)
    st = L.avs_paper_parameters(C.byref(sp), C.byref(cfg))
    if st != AVS_OK:
        raise AVSError(st, "avs_paper_parameters")


def paper_parameters(D, flow):
    """The library's Sec. 3.5 parameters for a workload's FlowSpec, as a dict
    (tree levels counted from the base forest)."""
    cfg = Config()
    _fill_paper_parameters(load(), D, flow, cfg)
    zones = [(tuple(cfg.zones[z].c[:D]), cfg.zones[z].r_in, cfg.zones[z].r_out, cfg.zones[z].level)
             for z in range(cfg.nzones)]
    return dict(base=tuple(cfg.base[:D]), vlo=tuple(cfg.vlo[:D]), vhi=tuple(cfg.vhi[:D]),
                max_refine=cfg.max_refine, zones=zones, outside=cfg.zone_outside_level,
                init_refine=cfg.init_refine, C1=cfg.C1, C2=cfg.C2)


def fma_peak_gflops(kind, iters=20000):
    """Measured FMA throughput of the current GPU in GFLOP/s; kind 0 FP32,
    1 FP64, 2 packed FP32 pairs (True / False still mean FP64 / FP32)."""
    out = C.c_double()
    st = load().avs_measure_fma_peak(int(kind), int(iters), C.byref(out))
    if st != AVS_OK:
        raise AVSError(st, "avs_measure_fma_peak")
    return out.value


def _is_torch(a):
    return a is not None and not isinstance(a, np.ndarray) and hasattr(a, "data_ptr")
