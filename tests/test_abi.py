"""The C-ABI library builds, loads without a GPU, exports every function that
include/avs.h declares, and rejects bad configurations before touching the
device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2212_05645_gb300 import build as B
from paper_2212_05645_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "avs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:avs_status|void|const char\s*\*|int|uint64_t)\s*\*?\s*([A-Za-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = C.CDLL(path)
    names = declared_functions()
    assert len(names) >= 18, names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in avs.h but not exported"
    from paper_2212_05645_gb300 import avs
    assert set(avs.EXPORTED) <= set(names)


def test_bad_configs_rejected_on_host():
    from paper_2212_05645_gb300 import avs
    B.build()
    L = avs.load()
    w = wl.cavity(n=4)

    def try_cfg(**kw):
        g = object.__new__(avs.AVS)
        cfg = avs.Config()
        cfg.dim = 2; cfg.base[0] = cfg.base[1] = 4; cfg.max_refine = 1
        cfg.vlo[0] = cfg.vlo[1] = -2.0; cfg.vhi[0] = cfg.vhi[1] = 2.0
        cfg.R = 0.5; cfg.Pr = 2 / 3; cfg.omega = 0.81; cfg.Kn = 0.1; cfg.T_ref = 1.0
        cfg.C1 = 1.0; cfg.C2 = 1e-4; cfg.W_inf[0] = 1.0; cfg.W_inf[3] = 1.0; cfg.limiter = 1; cfg.lim_K = 0.3
        cfg.corr_iters = 3
        for k, v in kw.items():
            setattr(cfg, k, v)
        m = w.mesh
        dp = C.POINTER(C.c_double); ip = C.POINTER(C.c_int)
        ms = avs.MeshS(m.D, m.Nc, m.Nf, m.bc.shape[0], m.faceL.ctypes.data_as(ip), m.faceR.ctypes.data_as(ip),
                       m.An.ctypes.data_as(dp), m.rL.ctypes.data_as(dp), m.rR.ctypes.data_as(dp),
                       m.vol.ctypes.data_as(dp), m.bc.ctypes.data_as(dp))
        h = C.c_void_p()
        return L.avs_create(C.byref(cfg), C.byref(ms), None, C.byref(h))

    assert try_cfg(dim=4) == -1
    assert try_cfg(C1=1e-5) == -1            # C1 must exceed C2
    assert try_cfg(precision=7) == -1
    assert try_cfg(limiter=5) == -1
    assert try_cfg(max_refine=20) == -1
    assert try_cfg(Kn=-1.0) == -1
