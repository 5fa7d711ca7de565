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
    # the options of the next rows are checked on the host too
    assert try_cfg(model=5) == -1
    assert try_cfg(model=1, Zrot=0.5) == -1              # Rykov: Z_rot >= 1
    assert try_cfg(model=1, Zrot=3.5, learned=1) != -1   # the diatomic gas takes the learned proposer
    assert try_cfg(nzones=9) == -1
    assert try_cfg(init_refine=2) == -1                  # beyond max_refine
    z = avs.Zone()
    z.r_in, z.r_out, z.level = 0.0, 1.0, 3              # level beyond max_refine
    cfgz = {"nzones": 1, "zones": (avs.Zone * avs.MAX_ZONES)(z)}
    assert try_cfg(**cfgz) == -1
    z.level, z.r_in, z.r_out = 1, 2.0, 1.0              # r_out must exceed r_in
    cfgz = {"nzones": 1, "zones": (avs.Zone * avs.MAX_ZONES)(z)}
    assert try_cfg(**cfgz) == -1


def test_paper_parameters_entry_point_on_host():
    """avs_paper_parameters is host code: it needs no GPU and rejects bad flow data."""
    from paper_2212_05645_gb300 import avs
    B.build()
    L = avs.load()
    sp = avs.FlowSpecS()
    sp.dim, sp.Ma, sp.gamma, sp.R, sp.T_inf, sp.T_w = 2, 5.0, 5.0 / 3.0, 0.5, 1.0, 1.0
    sp.dir[0], sp.h_std, sp.rdv_sigma = 1.0, 0.6, 4.0
    cfg = avs.Config()
    assert L.avs_paper_parameters(C.byref(sp), C.byref(cfg)) == 0
    assert (cfg.base[0], cfg.base[1], cfg.max_refine, cfg.init_refine, cfg.nzones) == (8, 8, 2, 1, 2)
    sp.Ma = -1.0
    assert L.avs_paper_parameters(C.byref(sp), C.byref(cfg)) == -1
    sp.Ma, sp.dir[0] = 5.0, 0.0                         # zero direction
    assert L.avs_paper_parameters(C.byref(sp), C.byref(cfg)) == -1


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: with the library missing, loading raises."""
    from paper_2212_05645_gb300 import avs
    monkeypatch.setattr(avs, "_lib", None)
    monkeypatch.setattr(avs, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        avs.load()


def test_binding_rejects_short_or_mistyped_buffers():
    """The binding checks every buffer it hands to the library for length,
    element type and contiguity before the call (the library reads or writes
    that many values through the pointer)."""
    import numpy as np
    import torch
    from paper_2212_05645_gb300.avs import _check_buf
    _check_buf(np.zeros((4, 5)), 20, "W")
    _check_buf(torch.zeros(20, dtype=torch.float64), 20, "W")
    _check_buf(None, 20, "W")
    for bad in (np.zeros((4, 4)), np.zeros((4, 5), np.float32), np.zeros((5, 4)).T,
                torch.zeros(19, dtype=torch.float64), torch.zeros(20, dtype=torch.float32),
                torch.zeros((5, 8), dtype=torch.float64)[:, :4], [0.0] * 20):
        with pytest.raises(ValueError):
            _check_buf(bad, 20, "W")


PARAM_FLOWS = [(2, dict(Ma=5.0)),
               (2, dict(Ma=8.0, separated=True)),
               (2, dict(Ma=20.2, gamma=1.4, T_w=290.0 / 13.32, dir=(0.9848, 0.1736, 0.0))),
               (3, dict(Ma=5.45, gamma=1.4, rdv_sigma=7.0)),
               (3, dict(Ma=4.25, gamma=1.4, dir=(1.0, 0.0, 1.0)))]


@pytest.mark.parametrize("D,kw", PARAM_FLOWS)
def test_library_paper_parameters_on_host(D, kw):
    """avs_paper_parameters is host code of the library (Sec. 3.5 rules): it
    runs without a GPU and gives the oracle's velocity space, zones and
    thresholds bit for bit."""
    import oracle as O
    from paper_2212_05645_gb300 import avs
    B.build()
    flow = wl.FlowSpec(**kw)
    g = avs.paper_parameters(D, flow)
    o = O.paper_parameters(D, flow.Ma, flow.gamma, flow.T_inf, flow.T_w, flow.dir, flow.h_std, flow.rdv_sigma,
                           flow.separated)
    for k in ("base", "vlo", "vhi", "max_refine", "outside", "init_refine", "C1", "C2"):
        assert g[k] == o[k], (k, g[k], o[k])
    assert len(g["zones"]) == len(o["zones"])
    for zg, zo in zip(g["zones"], o["zones"]):
        assert zg == (tuple(zo[0]), zo[1], zo[2], zo[3])


def test_bad_meshes_rejected_on_host():
    """The face list is checked on the host before any device work: cells out
    of range, a face joining a cell to itself, more than six faces on a cell,
    unknown boundary types, non-positive boundary temperatures and cell
    volumes are AVS_EINVAL; the untouched mesh passes the checks (and then
    fails only for want of a GPU here)."""
    from paper_2212_05645_gb300 import avs
    B.build()
    L = avs.load()
    w = wl.cavity(n=4)

    def try_mesh(edit=None):
        m = w.mesh
        a = {k: np.array(getattr(m, k), copy=True) for k in ("faceL", "faceR", "An", "rL", "rR", "vol", "bc")}
        if edit:
            edit(a)
        cfg = avs.Config()
        cfg.dim = 2; cfg.base[0] = cfg.base[1] = 4; cfg.max_refine = 1
        cfg.vlo[0] = cfg.vlo[1] = -2.0; cfg.vhi[0] = cfg.vhi[1] = 2.0
        cfg.R = 0.5; cfg.Pr = 2 / 3; cfg.omega = 0.81; cfg.Kn = 0.1; cfg.T_ref = 1.0
        cfg.C1 = 1.0; cfg.C2 = 1e-4; cfg.W_inf[0] = 1.0; cfg.W_inf[3] = 1.0; cfg.limiter = 1; cfg.lim_K = 0.3
        cfg.corr_iters = 3
        dp = C.POINTER(C.c_double); ip = C.POINTER(C.c_int)
        ms = avs.MeshS(m.D, m.Nc, len(a["faceL"]), a["bc"].shape[0], a["faceL"].ctypes.data_as(ip),
                       a["faceR"].ctypes.data_as(ip), a["An"].ctypes.data_as(dp), a["rL"].ctypes.data_as(dp),
                       a["rR"].ctypes.data_as(dp), a["vol"].ctypes.data_as(dp), a["bc"].ctypes.data_as(dp))
        h = C.c_void_p()
        return L.avs_create(C.byref(cfg), C.byref(ms), None, C.byref(h))

    def setv(key, idx, val):
        def e(a):
            a[key][idx] = val
        return e

    nc = w.mesh.Nc
    inner = int(np.nonzero(w.mesh.faceR >= 0)[0][0])
    assert try_mesh() != -1
    assert try_mesh(setv("faceL", 0, nc)) == -1                     # cell index out of range
    assert try_mesh(setv("faceL", 0, -1)) == -1
    assert try_mesh(setv("faceR", inner, nc)) == -1
    assert try_mesh(setv("faceR", 0, -1 - w.mesh.bc.shape[0])) == -1  # boundary row out of range
    assert try_mesh(setv("faceR", inner, int(w.mesh.faceL[inner]))) == -1   # a cell joined to itself
    assert try_mesh(setv("bc", (0, 0), 7.0)) == -1                  # unknown boundary type
    assert try_mesh(setv("bc", (0, 5), 0.0)) == -1                  # boundary temperature must be positive
    assert try_mesh(setv("vol", 3, 0.0)) == -1                      # non-positive cell volume

    def seven_faces(a):
        # three more faces between cells 0 and 1: cell 0 then has more than six
        for k in ("faceL", "faceR", "An", "rL", "rR"):
            extra = np.repeat(a[k][inner:inner + 1], 3, axis=0)
            a[k] = np.ascontiguousarray(np.concatenate([a[k], extra]))
    assert try_mesh(seven_faces) == -1
