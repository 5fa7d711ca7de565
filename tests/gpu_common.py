"""Shared helpers of the GPU parity tests (oracle side and CUDA side set up
from the same seeded inputs)."""
import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_05645_gb300 import build
    build.build()
    from paper_2212_05645_gb300 import avs
    return avs


def small_cylinder(n_theta=24, n_r=8, precision="fp64", C1=1.0, max_refine=2):
    w = wl.cylinder(n_theta=n_theta, n_r=n_r, C1=C1, max_refine=max_refine, precision=precision)
    return w


def small_sphere(precision="fp64"):
    return wl.sphere(n_r=4, n_theta=6, n_phi=6, C1=1.0, max_refine=1, precision=precision, learned=False)


def pair(w, avs, precision=None, amp=1e-3, seed=12345, limiter=None, corr_iters=3):
    """Oracle run and CUDA context with the same tree, f and W."""
    r = O.Run(w, limiter=limiter, corr_iters=corr_iters)
    r.init_field(amp=amp, seed=seed)
    g = avs.AVS(w, precision=precision, limiter=limiter, corr_iters=corr_iters)
    t = g.tree()
    assert np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
    g.set_f(r.f)
    g.set_W(r.Wc)
    return r, g


def rel_err(a, b):
    """max |a - b| / max |b| per leading index, then max."""
    a = np.asarray(a); b = np.asarray(b)
    axes = tuple(range(1, b.ndim))
    scale = np.abs(b).max(axis=axes, keepdims=True)
    scale[scale == 0] = 1.0
    return float((np.abs(a - b) / scale).max())


def field_err(Wg, Wo, D):
    """Macroscopic error by field: rho and E relative to their values,
    momentum relative to rho sqrt(2 R T) + |rho U| (the field's scale)."""
    rho = Wo[:, 0]
    e_rho = np.abs(Wg[:, 0] - rho) / np.abs(rho)
    m = Wo[:, 1:1 + D]
    RT = (Wo[:, D + 1] - 0.5 * (m * m).sum(1) / rho) / (1.5 * rho)
    mscale = np.sqrt((m * m).sum(1)) + rho * np.sqrt(2 * RT)
    e_m = np.abs(Wg[:, 1:1 + D] - m).max(1) / mscale
    e_E = np.abs(Wg[:, D + 1] - Wo[:, D + 1]) / np.abs(Wo[:, D + 1])
    return dict(rho=float(e_rho.max()), mom=float(e_m.max()), E=float(e_E.max()))
