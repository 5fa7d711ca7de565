"""Sampled parity at the configurations' full sizes, in the launch
configuration the benchmark uses.

The GPU advances the whole mesh; for a few sampled cells (nearest to and
farthest from the body, the poles in 3D, seeded random ones) the oracle then
recomputes the same step on the patch of cells within two face steps of
them, from the same f (copied out of the GPU with avs_get_f_cells) and W.
One step of a cell depends only on that patch (pinned on the CPU by
test_step_locality_two_face_rings), so the sampled cells must agree with the
oracle to the tolerance of the form: 1e-12 relative in FP64, 1e-5 on the
macroscopic fields in the mixed form.
"""
import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl

from gpu_common import field_err, need_gpu, patch_mesh, rel_err, sample_cells

pytestmark = pytest.mark.gpu


def _sampled_step(avs, w, precision, pre_steps, tol_f, tol_W):
    g = avs.AVS(w, precision=precision, learned=False)
    g.init_field(amp=1e-3, seed=17)
    dt = g.dt()
    if pre_steps:
        g.step(pre_steps, dt=dt)
    t = sample_cells(w.mesh)
    sub, cells, pos = patch_mesh(w.mesh, t)
    f0 = g.get_f_cells(cells)
    W0 = np.ascontiguousarray(g.moments()[0][cells])
    xi, wq = g.tree()["xi"], g.tree()["w"]
    g.step(1, dt=dt)
    f1 = g.get_f_cells(t)
    W1 = g.moments()[0][t]
    gas = O.gas(R=0.5, Pr=w.Pr, omega=w.omega, Kn=w.Kn, limiter=w.limiter, model=w.model, Zrot=w.Zrot)
    fo = O.step(O.MeshHandle(sub), gas, xi, wq, dt, f0, W0)
    e = field_err(W1, W0[pos], w.D)
    assert max(e.values()) < tol_W, e
    assert rel_err(f1, fo[pos]) < tol_f
    g.close()


def test_cylinder_full_size_fp64_sampled():
    avs = need_gpu()
    _sampled_step(avs, wl.cylinder(precision="fp64"), "fp64", 3, 1e-12, 1e-12)


def test_cylinder_full_size_mixed_sampled():
    avs = need_gpu()
    _sampled_step(avs, wl.cylinder(precision="mixed"), "mixed", 20, 1e-5, 1e-5)


def test_wedge_full_size_mixed_sampled():
    avs = need_gpu()
    _sampled_step(avs, wl.blunt_wedge(precision="mixed", learned=False), "mixed", 20, 1e-5, 1e-5)


def test_sphere_full_size_mixed_sampled():
    """147456 cells x ~21k octree nodes (FP32 f of 12.6 GB per buffer)."""
    avs = need_gpu()
    _sampled_step(avs, wl.sphere(precision="mixed", learned=False), "mixed", 5, 1e-5, 1e-5)


def _rykov(w):
    w.model = "rykov"
    w.learned = False
    return w


def test_rykov_cylinder_full_size_fp64_sampled():
    """The cylinder with the diatomic gas (G, H, R arrays, rotational exchange)."""
    avs = need_gpu()
    _sampled_step(avs, _rykov(wl.cylinder(precision="fp64")), "fp64", 2, 1e-12, 1e-12)


def test_rykov_cylinder_full_size_mixed_sampled():
    avs = need_gpu()
    _sampled_step(avs, _rykov(wl.cylinder(precision="mixed")), "mixed", 10, 1e-5, 1e-5)


def test_zoned_cylinder_full_size_mixed_sampled():
    """The cylinder with the velocity space of the Sec. 3.5 rules."""
    avs = need_gpu()
    _sampled_step(avs, wl.cylinder_zones(precision="mixed"), "mixed", 20, 1e-5, 1e-5)
