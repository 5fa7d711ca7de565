"""The FP32 face kernel for velocity meshes beyond its shared-memory cache.

Above 5888 nodes in 2D (G and H) and 11776 in 3D the foot values of one face
no longer fit the 48 KB cache, and the interior faces stream their foot
values (in 2D also the node coordinates and weights) through shared memory
in stages of asynchronous bulk copies, 1024 nodes in 2D and 2048 in 3D;
boundary faces keep direct loads.  These
cases put walls and far-field boundaries beside the staged interior faces,
with node counts that end on a stage boundary, in a ragged last stage and
just past the 32-node padding, and compare with the FP64 oracle.
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl

from gpu_common import field_err, need_gpu, pair, rel_err

pytestmark = pytest.mark.gpu


def _walled_box_2d(base):
    wall = wl._bc_row(wl.BC_WALL, T=1.0)
    hot = wl._bc_row(wl.BC_WALL, T=1.3)
    lid = wl._bc_row(wl.BC_WALL, U=(0.3, 0.0, 0.0), T=1.0)
    mesh = wl.cartesian_mesh((5, 4), (1.0, 1.0), bcs=[(wall, hot), (wall, lid)])
    v = 4.0 * wl.sqrt_RT(1.0)
    return wl.Workload("walled-box-5x4", mesh, 2, base, (-v, -v), (v, v), 0, Kn=0.05, omega=0.81,
                       Pr=2.0 / 3.0, C1=2.0, C2=wl.K_SIGMA * 2.0, W_inf=(1.0, 0.0, 0.0, 1.0),
                       W_init=wl.sweep_W(mesh), precision="mixed")


def _small_sphere_3d(base):
    w = wl.sphere(n_r=3, n_theta=4, n_phi=4, C1=1.0, max_refine=0, precision="mixed", learned=False)
    return dataclasses.replace(w, base=base)


def _check(w, D, nv, steps=3):
    avs = need_gpu()
    r, g = pair(w, avs, precision="mixed", amp=1e-2)
    assert g.Nv == nv
    dt = r.dt()
    for _ in range(steps):
        r.step(dt)
    g.step(steps, dt=dt)
    W, q = g.moments()
    Wo, qo = O.moments(D, r.xi, r.w, r.f)
    e = field_err(W, r.Wc, D)
    ef = field_err(g.f_moments(), Wo, D, q, qo)
    df = rel_err(g.get_f(), r.f)
    print(f"\n{w.name} Nv={nv}: carried W {e}, f moments {ef}, f {df:.2e}")
    assert max(e.values()) < 1e-5, e
    assert max(ef.values()) < 1e-5, ef
    assert df < 1e-5, df
    g.close()


@pytest.mark.parametrize("base", [(64, 96), (79, 79), (75, 79)])
def test_staged_face_2d_walls(base):
    """6144 nodes (6 full stages), 6241 (a padded last stage of 128 nodes)
    and 5925 (odd count: the last node pair half padding)."""
    _check(_walled_box_2d(base), 2, base[0] * base[1])


@pytest.mark.parametrize("base", [(23, 23, 23), (16, 24, 32)])
def test_staged_face_3d_sphere_walls_and_far_field(base):
    """12167 nodes (odd, ragged last stage) and 12288 (6 full stages)."""
    _check(_small_sphere_3d(base), 3, int(np.prod(base)))


def test_staged_copy_wait_is_bounded():
    """The mbarrier wait of the staged kernels' bulk copies: a copy completes
    it with the right bytes; a wait that nothing completes gives up within its
    limit, the call reports AVS_ETIMEOUT, and the context then runs a staged
    step that matches the oracle."""
    import time
    avs = need_gpu()
    w = _walled_box_2d((79, 79))
    r, g = pair(w, avs, precision="mixed", amp=1e-2)
    assert g.stage_wait_check(True) == 1
    t0 = time.perf_counter()
    with pytest.raises(avs.AVSError) as ei:
        g.stage_wait_check(False)
    assert ei.value.status == -4                     # AVS_ETIMEOUT
    assert time.perf_counter() - t0 < 60
    assert g.stage_wait_check(True) == 1             # the error word was cleared
    dt = r.dt()
    r.step(dt)
    g.step(1, dt=dt)
    e = field_err(g.f_moments(), O.moments(2, r.xi, r.w, r.f)[0], 2)
    assert max(e.values()) < 1e-5, e
    g.close()
