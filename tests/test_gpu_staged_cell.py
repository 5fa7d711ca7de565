"""The FP32 cell kernel for 3D velocity meshes above 1024 nodes.

There the cell kernel streams the cell's f row and its faces' flux rows
through shared memory in stages of asynchronous bulk copies, nodes by pairs
in a fixed thread order, and the raw-moment kernel that restores dropped
carried moments walks the nodes in the same order.  The carried moments must
equal the recomputed ones bit for bit, with node counts that end inside a
stage and on odd and even pads; the fields must match the FP64 oracle.  The
2D cases (direct cell kernel, two arrays and four faces) run the same checks
at the same node counts.
"""
import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl

from gpu_common import field_err, need_gpu, pair, rel_err, small_sphere

pytestmark = pytest.mark.gpu


def _box(base):
    wall = wl._bc_row(wl.BC_WALL, T=1.0)
    hot = wl._bc_row(wl.BC_WALL, T=1.3)
    mesh = wl.cartesian_mesh((6, 5), (1.0, 1.0), bcs=[(wall, hot), (wall, wall)])
    v = 4.0 * wl.sqrt_RT(1.0)
    return wl.Workload("walled-box-6x5", mesh, 2, base, (-v, -v), (v, v), 0, Kn=0.05, omega=0.81,
                       Pr=2.0 / 3.0, C1=2.0, C2=wl.K_SIGMA * 2.0, W_inf=(1.0, 0.0, 0.0, 1.0),
                       W_init=wl.sweep_W(mesh), precision="mixed")


def _sphere(base):
    import dataclasses
    w = wl.sphere(n_r=3, n_theta=4, n_phi=4, C1=1.0, max_refine=0, precision="mixed", learned=False)
    return dataclasses.replace(w, base=base)


CASES = [(_box, (33, 33), 2), (_box, (32, 40), 2), (_sphere, (11, 11, 11), 3), (_sphere, (10, 11, 12), 3)]


@pytest.mark.parametrize("make,base,D", CASES)
def test_staged_cell_carried_moments_bitwise(make, base, D):
    """1089 and 1280 nodes in 2D, 1331 and 1320 in 3D: three steps with the
    carried moments against three steps that drop them after every step."""
    avs = need_gpu()
    w = make(base)
    a = avs.AVS(w, precision="mixed")
    b = avs.AVS(w, precision="mixed")
    assert a.Nv == int(np.prod(base)) and a.Nv > 1024
    for g in (a, b):
        g.init_field(amp=1e-3, seed=5)
    dt = a.dt()
    a.step(3, dt=dt)
    for _ in range(3):
        b.step(1, dt=dt)
        b.set_W(b.moments()[0])
    assert np.array_equal(a.get_f(), b.get_f())
    assert np.array_equal(a.moments()[0], b.moments()[0])
    a.close(); b.close()


@pytest.mark.parametrize("make,base,D", CASES)
def test_staged_cell_against_oracle(make, base, D):
    avs = need_gpu()
    w = make(base)
    r, g = pair(w, avs, precision="mixed", amp=1e-2)
    dt = r.dt()
    for _ in range(3):
        r.step(dt)
    g.step(3, dt=dt)
    W, q = g.moments()
    Wo, qo = O.moments(D, r.xi, r.w, r.f)
    e = field_err(W, r.Wc, D)
    ef = field_err(g.f_moments(), Wo, D, q, qo)
    df = rel_err(g.get_f(), r.f)
    print(f"\n{w.name} Nv={g.Nv}: carried W {e}, f moments {ef}, f {df:.2e}")
    assert max(e.values()) < 1e-5, e
    assert max(ef.values()) < 1e-5, ef
    assert df < 1e-5, df
    g.close()
