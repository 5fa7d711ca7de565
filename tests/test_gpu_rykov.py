"""Rykov model (diatomic gas, Sec. 2.1) on the GPU against the oracle: the
explicit step with G, H, R (2D) and G, R (3D), the rotational energy
exchange, walls and far field, adaptation with the Rykov correction.  FP64
form within 1e-12, mixed form within 1e-5 on the fields."""
import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl

from gpu_common import field_err, need_gpu, pair_rykov, rel_err, small_cylinder, small_sphere

pytestmark = pytest.mark.gpu

CASES = {
    "box": lambda p: wl.sweep_box((7, 6), base=(10, 10), max_refine=1, precision=p),
    "omesh": lambda p: small_cylinder(precision=p),
    "triangles": lambda p: wl.triangle_box(precision=p),
    "sphere": lambda p: small_sphere(precision=p),
}


def rykov(w):
    w.model = "rykov"
    return w


def erot_err(Wg, Wo, D):
    return float((np.abs(Wg[:, D + 2] - Wo[:, D + 2]) / np.abs(Wo[:, D + 1])).max())


@pytest.mark.parametrize("case", sorted(CASES))
def test_rykov_fp64_steps_match_oracle(case):
    avs = need_gpu()
    w = rykov(CASES[case]("fp64"))
    r, g = pair_rykov(w, avs)
    dt = r.dt()
    assert g.dt() == dt
    for _ in range(2):
        r.step(dt)
    g.step(2, dt=dt)
    assert rel_err(g.moments()[0], r.Wc) < 1e-12
    assert rel_err(g.get_f(), r.f) < 1e-12
    g.close()


def test_rykov_init_field_matches_oracle():
    avs = need_gpu()
    w = rykov(CASES["omesh"]("fp64"))
    r = O.Run(w)
    g = avs.AVS(w)
    Wp = np.column_stack([w.W_init, 0.7 * w.W_init[:, 3]])
    r.init_field(Wp, amp=1e-2, seed=11)
    g.init_field(Wp, amp=1e-2, seed=11)
    assert rel_err(g.get_f(), r.f) < 1e-14
    assert rel_err(g.moments()[0], r.Wc) < 1e-13
    g.close()


@pytest.mark.parametrize("case", ["box", "omesh", "sphere"])
def test_rykov_mixed_fields_within_1e5(case):
    avs = need_gpu()
    w = rykov(CASES[case]("mixed"))
    r, g = pair_rykov(w, avs, precision="mixed")
    dt = r.dt()
    for _ in range(3):
        r.step(dt)
    g.step(3, dt=dt)
    Wg = g.moments()[0]
    e = field_err(Wg, r.Wc, w.D)
    assert max(e.values()) < 1e-5, e
    assert erot_err(Wg, r.Wc, w.D) < 1e-5
    g.close()


@pytest.mark.parametrize("D", [2, 3])
def test_rykov_adapt_topology_remap_and_correction(D):
    avs = need_gpu()
    w = rykov(small_cylinder(C1=0.6, max_refine=3) if D == 2 else small_sphere())
    r, g = pair_rykov(w, avs)
    dt = r.dt()
    r.step(dt)
    g.step(1, dt=dt)
    g.set_f(r.f)
    g.set_W(r.Wc)
    st_o = r.adapt()
    st_g = g.adapt()
    t = g.tree()
    assert st_g["Nv"] == st_o["Nv"]
    assert np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
    assert rel_err(g.get_f(), r.f) < 1e-12
    assert abs(st_g["gap"] - st_o["gap"]) <= 1e-12 + 1e-6 * st_o["gap"]
    # the equilibrium bypass on the Rykov model: f = (g^eq(T_t), (3-D) R T_t g, R T_r g)
    r.step(dt)
    g.step(1, dt=dt)
    g.set_f(r.f)
    g.set_W(r.Wc)
    r.adapt(bypass=True)
    g.adapt(bypass=True)
    assert rel_err(g.get_f(), r.f) < 1e-12
    g.close()


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("cfl", [0.8, 3.0])
def test_rykov_implicit_fp64_matches_oracle(case, cfl):
    """IUGKS with the Rykov model: Eqs. (SGS_w), (SGS_wrot), (SGS_phi)."""
    avs = need_gpu()
    w = rykov(CASES[case]("fp64"))
    r, g = pair_rykov(w, avs)
    dt = r.dt(cfl)
    for _ in range(2):
        r.step_implicit(dt)
    g.step_implicit(2, dt=dt)
    assert rel_err(g.moments()[0], r.Wc) < 1e-12
    assert rel_err(g.get_f(), r.f) < 1e-12
    g.close()


@pytest.mark.parametrize("case", ["box", "omesh"])
def test_rykov_implicit_mixed_fields_within_1e5(case):
    avs = need_gpu()
    w = rykov(CASES[case]("mixed"))
    r, g = pair_rykov(w, avs, precision="mixed")
    dt = r.dt(2.0)
    for _ in range(3):
        r.step_implicit(dt)
    g.step_implicit(3, dt=dt)
    Wg = g.moments()[0]
    e = field_err(Wg, r.Wc, w.D)
    assert max(e.values()) < 1e-5, e
    assert erot_err(Wg, r.Wc, w.D) < 1e-5
    g.close()


def test_rykov_carried_moments_equal_recomputed_bitwise():
    """Mixed form: the Rykov cell kernel sums the raw moments of f^{n+1} while
    writing it and the next explicit step takes them instead of re-reading f.
    Forcing the re-read after every step (set_W with the same W drops them)
    gives the same bits, and an implicit step in between leaves none behind."""
    avs = need_gpu()
    w = rykov(CASES["omesh"]("mixed"))
    a = avs.AVS(w, precision="mixed")
    b = avs.AVS(w, precision="mixed")
    Wp = np.column_stack([w.W_init, 0.8 * w.W_init[:, w.D + 1]])
    for g in (a, b):
        g.init_field(Wp, amp=1e-3, seed=5)
    dt = a.dt()
    for kind in ("e", "e", "i", "e", "e"):
        for g in (a, b):
            if kind == "e":
                g.step(1, dt=dt)
            else:
                g.step_implicit(1, dt=dt)
        b.set_W(b.moments()[0])
    assert np.array_equal(a.get_f(), b.get_f())
    assert np.array_equal(a.moments()[0], b.moments()[0])
    a.close(); b.close()
