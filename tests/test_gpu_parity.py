"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Tolerances: the velocity-mesh topology, node geometry and the time-step bound
are bit-exact; the FP64 form agrees to 1e-12 relative; the mixed form agrees
on the macroscopic fields to 1e-5 relative (field scale).
"""
import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl

from gpu_common import field_err, need_gpu, pair, q_err, rel_err, small_cylinder, small_sphere

pytestmark = pytest.mark.gpu


def test_step0_tree_geometry_and_dt_bitexact():
    avs = need_gpu()
    for w in (wl.cavity(), small_cylinder(), small_sphere()):
        r = O.Run(w)
        g = avs.AVS(w)
        t = g.tree()
        assert np.array_equal(t["level"], r.level)
        assert np.array_equal(t["base"], r.base)
        assert np.array_equal(t["key"], r.key)
        assert np.array_equal(t["xi"], r.xi)
        assert np.array_equal(t["w"], r.w)
        assert g.dt(0.8) == r.dt(0.8)
        g.close()


def test_init_field_and_moments():
    avs = need_gpu()
    w = wl.sweep_box((6, 5), base=(12, 12), max_refine=1)
    r = O.Run(w)
    r.init_field(amp=1e-3, seed=99)
    g = avs.AVS(w)
    g.init_field(amp=1e-3, seed=99)
    assert rel_err(g.get_f(), r.f) < 1e-14
    W, q = g.moments()
    Wo, qo = O.moments(2, r.xi, r.w, r.f)
    assert rel_err(W, Wo) < 1e-13
    assert np.abs(q - qo).max() < 1e-13 * np.abs(Wo).max()
    assert rel_err(g.f_moments(), Wo) < 1e-13


def test_init_field_mixed_within_fp32():
    """Mixed form: the Maxwellian start is evaluated in FP32 (f is stored in
    FP32); it stays within a few FP32 ulp of the FP64 oracle."""
    avs = need_gpu()
    w = wl.sweep_box((6, 5), base=(12, 12), max_refine=1, precision="mixed")
    r = O.Run(w)
    r.init_field(amp=1e-3, seed=99)
    g = avs.AVS(w, precision="mixed")
    g.init_field(amp=1e-3, seed=99)
    assert rel_err(g.get_f(), r.f) < 1e-6
    e = field_err(g.moments()[0], O.moments(2, r.xi, r.w, r.f)[0], 2)
    assert max(e.values()) < 1e-6, e
    g.close()


@pytest.mark.parametrize("limiter", [0, 1, 2])
def test_step_fp64_periodic(limiter):
    avs = need_gpu()
    w = wl.sweep_box((7, 6), base=(10, 10), max_refine=1)
    r, g = pair(w, avs, limiter=limiter)
    dt = r.dt()
    for _ in range(3):
        r.step(dt)
    g.step(3, dt=dt)
    assert rel_err(g.get_f(), r.f) < 1e-12
    W, _ = g.moments()
    assert rel_err(W, r.Wc) < 1e-12
    assert q_err(g, r, 2) < 1e-12


def test_step_fp64_cavity_walls_200_steps():
    """Config 1 (lid-driven cavity, FP64): all 200 steps against the oracle."""
    avs = need_gpu()
    w = wl.cavity()
    r, g = pair(w, avs, amp=0.0)
    dt = r.dt()
    assert g.dt() == dt
    for _ in range(200):
        r.step(dt)
    g.step(200, dt=dt)
    assert rel_err(g.get_f(), r.f) < 1e-11
    W, _ = g.moments()
    assert rel_err(W, r.Wc) < 1e-12
    assert q_err(g, r, 2) < 1e-11
    vol = w.mesh.vol
    m0 = (O.moments(2, r.xi, r.w, O.maxwell_init(2, r.xi, w.W_init))[0][:, 0] * vol).sum()
    assert abs((W[:, 0] * vol).sum() - m0) / m0 < 1e-12


def test_step_fp64_omesh_wall_farfield():
    avs = need_gpu()
    w = small_cylinder()
    r, g = pair(w, avs)
    dt = r.dt()
    for _ in range(4):
        r.step(dt)
    g.step(4, dt=dt)
    assert rel_err(g.get_f(), r.f) < 1e-12
    assert rel_err(g.moments()[0], r.Wc) < 1e-12
    assert q_err(g, r, 2) < 1e-12


def test_step_fp64_3d_sphere_shell():
    avs = need_gpu()
    w = small_sphere()
    r, g = pair(w, avs)
    dt = r.dt()
    for _ in range(2):
        r.step(dt)
    g.step(2, dt=dt)
    assert rel_err(g.get_f(), r.f) < 1e-12
    assert rel_err(g.moments()[0], r.Wc) < 1e-12
    assert q_err(g, r, 3) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_carried_moments_equal_recomputed_bitwise(precision):
    """The cell kernel sums the raw moments of f^{n+1} while writing it and the
    next step takes them instead of re-reading f.  Forcing the re-read (set_W
    with the same W drops the carried moments) gives the same bits."""
    avs = need_gpu()
    w = small_cylinder(precision=precision)
    a = avs.AVS(w, precision=precision)
    b = avs.AVS(w, precision=precision)
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


def test_state_replaced_between_steps_fp64():
    """f and W replaced between two steps (set_f, set_W): the second step
    starts from the new state, as in the oracle."""
    avs = need_gpu()
    w = small_cylinder()
    r, g = pair(w, avs)
    dt = r.dt()
    r.step(dt)
    g.step(1, dt=dt)
    k = np.arange(r.f.shape[2])
    r.f = np.ascontiguousarray(r.f * (1.0 + 1e-3 * np.cos(0.37 * k))[None, None, :])
    r.Wc = np.ascontiguousarray(r.Wc * 1.001)
    g.set_f(r.f)
    g.set_W(r.Wc)
    r.step(dt)
    g.step(1, dt=dt)
    assert rel_err(g.get_f(), r.f) < 1e-12
    assert rel_err(g.moments()[0], r.Wc) < 1e-12
    g.close()


@pytest.mark.parametrize("amp", [0.0, 1e-2])
def test_criterion_and_dt_bitexact_mixed_with_ties(amp):
    """Mixed form: the criterion (FP32 screening, FP64 at the pairs that can
    hold the maximum) equals the oracle's plain FP64 maximum bit for bit on
    the same FP32 f values, also when many cells are identical (amp 0: every
    cell of a uniform region ties at every node); the time-step bound too."""
    avs = need_gpu()
    w = wl.sweep_box((9, 7), base=(12, 12), max_refine=2, C1=3.0, precision="mixed")
    g = avs.AVS(w, precision="mixed")
    g.init_field(amp=amp, seed=9)
    r = O.Run(w)
    t = g.tree()
    assert np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
    f = g.get_f()                                  # the FP32 values, exactly, as float64
    Wf, _ = O.moments(2, r.xi, r.w, f)
    assert np.array_equal(g.criterion(Wf), O.criterion(2, r.xi, r.w, f, Wf))
    assert g.dt() == r.dt()
    g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_unstructured_triangles_steps_and_adaptation(precision, tol):
    """Unstructured physical mesh (Delaunay triangles, 3 faces per cell,
    walls on the boundary): steps and one adaptation against the oracle."""
    avs = need_gpu()
    w = wl.triangle_box(precision=precision)
    r, g = pair(w, avs, precision=precision, amp=1e-2)
    dt = r.dt()
    assert g.dt() == dt
    for _ in range(4):
        r.step(dt)
    g.step(4, dt=dt)
    e = field_err(g.moments()[0], r.Wc, 2)
    assert max(e.values()) < tol, e
    if precision == "fp64":
        assert rel_err(g.get_f(), r.f) < tol
        o = r.adapt()
        st = g.adapt()
        t = g.tree()
        assert st["Nv"] == o["Nv"]
        assert np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
        assert rel_err(g.get_f(), r.f) < 1e-12
    g.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_adapt_equilibrium_bypass(precision, tol):
    """Adaptation with the equilibrium bypass (end of Sec. 3.3): same tree as
    the oracle and f = g^eq(W) of the carried W on it."""
    avs = need_gpu()
    w = wl.sweep_box((7, 6), base=(10, 10), max_refine=2, C1=2.0, precision=precision)
    r, g = pair(w, avs, precision=precision, amp=1e-2)
    dt = r.dt()
    for _ in range(3):
        r.step(dt)
    g.step(3, dt=dt)
    g.set_W(r.Wc)
    g.set_f(r.f)
    r.f = g.get_f()              # the same (FP32-rounded in the mixed form) inputs to the criterion
    o = r.adapt(bypass=True)
    st = g.adapt(bypass=True)
    t = g.tree()
    assert st["Nv"] == o["Nv"]
    assert np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
    assert rel_err(g.get_f(), r.f) < tol
    assert np.array_equal(g.moments()[0], r.Wc)
    g.close()


def test_criterion_bitexact_given_W():
    avs = need_gpu()
    w = small_cylinder()
    r, g = pair(w, avs, amp=1e-2)
    Wf, _ = O.moments(2, r.xi, r.w, r.f)
    M_o = O.criterion(2, r.xi, r.w, r.f, Wf)
    M_g = g.criterion(Wf)
    assert np.array_equal(M_g, M_o)


@pytest.mark.parametrize("D", [2, 3])
def test_adapt_topology_remap_bitexact_and_correction(D):
    avs = need_gpu()
    w = small_cylinder(C1=0.6, max_refine=3) if D == 2 else small_sphere()
    r, g = pair(w, avs, amp=1e-2)
    r.step(r.dt()); g.step(1, dt=r.dt())
    f_now = r.f.copy()
    g.set_f(f_now)
    Wf, _ = O.moments(D, r.xi, r.w, f_now)
    # remap only: bit-exact
    st_o = r.adapt(Wc_override=Wf, correct_f=False)
    st_g = g.adapt(W_override=Wf, skip_correction=True)
    t = g.tree()
    assert st_g["Nv"] == st_o["Nv"]
    assert np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
    assert np.array_equal(t["base"], r.base)
    assert np.array_equal(g.get_f(), r.f)
    # with the conservation correction
    r2, g2 = pair(w, avs, amp=1e-2)
    r2.f = f_now.copy(); g2.set_f(f_now)
    st_o = r2.adapt(Wc_override=Wf)
    st_g = g2.adapt(W_override=Wf)
    assert rel_err(g2.get_f(), r2.f) < 1e-12
    assert abs(st_g["gap"] - st_o["gap"]) <= 1e-12 + 1e-6 * st_o["gap"]


@pytest.mark.parametrize("D", [2, 3])
def test_mixed_adaptation_correction_gap(D):
    """Mixed form: the adaptation's correction (Sec. 3.3) sums the moments of
    the FP32 f with compensated per-thread sums and FP64 across threads, and
    applies g(W) - g(W') in a form free of cancellation, so after the remap the
    moments of f come back to their pre-adaptation values to within the FP32
    storage of f: the reported gap is below 1e-6, and the corrected f's
    moments stay within 1e-5 of the FP64 oracle's after the same adaptation
    (per-field errors printed)."""
    avs = need_gpu()
    w = (wl.sweep_box((8, 7), base=(10, 10), max_refine=2, C1=2.0, precision="mixed") if D == 2 else
         wl.sweep_box((5, 4, 3), base=(8, 8, 8), max_refine=1, C1=2.0, precision="mixed"))
    r, g = pair(w, avs, precision="mixed", amp=1e-2)
    dt = r.dt()
    for _ in range(3):
        r.step(dt)
    g.step(3, dt=dt)
    W_pre = g.f_moments()
    st = g.adapt()
    o = r.adapt()
    t = g.tree()
    same = np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
    e_gap = field_err(g.f_moments(), W_pre, D)
    e_or = field_err(g.f_moments(), O.moments(D, r.xi, r.w, r.f)[0], D) if same else None
    print(f"\nmixed adaptation D={D}: {st['splits']} splits, {st['merges']} merges, gap {st['gap']:.2e}, "
          f"moments of f against their pre-adaptation values {e_gap}, against the oracle {e_or}")
    assert st["splits"] + st["merges"] > 0
    assert st["gap"] < 1e-6
    assert max(e_gap.values()) < 1e-6
    assert same and max(e_or.values()) < 1e-5
    g.close()


def test_adapt_learned_off_counts_and_stats():
    avs = need_gpu()
    w = small_cylinder(C1=0.6, max_refine=3)
    r, g = pair(w, avs, amp=1e-2)
    st = g.adapt()
    o = r.adapt()
    assert st["Nv"] == o["Nv"]
    assert st["Nv"] == g.Nv
    assert st["splits"] * 3 - st["merges"] * 3 == st["Nv"] - st["Nv_old"]


def test_mixed_precision_fields_within_1e5():
    """Mixed form (FP32 f, FP64 sums): macroscopic fields within 1e-5 of the
    FP64 oracle after 20 steps on the O-mesh with wall and far field."""
    avs = need_gpu()
    w = small_cylinder(precision="mixed")
    r, g = pair(w, avs, precision="mixed")
    dt = r.dt()
    for _ in range(20):
        r.step(dt)
    g.step(20, dt=dt)
    W, q = g.moments()
    Wo, qo = O.moments(2, r.xi, r.w, r.f)
    e = field_err(W, r.Wc, 2, q, qo)
    print(f"\nmixed O-mesh, 20 steps, per-field error against the FP64 oracle: {e}")
    assert max(e.values()) < 1e-5, e
    assert rel_err(g.get_f(), r.f) < 1e-4


def test_mixed_cavity_fields_and_mass_over_1000_steps_with_adaptations():
    """Config 1 geometry (lid-driven cavity) in the mixed form.
    - After 200 steps every macroscopic field, the heat flux of f included,
      is within 1e-5 of the FP64 oracle (per-field errors printed).
    - Then 1000 steps with an adaptation every 50 (criterion, consanguinity
      remap, correction), run by the mixed form and by the FP64 oracle from
      the same state: the total mass of the carried W changes by less than
      1e-10 in both (zero net mass flux through the walls, telescoping
      fluxes), and the total mass of f itself (the moments of the FP32 f,
      summed in FP64) changes by no more than the FP64 oracle's f does plus
      1e-9: the method's own quadrature drift, with nothing added by the
      FP32 storage."""
    avs = need_gpu()
    w = wl.cavity(precision="mixed")
    r, g = pair(w, avs, precision="mixed", amp=0.0)
    dt = r.dt()
    for _ in range(200):
        r.step(dt)
    g.step(200, dt=dt)
    W, q = g.moments()
    Wo, qo = O.moments(2, r.xi, r.w, r.f)
    e = field_err(W, r.Wc, 2, q, qo)
    print(f"\nmixed cavity, 200 steps, per-field error against the FP64 oracle: {e}")
    assert max(e.values()) < 1e-5, e
    vol = w.mesh.vol

    def masses_gpu():
        return (g.moments()[0][:, 0] * vol).sum(), (g.f_moments()[:, 0] * vol).sum()

    def masses_oracle():
        return (r.Wc[:, 0] * vol).sum(), (O.moments(2, r.xi, r.w, r.f)[0][:, 0] * vol).sum()

    mg0, fg0 = masses_gpu()
    mo0, fo0 = masses_oracle()
    for cycle in range(20):
        g.step(50, dt=dt)
        for _ in range(50):
            r.step(dt)
        g.adapt()
        r.adapt()
        dt = r.dt()
    mg1, fg1 = masses_gpu()
    mo1, fo1 = masses_oracle()
    dW_g, dW_o = abs(mg1 - mg0) / mg0, abs(mo1 - mo0) / mo0
    df_g, df_o = abs(fg1 - fg0) / fg0, abs(fo1 - fo0) / fo0
    print(f"1000 steps, 20 adaptations: carried-W mass drift mixed {dW_g:.2e} FP64 {dW_o:.2e}; "
          f"f mass drift mixed {df_g:.2e} FP64 {df_o:.2e}; nodes {g.Nv} / {r.Nv}")
    assert dW_g < 1e-10 and dW_o < 1e-10
    assert df_g <= df_o + 1e-9
    g.close()


def test_edge_cases_zero_steps_single_cell_row():
    avs = need_gpu()
    w = wl.sweep_box((3, 2), base=(5, 3), max_refine=0)
    r, g = pair(w, avs)
    g.step(0, dt=1e-3)
    assert np.array_equal(g.get_f(), r.f)
    dt = r.dt()
    r.step(dt); g.step(1, dt=dt)
    assert rel_err(g.get_f(), r.f) < 1e-12
