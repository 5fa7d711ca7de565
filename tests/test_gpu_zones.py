"""Adaptive-parameter zones (Sec. 3.5) on the GPU against the oracle: the
library's parameter rules equal the oracle's, and the step-0 tree, steps and
adaptations of a zoned velocity space keep a bit-identical topology."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp
from paper_2212_05645_gb300 import workloads as wl

from gpu_common import field_err, need_gpu, pair, rel_err

pytestmark = pytest.mark.gpu

FLOWS = [(2, wl.FlowSpec(Ma=5.0)),
         (2, wl.FlowSpec(Ma=8.0, separated=True)),
         (2, wl.FlowSpec(Ma=20.2, gamma=1.4, T_w=290.0 / 13.32, dir=(0.9848, 0.1736, 0.0))),
         (3, wl.FlowSpec(Ma=5.45, gamma=1.4, rdv_sigma=7.0)),
         (3, wl.FlowSpec(Ma=4.25, gamma=1.4, dir=(1.0, 0.0, 1.0)))]


@pytest.mark.parametrize("D,flow", FLOWS)
def test_library_parameters_equal_the_oracle(D, flow):
    avs = need_gpu()
    g = avs.paper_parameters(D, flow)
    o = O.paper_parameters(D, flow.Ma, flow.gamma, flow.T_inf, flow.T_w, flow.dir, flow.h_std, flow.rdv_sigma,
                           flow.separated)
    for k in ("base", "vlo", "vhi", "max_refine", "outside", "init_refine", "C1", "C2"):
        assert g[k] == o[k], (k, g[k], o[k])
    assert len(g["zones"]) == len(o["zones"])
    for zg, zo in zip(g["zones"], o["zones"]):
        assert zg == (tuple(zo[0]), zo[1], zo[2], zo[3])


def hot_rest(w, T=6.0):
    W = np.zeros((w.mesh.Nc, w.D + 2))
    W[:, 0] = 1.0
    W[:, w.D + 1] = T
    return W


@pytest.mark.parametrize("case", ["cyl", "cyl-sep", "sphere"])
def test_zoned_tree_steps_and_adaptation_fp64(case):
    avs = need_gpu()
    if case == "sphere":
        w = wl.sphere_zones(n_r=3, n_theta=4, n_phi=4, Ma=4.25, precision="fp64")
    else:
        w = wl.cylinder_zones(n_theta=16, n_r=5, Ma=5.0, separated=(case == "cyl-sep"), precision="fp64")
    r, g = pair(w, avs, amp=1e-2)           # asserts the step-0 tree
    dt = r.dt()
    assert g.dt() == dt
    for _ in range(2):
        r.step(dt)
    g.step(2, dt=dt)
    assert rel_err(g.get_f(), r.f) < 1e-12
    # a hot stagnation state: its tail outside the zones is where the caps act
    r.init_field(hot_rest(w))
    g.set_f(r.f)
    g.set_W(r.Wc)
    o = r.adapt()
    st = g.adapt()
    t = g.tree()
    assert st["Nv"] == o["Nv"]
    assert np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
    assert np.array_equal(t["base"], r.base)
    assert rel_err(g.get_f(), r.f) < 1e-12
    g.close()


def test_zoned_mixed_fields_and_topology():
    avs = need_gpu()
    w = wl.cylinder_zones(n_theta=16, n_r=5, Ma=5.0, precision="mixed")
    r, g = pair(w, avs, precision="mixed", amp=1e-2)
    dt = r.dt()
    for _ in range(3):
        r.step(dt)
    g.step(3, dt=dt)
    e = field_err(g.moments()[0], r.Wc, 2)
    assert max(e.values()) < 1e-5, e
    g.set_W(r.Wc)
    g.set_f(r.f)
    r.f = g.get_f()                         # identical (FP32-rounded) inputs to the criterion
    o = r.adapt()
    g.adapt()
    t = g.tree()
    assert np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
    g.close()


def test_zoned_labels_use_the_node_caps():
    """The proposer's split-witness label counts only nodes below their zone
    cap; the labels equal the oracle's with the per-node caps bit for bit
    (the oracle's labels taken from the same W, the moments of f the GPU uses)."""
    avs = need_gpu()
    w = wl.cylinder_zones(n_theta=16, n_r=5, Ma=5.0, precision="fp64", learned=True)
    r, g = pair(w, avs, amp=1e-2)
    r.init_field(hot_rest(w, T=3.0), amp=1e-2)
    g.set_f(r.f)
    g.set_W(r.Wc)
    X, Y = g.features()
    Wg = g.f_moments()
    m = mlp.criterion_values(2, r.xi, r.w, r.f, Wg, r.s)
    Yo = mlp.labels(m, m.max(0), r.level, r.p["C1"], r.p["C2"], r.ncap)
    assert np.array_equal(Y, Yo)
    Yflat = mlp.labels(m, m.max(0), r.level, r.p["C1"], r.p["C2"], r.p["max_refine"])
    assert Yflat[:, 0].sum() >= Yo[:, 0].sum()
    g.close()
