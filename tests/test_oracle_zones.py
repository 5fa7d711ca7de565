"""Pins of the oracle's adaptive-parameter rules (Sec. 3.5) and of the
refinement zones, against the values the paper prints (tests/golden/) and
against properties of the rules."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2212_05645_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def rows(name):
    out = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                out.append(line.split())
    return out


def test_max_level_against_the_cylinder_table():
    """L_max for every Mach number of the cylinder table: pins T_0, sigma_0 =
    sqrt(R T_0) with R = 1/2, R_dv = 4 sigma_0 and the 2^L >= 2 R_dv / h_std rule."""
    rs = rows("avs_levels_cylinder.txt")
    assert len(rs) == 16
    for Ma, L in rs:
        p = O.paper_parameters(2, float(Ma), 5.0 / 3.0)
        assert p["L_max"] == int(L), (Ma, p["L_max"], L)


def test_smallest_interval_against_the_sphere_table():
    for Ma, k, h in rows("avs_hinf_sphere.txt"):
        p = O.paper_parameters(3, float(Ma), 7.0 / 5.0, rdv_sigma=float(k))
        assert abs(p["h_inf"] - float(h)) <= 5e-4, (k, p["h_inf"], h)


def test_c1_law_against_the_quoted_thresholds():
    for Ma, C1, *_ in rows("c1_law.txt"):
        p = O.paper_parameters(2, float(Ma), 5.0 / 3.0)
        assert abs(p["C1"] - float(C1)) <= 5e-3, (Ma, p["C1"], C1)
        assert p["C2"] == 3.3546e-4 * p["C1"]


def test_total_temperature_against_the_sphere_cases():
    for Ma, T0, Tinf in rows("total_temperature.txt"):
        p = O.paper_parameters(3, float(Ma), 7.0 / 5.0)      # T_inf = 1: T0 is the ratio T_0 / T_inf
        assert abs(float(T0) / p["T0"] - float(Tinf)) <= 5e-3


def test_level_rules():
    """L_w drops by one when the wall is hot (T_w / T_inf >= 4); L_min is 4
    only for D = 2 above Ma 5; the separated zone sits one level below L_w
    but not below L_min; Ma 5 gives the paper's complete level-5 mesh of
    1024 elements (Sec. 4.1) as the base forest refined to max_refine."""
    p = O.paper_parameters(2, 5.0, 5.0 / 3.0)
    assert (p["L_max"], p["L_w"], p["L_min"], p["L_sep"]) == (5, 5, 3, 4)
    assert np.prod(p["base"]) * (4 ** p["max_refine"]) == 1024
    assert p["init_refine"] == 1                         # root split L_w - 1 = 4 times, base at level 3
    hot = O.paper_parameters(2, 20.2, 7.0 / 5.0, T_inf=1.0, T_w=290.0 / 13.32)
    assert hot["L_w"] == hot["L_max"] - 1
    assert O.paper_parameters(2, 6.0, 5.0 / 3.0)["L_min"] == 4
    assert O.paper_parameters(3, 6.0, 5.0 / 3.0)["L_min"] == 3
    sep = O.paper_parameters(2, 5.0, 5.0 / 3.0, separated=True)
    assert sep["zones"][2][3] == sep["L_sep"] - sep["L_min"] == 1
    # domain: square of half-width R_dv about 0.4 U_inf
    U = 5.0 * math.sqrt(5.0 / 3.0 * 0.5)
    assert abs(0.5 * (p["vlo"][0] + p["vhi"][0]) - 0.4 * U) < 1e-12
    assert abs(p["vhi"][0] - p["vlo"][0] - 2 * p["R_dv"]) < 1e-12


def test_node_caps_by_zone():
    p = O.paper_parameters(2, 5.0, 5.0 / 3.0, separated=True)
    U = p["U"]
    xi = np.array([[U[0], 0.0],                    # free-stream centre
                   [0.0, 0.0],                     # stationary centre
                   [0.0, 4.0 * p["sigma_w"]],      # separated ring, outside the free-stream zone
                   [0.0, -6.0]])                   # no zone
    cap = O.node_caps(2, xi, p["zones"], p["outside"], p["max_refine"])
    assert list(cap) == [p["L_max"] - p["L_min"], p["L_w"] - p["L_min"], p["L_sep"] - p["L_min"], 0]
    assert list(O.node_caps(2, xi, [], 0, 3)) == [3, 3, 3, 3]


@pytest.fixture(scope="module")
def zone_run():
    w = wl.cylinder_zones(n_theta=12, n_r=4, Ma=5.0, precision="fp64")
    return O.Run(w)


def split_from_a_zone(r):
    """Every node finer than the uniform step came from splitting a parent
    whose centre lies in a zone of at least the node's level: the parent
    centre is sqrt(D) h_l / 2 away from the node's (h_l its edge), so the node
    is within r_out + sqrt(D) h_l / 2 of such a zone's centre."""
    p = r.p
    D = r.D
    hb = (np.array(p["vhi"]) - np.array(p["vlo"])) / np.array(p["base"])
    for k in np.nonzero(r.level > p["init_refine"])[0]:
        l = r.level[k]
        reach = math.sqrt(D) * hb[0] / 2 ** (l + 1)
        ok = False
        for c, r_in, r_out, lev in p["zones"]:
            d = math.sqrt(sum((r.xi[k, i] - c[i]) ** 2 for i in range(D)))
            if lev >= l and r_in - reach <= d < r_out + reach:
                ok = True
        if not ok:
            return False
    return True


def test_initial_tree_respects_the_zones(zone_run):
    """Step 0 (Sec. 3.5): the base forest (level L_min) split init_refine times
    everywhere, then adapted on the two pseudo cells: nodes finer than the
    uniform step only where a zone allows, the free-stream zone reaches L_max."""
    r = zone_run
    p = r.p
    assert split_from_a_zone(r)
    top = r.level == p["max_refine"]
    assert top.any()
    d = np.sqrt(((r.xi[top] - np.array(p["U"])) ** 2).sum(1))
    assert (d < 3.0 * p["sigma_inf"]).any()
    # the outer region merged below the uniform level where g^eq is negligible
    assert (r.level < p["init_refine"]).any()


def test_adaptation_keeps_the_caps(zone_run):
    r = zone_run
    r.init_field(amp=1e-2, seed=3)
    dt = r.dt()
    r.step(dt)
    out = r.adapt()
    assert split_from_a_zone(r)
    assert out["Nv"] == r.Nv


def test_zones_change_the_tree():
    """Gas at rest at 6 T_inf (a stagnation state, wider than the zones around
    0 and U_inf): with the zones its tail outside them stays at the outside
    level; with every node capped at max_refine instead it refines there too."""
    w = wl.cylinder_zones(n_theta=12, n_r=4, Ma=5.0, precision="fp64")
    hot = np.zeros((w.mesh.Nc, 4))
    hot[:, 0] = 1.0
    hot[:, 3] = 6.0
    out = []
    for zones in (True, False):
        r = O.Run(w, build_tree=False)
        if not zones:
            r.p = dict(r.p, zones=[])
        r._geom()
        r.initial_tree()
        r.init_field(hot)
        r.adapt()
        out.append(r)
    rz, rn = out
    assert rn.Nv > rz.Nv
    assert split_from_a_zone(rz)
    assert not split_from_a_zone(rn)
