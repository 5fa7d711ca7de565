"""Learned proposer on the GPU against the FP64 MLP oracle (oracle/mlp.py).

The kernels run BF16 tensor-core products with FP32 accumulation, so the
comparison is against the oracle evaluated on the BF16-rounded weights and
inputs, with a tolerance set by the BF16 rounding of the intermediate
activations (2^-9 relative per rounding, a few roundings deep).
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp
from oracle.mlp_params import flatten, unflatten
from paper_2212_05645_gb300 import workloads as wl

from gpu_common import need_gpu, pair, pair_rykov, small_sphere

pytestmark = pytest.mark.gpu


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    return mlp.bf16_round(x)


def rounded_params(P32):
    p = unflatten(P32.astype(np.float64))
    for k in ("W1", "W2", "W3"):
        p[k] = bf16(p[k])
    return p


def small_ctx(avs, learned=True):
    w = wl.sweep_box((6, 6), base=(8, 8), max_refine=1)
    return avs.AVS(w, learned=learned)


def test_mlp_forward_and_gradients_match_oracle():
    """Logits and every parameter gradient, element by element: within the
    first-order BF16 rounding bound of the FP64 oracle (mlp.gradient_error_bound,
    pinned on the CPU), and within 2 % of that bound of the same BF16 pipeline
    emulated in numpy (the GPU differs from it only in the FP32 summation order)."""
    avs = need_gpu()
    g = small_ctx(avs)
    rng = np.random.default_rng(11)
    P32 = flatten(mlp.init_params(5)).astype(np.float32)
    P32[mlp.H * mlp.NF:mlp.H * mlp.NF + mlp.H] = 0.1 * rng.standard_normal(mlp.H)    # non-zero b1
    g.mlp_set_params(P32)
    assert np.array_equal(g.mlp_get_params(), P32)
    n = 301                                   # ragged: not a multiple of the 16-row tile
    X = rng.standard_normal((n, 8)).astype(np.float32)
    Y = (rng.random((n, 4)) > 0.6).astype(np.float32)
    pr = rounded_params(P32)
    Xr = bf16(X)
    Yd = Y.astype(np.float64)
    z_ref, _ = mlp.forward(pr, Xr)
    bound, ez3 = mlp.gradient_error_bound(pr, Xr, Yd)
    emu, z_emu = mlp.backward_bf16_emulated(pr, Xr, Yd)
    z = g.mlp_forward(X)
    assert np.all(np.abs(z - z_ref) <= ez3)
    assert np.all(np.abs(z - z_emu) <= 0.02 * ez3 + 1e-6 * np.abs(z_ref))
    gr, loss = g.mlp_grad(X, Y, lr=0.0)
    assert abs(loss - mlp.loss(pr, Xr, Yd)) < 1e-2 * mlp.loss(pr, Xr, Yd)
    ref = mlp.backward(pr, Xr, Yd)
    gd = unflatten(gr.astype(np.float64))
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        d = np.abs(gd[k] - ref[k])
        assert np.all(d <= bound[k]), (k, float((d / np.maximum(bound[k], 1e-300)).max()))
        de = np.abs(gd[k] - emu[k])
        tol = 0.02 * bound[k] + 1e-6 * np.abs(ref[k]).max()
        assert np.all(de <= tol), (k, float((de / tol).max()))
    g.close()


def test_mlp_sgd_tracks_oracle():
    avs = need_gpu()
    g = small_ctx(avs)
    rng = np.random.default_rng(12)
    p = mlp.init_params(6)
    P32 = flatten(p).astype(np.float32)
    g.mlp_set_params(P32)
    n = 512
    X = rng.standard_normal((n, 8)).astype(np.float32)
    Y = (X[:, :4] + 0.3 * X[:, 4:] > 0).astype(np.float32)
    pr = rounded_params(P32)
    Xr = bf16(X)
    l0 = mlp.loss(pr, Xr, Y)
    for _ in range(60):
        g.mlp_grad(X, Y, lr=0.5)
        pr = mlp.sgd(pr, mlp.backward(pr, Xr, Y), 0.5)
    _, lg = g.mlp_grad(X, Y, lr=0.0)
    lo = mlp.loss(pr, Xr, Y)
    assert lg < 0.7 * l0 and lo < 0.7 * l0
    assert abs(lg - lo) < 0.1 * lo


def test_features_and_labels_match_oracle():
    """Features within FP32 rounding of the oracle's; labels bit-exact against
    the oracle's labels of the same f and the same W (the moments of f the
    GPU uses, so that the equality test of the dominant label sees the same
    values on both sides)."""
    avs = need_gpu()
    w = wl.sweep_box((8, 8), base=(10, 10), max_refine=1, C1=2.0)
    r, g = pair(w, avs, amp=1e-2)
    X, Y = g.features()
    Wf, q = O.moments(2, r.xi, r.w, r.f)
    Xo = mlp.features(2, Wf, q, w.mesh.vol, w.mesh.faceL, w.mesh.faceR,
                      mu_ref=O.mu_ref_from_Kn(w.Kn, w.omega), omega=w.omega)
    assert np.allclose(X, Xo, rtol=2e-5, atol=2e-6)
    Wg = g.f_moments()
    m = mlp.criterion_values(2, r.xi, r.w, r.f, Wg, float(np.prod(w.base)))
    Yo = mlp.labels(m, m.max(0), r.level, w.C1, w.C2, w.max_refine)
    assert np.array_equal(Y, Yo)
    assert Yo[:, 1].sum() >= 1 and Yo[:, 1].sum() < len(Yo)


RYKOV_FEATURE_CASES = {
    "box": lambda: wl.sweep_box((8, 8), base=(10, 10), max_refine=1, C1=2.0),
    "sphere": lambda: small_sphere(),
}


@pytest.mark.parametrize("case", sorted(RYKOV_FEATURE_CASES))
def test_features_and_labels_match_oracle_rykov(case):
    """Diatomic gas (Rykov model, T_r = 0.8 T_t): features of the
    translational temperature and the total heat flux q_t + q_r within FP32
    rounding of the oracle's; labels bit-exact against the oracle's labels of
    the same f (G decides the criterion) and the same W, 2D (G, H, R) and 3D
    (G, R)."""
    avs = need_gpu()
    w = RYKOV_FEATURE_CASES[case]()
    w.model = "rykov"
    D = w.D
    r, g = pair_rykov(w, avs, amp=1e-2)
    X, Y = g.features()
    Wf, qt, qr = O.moments_rykov(D, r.xi, r.w, r.f)
    Xo = mlp.features(D, Wf, qt + qr, w.mesh.vol, w.mesh.faceL, w.mesh.faceR,
                      mu_ref=O.mu_ref_from_Kn(w.Kn, w.omega), omega=w.omega, rykov=True)
    assert np.allclose(X, Xo, rtol=2e-5, atol=2e-6)
    Wg = g.f_moments()
    assert Wg.shape[1] == D + 3
    m = mlp.criterion_values(D, r.xi, r.w, r.f, Wg, r.s)
    Yo = mlp.labels(m, m.max(0), r.level, w.C1, w.C2, w.max_refine)
    assert np.array_equal(Y, Yo)
    assert Yo[:, 1].sum() >= 1 and Yo[:, 1].sum() < len(Yo)
    g.close()


@pytest.mark.parametrize("model", ["shakhov", "rykov"])
def test_learned_adaptation_check_set_and_misses(model):
    """A learned adaptation applies exactly the decisions of the criterion
    restricted to its check set (a strict subset of the cells); a full one
    right after applies the decisions of the whole criterion and reports as
    misses exactly the nodes whose split or merge test the check set would
    have decided differently.  Both judged against the oracle's criterion on
    the same f and W, with the check set the library reports; for the
    monatomic gas and for the diatomic one (Rykov model, W with rho E_rot)."""
    avs = need_gpu()
    w = wl.sweep_box((16, 16), base=(10, 10), max_refine=2, C1=2.0)
    w.learned = True
    w.model = model
    r, g = pair_rykov(w, avs, amp=1e-3) if model == "rykov" else pair(w, avs, amp=1e-3)
    loss = g.mlp_train(400, lr=0.2)
    assert np.isfinite(loss)
    s, C1, C2 = r.s, w.C1, w.C2
    kinds = []
    for force_full in (False, False, True):
        t0 = g.tree()
        f = g.get_f()
        Wg = g.f_moments()
        st = g.adapt(force_full=force_full)
        full = bool(st["full"])
        kinds.append(full)
        cells = g.check_set()
        assert cells is not None and 0 < len(cells) < g.Nc
        assert np.array_equal(np.unique(cells), cells)
        M_full = O.criterion(2, t0["xi"], t0["w"], f, Wg)
        M_chk = O.criterion(2, t0["xi"], t0["w"], f[cells], Wg[cells])
        a, b = s * M_full, s * M_chk
        flips = int((((a > C1) != (b > C1)) | ((a < C2) != (b < C2))).sum())
        M_used = M_full if full else M_chk
        lv, bs, ky, _, _ = O.adapt_tree(2, t0["level"], t0["base"], t0["key"], M_used, s, C1, C2, w.max_refine)
        t1 = g.tree()
        assert np.array_equal(t1["level"], lv) and np.array_equal(t1["base"], bs) and np.array_equal(t1["key"], ky)
        if full:
            assert st["missed_nodes"] == flips
            assert st["checked_cells"] == g.Nc
        else:
            assert st["missed_nodes"] == 0 and st["checked_cells"] == len(cells)
    assert kinds[-1] and not all(kinds), kinds          # at least one learned and the forced full one
    g.close()


def _walled_box(n=32, precision="mixed"):
    wall = wl._bc_row(wl.BC_WALL, T=1.0)
    hot = wl._bc_row(wl.BC_WALL, T=1.3)
    mesh = wl.cartesian_mesh((n, n), (1.0, 1.0), bcs=[(wall, hot), (wall, wall)])
    v = 4.0 * wl.sqrt_RT(1.0)
    return wl.Workload(f"walled-box-{n}", mesh, 2, (12, 12), (-v, -v), (v, v), 2, Kn=0.05, omega=0.81,
                       Pr=2.0 / 3.0, C1=2.0, C2=wl.K_SIGMA * 2.0, W_inf=(1.0, 0.0, 0.0, 1.0),
                       W_init=wl.sweep_W(mesh), precision=precision, learned=True)


def _wall_heat_flux(w, q):
    """q . n at the cells next to a wall (outward normals of the boundary faces)."""
    m = w.mesh
    b = m.faceR < 0
    n = m.An[b] / np.linalg.norm(m.An[b], axis=1, keepdims=True)
    return (q[m.faceL[b]] * n).sum(1)


@pytest.mark.parametrize("model", ["shakhov", "rykov"])
def test_learned_proposer_gain_over_plain_criterion(model):
    """What the trained network gains, and what it costs, over four
    adaptations 10 steps apart.  The first adaptation of a context and the
    forced last one run the full criterion (the fallback and judge); the two
    between are learned.  Gain: the learned adaptations evaluate the criterion
    on at most half of the cells (budget a quarter, doubled once when the first
    full adaptation finds more than 1 % of the nodes decided wrongly by the
    check set).  Cost, judged by the plain criterion and by a plain run from
    the same start over the same steps: on the forced full adaptation the check
    set would have decided at most 1 % of the nodes differently (the
    fallback's own widening trigger), and the learned run's f-moments and wall
    heat flux differ from the plain run's by less than 1e-4 and 1 % (L1,
    relative), a fifth of the 5 % the paper takes as its accuracy standard
    (Sec. 4.6)."""
    avs = need_gpu()
    import time
    w = _walled_box()
    w.model = model
    gl = avs.AVS(w, learned=True, full_every=1000)
    gp = avs.AVS(w, learned=False)
    for g in (gl, gp):
        g.init_field(amp=1e-3, seed=21)
    loss = gl.mlp_train(400, lr=0.2)
    fracs, misses, tl, tp = [], [], 0.0, 0.0
    dt = gp.dt()
    for cycle in range(4):
        for g in (gl, gp):
            g.step(10, dt=dt)
        t0 = time.perf_counter(); sl = gl.adapt(force_full=(cycle == 3)); tl += time.perf_counter() - t0
        t0 = time.perf_counter(); sp = gp.adapt(); tp += time.perf_counter() - t0
        if not sl["full"]:
            fracs.append(sl["checked_cells"] / gl.Nc)
        else:
            misses.append(sl["missed_nodes"])
    Wl, ql = gl.moments()
    Wp, qp = gp.moments()
    l1_mom = np.abs(Wl - Wp).sum() / np.abs(Wp).sum()
    hf = np.abs(_wall_heat_flux(w, ql) - _wall_heat_flux(w, qp)).sum() / np.abs(_wall_heat_flux(w, qp)).sum()
    print(f"\nlearned proposer ({model}): loss {loss:.4f}, checked fraction {np.mean(fracs):.3f}, misses {misses} of "
          f"{gl.Nv} nodes, L1 f-moment gap {l1_mom:.2e}, wall heat-flux gap {hf:.2e}, "
          f"adapt time learned {tl:.3f}s plain {tp:.3f}s")
    assert len(fracs) == 2 and len(misses) == 2
    assert max(fracs) <= 0.5
    assert misses[-1] <= 0.01 * gl.Nv
    assert l1_mom < 1e-4 and hf < 1e-2
    gl.close(); gp.close()
