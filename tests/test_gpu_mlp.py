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

from gpu_common import need_gpu, pair

pytestmark = pytest.mark.gpu


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def rounded_params(P32):
    p = unflatten(P32.astype(np.float64))
    for k in ("W1", "W2", "W3"):
        p[k] = bf16(p[k])
    return p


def relnorm(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def small_ctx(avs, learned=True):
    w = wl.sweep_box((6, 6), base=(8, 8), max_refine=1)
    return avs.AVS(w, learned=learned)


def test_mlp_forward_and_gradients_match_oracle():
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
    z_ref, _ = mlp.forward(pr, Xr)
    z = g.mlp_forward(X)
    assert relnorm(z, z_ref) < 2e-2
    gr, loss = g.mlp_grad(X, Y, lr=0.0)
    assert abs(loss - mlp.loss(pr, Xr, Y)) < 1e-2 * mlp.loss(pr, Xr, Y)
    ref = mlp.backward(pr, Xr, Y)
    gd = unflatten(gr.astype(np.float64))
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, b = gd[k].reshape(-1), ref[k].reshape(-1)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        assert relnorm(a, b) < 6e-2 and cos > 0.998, (k, relnorm(a, b), cos)
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
    avs = need_gpu()
    w = wl.sweep_box((8, 8), base=(10, 10), max_refine=1, C1=2.0)
    r, g = pair(w, avs, amp=1e-2)
    X, Y = g.features()
    Wf, q = O.moments(2, r.xi, r.w, r.f)
    Xo = mlp.features(2, Wf, q, w.mesh.vol, w.mesh.faceL, w.mesh.faceR,
                      mu_ref=O.mu_ref_from_Kn(w.Kn, w.omega), omega=w.omega)
    assert np.allclose(X, Xo, rtol=2e-5, atol=2e-6)
    m = mlp.criterion_values(2, r.xi, r.w, r.f, Wf, float(np.prod(w.base)))
    Yo = mlp.labels(m, m.max(0), r.level, w.C1, w.C2, w.max_refine)
    assert (Y == Yo).mean() > 0.995
    assert Yo[:, 1].sum() >= 1


def test_learned_adaptation_check_set_and_misses():
    """After training on the criterion's own labels the proposer's check set is
    a strict subset of the cells; a full adaptation right after reports the
    misses of the check set, and decisions with the full criterion stay exact."""
    avs = need_gpu()
    w = wl.sweep_box((16, 16), base=(10, 10), max_refine=2, C1=2.0)
    w.learned = True
    r, g = pair(w, avs, amp=1e-3)
    loss = g.mlp_train(400, lr=0.2)
    assert np.isfinite(loss)
    st_l = g.adapt()                          # learned step (trained network, not a full step)
    assert st_l["full"] in (0, 1)
    assert 0 < st_l["checked_cells"] <= g.Nc
    # the plain oracle adaptation from the same state gives the same tree when no node was missed
    o = r.adapt()
    if st_l["full"] == 1 or st_l["missed_nodes"] == 0:
        assert st_l["Nv"] == o["Nv"]
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


def test_learned_proposer_gain_over_plain_criterion():
    """What the trained network gains: the criterion runs on a quarter of the
    cells (the proposer's budget).  The plain criterion stays the judge: it
    counts the nodes whose decision the check set got wrong, and the learned
    run and the plain run (same start, same steps) are compared by the L1 gap
    of their f-moments and wall heat flux."""
    avs = need_gpu()
    import time
    w = _walled_box()
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
    print(f"\nlearned proposer: loss {loss:.4f}, checked fraction {np.mean(fracs):.3f}, misses {misses}, "
          f"L1 f-moment gap {l1_mom:.2e}, wall heat-flux gap {hf:.2e}, adapt time learned {tl:.3f}s plain {tp:.3f}s")
    assert np.mean(fracs) <= 0.6
    assert misses[-1] < 0.5 * gl.Nv
    assert l1_mom < 1e-2 and hf < 0.2
    gl.close(); gp.close()
