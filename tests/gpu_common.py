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


def pair_rykov(w, avs, precision=None, amp=1e-2, seed=7):
    """Oracle run and CUDA context of the diatomic gas (Rykov model), same
    tree, same f with the rotational temperature T_r = 0.8 T_t."""
    r = O.Run(w)
    g = avs.AVS(w, precision=precision)
    t = g.tree()
    assert np.array_equal(t["level"], r.level) and np.array_equal(t["key"], r.key)
    Wp = np.column_stack([w.W_init, 0.8 * w.W_init[:, w.D + 1]])
    r.init_field(Wp, amp=amp, seed=seed)
    g.set_f(r.f)
    g.set_W(r.Wc)
    assert r.f.shape[1] == g.NA and r.Wc.shape[1] == g.NW
    return r, g


def rel_err(a, b):
    """max |a - b| / max |b| per leading index, then max."""
    a = np.asarray(a); b = np.asarray(b)
    axes = tuple(range(1, b.ndim))
    scale = np.abs(b).max(axis=axes, keepdims=True)
    scale[scale == 0] = 1.0
    return float((np.abs(a - b) / scale).max())


def field_err(Wg, Wo, D, qg=None, qo=None):
    """Macroscopic error by field: rho and E relative to their values,
    momentum relative to rho sqrt(2 R T) + |rho U| (the field's scale), and,
    when given, the heat flux q (Eq. 8) relative to rho (2 R T)^(3/2) (the
    scale of a third velocity moment)."""
    rho = Wo[:, 0]
    e_rho = np.abs(Wg[:, 0] - rho) / np.abs(rho)
    m = Wo[:, 1:1 + D]
    RT = (Wo[:, D + 1] - 0.5 * (m * m).sum(1) / rho) / (1.5 * rho)
    mscale = np.sqrt((m * m).sum(1)) + rho * np.sqrt(2 * RT)
    e_m = np.abs(Wg[:, 1:1 + D] - m).max(1) / mscale
    e_E = np.abs(Wg[:, D + 1] - Wo[:, D + 1]) / np.abs(Wo[:, D + 1])
    out = dict(rho=float(e_rho.max()), mom=float(e_m.max()), E=float(e_E.max()))
    if qg is not None:
        qscale = rho * (2.0 * RT) ** 1.5
        out["q"] = float((np.abs(np.asarray(qg) - np.asarray(qo)).max(1) / qscale).max())
    return out


def q_err(g, r, D):
    """Heat flux of the GPU's f against the oracle's, both about the mean
    velocity of their own f (Eq. 8), relative to rho (2 R T)^(3/2)."""
    _, qg = g.moments()
    Wo, qo = O.moments(D, r.xi, r.w, r.f)
    return field_err(Wo, Wo, D, qg, qo)["q"]


def patch_mesh(mesh, targets, rings=2):
    """Sub-mesh of the cells within `rings` face-neighbour steps of `targets`.

    Faces are kept, in their original order, when both cells are in the patch
    or when the face is a boundary face of a patch cell, so every cell within
    rings - 1 steps keeps all its faces and neighbours.  One explicit step of
    a target cell depends only on the cells within two steps (its faces'
    upwind cells and their gradients), so on the patch it computes the same
    update as on the whole mesh.  Returns (sub-mesh, patch cell indices,
    positions of the targets in the patch)."""
    from paper_2212_05645_gb300 import workloads as wl
    L, R = mesh.faceL, mesh.faceR
    inner = R >= 0
    a = np.concatenate([L[inner], R[inner]])
    b = np.concatenate([R[inner], L[inner]])
    order = np.argsort(a, kind="stable")
    a, b = a[order], b[order]
    start = np.searchsorted(a, np.arange(mesh.Nc + 1))
    cells = set(int(t) for t in targets)
    frontier = list(cells)
    for _ in range(rings):
        nxt = []
        for c in frontier:
            for n in b[start[c]:start[c + 1]]:
                n = int(n)
                if n not in cells:
                    cells.add(n)
                    nxt.append(n)
        frontier = nxt
    cells = np.array(sorted(cells), dtype=np.int64)
    inv = -np.ones(mesh.Nc, dtype=np.int64)
    inv[cells] = np.arange(len(cells))
    keep = (inv[L] >= 0) & ((R < 0) | (inv[np.maximum(R, 0)] >= 0))
    fL = inv[L[keep]].astype(np.int32)
    fR = np.where(R[keep] >= 0, inv[np.maximum(R[keep], 0)], R[keep]).astype(np.int32)
    sub = wl.Mesh(mesh.D, fL, fR, mesh.An[keep], mesh.rL[keep], mesh.rR[keep], mesh.vol[cells], mesh.xc[cells],
                  mesh.bc, name="patch").contiguous()
    return sub, cells, inv[np.asarray(targets, dtype=np.int64)]


def sample_cells(mesh, n_random=2, seed=7):
    """Cells to sample at full size: nearest to and farthest from the body
    centre, the ones closest to the +z / +y axis direction (3D poles), and a
    few seeded random ones."""
    x = mesh.xc - mesh.xc.mean(0)
    r = np.linalg.norm(x, axis=1)
    pick = [int(np.argmin(r)), int(np.argmax(r))]
    ax = x[:, -1] / np.maximum(r, 1e-30)
    pick += [int(np.argmax(ax)), int(np.argmin(ax))]
    rng = np.random.default_rng(seed)
    pick += [int(i) for i in rng.integers(0, mesh.Nc, n_random)]
    return sorted(set(pick))
