"""avs_criterion_noalloc, the entry point that allocates no device memory.

It serves callers that cannot allocate on demand (an embedder whose device
memory belongs to another allocator, or a latency-sensitive loop that cannot
afford cudaMalloc's synchronisation).  Its output must equal that of the
regular criterion entry point (avs_criterion), which is bit-exact against the
oracle, on two calls in a row with different inputs (the shared scratch must
not leak the first call's values into the second).  This file is named so that
pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O

from gpu_common import need_gpu, small_cylinder, small_sphere

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dim", [2, 3])
def test_noalloc_criterion_matches_regular_entry_point_twice(dim):
    """2D (G and H per node, a quadtree) and 3D (G only, an octree): two calls
    in a row with different f and W, each bit-exact with avs_criterion."""
    avs = need_gpu()
    import torch
    L = avs.load()
    fn = L.avs_criterion_noalloc
    fn.restype = C.c_int
    fn.argtypes = [C.c_int, C.c_int, C.c_int] + [C.c_void_p] * 6
    w = small_cylinder() if dim == 2 else small_sphere()
    r = O.Run(w)
    g = avs.AVS(w, precision="fp64")
    t = g.tree()
    xi = torch.from_numpy(t["xi"]).cuda()
    wt = torch.from_numpy(t["w"]).cuda()
    stream = torch.cuda.current_stream()
    for seed, amp in ((3, 1e-2), (11, 5e-2)):
        r.init_field(amp=amp, seed=seed)
        g.set_f(r.f)
        Wf, _ = O.moments(dim, r.xi, r.w, r.f)
        M_ref = g.criterion(Wf)                       # existing entry point
        f_d = torch.from_numpy(np.ascontiguousarray(r.f)).cuda()
        W_d = torch.from_numpy(np.ascontiguousarray(Wf)).cuda()
        M_d = torch.full((g.Nv,), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(dim, g.Nc, g.Nv, f_d.data_ptr(), xi.data_ptr(), wt.data_ptr(), W_d.data_ptr(),
                M_d.data_ptr(), stream.cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        assert np.array_equal(M_d.cpu().numpy(), M_ref)
    # sizes beyond the fixed scratch are rejected before any work
    st = fn(dim, (1 << 18) + 1, 8, f_d.data_ptr(), xi.data_ptr(), wt.data_ptr(), W_d.data_ptr(),
            M_d.data_ptr(), stream.cuda_stream)
    assert st == -7
    st = fn(dim, 8, (1 << 17) + 1, f_d.data_ptr(), xi.data_ptr(), wt.data_ptr(), W_d.data_ptr(),
            M_d.data_ptr(), stream.cuda_stream)
    assert st == -7
    g.close()
