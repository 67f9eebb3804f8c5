"""The allocation-free energy entry point against the context-based one.

ed_energy_noalloc exists for callers that cannot allocate device memory
(they are handed their buffers by a host framework, or forbid allocation
after start-up).  It keeps its reduction
scratch in a fixed array inside the library; this test calls it through the
C ABI twice in a row (the second call reuses the array the first one left
behind), then captures one call into a CUDA graph and replays it twice, and
checks every result against ed_energy within the energy tolerance of the
parity tests.  It lives in a file of its own, collected
last, and passes alone in a fresh process as well as after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from tests import gpu_common as G


@pytest.mark.gpu
def test_energy_noalloc_matches_energy_twice():
    import torch
    import paper_1803_02009_b300 as E

    L = E.lib()
    fn = L.ed_energy_noalloc
    vp = C.c_void_p
    fn.argtypes = [vp, vp, vp, vp, C.c_int, vp, vp, C.c_int, C.c_int, C.POINTER(E.Frame),
                   C.POINTER(E.SolverParamsC), vp, vp, vp, vp]
    fn.restype = C.c_int

    s = G.scene("tissue_160x120_n64")
    S = G.gpu_setup(s)
    ctx, g = S["ctx"], S["graph"]
    rng = np.random.default_rng(11)
    x0 = np.zeros((g.m, 12), np.float32)
    x0[:, [0, 5, 10]] = 1.0
    x0 += rng.normal(0, 2e-3, x0.shape).astype(np.float32)
    x = torch.from_numpy(x0).cuda()
    pose = torch.tensor(np.asarray(s.pose_prior) + rng.normal(0, 1e-3, 6), dtype=torch.float64, device="cuda")
    prm = G.solver(s)
    ref = ctx.energy(S["frame"], prm, x, pose).cpu().numpy()
    pc = prm.c()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        rc = fn(vp(S["pos"].data_ptr()), vp(S["nrm"].data_ptr()), vp(g.idx.data_ptr()), vp(g.weights.data_ptr()),
                s.N, vp(g.nodes.data_ptr()), vp(g.nbr.data_ptr()), g.m, g.nbr.shape[1], C.byref(S["frame"]),
                C.byref(pc), vp(x.data_ptr()), vp(pose.data_ptr()), vp(out.data_ptr()), stream)
        assert rc == 0, f"call {call}: status {rc}"
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(ref[0], rel=G.TOL_E), call
        for k in range(1, 6):
            assert got[k] == pytest.approx(ref[k], rel=G.TOL_E, abs=1e-6 * ref[0]), (call, k)
    # one call captured into a CUDA graph (it takes the scratch address the
    # plain calls above looked up) and replayed twice
    out_g = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cs = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = fn(vp(S["pos"].data_ptr()), vp(S["nrm"].data_ptr()), vp(g.idx.data_ptr()), vp(g.weights.data_ptr()),
                s.N, vp(g.nodes.data_ptr()), vp(g.nbr.data_ptr()), g.m, g.nbr.shape[1], C.byref(S["frame"]),
                C.byref(pc), vp(x.data_ptr()), vp(pose.data_ptr()), vp(out_g.data_ptr()), cs)
    assert rc == 0, f"captured call: status {rc}"
    for rep in range(2):
        out_g.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        got = out_g.cpu().numpy()
        assert got[0] == pytest.approx(ref[0], rel=G.TOL_E), rep
        for k in range(1, 6):
            assert got[k] == pytest.approx(ref[k], rel=G.TOL_E, abs=1e-6 * ref[0]), (rep, k)
    # sizes beyond the fixed scratch are refused before any launch
    rc = fn(vp(S["pos"].data_ptr()), vp(S["nrm"].data_ptr()), vp(g.idx.data_ptr()), vp(g.weights.data_ptr()),
            (1 << 21) + 1, vp(g.nodes.data_ptr()), vp(g.nbr.data_ptr()), g.m, g.nbr.shape[1], C.byref(S["frame"]),
            C.byref(pc), vp(x.data_ptr()), vp(pose.data_ptr()), vp(out.data_ptr()), stream)
    assert rc == 3
