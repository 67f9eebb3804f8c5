"""Model maintenance across frames on the GPU against the FP64 oracle: box
downsampling (Sec. III.A, Algorithm 3), the back-projection error (Sec. III)
and the frame loop of Algorithm 2 (Tracker) over synthetic push sequences.

Downsampling: the box of every point is an FP32 decision taken by the same
rule on both sides, so the merged point count and the output order are
compared exactly; the merged values (FP32 sums on the GPU, FP64 in the
oracle) within 2e-5 mm / 1e-5.  The frame loop is checked in lock step: each
stage of a GPU frame is recomputed by the oracle from the GPU's own input to
that stage (nodes, fusion, downsampling, error), and the whole frame is
compared with the oracle's frame from the same model (error within
0.02 mm)."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
from tests import gpu_common as C

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _E():
    import paper_1803_02009_b300 as E
    return E


def _fused_like(name, seed=1):
    """A model as fusion leaves it: the scene's model points (omega 5) and the
    back-projected pixels of its target depth (omega 1, newer time stamp)."""
    s = C.scene(name, seed)
    fx, fy, cx, cy, W, H = s.intr
    d = s.tgt_depth
    v, u = np.nonzero(d > 0)
    z = d[v, u].astype(np.float64)
    lifted = np.stack([(u - cx) * z / fx, (v - cy) * z / fy, z, np.ones_like(z)], 1).astype(np.float32)
    pos = np.concatenate([s.model_pos, lifted])
    nrm = np.concatenate([s.model_nrm, np.tile(np.array([0, 0, -1, 0], np.float32), (len(z), 1))])
    col = np.concatenate([s.model_col, s.tgt_color[v, u]])
    t = np.concatenate([s.model_t, np.full(len(z), 3, np.int32)])
    return s, pos, nrm, col, t


@pytest.mark.parametrize("name,box", [("tissue_160x120_n64", 0.5), ("tissue_640x480_n2048", 0.2)])
def test_downsample_matches_oracle(name, box):
    torch, E = _torch(), _E()
    s, pos, nrm, col, t = _fused_like(name)
    n = pos.shape[0]
    fx, fy, cx, cy, W, H = s.intr
    ctx = E.Context(max_points=n, max_nodes=64, max_width=W, max_height=H)
    dev = "cuda"
    out = ctx.downsample(torch.from_numpy(pos).to(dev), torch.from_numpy(nrm).to(dev), torch.from_numpy(col).to(dev),
                         torch.from_numpy(t).to(dev), box, omega_max=20.0, tau_weight=3.0)
    cnt = out["counts"].cpu().numpy()
    po, no, co, to, ko = oracle.downsample(pos, nrm, col, t, box, 20.0, 3.0)
    k = int(cnt[0])
    assert cnt[1] == 0 and k == po.shape[0] and 0 < k < n
    gp, gn, gc, gt = (out[key][:k].cpu().numpy() for key in ("pos", "nrm", "col", "t"))
    assert np.array_equal(gt, to)
    assert np.array_equal(gp[:, 3], po[:, 3]) and np.array_equal(gn[:, 3], no[:, 3])
    assert np.abs(gp[:, :3] - po[:, :3]).max() < 2e-5
    assert np.abs(gn[:, :3] - no[:, :3]).max() < 1e-5
    assert np.abs(gc - co).max() < 1e-5
    # capacity: truncated output, status set
    out2 = ctx.downsample(torch.from_numpy(pos).to(dev), torch.from_numpy(nrm).to(dev),
                          torch.from_numpy(col).to(dev), torch.from_numpy(t).to(dev), box, capacity=k - 7)
    c2 = out2["counts"].cpu().numpy()
    assert c2[0] == k - 7 and c2[1] == 3   # ED_ERR_CAPACITY
    assert np.array_equal(out2["pos"][:k - 7].cpu().numpy(), gp[:k - 7])


@pytest.mark.parametrize("name", ["tissue_160x120_n64", "tissue_640x480_n2048"])
def test_depth_error_matches_oracle(name):
    torch, E = _torch(), _E()
    s = C.scene(name)
    fx, fy, cx, cy, W, H = s.intr
    ctx = E.Context(max_points=s.N, max_nodes=64, max_width=W, max_height=H)
    # the source model seen against the (deformed, moved) target depth
    got = ctx.depth_error(torch.from_numpy(s.model_pos).cuda(), torch.from_numpy(s.tgt_depth).cuda(),
                          s.intr).cpu().numpy()
    mean, cnt, mx, rms = oracle.depth_error(s.model_pos, s.tgt_depth, s.intr)
    assert got[1] == cnt and got[2] == mx
    assert got[0] / got[1] == pytest.approx(mean, rel=1e-12)
    assert np.sqrt(got[3] / got[1]) == pytest.approx(rms, rel=1e-12)


def _tracker(seq_name, n_frames, box, max_nodes, seed=1):
    E = _E()
    S = synth.make_push_sequence(seq_name, n_frames, seed=seed)
    cfg = S.cfg
    radius = oracle.calibrate_radius(S.model_pos, max_nodes)
    tc = E.TrackerConfig(node_radius=radius, max_nodes=max_nodes, box=box, n_gn=cfg.n_gn,
                         normal_half_width=cfg.normal_half_width,
                         solver=E.SolverParams(n_pcg=cfg.n_pcg), fuse=E.FuseParams())
    cap = S.model_pos.shape[0] + 2 * cfg.W * cfg.H
    import torch
    T = E.Tracker(torch.from_numpy(S.model_pos).cuda(), torch.from_numpy(S.model_nrm).cuda(),
                  torch.from_numpy(S.model_col).cuda(), torch.from_numpy(S.model_t).cuda(), S.intr, tc, cap)
    return S, T, tc, radius


def test_tracker_lockstep_push_sequence_small():
    torch = _torch()
    S, T, tc, radius = _tracker("push_160x120", 3, 0.5, 128)
    for f in S.frames:
        m_in = {k: v.cpu().numpy() for k, v in T.model().items()}
        dev = lambda a: torch.from_numpy(a).cuda()   # noqa: E731
        info = T.process(dev(f.depth), dev(f.color), f.index, truth_depth=dev(f.depth_clean))
        assert info["status"] == 0 and info["gn"]["status"] == 0
        # nodes regenerated on the frame's input model (bit-exact)
        node_pt, _ = oracle.poisson_nodes(m_in["pos"], radius, 128)
        g = T.ctx.graph
        assert g.m == len(node_pt)
        assert np.array_equal(g.nodes[:g.m, :3].cpu().numpy(), m_in["pos"][node_pt, :3])
        # fusion of the GPU's warped model
        n = m_in["pos"].shape[0]
        wpos, wnrm = T.wpos[:n].cpu().numpy(), T.wnrm[:n].cpu().numpy()
        nm = T.nmap.cpu().numpy()
        F = dataclasses.replace(oracle.FuseParams(), frame=f.index)
        fp, fn, fc, ft, _ = oracle.fuse(m_in["pos"], m_in["nrm"], m_in["col"], m_in["t"], wpos, wnrm, f.depth, nm,
                                        f.color, S.intr, F, T.capacity)
        nf = info["fused"]
        assert nf == fp.shape[0]
        B = {k: T.B[k][:nf].cpu().numpy() for k in ("pos", "nrm", "col", "t")}
        assert np.array_equal(B["t"], ft) and np.array_equal(B["pos"][:, 3], fp[:, 3])
        assert np.abs(B["pos"][:, :3] - fp[:, :3]).max() < 2e-4
        # downsampling of the GPU's fused model
        dp, dn, dc, dt, _ = oracle.downsample(B["pos"], B["nrm"], B["col"], B["t"], tc.box, 20.0, 3.0)
        m_out = {k: v.cpu().numpy() for k, v in T.model().items()}
        assert m_out["pos"].shape[0] == dp.shape[0] == info["model"]
        assert np.array_equal(m_out["t"], dt) and np.array_equal(m_out["pos"][:, 3], dp[:, 3])
        assert np.abs(m_out["pos"][:, :3] - dp[:, :3]).max() < 2e-5
        # back-projection error of the GPU's warped model
        mean, cnt, mx, rms = oracle.depth_error(wpos, f.depth_clean, S.intr)
        assert info["error_pixels"] == cnt and info["error_mean_mm"] == pytest.approx(mean, rel=1e-12)
        # the whole frame against the oracle's frame from the same model
        _, oinfo = oracle.track_frame((m_in["pos"], m_in["nrm"], m_in["col"], m_in["t"]), f.depth, f.color, S.intr,
                                      radius, 128, tc.box, tc.n_gn, tc.solver.n_pcg, f.index, tc.normal_half_width,
                                      truth_depth=f.depth_clean)
        assert abs(info["error_mean_mm"] - oinfo["error_mean_mm"]) < 0.02
        assert abs(info["model"] - oinfo["model"]) <= 0.01 * oinfo["model"]
        assert info["error_mean_mm"] < 0.6


def test_tracker_push_sequence_full_size():
    torch = _torch()
    S, T, tc, radius = _tracker("push_640x480_n2048", 3, 0.2, 2048)
    dev = lambda a: torch.from_numpy(a).cuda()   # noqa: E731
    first = None
    for f in S.frames:
        m_in = {k: v.cpu().numpy() for k, v in T.model().items()} if first is None else None
        info = T.process(dev(f.depth), dev(f.color), f.index, truth_depth=dev(f.depth_clean))
        assert info["status"] == 0 and info["gn"]["status"] == 0 and info["nodes"] == 2048
        assert info["error_mean_mm"] < 0.3
        if first is None:
            first = info
            _, oinfo = oracle.track_frame((m_in["pos"], m_in["nrm"], m_in["col"], m_in["t"]), f.depth, f.color,
                                          S.intr, radius, 2048, tc.box, tc.n_gn, tc.solver.n_pcg, f.index,
                                          tc.normal_half_width, truth_depth=f.depth_clean)
            assert abs(info["error_mean_mm"] - oinfo["error_mean_mm"]) < 0.01
            assert abs(info["model"] - oinfo["model"]) <= 0.005 * oinfo["model"]
