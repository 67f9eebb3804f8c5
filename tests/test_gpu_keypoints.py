"""The sparse key-correspondence term E_corr (Sec. II.E, w_corr = 10) on the
GPU against the FP64 oracle: key-point skinning, energy, normal equations,
the PCG update and the gradient."""
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


def _setup(name, nk, radius=None, max_nodes=None):
    torch, E = _torch(), _E()
    s = C.scene(name)
    kp, tgt, _ = synth.make_keypoints(s, nk, seed=3)
    fx, fy, cx, cy, W, H = s.intr
    cap = max(64, max_nodes or 64)
    ctx = E.Context(max_points=s.N + 3 * nk, max_nodes=cap, max_width=W, max_height=H, max_cells=1 << 24)
    pos = torch.from_numpy(s.model_pos).cuda()
    nrm = torch.from_numpy(s.model_nrm).cuda()
    depth = torch.from_numpy(s.tgt_depth).cuda()
    nmap = ctx.compute_normals(depth, s.intr, s.cfg.normal_half_width)
    kpt = torch.from_numpy(kp).cuda()
    tgtt = torch.from_numpy(tgt).cuda()
    ctx.set_keypoints(kpt, tgtt, oracle.W_CORR)
    if radius is None:
        g = ctx.build_graph(pos, nrm, nodes=torch.from_numpy(s.nodes).cuda(), sigma=s.sigma)
        sig = s.sigma
    else:
        g = ctx.build_graph(pos, nrm, node_radius=radius, max_nodes=max_nodes, sigma=radius)
        sig = radius
    torch.cuda.synchronize()
    G = dict(ctx=ctx, graph=g, nmap=nmap, frame=E.make_frame(depth, nmap, s.intr), pos=pos, nrm=nrm,
             keep=(kpt, tgtt, depth))
    og = C.oracle_graph_from_gpu(G)
    og = oracle.Graph(g=og.g, idx=og.idx[:s.N], idx_k1=None, key=None, w=og.w[:s.N], nbr=og.nbr, node_pt=None,
                      m_total=og.m_total)
    K = oracle.keypoints(kp, tgt[:, :3].astype(np.float64), og.g, K=4, mode=0, sigma=sig)
    P = oracle.Problem(s.model_pos, s.model_nrm, og, s.tgt_depth, nmap.cpu().numpy(), s.intr, s.pose_prior,
                       keypoints=K)
    return s, G, P, K


def _step(s, G, P, seed=0):
    torch, E = _torch(), _E()
    ctx, m = G["ctx"], G["graph"].m
    rng = np.random.default_rng(seed)
    x0 = np.zeros((m, 12))
    x0[:, [0, 5, 10]] = 1.0
    x0 = (x0 + rng.normal(0, 1e-3, x0.shape)).astype(np.float32)
    pose0 = np.asarray(s.pose_prior) + rng.normal(0, 1e-3, 6)
    x = torch.from_numpy(x0).cuda()
    pose = torch.from_numpy(pose0.copy()).cuda()
    wpos = torch.empty((s.N, 4), dtype=torch.float32, device="cuda")
    wnrm = torch.empty_like(wpos)
    pix = torch.empty(s.N + 3 * P.s.NK, dtype=torch.int32, device="cuda")
    ctx.set_debug(wpos, wnrm, pix)
    st = E.new_stats()
    prm = C.solver(s)
    ctx.gn_step(G["frame"], prm, x, pose, stats=st)
    sysd = {k: v.cpu().numpy() for k, v in ctx.export_system().items()}
    ctx.set_debug(None, None, None)
    return dict(x0=x0, pose0=pose0, x1=x.cpu().numpy(), pose1=pose.cpu().numpy(), pix=pix.cpu().numpy()[:s.N],
                wpos=wpos.cpu().numpy(), wnrm=wnrm.cpu().numpy(), stats=E.read_stats(st)[0], sys=sysd, prm=prm)


def _check(s, G, P, K, o):
    st = o["stats"]
    assert st["status"] == 0
    # key-point skinning: the rows after the model points, three per key point
    idx = G["graph"].idx_long().cpu().numpy()
    assert np.array_equal(idx[s.N::3][:K.idx.shape[0]], K.idx)
    # association of the model points: bit-exact on the GPU's warped floats
    ref_pix = oracle.associate_f32(o["wpos"], o["wnrm"], s.tgt_depth, G["nmap"].cpu().numpy(), s.intr)
    assert np.array_equal(ref_pix, o["pix"])
    Q = oracle.NormalEq(P, o["x0"].astype(np.float64), o["pose0"], pix_in=o["pix"])
    assert Q.E[5] > 0.0
    assert st["e_corr"] == pytest.approx(Q.E[5], rel=C.TOL_E)
    assert st["energy"] == pytest.approx(Q.energy, rel=C.TOL_E)
    assert st["n_valid"] == Q.n_valid
    sd = o["sys"]
    assert np.array_equal(sd["row_ptr"], Q.row_ptr) and np.array_equal(sd["col"], Q.col)
    assert np.abs(sd["blocks"] - Q.blk).max() <= 3e-4 * np.abs(Q.blk).max()
    assert np.abs(sd["grad"] - Q.g).max() <= 3e-4 * np.abs(Q.g).max()
    d, _, _, _ = Q.pcg(-Q.g, o["prm"].n_pcg, jitter=o["prm"].jitter)
    m = P.m
    x_ref = o["x0"].astype(np.float64) + d[:12 * m].reshape(m, 12)
    err = np.abs(o["x1"] - x_ref) / np.maximum(1.0, np.abs(x_ref))
    assert err.max() <= C.TOL_X, err.max()
    assert np.abs(o["pose1"] - (o["pose0"] + d[12 * m:])).max() <= C.TOL_X


def test_keypoint_step_small():
    s, G, P, K = _setup("tissue_160x120_n64", 60)
    _check(s, G, P, K, _step(s, G, P))


def test_keypoint_step_full_size():
    s, G, P, K = _setup("tissue_640x480_n2048", 500, radius=C.radius_for("tissue_640x480_n2048"), max_nodes=2048)
    _check(s, G, P, K, _step(s, G, P, 1))


def test_keypoint_energy_and_gradient():
    torch, E = _torch(), _E()
    s, G, P, K = _setup("tissue_160x120_n64", 60)
    o = _step(s, G, P, 2)
    ctx = G["ctx"]
    x = torch.from_numpy(o["x0"]).cuda().requires_grad_(True)
    pose = torch.from_numpy(o["pose0"].copy()).cuda().requires_grad_(True)
    e = E.EDEnergy.apply(x, pose, ctx, G["frame"], o["prm"])
    e.backward()
    E_ref, terms, _ = oracle.energy(P, o["x0"].astype(np.float64), o["pose0"], pix_in=o["pix"])
    assert float(e.detach()) == pytest.approx(E_ref, rel=C.TOL_E)
    eo = ctx.energy(G["frame"], o["prm"], torch.from_numpy(o["x0"]).cuda(), torch.from_numpy(o["pose0"]).cuda())
    assert float(eo[6]) == pytest.approx(terms[5], rel=C.TOL_E)
    g_ref = oracle.gradient(P, o["x0"].astype(np.float64), o["pose0"], o["pix"])
    m = P.m
    sc = np.abs(g_ref).max()
    assert np.abs(x.grad.cpu().numpy().ravel() - g_ref[:12 * m]).max() <= 3e-4 * sc
    assert np.abs(pose.grad.cpu().numpy() - g_ref[12 * m:]).max() <= 3e-4 * max(sc, 1.0)


def test_keypoints_removed_restore_plain_energy():
    torch, E = _torch(), _E()
    s, G, P, K = _setup("tissue_160x120_n64", 60)
    ctx = G["ctx"]
    ctx.set_keypoints(None)
    g = ctx.build_graph(G["pos"], G["nrm"], nodes=torch.from_numpy(s.nodes).cuda(), sigma=s.sigma)
    x = ctx.identity_x()
    pose = torch.tensor(s.pose_prior, dtype=torch.float64, device="cuda")
    st = E.new_stats()
    ctx.gn_step(G["frame"], C.solver(s), x, pose, stats=st)
    assert E.read_stats(st)[0]["e_corr"] == 0.0
    assert g.idx.shape[0] == s.N
