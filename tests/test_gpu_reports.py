"""Error reports against the FP64 oracle at the full workload sizes.

Differentiation (640x480, 2048 nodes): the autograd energy's hand-written
backward against the oracle gradient, against central finite differences of
the oracle's FP64 energy (h = 1e-4) at 100 seeded node coordinates and the 6
pose coordinates, and against the J^T r that the Gauss-Newton step assembles
with its own kernels.

Precision (160x120 over the whole 5-iteration trajectory, 640x480 / 2048
nodes over 3 iterations, 1280x720 / 4096 nodes for one iteration): plain
FP32 and the two mixed forms (compensated block reductions and an FP64
node-parameter master copy, with the PCG dot products and norms in
float-float or in FP64), each result's error against the oracle stated:
energy, node parameters, warped points in mm.

With ED_REPORT_DIR set, every test also writes its figures there as JSON."""
import json
import os

import numpy as np
import pytest

import oracle
from tests import gpu_common as C

pytestmark = pytest.mark.gpu

SMALL = "tissue_160x120_n64"
METRIC = "tissue_640x480_n2048"
LARGE = "tissue_1280x720_n4096"


def _torch():
    import torch
    return torch


def _E():
    import paper_1803_02009_b300 as E
    return E


def _report(name, data):
    d = os.environ.get("ED_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, name + ".json"), "w") as f:
            json.dump(data, f, indent=1, default=float)
    print(name, json.dumps(data, default=float))


def _start(s, m, seed):
    rng = np.random.default_rng(seed)
    x0 = np.zeros((m, 12))
    x0[:, [0, 5, 10]] = 1.0
    x0 = (x0 + rng.normal(0, 1e-3, x0.shape)).astype(np.float32)
    pose0 = np.asarray(s.pose_prior) + rng.normal(0, 1e-3, 6)
    return x0, pose0


def _sub_problem(P, G, s, sel):
    """The same problem restricted to the points `sel` (every node kept): with
    the association frozen, the data terms of the other points are equal on
    both sides of a central difference in a coordinate of a node they do not
    depend on, so the finite difference is unchanged."""
    og = C.oracle_graph_from_gpu(G)
    sub = oracle.Graph(g=og.g, idx=og.idx[sel], idx_k1=None, key=None, w=og.w[sel], nbr=og.nbr, node_pt=None,
                       m_total=og.m_total)
    return oracle.Problem(s.model_pos[sel], s.model_nrm[sel], sub, s.tgt_depth, G["nmap"].cpu().numpy(), s.intr,
                          s.pose_prior)


def test_differentiation_full_size():
    torch, E = _torch(), _E()
    s = C.scene(METRIC)
    G = C.gpu_setup(s, radius=C.radius_for(METRIC), max_nodes=2048)
    ctx, m = G["ctx"], G["graph"].m
    x0, pose0 = _start(s, m, 4)
    prm = C.solver(s)
    # forward + hand-written backward through the autograd function
    xg = torch.from_numpy(x0).cuda().requires_grad_(True)
    pg = torch.from_numpy(pose0.copy()).cuda().requires_grad_(True)
    e = E.EDEnergy.apply(xg, pg, ctx, G["frame"], prm)
    e.backward()
    gx = xg.grad.cpu().numpy().ravel().astype(np.float64)
    gp = pg.grad.cpu().numpy().astype(np.float64)
    g_gpu = np.concatenate([gx, gp])
    # the association at the same point and the assembled J^T r of one step
    wpos = torch.empty((s.N, 4), dtype=torch.float32, device="cuda")
    wnrm = torch.empty_like(wpos)
    pix_t = torch.empty(s.N, dtype=torch.int32, device="cuda")
    ctx.set_debug(wpos, wnrm, pix_t)
    ctx.gn_step(G["frame"], prm, torch.from_numpy(x0).cuda(), torch.from_numpy(pose0.copy()).cuda())
    jtr = ctx.export_system()["grad"].cpu().numpy().astype(np.float64)
    ctx.set_debug(None, None, None)
    pix = pix_t.cpu().numpy()
    P = C.oracle_problem_from_gpu(s, G)
    E_ref, _, _ = oracle.energy(P, x0.astype(np.float64), pose0, pix_in=pix)
    g_ref = oracle.gradient(P, x0.astype(np.float64), pose0, pix)
    sc = np.abs(g_ref).max()
    # central differences of the FP64 oracle energy, association frozen
    h = 1e-4
    rng = np.random.default_rng(7)
    coords = np.sort(rng.choice(12 * m, 100, replace=False))
    idx = C.oracle_graph_from_gpu(G).idx
    fd = []
    for k in coords:
        j = k // 12
        sel = np.nonzero((idx == j).any(axis=1))[0]
        Ps = _sub_problem(P, G, s, sel)
        xp = x0.astype(np.float64).copy()
        xp.ravel()[k] += h
        xm = x0.astype(np.float64).copy()
        xm.ravel()[k] -= h
        ep, _, _ = oracle.energy(Ps, xp, pose0, pix_in=pix[sel])
        em, _, _ = oracle.energy(Ps, xm, pose0, pix_in=pix[sel])
        fd.append((ep - em) / (2 * h))
    fd_pose = []
    for q in range(6):
        pp, pm = pose0.copy(), pose0.copy()
        pp[q] += h
        pm[q] -= h
        ep, _, _ = oracle.energy(P, x0.astype(np.float64), pp, pix_in=pix)
        em, _, _ = oracle.energy(P, x0.astype(np.float64), pm, pix_in=pix)
        fd_pose.append((ep - em) / (2 * h))
    fd, fd_pose = np.array(fd), np.array(fd_pose)
    rep = {
        "workload": METRIC, "nodes": m, "unknowns": 12 * m + 6, "fd_h": h, "fd_coordinates": 100 + 6,
        "energy_rel_err": abs(float(e.detach()) - E_ref) / E_ref,
        "grad_scale_max_abs": sc,
        "gpu_vs_oracle_grad_max_err_over_scale": float(np.abs(g_gpu - g_ref).max() / sc),
        "gpu_vs_fd_max_err_over_scale": float(max(np.abs(gx[coords] - fd).max(), np.abs(gp - fd_pose).max()) / sc),
        "oracle_vs_fd_max_err_over_scale": float(max(np.abs(g_ref[coords] - fd).max(),
                                                     np.abs(g_ref[12 * m:] - fd_pose).max()) / sc),
        "backward_vs_2JTr_max_err_over_scale": float(np.abs(g_gpu - 2.0 * jtr).max() / sc),
        "skinning_weights": "recomputed in the backward (Gaussian), not read from the graph",
    }
    _report("differentiation_640x480_n2048", rep)
    assert rep["energy_rel_err"] <= C.TOL_E
    assert rep["oracle_vs_fd_max_err_over_scale"] <= 1e-6
    assert rep["gpu_vs_fd_max_err_over_scale"] <= 3e-4
    assert rep["gpu_vs_oracle_grad_max_err_over_scale"] <= 3e-4
    # the step and the energy take the same association from the same FP32 warp,
    # and both sum the same products: they agree far below the FP32 accumulation error
    assert rep["backward_vs_2JTr_max_err_over_scale"] <= 1e-5


def _trajectory_errors(name, precision, n_it, radius=None, max_nodes=None):
    """GPU GN iterations; each compared with the oracle's step from the GPU's
    own state and association (the locked protocol)."""
    torch, E = _torch(), _E()
    s = C.scene(name)
    G = C.gpu_setup(s, radius=radius, max_nodes=max_nodes)
    ctx, m = G["ctx"], G["graph"].m
    x = ctx.identity_x() if radius is None else torch.from_numpy(_start(s, m, 1)[0]).cuda()
    xm = x.double().clone()
    pose = torch.tensor(s.pose_prior, dtype=torch.float64, device="cuda")
    prm = C.solver(s, precision=precision)
    wpos = torch.empty((s.N, 4), dtype=torch.float32, device="cuda")
    wnrm = torch.empty_like(wpos)
    pix = torch.empty(s.N, dtype=torch.int32, device="cuda")
    P = C.oracle_problem_from_gpu(s, G)
    st = E.new_stats(n_it)
    rows = []
    for it in range(n_it):
        xin = (xm if precision else x).cpu().numpy().astype(np.float64)
        pin = pose.cpu().numpy().copy()
        ctx.set_debug(wpos, wnrm, pix)
        ctx.gn_step(G["frame"], prm, x, pose, x_master=xm, stats=st[it:it + 1])
        ctx.set_debug(None, None, None)
        p_np = pix.cpu().numpy()
        Q = oracle.NormalEq(P, xin, pin, pix_in=p_np)
        d, _, _, _ = Q.pcg(-Q.g, prm.n_pcg, jitter=prm.jitter)
        x_ref = xin + d[:12 * m].reshape(m, 12)
        pose_ref = pin + d[12 * m:]
        x_gpu = (xm if precision else x).cpu().numpy().astype(np.float64)
        # warped points (mm) of the new parameters: the library's FP32 warp vs the FP64 warp
        wp_gpu, _ = ctx.warp(x.contiguous(), pose, G["pos"], G["nrm"])
        wp_ref, _, _ = oracle.warp(P, x_ref, pose_ref)
        stt = E.read_stats(st[it:it + 1])[0]
        rows.append({
            "iter": it, "status": stt["status"],
            "energy_rel_err": abs(stt["energy"] - Q.energy) / Q.energy,
            "node_param_max_rel_err": float((np.abs(x_gpu - x_ref) / np.maximum(1.0, np.abs(x_ref))).max()),
            "node_param_l2_rel_err": float(np.linalg.norm(x_gpu - x_ref) / np.linalg.norm(x_ref)),
            "pose_max_abs_err": float(np.abs(pose.cpu().numpy() - pose_ref).max()),
            "warped_points_max_err_mm": float(np.abs(wp_gpu.cpu().numpy()[:, :3] - wp_ref).max()),
        })
    return rows


@pytest.mark.parametrize("name,n_it", [(SMALL, 5), (METRIC, 3), (LARGE, 1)])
def test_precision_report(name, n_it):
    out = {}
    for precision, label in ((0, "fp32"), (1, "mixed"), (2, "mixed_fp64")):
        if name != SMALL:
            m = 4096 if name == LARGE else 2048
            rows = _trajectory_errors(name, precision, n_it, radius=C.radius_for(name), max_nodes=m)
        else:
            rows = _trajectory_errors(name, precision, n_it)
        out[label] = {"per_iteration": rows,
                      "max": {k: max(r[k] for r in rows) for k in rows[0] if k not in ("iter", "status")}}
        for r in rows:
            assert r["status"] == 0
            assert r["energy_rel_err"] <= C.TOL_E
            assert r["node_param_max_rel_err"] <= C.TOL_X
    _report(f"precision_{name}", out)
