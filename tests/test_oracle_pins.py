"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test states the passage of the paper it exercises (Sec. / Eq. / Alg.)
and what fixes the expected value: a closed form, an invariant of the
formulation, an independent brute-force implementation on a tiny input, a
library routine (numpy LAPACK), or finite differences.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import scenes_exact as X

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# constants printed in the paper (Sec. III.B)
# ----------------------------------------------------------------------------

def test_paper_constants():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        c = json.load(f)
    assert (oracle.W_ROT, oracle.W_REG, oracle.W_DATA, oracle.W_R, oracle.W_P) == (
        c["w_rot"]["value"], c["w_reg"]["value"], c["w_data"]["value"], c["w_r"]["value"], c["w_p"]["value"])
    assert oracle.EPS_D_MM == c["eps_d_mm"]["value"]
    assert oracle.EPS_N_DEG == c["eps_n_deg"]["value"]
    assert oracle.FuseParams().tau_d == c["reg_dist_mm"]["value"]
    assert oracle.FuseParams().delta_deg == c["reg_angle_deg"]["value"]
    assert oracle.FuseParams().omega_max == c["omega_max"]["value"]
    assert oracle.FuseParams().tau_time == c["tau_time"]["value"]


# ----------------------------------------------------------------------------
# rotation parameterisation
# ----------------------------------------------------------------------------

def test_rotation_orthonormal_and_derivative_fd():
    pose = np.array([0.3, -0.2, 0.7, 0, 0, 0])
    R, dR = oracle.rotation(pose)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1) < 1e-14
    # R = Rz Ry Rx: the z-y-x composition written out with numpy
    a, b, c = pose[:3]
    Rx = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rz = np.array([[math.cos(c), -math.sin(c), 0], [math.sin(c), math.cos(c), 0], [0, 0, 1]])
    assert np.allclose(R, Rz @ Ry @ Rx, atol=1e-15)
    h = 1e-6
    for t in range(3):
        e = np.zeros(6)
        e[t] = h
        fd = (oracle.rotation(pose + e)[0] - oracle.rotation(pose - e)[0]) / (2 * h)
        assert np.abs(fd - dR[t]).max() < 1e-9


# ----------------------------------------------------------------------------
# target normals (data term n(u))
# ----------------------------------------------------------------------------

def test_normals_of_a_plane_are_the_plane_normal():
    # a true 3D plane n.X = c rendered in FP64: D(u,v) = c / (n . r(u,v))
    W, H, f = 64, 48, 64.0
    intr = (f, f, W / 2.0, H / 2.0, W, H)
    n = np.array([0.2, 0.1, -1.0])
    n /= np.linalg.norm(n)
    c = n @ np.array([0.0, 0.0, 60.0])
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    dot = n[0] * (u - W / 2.0) / f + n[1] * (v - H / 2.0) / f + n[2]
    depth = (c / dot).astype(np.float32)
    nm = oracle.normals(depth, intr, 2)
    val = nm[..., 3] > 0
    assert val.sum() == (64 - 4) * (48 - 4)
    assert np.abs(nm[val][:, :3] - n).max() < 2e-5
    # stencil touching a hole -> invalid
    d2 = depth.copy()
    d2[20, 30] = 0
    nm2 = oracle.normals(d2, intr, 2)
    for (v, u) in [(20, 30), (20, 28), (20, 32), (18, 30), (22, 30)]:
        assert nm2[v, u, 3] == 0
    assert nm2[20, 31, 3] == 1


# ----------------------------------------------------------------------------
# node sampling, k nearest nodes, node graph (Sec. II.D, II.E)
# ----------------------------------------------------------------------------

def _key32(p, q):
    d = (p[..., :3] - q[..., :3]).astype(np.float32)
    s = d[..., 0] * d[..., 0]
    s = s + d[..., 1] * d[..., 1]
    s = s + d[..., 2] * d[..., 2]
    return s


def _poisson_bruteforce(pos, r):
    """Phase-ordered Poisson disk by brute force against every chosen node."""
    pos = pos.astype(np.float32)
    mn = pos[:, :3].min(0)
    mx = pos[:, :3].max(0)
    cs = np.float32(r) * np.float32(0.577350269)
    inv = np.float32(1.0) / cs
    dim = (np.floor((mx - mn) * inv)).astype(np.int64) + 1
    c3 = np.clip(np.floor((pos[:, :3] - mn) * inv).astype(np.int64), 0, dim - 1)
    lin = c3[:, 0] + dim[0] * (c3[:, 1] + dim[1] * c3[:, 2])
    phase = (c3[:, 0] % 3) + 3 * (c3[:, 1] % 3) + 9 * (c3[:, 2] % 3)
    r2 = np.float32(r) * np.float32(r)
    nodes = []
    for ph in range(27):
        cells = sorted(set(lin[phase == ph].tolist()))
        for c in cells:
            for i in np.nonzero(lin == c)[0]:
                if not nodes or _key32(pos[i][None], pos[nodes]).min() >= r2:
                    nodes.append(int(i))
                    break
    return nodes


def test_poisson_matches_bruteforce_and_is_maximal():
    s = synth.make_scene("tissue_160x120_n64", 3)
    pos = s.model_pos[::9].copy()            # ~2k points
    r = 4.0
    nodes, mt = oracle.poisson_nodes(pos, r, 100000)
    assert mt == len(nodes)
    assert nodes.tolist() == _poisson_bruteforce(pos, r)
    g = pos[nodes]
    K = _key32(g[:, None, :], g[None, :, :])
    np.fill_diagonal(K, np.inf)
    assert K.min() >= np.float32(r) * np.float32(r)
    # every point lies within one cell diagonal (~ r) of a node
    kmin = _key32(pos[:, None, :], g[None, :, :]).min(1)
    assert kmin.max() <= np.float32(r) ** 2 * 1.000001
    # truncation keeps the first nodes in selection order
    n10, mt10 = oracle.poisson_nodes(pos, r, 10)
    assert mt10 == mt and n10.tolist() == nodes[:10].tolist()


def test_knn_matches_numpy_bruteforce():
    s = synth.make_scene("tissue_160x120_n64", 2)
    pos = s.model_pos[::17]
    g = s.nodes
    idx, key = oracle.knn(pos, g, 5)
    kk = _key32(pos[:, None, :], g[None, :, :])
    for i in range(pos.shape[0]):
        order = np.lexsort((np.arange(g.shape[0]), kk[i]))[:5]
        assert idx[i].tolist() == order.tolist()
        assert np.array_equal(key[i], kk[i][order])


def test_knn_tie_goes_to_lower_index():
    g = np.zeros((6, 4), np.float32)
    g[:, 0] = [1, -1, 1, 2, -1, 0]
    pos = np.zeros((1, 4), np.float32)
    idx, key = oracle.knn(pos, g, 4)
    assert idx[0].tolist() == [5, 0, 1, 2]


def test_node_graph_matches_numpy():
    s = synth.make_scene("tissue_160x120_n64", 1)
    g = s.nodes
    nbr = oracle.node_graph(g, 4)
    kk = _key32(g[:, None, :], g[None, :, :])
    for j in range(g.shape[0]):
        kk[j, j] = np.inf
        order = np.lexsort((np.arange(g.shape[0]), kk[j]))[:4]
        assert nbr[j].tolist() == order.tolist()


def test_weights_gaussian_and_eq2():
    s = synth.make_scene("tissue_160x120_n64", 1)
    pos = s.model_pos[:500]
    idx5, _ = oracle.knn(pos, s.nodes, 5)
    wg = oracle.skin_weights(pos, s.nodes, idx5, 4, 0, 8.0)
    we = oracle.skin_weights(pos, s.nodes, idx5, 4, 1, 8.0)
    d = np.linalg.norm(pos[:, None, :3].astype(np.float64) - s.nodes[idx5][:, :, :3].astype(np.float64), axis=2)
    g_exp = np.exp(-d[:, :4] ** 2 / 128.0)
    assert np.allclose(wg, g_exp / g_exp.sum(1, keepdims=True), rtol=1e-13)
    e2 = 1 - d[:, :4] / d[:, 4:5]                    # Eq. (2)
    assert np.allclose(we, e2 / e2.sum(1, keepdims=True), rtol=1e-13)
    assert np.allclose(wg.sum(1), 1) and np.allclose(we.sum(1), 1)


# ----------------------------------------------------------------------------
# warp (Eq. 1)
# ----------------------------------------------------------------------------

def _small_problem(seed=1, prior=None):
    s = synth.make_scene("tissue_160x120_n64", seed)
    nm = oracle.normals(s.tgt_depth, s.intr, s.cfg.normal_half_width)
    G = oracle.build_graph(s.model_pos, nodes=s.nodes, K=4, KG=4, mode=0, sigma=s.sigma)
    P = oracle.Problem(s.model_pos, s.model_nrm, G, s.tgt_depth, nm, s.intr,
                       s.pose_prior if prior is None else prior)
    return s, G, P


def test_identity_warp_is_identity():
    s, G, P = _small_problem()
    wpos, wnrm, _ = oracle.warp(P, P.identity_x(), np.zeros(6))
    assert np.abs(wpos - P.pos[:, :3]).max() < 1e-12
    n = P.nrm[:, :3] / np.linalg.norm(P.nrm[:, :3], axis=1, keepdims=True)
    assert np.abs(wnrm - n).max() < 1e-12


def test_rigid_params_give_rigid_warp_and_zero_rot_reg():
    s, G, P = _small_problem()
    Rg = synth.scene.euler_matrix(0.2, -0.1, 0.3)
    Tg = np.array([1.0, 2.0, -3.0])
    x = np.zeros((P.m, 12))
    for j in range(P.m):
        gj = P.g[j, :3]
        t = Rg @ gj + Tg - gj                       # A_j = R, t_j = R g_j + T - g_j
        x[j] = np.concatenate([np.c_[Rg, t].ravel()])
    wpos, wnrm, _ = oracle.warp(P, x, np.zeros(6))
    assert np.abs(wpos - (P.pos[:, :3] @ Rg.T + Tg)).max() < 1e-12
    n = P.nrm[:, :3] / np.linalg.norm(P.nrm[:, :3], axis=1, keepdims=True)
    assert np.abs(wnrm - n @ Rg.T).max() < 1e-12
    E, terms, nv = oracle.energy(P, x, P.s.prior[:], pix_in=np.full(P.N, -1, np.int32))
    assert terms[1] < 1e-20 and terms[2] < 1e-18


def test_rot_term_closed_form():
    s, G, P = _small_problem()
    none = np.full(P.N, -1, np.int32)
    prior = np.array(P.s.prior[:])
    x = np.zeros((P.m, 12))
    x[:, 0] = x[:, 5] = x[:, 10] = 2.0               # A = 2I: (c.c - 1) = 3 on each column
    # translations chosen so that every E_reg residual vanishes: t_j = -g_j
    x[:, 3], x[:, 7], x[:, 11] = -P.g[:, 0], -P.g[:, 1], -P.g[:, 2]
    E, terms, _ = oracle.energy(P, x, prior, pix_in=none)
    assert terms[1] == pytest.approx(oracle.W_ROT * 27.0 * P.m, rel=1e-14)
    # A_j(g_k - g_j) + g_j + t_j - g_k - t_k with A = 2I, t = -g: 2(g_k - g_j) + 0 - 0 ... not 0
    # -> compute the reg energy in closed form from the graph
    e = 0.0
    for j in range(P.m):
        for k in P.nbr[j]:
            d = P.g[k, :3] - P.g[j, :3]
            e += np.sum((2 * d + P.g[j, :3] - P.g[j, :3] - P.g[k, :3] + P.g[k, :3]) ** 2)
    assert terms[2] == pytest.approx(oracle.W_REG * e, rel=1e-12)
    # pose prior closed form
    pose = prior + np.array([0.01, 0, 0, 0, 0.5, 0])
    E2, t2, _ = oracle.energy(P, P.identity_x(), pose, pix_in=none)
    assert t2[3] == pytest.approx(oracle.W_R * 1e-4, rel=1e-9)
    assert t2[4] == pytest.approx(oracle.W_P * 0.25, rel=1e-9)
    # a rotation matrix has Rot = 0
    Rg = synth.scene.euler_matrix(0.4, 0.1, -0.5)
    x3 = P.identity_x()
    for r in range(3):
        x3[:, 4 * r:4 * r + 3] = Rg[r]
    E3, t3, _ = oracle.energy(P, x3, prior, pix_in=none)
    assert t3[1] < 1e-24


# ----------------------------------------------------------------------------
# association and data term on a self-registered surface (Sec. II.E)
# ----------------------------------------------------------------------------

def _exact_selfreg():
    depth, intr = X.exact_plane()
    nm = oracle.normals(depth, intr, 1)
    V = X.backproject64(depth, intr).reshape(-1, 3)
    pix = np.nonzero(nm.reshape(-1, 4)[:, 3] > 0)[0]
    pos = np.concatenate([V[pix], np.ones((len(pix), 1))], 1).astype(np.float32)
    assert np.array_equal(pos[:, :3].astype(np.float64), V[pix])       # exact in FP32
    nrm = nm.reshape(-1, 4)[pix].copy()
    return depth, intr, nm, pos, nrm, pix


def test_selfregistered_association_and_zero_data_energy():
    depth, intr, nm, pos, nrm, pix = _exact_selfreg()
    got = oracle.associate_f32(pos, nrm, depth, nm, intr)
    assert np.array_equal(got, pix)
    g, sp = X.grid_nodes(pos[:, :3].astype(np.float64), 3, 3)
    G = oracle.build_graph(pos, nodes=g, K=4, KG=4, mode=0, sigma=sp)
    P = oracle.Problem(pos, nrm, G, depth, nm, intr, np.zeros(6))
    E, terms, nv = oracle.energy(P, P.identity_x(), np.zeros(6))
    assert nv == len(pix)
    assert terms[0] < 1e-20 and E < 1e-20


def test_association_gates():
    depth, intr, nm, pos, nrm, pix = _exact_selfreg()
    p2 = pos.copy()
    p2[0, :3] *= 1.3                   # same ray, 19 mm deeper: fails ||v - Gamma|| < 15 mm
    p2[1, 2] += 100.0                  # projects elsewhere / fails distance
    n2 = nrm.copy()
    ang = math.radians(11.0)           # normal rotated by 11 degrees about x: fails 10 degree gate
    c, s_ = math.cos(ang), math.sin(ang)
    n = n2[2, :3].astype(np.float64)
    n2[2, :3] = np.array([n[0], c * n[1] - s_ * n[2], s_ * n[1] + c * n[2]])
    ang = math.radians(9.0)
    c, s_ = math.cos(ang), math.sin(ang)
    n = n2[3, :3].astype(np.float64)
    n2[3, :3] = np.array([n[0], c * n[1] - s_ * n[2], s_ * n[1] + c * n[2]])
    p2[4, 2] = -1.0                    # behind the camera
    got = oracle.associate_f32(p2, n2, depth, nm, intr)
    assert got[0] == -1 and got[1] == -1 and got[2] == -1 and got[4] == -1
    assert got[3] == pix[3]
    assert np.array_equal(got[5:], pix[5:])


# ----------------------------------------------------------------------------
# Jacobian, J^T J, gradient (Sec. II.E-F)
# ----------------------------------------------------------------------------

def _perturbed(P, seed=0, scale=0.02):
    rng = np.random.default_rng(seed)
    x = P.identity_x() + rng.normal(0, scale, (P.m, 12)) * np.tile([1, 1, 1, 20] * 3, 1)
    pose = np.array(P.s.prior[:]) + rng.normal(0, 0.01, 6)
    return x, pose


def test_jacobian_matches_central_differences():
    s, G, P = _small_problem()
    x, pose = _perturbed(P)
    pix = oracle.NormalEq(P, x, pose).pix
    r0, J = oracle.residuals(P, x, pose, pix, jacobian=True)
    rng = np.random.default_rng(5)
    cols = list(rng.choice(12 * P.m, 60, replace=False)) + list(range(12 * P.m, 12 * P.m + 6))
    for c in cols:
        xp, xm = x.copy().ravel(), x.copy().ravel()
        pp, pm = pose.copy(), pose.copy()
        h = 1e-6 * max(1.0, abs(np.concatenate([x.ravel(), pose])[c]))
        if c < 12 * P.m:
            xp[c] += h
            xm[c] -= h
        else:
            pp[c - 12 * P.m] += h
            pm[c - 12 * P.m] -= h
        fd = (oracle.residuals(P, xp.reshape(P.m, 12), pp, pix) - oracle.residuals(P, xm.reshape(P.m, 12), pm, pix)) / (2 * h)
        scale = max(1.0, np.abs(J[:, c]).max())
        assert np.abs(fd - J[:, c]).max() <= 1e-6 * scale, c


def test_normal_equations_equal_dense_JtJ_symmetric_psd():
    s, G, P = _small_problem()
    x, pose = _perturbed(P, 1)
    Q = oracle.NormalEq(P, x, pose)
    r, J = oracle.residuals(P, x, pose, Q.pix, jacobian=True)
    H = Q.dense()
    JtJ = J.T @ J
    assert np.abs(H - JtJ).max() <= 1e-10 * np.abs(JtJ).max()
    assert np.abs(Q.g - J.T @ r).max() <= 1e-10 * np.abs(J.T @ r).max()
    assert np.abs(H - H.T).max() <= 1e-13 * np.abs(H).max()
    ev = np.linalg.eigvalsh(H)
    assert ev.min() >= -1e-10 * ev.max()
    assert Q.energy == pytest.approx(float(r @ r), rel=1e-12)


def test_gradient_matches_energy_finite_differences():
    s, G, P = _small_problem()
    x, pose = _perturbed(P, 2)
    pix = oracle.NormalEq(P, x, pose).pix
    grad = oracle.gradient(P, x, pose, pix)
    rng = np.random.default_rng(9)
    cols = list(rng.choice(12 * P.m, 40, replace=False)) + list(range(12 * P.m, 12 * P.m + 6))
    flat = np.concatenate([x.ravel(), pose])
    for c in cols:
        h = 1e-5 * max(1.0, abs(flat[c]))
        fp, fm = flat.copy(), flat.copy()
        fp[c] += h
        fm[c] -= h
        Ep = oracle.energy(P, fp[:-6].reshape(P.m, 12), fp[-6:], pix)[0]
        Em = oracle.energy(P, fm[:-6].reshape(P.m, 12), fm[-6:], pix)[0]
        fd = (Ep - Em) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-5 * max(1.0, abs(grad[c])), (c, fd, grad[c])


# ----------------------------------------------------------------------------
# linear solve
# ----------------------------------------------------------------------------

def test_pcg_converges_to_dense_cholesky_and_lapack():
    s = synth.make_scene("tissue_160x120_n64", 4)
    nm = oracle.normals(s.tgt_depth, s.intr, s.cfg.normal_half_width)
    sel = s.nodes[[0, 1, 2, 3, 8, 9, 10, 11, 16, 17, 18, 19, 24, 25, 26, 27]]   # 16 nodes: tiny graph
    keep = (s.model_pos[:, 0] < sel[:, 0].max() + 2) & (s.model_pos[:, 1] < sel[:, 1].max() + 2)
    G = oracle.build_graph(s.model_pos[keep], nodes=sel, K=4, KG=4, mode=0, sigma=s.sigma)
    P = oracle.Problem(s.model_pos[keep], s.model_nrm[keep], G, s.tgt_depth, nm, s.intr, s.pose_prior)
    x, pose = _perturbed(P, 3)
    Q = oracle.NormalEq(P, x, pose)
    b = -Q.g
    d_chol = Q.dense_solve(b)
    d_np = np.linalg.solve(Q.dense(), b)
    assert np.abs(d_chol - d_np).max() <= 1e-9 * np.abs(d_np).max()
    d_pcg, it, st, hist = Q.pcg(b, 5000, tol=1e-15)
    assert st == 0
    assert np.linalg.norm(d_pcg - d_chol) <= 1e-10 * np.linalg.norm(d_chol)
    # fixed iteration count: residual decreases overall and the first step is the
    # preconditioned steepest-descent step
    d1, it1, st1, _ = Q.pcg(b, 1)
    assert it1 == 1


# ----------------------------------------------------------------------------
# Gauss-Newton (Sec. II.F)
# ----------------------------------------------------------------------------

def test_pure_rigid_motion_is_recovered():
    pr = X.rigid_problem()
    pos = pr["pos"]
    g, sp = X.grid_nodes(pos[:, :3], 4, 3)
    G = oracle.build_graph(pos.astype(np.float32), nodes=g, K=4, KG=4, mode=0, sigma=sp)
    P = oracle.Problem(pos, pr["nrm"], G, pr["depth"], pr["nmap"], pr["intr"], pr["pose"])
    pose0 = pr["pose"] + np.array([0.004, -0.003, 0.005, 0.3, -0.2, 0.25])
    x, pose, hist, st = oracle.gn_solve(P, P.identity_x(), pose0, 12, 0, dense=True)
    assert st == 0
    assert np.abs(pose - pr["pose"]).max() < 1e-9
    assert np.abs(x - P.identity_x()).max() < 1e-9
    wpos, _, _ = oracle.warp(P, x, pose)
    assert np.abs(wpos - pr["target"]).max() < 1e-9
    assert hist[-1, :5].sum() < 1e-15


def test_gn_energy_nonincreasing_with_lm_and_noise_free_gn():
    s, G, P = _small_problem(1)
    x, pose, hist, st = oracle.gn_solve(P, P.identity_x(), np.array(P.s.prior[:]), 6, 10, lam=1e-4,
                                        lm_accept=True)
    E = hist[:, :5].sum(1)
    assert st == 0 and np.all(np.diff(E) <= 1e-9 * E[0])
    # noise-free, hole-free small scene, plain GN (lambda = 0)
    cfg = synth.scene.CONFIGS["tissue_160x120_n64"]
    import dataclasses
    cfg0 = dataclasses.replace(cfg, noise_mm=0.0, p_hole=0.0, prior_noise_mm=0.0, prior_noise_rad=0.0)
    s0 = synth.make_scene(cfg0, 1)
    nm = oracle.normals(s0.tgt_depth, s0.intr, cfg0.normal_half_width)
    G0 = oracle.build_graph(s0.model_pos, nodes=s0.nodes, K=4, KG=4, mode=0, sigma=s0.sigma)
    P0 = oracle.Problem(s0.model_pos, s0.model_nrm, G0, s0.tgt_depth, nm, s0.intr, s0.pose_prior)
    x, pose, hist, st = oracle.gn_solve(P0, P0.identity_x(), s0.pose_prior, 5, 10)
    E = hist[:, :5].sum(1)
    assert st == 0 and np.all(np.diff(E) <= 0)


# ----------------------------------------------------------------------------
# fusion (Sec. II.G, Alg. 1-3, Eqs. fusion1-4)
# ----------------------------------------------------------------------------

def test_fuse_identity_same_frame():
    depth, intr, nm, pos, nrm, pix = _exact_selfreg()
    fx, fy, cx, cy, W, H = intr
    n = pos.shape[0]
    pos[:, 3] = 5.0
    col = np.tile(np.array([0.2, 0.4, 0.6, 1.0], np.float32), (n, 1))
    color = np.tile(np.array([0.8, 0.4, 0.0, 1.0], np.float32), (H, W, 1))
    t = np.zeros(n, np.int32)
    F = oracle.FuseParams(frame=3)
    po, no, co, to, reg = oracle.fuse(pos, nrm, col, t, pos, nrm, depth, nm, color, intr, F, 4 * n)
    assert po.shape[0] == n                      # every point registered, nothing lifted
    assert np.array_equal(reg[pix], np.arange(n))
    assert np.array_equal(po[:, :3], pos[:, :3])  # D' = (5 z + z) / 6 = z
    assert np.all(po[:, 3] == 6.0) and np.all(to == 3)
    assert np.allclose(co, (col * 5 + color[0, 0]) / 6, atol=1e-7)
    assert np.allclose(no[:, :3], nrm[:, :3], atol=1e-7)


def _fuse_unequal_case():
    """Four model points registered to a fronto-parallel depth map D = 60 mm
    (16x12 pixels, f = 16, principal point (8, 6), every target normal
    (0, 0, -1)) with warped depths different from D, unequal weights and one
    tilted normal.  The values below were worked out by hand from Eqs.
    fusion1-4 (Sec. II.G) with observation weight 1, the registered point
    moved along its own ray, omega_max = 20 (Sec. III.B)."""
    W, H, f = 16, 12, 16.0
    intr = (f, f, 8.0, 6.0, W, H)
    depth = np.full((H, W), 60.0, np.float32)
    nm = np.zeros((H, W, 4), np.float32)
    nm[..., 2] = -1.0
    nm[..., 3] = 1.0
    color = np.zeros((H, W, 4), np.float32)
    color[..., :] = (1.0, 0.0, 0.2, 1.0)
    # warped positions (x, y, z~) and weights omega; pixels by P:
    # A (0, 0, 62) -> (8, 6); B (7, 0, 56) -> (10, 6); C (-16, -12, 64) -> (4, 3);
    # D (14.5, 10.875, 58) -> (12, 9)
    wpos = np.array([[0.0, 0.0, 62.0, 3.0], [7.0, 0.0, 56.0, 1.0], [-16.0, -12.0, 64.0, 19.5],
                     [14.5, 10.875, 58.0, 20.0]], np.float32)
    wnrm = np.array([[0.6, 0.0, -0.8, 0.0], [0.0, 0.0, -1.0, 0.0], [0.0, 0.0, -1.0, 0.0],
                     [0.0, 0.0, -1.0, 0.0]], np.float32)
    col = np.tile(np.array([0.2, 0.4, 0.6, 1.0], np.float32), (4, 1))
    t = np.zeros(4, np.int32)
    # the tilted normal of A is 36.87 degrees off the target normal: a 60 degree gate lets it through
    F = oracle.FuseParams(frame=7, delta_deg=60.0)
    return dict(intr=intr, depth=depth, nm=nm, color=color, wpos=wpos, wnrm=wnrm, col=col, t=t, F=F)


def test_fuse_unequal_depths_weights_and_normals():
    c = _fuse_unequal_case()
    po, no, co, to, reg = oracle.fuse(c["wpos"], c["wnrm"], c["col"], c["t"], c["wpos"], c["wnrm"], c["depth"],
                                      c["nm"], c["color"], c["intr"], c["F"], 400)
    W = 16
    assert reg[6 * W + 8] == 0 and reg[6 * W + 10] == 1 and reg[3 * W + 4] == 2 and reg[9 * W + 12] == 3
    assert po.shape[0] == 16 * 12                    # 4 fused + 188 lifted pixels
    # Eq. fusion1: D' = (z~ omega + D) / (omega + 1), along the point's ray
    #   A: (62*3 + 60)/4 = 61.5
    #   B: (56*1 + 60)/2 = 58;  x' = 7 * 58/56 = 7.25
    #   C: (64*19.5 + 60)/20.5 = 2616/41;  x' = -16 (2616/41)/64 = -654/41, y' = -12 (2616/41)/64 = -1962/164
    #   D: (58*20 + 60)/21 = 1220/21;  x' = 14.5 (1220/21)/58 = 14.5 * 1220/1218, y' = 10.875 * 1220/1218
    exp_pos = np.array([[0.0, 0.0, 61.5], [7.25, 0.0, 58.0],
                        [-654.0 / 41.0, -1962.0 / 164.0, 2616.0 / 41.0],
                        [14.5 * 1220.0 / 1218.0, 10.875 * 1220.0 / 1218.0, 1220.0 / 21.0]])
    assert np.abs(po[:4, :3] - exp_pos).max() < 1e-5
    # Eq. fusion4: omega' = min(omega + 1, 20): 3 -> 4, 1 -> 2, 19.5 -> 20, 20 -> 20
    assert np.array_equal(po[:4, 3], np.array([4.0, 2.0, 20.0, 20.0], np.float32))
    # Eq. fusion3: A's normal (3 (0.6, 0, -0.8) + (0, 0, -1)) / 4 = (0.45, 0, -0.85), renormalised:
    # (1.8, 0, -3.4) / sqrt(14.8)
    s148 = 14.8 ** 0.5
    assert np.abs(no[0, :3] - np.array([1.8 / s148, 0.0, -3.4 / s148])).max() < 1e-6
    assert np.abs(no[1:4, :3] - np.array([0.0, 0.0, -1.0])).max() < 1e-7
    # stability flags omega' >= tau_weight = 3: all but B (omega' = 2)
    assert np.array_equal(no[:4, 3], np.array([1.0, 0.0, 1.0, 1.0], np.float32))
    # Eq. fusion2 (colour), A: ((0.2, 0.4, 0.6, 1) 3 + (1, 0, 0.2, 1)) / 4 = (0.4, 0.3, 0.5, 1)
    assert np.abs(co[0] - np.array([0.4, 0.3, 0.5, 1.0])).max() < 1e-6
    # C: (c 19.5 + (1, 0, 0.2, 1)) / 20.5: red (3.9 + 1) / 20.5 = 4.9 / 20.5
    assert abs(co[2, 0] - 4.9 / 20.5) < 1e-6
    assert np.array_equal(to[:4], np.full(4, 7))
    # the first lifted pixel (0, 0): Pi(u, 60) = ((0 - 8) 60 / 16, (0 - 6) 60 / 16, 60), omega 1, frame 7
    assert np.abs(po[4] - np.array([-30.0, -22.5, 60.0, 1.0])).max() < 1e-6
    assert to[4] == 7 and np.array_equal(no[4], np.array([0.0, 0.0, -1.0, 0.0], np.float32))


def test_fuse_zbuffer_lift_delete_conservation():
    rng = np.random.default_rng(0)
    depth, intr = X.exact_plane(16, 12, 16.0)
    fx, fy, cx, cy, W, H = intr
    nm = oracle.normals(depth, intr, 1)
    n = 300
    wpos = np.zeros((n, 4), np.float32)
    wpos[:, 2] = rng.uniform(55, 75, n).astype(np.float32)
    wpos[:, 0] = (rng.uniform(-8, 8, n) * wpos[:, 2] / fx).astype(np.float32)
    wpos[:, 1] = (rng.uniform(-6, 6, n) * wpos[:, 2] / fy).astype(np.float32)
    wnrm = np.tile(np.array([0, 0, -1, 0], np.float32), (n, 1))
    pos = wpos.copy()
    pos[:, 3] = rng.choice([1.0, 2.0, 8.0], n).astype(np.float32)
    t = rng.choice([0, 20], n).astype(np.int32)
    col = np.ones((n, 4), np.float32)
    color = np.zeros((H, W, 4), np.float32)
    F = oracle.FuseParams(frame=25, tau_d=1e6, delta_deg=90.0)     # register every visible winner
    po, no, co, to, reg = oracle.fuse(pos, wnrm, col, t, wpos, wnrm, depth, nm, color, intr, F, 10 * n)
    # z-buffer by brute force: FP32 projection, then smallest (z, index)
    win = {}
    for i in range(n):
        x, y, z = wpos[i, :3]
        u = int(np.floor(np.float32(np.float32(np.float32(fx) * np.float32(x / z)) + np.float32(cx)) + np.float32(0.5)))
        v = int(np.floor(np.float32(np.float32(np.float32(fy) * np.float32(y / z)) + np.float32(cy)) + np.float32(0.5)))
        if 0 <= u < W and 0 <= v < H:
            q = v * W + u
            if q not in win or (z, i) < (wpos[win[q], 2], win[q]):
                win[q] = i
    valid_px = {q for q in range(W * H) if depth.reshape(-1)[q] > 0 and nm.reshape(-1, 4)[q, 3] > 0}
    expect_reg = {q: i for q, i in win.items() if q in valid_px}
    got_reg = {q: int(i) for q, i in enumerate(reg) if i >= 0}
    assert got_reg == expect_reg
    registered = set(expect_reg.values())
    deleted = [i for i in range(n) if i not in registered and 25 - t[i] > 10 and pos[i, 3] < 3.0]
    lifted = len(valid_px) - len(expect_reg)
    assert po.shape[0] == n - len(deleted) + lifted
    kept = [i for i in range(n) if i not in deleted]
    assert np.array_equal(to[:len(kept)], np.where(np.isin(kept, list(registered)), 25, t[kept]))
    assert np.all(po[len(kept):, 3] == 1.0) and np.all(to[len(kept):] == 25)


# ----------------------------------------------------------------------------
# sparse key correspondences, E_corr (Sec. II.E "Correspondence", w_corr = 10)
# ----------------------------------------------------------------------------

def _keypoint_problem(seed=0, nk=40, shift=None):
    """The small problem plus nk key points drawn from the model, their targets
    the key points themselves moved by `shift` (or by seeded noise)."""
    s, G, P0 = _small_problem()
    rng = np.random.default_rng(100 + seed)
    sel = rng.choice(s.N, nk, replace=False)
    kp = s.model_pos[sel].astype(np.float32)
    d = rng.normal(0, 0.5, (nk, 3)) if shift is None else np.broadcast_to(np.asarray(shift, float), (nk, 3))
    tgt = kp[:, :3].astype(np.float64) + d
    K = oracle.keypoints(kp, tgt, G.g, K=4, mode=0, sigma=s.sigma)
    nm = oracle.normals(s.tgt_depth, s.intr, s.cfg.normal_half_width)
    P = oracle.Problem(s.model_pos, s.model_nrm, G, s.tgt_depth, nm, s.intr, s.pose_prior, keypoints=K)
    return s, G, P, d


def test_corr_energy_closed_form_at_identity():
    s, G, P, d = _keypoint_problem(shift=None)
    zero_pose = np.zeros(6)
    # identity warp and pose: the warped key point is the key point, so
    # E_corr = w_corr sum_k |target_k - p_k|^2
    _, terms, _ = oracle.energy(P, P.identity_x(), zero_pose)
    assert terms[5] == pytest.approx(oracle.W_CORR * float((d ** 2).sum()), rel=1e-12)
    # the key points at their targets: E_corr vanishes
    s2, G2, P2, d2 = _keypoint_problem(shift=(0.0, 0.0, 0.0))
    _, terms2, _ = oracle.energy(P2, P2.identity_x(), zero_pose)
    assert terms2[5] < 1e-20     # the identity warp up to the rounding of the normalised weights
    # a pure translation T of the pose moves every key point by T
    T = np.array([0.0, 0.0, 0.0, 0.7, -0.4, 1.1])
    _, terms3, _ = oracle.energy(P2, P2.identity_x(), T)
    assert terms3[5] == pytest.approx(oracle.W_CORR * 40 * float((T[3:] ** 2).sum()), rel=1e-12)


def test_corr_jacobian_and_normal_equations():
    s, G, P, d = _keypoint_problem(seed=1)
    x, pose = _perturbed(P, 4)
    Q = oracle.NormalEq(P, x, pose)
    r, J = oracle.residuals(P, x, pose, Q.pix, jacobian=True)
    nv = int((Q.pix >= 0).sum())
    kr = slice(nv, nv + 3 * 40)                      # the key-point rows
    assert float(r[kr] @ r[kr]) == pytest.approx(Q.E[5], rel=1e-12)
    # explicit Jacobian rows of the key points against central differences
    rng = np.random.default_rng(6)
    nodes = np.unique(P.kp_idx)
    cols = [12 * j + c for j in rng.choice(nodes, 6, replace=False) for c in range(12)]
    cols += list(range(12 * P.m, 12 * P.m + 6))
    flat = np.concatenate([x.ravel(), pose])
    for c in cols:
        h = 1e-6 * max(1.0, abs(flat[c]))
        fp, fm = flat.copy(), flat.copy()
        fp[c] += h
        fm[c] -= h
        rp = oracle.residuals(P, fp[:-6].reshape(P.m, 12), fp[-6:], Q.pix)[kr]
        rm = oracle.residuals(P, fm[:-6].reshape(P.m, 12), fm[-6:], Q.pix)[kr]
        fd = (rp - rm) / (2 * h)
        assert np.abs(fd - J[kr, c]).max() <= 1e-6 * max(1.0, np.abs(J[kr, c]).max()), c
    # the assembled normal equations still equal J^T J and J^T r
    H = Q.dense()
    assert np.abs(H - J.T @ J).max() <= 1e-10 * np.abs(J.T @ J).max()
    assert np.abs(Q.g - J.T @ r).max() <= 1e-10 * np.abs(J.T @ r).max()
    # and E_corr shows in the gradient: 2 J^T r against the energy's differences
    grad = 2.0 * Q.g
    for c in cols[:20] + cols[-6:]:
        h = 1e-5 * max(1.0, abs(flat[c]))
        fp, fm = flat.copy(), flat.copy()
        fp[c] += h
        fm[c] -= h
        Ep = oracle.energy(P, fp[:-6].reshape(P.m, 12), fp[-6:], Q.pix)[0]
        Em = oracle.energy(P, fm[:-6].reshape(P.m, 12), fm[-6:], Q.pix)[0]
        assert abs((Ep - Em) / (2 * h) - grad[c]) <= 1e-5 * max(1.0, abs(grad[c])), c


def test_rigid_motion_recovered_with_consistent_keypoints():
    pr = X.rigid_problem()
    pos = pr["pos"]
    g, sp = X.grid_nodes(pos[:, :3], 4, 3)
    G = oracle.build_graph(pos.astype(np.float32), nodes=g, K=4, KG=4, mode=0, sigma=sp)
    R, _ = oracle.rotation(pr["pose"])
    rng = np.random.default_rng(3)
    sel = rng.choice(pos.shape[0], 30, replace=False)
    kp = pos[sel].astype(np.float32)
    tgt = kp[:, :3].astype(np.float64) @ R.T + pr["pose"][3:]     # the true rigid motion of the key points
    K = oracle.keypoints(kp, tgt, G.g, K=4, mode=0, sigma=sp)
    P = oracle.Problem(pos, pr["nrm"], G, pr["depth"], pr["nmap"], pr["intr"], pr["pose"], keypoints=K)
    pose0 = pr["pose"] + np.array([0.004, -0.003, 0.005, 0.3, -0.2, 0.25])
    x, pose, hist, st = oracle.gn_solve(P, P.identity_x(), pose0, 12, 0, dense=True)
    assert st == 0
    assert np.abs(pose - pr["pose"]).max() < 1e-9
    assert np.abs(x - P.identity_x()).max() < 1e-9


# ----------------------------------------------------------------------------
# model maintenance: box downsampling (Sec. III.A, Alg. 3), back-projection
# error (Sec. III)
# ----------------------------------------------------------------------------

def _lattice(nx, ny, nz, box, rng, jitter=0.3):
    """One point inside each box of an nx x ny x nz grid of edge `box` whose
    origin is a corner point, so the bounding box starts at the origin."""
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    c = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1).astype(np.float64)
    off = 0.5 + rng.uniform(-jitter, jitter, c.shape)
    off[0] = 0.0          # the first point sits on the origin (the bbox minimum)
    p = (c + off) * box
    return c, p


def test_downsample_one_point_per_box_keeps_every_point():
    rng = np.random.default_rng(3)
    box = 0.5
    c, p = _lattice(5, 4, 3, box, rng)
    n = p.shape[0]
    perm = rng.permutation(n)
    pos = np.concatenate([p[perm], rng.uniform(1, 4, (n, 1))], 1).astype(np.float32)
    nrm = np.concatenate([rng.normal(size=(n, 3)), np.ones((n, 1))], 1)
    nrm[:, :3] /= np.linalg.norm(nrm[:, :3], axis=1, keepdims=True)
    nrm = nrm.astype(np.float32)
    col = rng.random((n, 4)).astype(np.float32)
    t = rng.integers(0, 9, n).astype(np.int32)
    po, no, co, to, ko = oracle.downsample(pos, nrm, col, t, box, omega_max=20.0, tau_weight=3.0)
    assert po.shape[0] == n
    # output in box order: x fastest, then y, then z; the key of box (i, j, k) is i + 5 (j + 4 k)
    cp = c[perm]
    key = (cp[:, 0] + 5 * (cp[:, 1] + 4 * cp[:, 2])).astype(np.uint32)
    order = np.argsort(key)
    assert np.array_equal(ko, key[order])
    assert np.array_equal(po, pos[order])               # a single point is its own mean
    assert np.allclose(no[:, :3], nrm[order, :3], atol=1e-7)
    assert np.array_equal(no[:, 3], (pos[order, 3] >= 3.0).astype(np.float32))
    assert np.array_equal(co, col[order]) and np.array_equal(to, t[order])


def test_downsample_merges_a_box_to_its_weighted_mean():
    rng = np.random.default_rng(4)
    box = 1.0
    anchor = np.array([[0.0, 0.0, 0.0, 1.0]], np.float32)   # fixes the bounding-box minimum
    pts = np.array([[2.2, 3.1, 4.4], [2.7, 3.9, 4.05], [2.05, 3.5, 4.95]], np.float64)
    w = np.array([1.0, 2.0, 3.0])
    pos = np.concatenate([anchor, np.concatenate([pts, w[:, None]], 1).astype(np.float32)])
    nrm = np.array([[0, 0, -1, 1], [0.6, 0, -0.8, 1], [0, 0.6, -0.8, 1], [0, 0, -1, 1]], np.float32)
    col = np.array([[0, 0, 0, 1], [1, 0, 0, 1], [0, 1, 0, 1], [0, 0, 1, 1]], np.float32)
    t = np.array([0, 4, 9, 2], np.int32)
    po, no, co, to, ko = oracle.downsample(pos, nrm, col, t, box, omega_max=5.0, tau_weight=3.0)
    assert po.shape[0] == 2
    assert np.array_equal(po[0], anchor[0]) and ko[0] == 0
    p32 = pos[1:, :3].astype(np.float64)
    assert np.allclose(po[1, :3], (w[:, None] * p32).sum(0) / 6.0, rtol=0, atol=1e-6)
    assert po[1, 3] == 5.0                                   # min(1 + 2 + 3, omega_max)
    nsum = (w[:, None] * nrm[1:, :3]).sum(0)
    assert np.allclose(no[1, :3], nsum / np.linalg.norm(nsum), atol=1e-7) and no[1, 3] == 1.0
    assert np.allclose(co[1], (w[:, None] * col[1:]).sum(0) / 6.0, atol=1e-7)
    assert to[1] == 9
    # box (2, 3, 4) of the 3 x 4 x 5 grid: floor(max / box) + 1 boxes per axis
    dims = np.floor(np.max(pos[:, :3], 0) / np.float32(box)).astype(int) + 1
    assert ko[1] == 2 + dims[0] * (3 + dims[1] * 4)


def test_downsample_keeps_the_weighted_sum_and_ignores_input_order():
    rng = np.random.default_rng(5)
    n = 4000
    pos = np.concatenate([rng.uniform(0, 6, (n, 3)), rng.integers(1, 4, (n, 1))], 1).astype(np.float32)
    nrm = np.tile(np.array([0, 0, -1, 1], np.float32), (n, 1))
    col = rng.random((n, 4)).astype(np.float32)
    t = rng.integers(0, 5, n).astype(np.int32)
    po, no, co, to, ko = oracle.downsample(pos, nrm, col, t, 0.8, omega_max=1e9, tau_weight=3.0)
    w = pos[:, 3].astype(np.float64)
    assert np.isclose(po[:, 3].astype(np.float64).sum(), w.sum())
    assert np.allclose((po[:, 3:4] * po[:, :3]).sum(0), (w[:, None] * pos[:, :3]).sum(0), rtol=1e-6)
    assert np.all(np.diff(ko.astype(np.int64)) > 0)
    perm = rng.permutation(n)
    qo, qn, qc, qt, qk = oracle.downsample(pos[perm], nrm[perm], col[perm], t[perm], 0.8, omega_max=1e9)
    assert np.array_equal(qk, ko) and np.array_equal(qt, to) and np.array_equal(qo[:, 3], po[:, 3])
    assert np.allclose(qo, po, atol=1e-6) and np.allclose(qc, co, atol=1e-6)


def test_downsample_box_without_weight_is_a_plain_mean():
    pos = np.array([[0, 0, 0, 0], [0.2, 0.4, 0.1, 0]], np.float32)
    nrm = np.array([[0, 0, -1, 0], [0, 0, -1, 0]], np.float32)
    col = np.array([[1, 0, 0, 1], [0, 1, 0, 1]], np.float32)
    po, no, co, to, ko = oracle.downsample(pos, nrm, col, np.zeros(2, np.int32), 1.0)
    assert po.shape[0] == 1
    assert np.allclose(po[0, :3], [0.1, 0.2, 0.05], atol=1e-7) and po[0, 3] == 0.0 and no[0, 3] == 0.0
    assert np.allclose(co[0], [0.5, 0.5, 0, 1])


def test_depth_error_zero_for_the_depth_itself_and_equal_to_a_shift_along_rays():
    depth, intr, nm, pos, nrm, pix = _exact_selfreg()
    mean, cnt, mx, rms = oracle.depth_error(pos, depth, intr)
    assert cnt == pos.shape[0] and mean == 0.0 and mx == 0.0
    # every point moved along its ray by 0.5 mm: the same pixel, z + 0.5
    d = 0.5
    s = (pos[:, 2].astype(np.float64) + d) / pos[:, 2]
    moved = pos.copy()
    moved[:, :3] = (pos[:, :3] * s[:, None]).astype(np.float32)
    got = oracle.associate_f32(moved, nrm, depth, nm, intr, eps_d=1e6, cos_eps_n=np.float32(-2.0))
    keep = got == pix                                     # points that stayed on their pixel
    assert keep.mean() > 0.9
    mean, cnt, mx, rms = oracle.depth_error(moved[keep], depth, intr)
    zerr = np.abs(moved[keep, 2].astype(np.float64) - depth.reshape(-1)[pix[keep]])
    assert cnt == keep.sum() and np.isclose(mean, zerr.mean()) and abs(mean - d) < 1e-5
    # a second copy of the surface 5 mm behind it is hidden by the z-buffer
    behind = pos.copy()
    behind[:, :3] = (pos[:, :3] * ((pos[:, 2:3] + 5.0) / pos[:, 2:3])).astype(np.float32)
    mean, cnt, mx, rms = oracle.depth_error(np.concatenate([pos, behind]), depth, intr)
    assert mx == 0.0 and cnt == pos.shape[0]
