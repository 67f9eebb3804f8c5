"""Levenberg-Marquardt acceptance on the device (Sec. II.F solves Eq. (3)
with LM): every step is checked against the FP64 oracle run through the same
decision rule in lock step.  At each step the oracle takes the GPU's input
point and association, decides accept / reject from its own FP64 energies,
linearises at the accepted point, damps the normal equations by
(1 + lambda) on the diagonal and solves them with its block-Jacobi PCG; the
GPU's decision, lambda, reported energy and updated parameters must agree.
A host-side perturbation of the parameters between two steps forces a
rejection (the energy rises by orders of magnitude), so the restore path
runs on every call."""
import numpy as np
import pytest

import oracle
from tests import gpu_common as C

pytestmark = pytest.mark.gpu

SMALL = "tissue_160x120_n64"


def _torch():
    import torch
    return torch


def _E():
    import paper_1803_02009_b300 as E
    return E


def _start(s, m, seed):
    rng = np.random.default_rng(seed)
    x0 = np.zeros((m, 12))
    x0[:, [0, 5, 10]] = 1.0
    x0 = (x0 + rng.normal(0, 1e-3, x0.shape)).astype(np.float32)
    pose0 = np.asarray(s.pose_prior) + rng.normal(0, 1e-3, 6)
    return x0, pose0


class _OracleLM:
    """The oracle side of the lock-step comparison: the LM state machine of
    the oracle's GN driver, fed with the GPU's input point and association."""

    def __init__(self, P, prm, lam0):
        self.P, self.prm, self.lam = P, prm, float(lam0)
        self.have = False
        self.E_prev = None
        self.acc = None          # (x, pose, pix) of the last accepted point

    def step(self, x_in, pose_in, pix, gpu_rejected):
        Q = oracle.NormalEq(self.P, x_in, pose_in, pix_in=pix)
        E = Q.energy
        if self.have:
            margin = abs(E - self.E_prev) / self.E_prev
            reject = E > self.E_prev
            if margin > 1e-6:
                assert bool(gpu_rejected) == reject, (E, self.E_prev)
            else:
                reject = bool(gpu_rejected)   # a tie within rounding: either decision is correct
        else:
            reject = False
        if reject:
            self.lam = self.lam * 10.0 if self.lam > 0 else 1e-4
            x_in, pose_in, pix = self.acc
            Q = oracle.NormalEq(self.P, x_in, pose_in, pix_in=pix)
        else:
            if self.have:
                self.lam *= 0.1
            self.have = True
            self.E_prev = E
            self.acc = (x_in.copy(), pose_in.copy(), pix.copy())
        E_lin = Q.energy
        if self.lam:
            Q.damp(self.lam)
        d, _, _, _ = Q.pcg(-Q.g, self.prm.n_pcg, jitter=self.prm.jitter)
        m = self.P.m
        return reject, E_lin, x_in + d[:12 * m].reshape(m, 12), pose_in + d[12 * m:]


def _run(precision, lam0, perturb_before, n_it=5, seed=5):
    torch, E = _torch(), _E()
    s = C.scene(SMALL)
    G = C.gpu_setup(s)
    ctx, m = G["ctx"], G["graph"].m
    x0, pose0 = _start(s, m, seed)
    x = torch.from_numpy(x0).cuda()
    xm = x.double().clone()
    pose = torch.from_numpy(pose0.copy()).cuda()
    prm = C.solver(s, precision=precision, lm_accept=True)
    P = C.oracle_problem_from_gpu(s, G)
    ref = _OracleLM(P, prm, lam0)
    wpos = torch.empty((s.N, 4), dtype=torch.float32, device="cuda")
    wnrm = torch.empty_like(wpos)
    pix = torch.empty(s.N, dtype=torch.int32, device="cuda")
    st = E.new_stats(n_it)
    ctx.lm_reset(lam0)
    rng = np.random.default_rng(11)
    rows = []
    for it in range(n_it):
        if it in perturb_before:
            # a large host-side change of the affine parts: Rot(A) and the
            # regulariser blow up, so the next step must undo it
            dA = np.zeros((m, 12), np.float32)
            dA[:, [0, 1, 2, 4, 5, 6, 8, 9, 10]] = rng.normal(0, 0.2, (m, 9))
            x += torch.from_numpy(dA).cuda()
            xm.copy_(x.double())
        xin = (xm if precision else x).cpu().numpy().astype(np.float64)
        pin = pose.cpu().numpy().copy()
        ctx.set_debug(wpos, wnrm, pix)
        ctx.gn_step(G["frame"], prm, x, pose, x_master=xm, stats=st[it:it + 1])
        ctx.set_debug(None, None, None)
        stt = E.read_stats(st[it:it + 1])[0]
        assert stt["status"] == 0, stt
        reject, E_lin, x_ref, pose_ref = ref.step(xin, pin, pix.cpu().numpy(), stt["lm_rejected"])
        assert stt["lm_rejected"] == int(reject), it
        assert stt["lam"] == pytest.approx(ref.lam, rel=1e-6), it
        assert stt["energy"] == pytest.approx(E_lin, rel=C.TOL_E), it
        x_gpu = (xm if precision else x).cpu().numpy().astype(np.float64)
        err = (np.abs(x_gpu - x_ref) / np.maximum(1.0, np.abs(x_ref))).max()
        assert err <= C.TOL_X, (it, err)
        assert np.abs(pose.cpu().numpy() - pose_ref).max() <= C.TOL_X, it
        if precision:
            assert np.array_equal(x.cpu().numpy(), xm.cpu().numpy().astype(np.float32))
        rows.append(stt)
    return rows


@pytest.mark.parametrize("precision", [0, 1])
def test_lm_accepts_and_rejects_in_lock_step_with_oracle(precision):
    rows = _run(precision, lam0=1e-3, perturb_before={2})
    flags = [r["lm_rejected"] for r in rows]
    assert flags[0] == 0 and flags[2] == 1, flags
    # the rejected step reports the energy of the restored point, bit for bit
    assert rows[2]["energy"] == rows[1]["energy"]
    assert rows[2]["n_valid"] == rows[1]["n_valid"]
    assert rows[2]["lam"] == pytest.approx(10.0 * rows[1]["lam"], rel=1e-12)
    # accepted energies never rise
    acc = [r["energy"] for r in rows if not r["lm_rejected"]]
    assert all(b <= a for a, b in zip(acc, acc[1:])), acc


def test_lm_from_zero_damping_rejects_to_1e4():
    rows = _run(0, lam0=0.0, perturb_before={1}, n_it=3)
    assert rows[0]["lam"] == 0.0 and rows[1]["lm_rejected"] == 1
    assert rows[1]["lam"] == pytest.approx(1e-4, rel=1e-12)


def test_lm_argument_checks():
    E = _E()
    s = C.scene(SMALL)
    G = C.gpu_setup(s)
    ctx = G["ctx"]
    with pytest.raises(E.EDError):
        ctx.lm_reset(-1.0)
    with pytest.raises(E.EDError):
        ctx.lm_reset(float("nan"))
    prm = C.solver(s)
    p = prm.c()
    p.lm_accept = 2
    torch = _torch()
    x = ctx.identity_x()
    pose = torch.tensor(s.pose_prior, dtype=torch.float64, device="cuda")
    import ctypes
    from paper_1803_02009_b300 import lib, _ptr, _stream
    rc = lib().ed_gn_step(ctx.h, ctypes.byref(G["frame"]), ctypes.byref(p), _ptr(x), None, _ptr(pose), None,
                          _stream(None))
    assert rc == 1   # ED_ERR_ARG


def test_lm_batched_and_graph_replay_match_single_problem():
    """Two problems in one batch with LM acceptance (a perturbation forces a
    rejection in both) against each problem alone; a captured graph of the
    last two iterations replays the eager batched run bit for bit."""
    torch, E = _torch(), _E()
    probs = []
    for seed in (1, 2):
        s = C.scene(SMALL, seed)
        G = C.gpu_setup(s)
        x0, pose0 = _start(s, G["graph"].m, 20 + seed)
        probs.append(dict(s=s, G=G, x0=x0, pose0=pose0, prm=C.solver(s, lm_accept=True)))
    K = len(probs)
    dA = [torch.from_numpy(np.random.default_rng(30 + k).normal(0, 0.2, (p["G"]["graph"].m, 12))
                           .astype(np.float32)).cuda() for k, p in enumerate(probs)]
    xs = [torch.from_numpy(p["x0"]).cuda() for p in probs]
    ps = [torch.from_numpy(p["pose0"].copy()).cuda() for p in probs]

    def reset():
        for p, x, q in zip(probs, xs, ps):
            x.copy_(torch.from_numpy(p["x0"]))
            q.copy_(torch.from_numpy(p["pose0"]))
            p["G"]["ctx"].lm_reset(1e-3)

    # each problem alone: 2 steps, perturbation, 2 steps
    single = []
    reset()
    for k, p in enumerate(probs):
        for it in range(4):
            if it == 2:
                xs[k] += dA[k]
            p["G"]["ctx"].gn_step(p["G"]["frame"], p["prm"], xs[k], ps[k])
        single.append((xs[k].cpu().numpy(), ps[k].cpu().numpy()))
    # batched, eager
    stats = [E.new_stats(2) for _ in probs]   # eager steps write entry 0; the 2-iteration graph entries 0, 1
    B = E.Batch([p["G"]["ctx"] for p in probs])
    B.bind([p["G"]["frame"] for p in probs], [p["prm"] for p in probs], xs, ps, stats=stats)
    reset()
    rej = []
    for it in range(4):
        if it == 2:
            for k in range(K):
                xs[k] += dA[k]
        B.gn_step()
        torch.cuda.synchronize()
        rej.append([E.read_stats(st)[0]["lm_rejected"] for st in stats])
    assert rej[2] == [1] * K, rej
    eager = [(x.cpu().numpy(), q.cpu().numpy()) for x, q in zip(xs, ps)]
    for k in range(K):
        assert (np.abs(eager[k][0] - single[k][0]) / np.maximum(1.0, np.abs(single[k][0]))).max() <= C.TOL_X
        assert np.abs(eager[k][1] - single[k][1]).max() <= C.TOL_X
    # the same run with the last two iterations (reject, then accept) as one graph
    reset()
    for it in range(2):
        B.gn_step()
    for k in range(K):
        xs[k] += dA[k]
    B.capture(n_iters=2)
    B.launch()
    torch.cuda.synchronize()
    for k in range(K):
        assert np.array_equal(xs[k].cpu().numpy(), eager[k][0]), k
        assert np.array_equal(ps[k].cpu().numpy(), eager[k][1]), k
