"""Edge cases of the C ABI on the GPU: empty inputs, call order, invalid
arguments, degenerate graphs, the parameter reset, and capacity limits.
Every error is a synchronous ed_status or a device status word; none of
these cases faults or waits."""
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


def _ctx(s, max_nodes=64):
    E = _E()
    fx, fy, cx, cy, W, H = s.intr
    return E.Context(max_points=s.N + W * H, max_nodes=max_nodes, max_width=W, max_height=H)


def test_call_order_and_argument_errors():
    torch, E = _torch(), _E()
    s = C.scene(SMALL)
    ctx = _ctx(s)
    depth = torch.from_numpy(s.tgt_depth).cuda()
    nmap = ctx.compute_normals(depth, s.intr, s.cfg.normal_half_width)
    frame = E.make_frame(depth, nmap, s.intr)
    x = torch.zeros((64, 12), dtype=torch.float32, device="cuda")
    pose = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EDError) as ei:            # no graph yet
        ctx.gn_step(frame, E.SolverParams(), x, pose)
    assert ei.value.status == 7
    with pytest.raises(E.EDError) as ei:
        ctx.reset_params(x, pose)
    assert ei.value.status == 7
    pos = torch.from_numpy(s.model_pos).cuda()
    nrm = torch.from_numpy(s.model_nrm).cuda()
    with pytest.raises(E.EDError) as ei:            # no points
        ctx.build_graph(pos[:0], nrm[:0], node_radius=2.0, max_nodes=64, sigma=2.0)
    assert ei.value.status == 1
    with pytest.raises(E.EDError) as ei:            # a radius so large that fewer than k + 1 nodes are sampled
        ctx.build_graph(pos, nrm, node_radius=500.0, max_nodes=64, sigma=500.0)
    assert ei.value.status == 1
    col = torch.from_numpy(s.model_col).cuda()
    t = torch.from_numpy(s.model_t).cuda()
    with pytest.raises(E.EDError):                  # box edge must be positive
        ctx.downsample(pos, nrm, col, t, 0.0)
    with pytest.raises(E.EDError):                  # output may not alias the input
        ctx.downsample(pos, nrm, col, t, 0.5, out=dict(pos=pos, nrm=nrm.clone(), col=col.clone(), t=t.clone(),
                                                       counts=torch.zeros(2, dtype=torch.int32, device="cuda")))


def test_empty_inputs():
    torch, E = _torch(), _E()
    s = C.scene(SMALL)
    ctx = _ctx(s)
    fx, fy, cx, cy, W, H = s.intr
    dev = "cuda"
    empty4 = torch.zeros((0, 4), dtype=torch.float32, device=dev)
    empty_t = torch.zeros(0, dtype=torch.int32, device=dev)
    out = ctx.downsample(empty4, empty4, empty4, empty_t, 0.5, capacity=8)
    assert out["counts"].cpu().tolist() == [0, 0]
    depth = torch.from_numpy(s.tgt_depth).to(dev)
    err = ctx.depth_error(empty4, depth, s.intr).cpu().numpy()
    assert err.tolist() == [0.0, 0.0, 0.0, 0.0]
    # fusing an empty model lifts every observed pixel with a valid normal
    nmap = ctx.compute_normals(depth, s.intr, s.cfg.normal_half_width)
    color = torch.from_numpy(np.ascontiguousarray(s.tgt_color)).to(dev)
    fr = E.make_frame(depth, nmap, s.intr, color)
    fo = ctx.fuse(empty4, empty4, empty4, empty_t, empty4, empty4, fr, E.FuseParams(frame=2), W * H)
    n = int(fo["counts"][0])
    ref = oracle.fuse(np.zeros((0, 4), np.float32), np.zeros((0, 4), np.float32), np.zeros((0, 4), np.float32),
                      np.zeros(0, np.int32), np.zeros((0, 4), np.float32), np.zeros((0, 4), np.float32),
                      s.tgt_depth, nmap.cpu().numpy(), s.tgt_color, s.intr, oracle.FuseParams(frame=2), W * H)
    assert n == ref[0].shape[0] == int(((s.tgt_depth > 0) & (nmap.cpu().numpy()[..., 3] > 0)).sum())
    assert np.abs(fo["pos"][:n].cpu().numpy() - ref[0]).max() < 1e-4
    assert np.array_equal(fo["t"][:n].cpu().numpy(), ref[3])


def test_fuse_capacity_truncates_and_flags():
    torch, E = _torch(), _E()
    s = C.scene(SMALL)
    G = C.gpu_setup(s)
    ctx = G["ctx"]
    x = ctx.identity_x()
    pose = torch.zeros(6, dtype=torch.float64, device="cuda")
    wp, wn = ctx.warp(x, pose, G["pos"], G["nrm"])
    col = torch.from_numpy(s.model_col).cuda()
    t = torch.from_numpy(s.model_t).cuda()
    full = ctx.fuse(G["pos"], G["nrm"], col, t, wp, wn, G["frame"], E.FuseParams(frame=1), s.N + 160 * 120)
    n = int(full["counts"][0])
    cap = n - 100
    part = ctx.fuse(G["pos"], G["nrm"], col, t, wp, wn, G["frame"], E.FuseParams(frame=1), cap)
    c = part["counts"].cpu().tolist()
    assert c == [cap, 3]                            # truncated, ED_ERR_CAPACITY
    assert np.array_equal(part["pos"][:cap].cpu().numpy(), full["pos"][:cap].cpu().numpy())


def test_reset_params_sets_identity_master_and_prior():
    torch, E = _torch(), _E()
    s = C.scene(SMALL)
    G = C.gpu_setup(s)
    ctx, m = G["ctx"], G["graph"].m
    x = torch.full((m, 12), 7.0, dtype=torch.float32, device="cuda")
    xm = torch.full((m, 12), 7.0, dtype=torch.float64, device="cuda")
    pose = torch.full((6,), 7.0, dtype=torch.float64, device="cuda")
    prior = (0.01, -0.02, 0.03, 1.5, -2.5, 0.25)
    ctx.reset_params(x, pose, x_master=xm, prior=prior)
    eye = np.zeros((m, 12))
    eye[:, [0, 5, 10]] = 1.0
    assert np.array_equal(x.cpu().numpy(), eye.astype(np.float32))
    assert np.array_equal(xm.cpu().numpy(), eye)
    assert np.array_equal(pose.cpu().numpy(), np.array(prior))
    ctx.reset_params(x, pose)                       # no prior: zeros
    assert np.array_equal(pose.cpu().numpy(), np.zeros(6))


def test_graph_node_cap_truncates_in_selection_order():
    torch, E = _torch(), _E()
    s = C.scene(SMALL)
    ctx = _ctx(s, max_nodes=128)
    pos = torch.from_numpy(s.model_pos).cuda()
    nrm = torch.from_numpy(s.model_nrm).cuda()
    r = 2.0
    full_pt, mt = oracle.poisson_nodes(s.model_pos, r, 100000)
    cap = min(100, len(full_pt) - 5)
    g = ctx.build_graph(pos, nrm, node_radius=r, max_nodes=cap, sigma=r)
    counts = g.counts.cpu().numpy()
    assert g.m == cap and counts[0] == cap and counts[1] == len(full_pt)
    assert np.array_equal(g.nodes[:cap, :3].cpu().numpy(), s.model_pos[full_pt[:cap], :3])


def test_block_capacity_is_an_error_not_a_fault():
    # a context whose block budget (max_pairs_per_node) is below the graph's
    # row lengths: the pattern kernels queued before the host sees the block
    # count check it themselves; the build reports ED_ERR_CAPACITY and the
    # context stays usable (no graph: a GN step is refused)
    torch, E = _torch(), _E()
    s = C.scene(SMALL)
    fx, fy, cx, cy, W, H = s.intr
    ctx = E.Context(max_points=s.N, max_nodes=64, max_width=W, max_height=H, max_pairs_per_node=4)
    pos = torch.from_numpy(s.model_pos).cuda()
    nrm = torch.from_numpy(s.model_nrm).cuda()
    r = C.radius_for(SMALL)
    # the build queues the pattern and returns; the capacity error comes with
    # the first read of the pattern's size
    g = ctx.build_graph(pos, nrm, node_radius=r, max_nodes=64, sigma=r)
    assert g.m > 0
    with pytest.raises(E.EDError) as ei:
        g.nnzb
    assert ei.value.status == 3
    depth = torch.from_numpy(s.tgt_depth).cuda()
    nmap = ctx.compute_normals(depth, s.intr, s.cfg.normal_half_width)
    frame = E.make_frame(depth, nmap, s.intr)
    x = torch.zeros((64, 12), dtype=torch.float32, device="cuda")
    pose = torch.zeros(6, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EDError) as ei:
        ctx.gn_step(frame, E.SolverParams(), x, pose)
    assert ei.value.status == 7
    torch.cuda.synchronize()
    # the same build with the default budget succeeds
    G = C.gpu_setup(s, radius=r, max_nodes=64)
    assert G["graph"].m > 0


@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed_fp64"])
def test_zero_pcg_iterations_keep_the_parameters_and_report_b(precision):
    # n_pcg = 0: no PCG iteration, x and the pose unchanged, d = 0; ||b||
    # (the norm of the assembled gradient) is still reported, the same as a
    # solve with iterations reports for the same system
    torch, E = _torch(), _E()
    s = C.scene(SMALL)
    G = C.gpu_setup(s)
    ctx, m = G["ctx"], G["graph"].m
    prec = {"fp32": E.ED_PRECISION_FP32, "mixed": E.ED_PRECISION_MIXED,
            "mixed_fp64": E.ED_PRECISION_MIXED_FP64}[precision]
    x = ctx.identity_x()
    xm = x.double().clone()
    pose = torch.zeros(6, dtype=torch.float64, device="cuda")
    st = E.new_stats(1)
    ctx.gn_step(G["frame"], E.SolverParams(n_pcg=0, precision=prec), x, pose, x_master=xm, stats=st)
    r0 = E.read_stats(st)[0]
    assert r0["status"] == 0 and r0["pcg_iters"] == 0
    assert torch.equal(x, ctx.identity_x()) and torch.equal(pose, torch.zeros_like(pose))
    sysm = ctx.export_system()
    assert float(sysm["delta"].abs().max()) == 0.0
    gnorm = float(sysm["grad"].double().norm())
    assert r0["pcg_res0"] == pytest.approx(gnorm, rel=1e-5) and r0["pcg_res"] == pytest.approx(gnorm, rel=1e-5)
    # the same system solved with iterations reports the same ||b||
    ctx.gn_step(G["frame"], E.SolverParams(n_pcg=10, precision=prec), x, pose, x_master=xm, stats=st)
    r1 = E.read_stats(st)[0]
    assert r1["status"] == 0 and r1["pcg_iters"] == 10
    assert r1["pcg_res0"] == pytest.approx(gnorm, rel=1e-5)
    assert r1["pcg_res"] < r1["pcg_res0"]


def test_sampled_timing_hook_records_every_nth_launch():
    """ed_set_timing_every: of 7 PCG solves with every = 3 only launches 2 and
    5 are recorded (two pairs, each a positive duration); every = 0 is an
    argument error; the solves' results do not depend on the hook."""
    torch, E = _torch(), _E()
    s = C.scene(SMALL)
    G = C.gpu_setup(s)
    ctx, g = G["ctx"], G["graph"]
    prm = C.solver(s)

    def run(events, every):
        x = torch.empty((g.m, 12), dtype=torch.float32, device="cuda")
        pose = torch.empty(6, dtype=torch.float64, device="cuda")
        ctx.reset_params(x, pose, prior=s.pose_prior)
        if events is not None:
            ctx.set_timing(E.ED_KERNEL_PCG, events, every=every)
        for _ in range(7):
            ctx.gn_step(G["frame"], prm, x, pose)
        torch.cuda.synchronize()
        n = ctx.timing_count() if events is not None else 0
        ctx.set_timing(E.ED_KERNEL_PCG, [])
        return x.cpu(), n

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
    x_hook, n = run(ev, 3)
    assert n == 2
    assert all(ev[2 * i].elapsed_time(ev[2 * i + 1]) > 0 for i in range(n))
    x_plain, _ = run(None, 1)
    assert torch.equal(x_hook, x_plain)
    with pytest.raises(E.EDError) as ei:
        ctx.set_timing(E.ED_KERNEL_PCG, ev, every=0)
    assert ei.value.status == 1
