#!/usr/bin/env python
"""Benchmark of the ED Gauss-Newton registration hot path on B300.

One step = one frame of the whole hot path on the 640x480 / 2048-node
workload: target normal map, deformation graph (Poisson nodes, nearest
nodes, weights, node graph, block structure), 10 Gauss-Newton iterations of
20 block-Jacobi PCG iterations each, final warp and fusion.  The metric is
Gauss-Newton iterations per second over the whole step (10 per frame), with
the inputs resident in HBM; L2 is flushed between steps by writing a buffer
larger than L2.  `e2e` repeats the measurement with the frame's depth and
colour maps copied from pinned host memory every step and the solved node
parameters and statistics copied back.

--impl reference times the FP64 CPU oracle (the reference arm of this
build) on the same workload, one frame per step.
Multi-GPU: every rank solves its own frame (independent problems, weak
scaling, no collective on the data path).
"""
import argparse
import contextlib
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ED Gauss-Newton iters/s @640x480, 2048 nodes; fraction of HBM roofline"
WORKLOAD = "tissue_640x480_n2048"


def metric_for(W, H, nodes):
    """The headline metric's name for a workload of W x H pixels and this many
    nodes (the 640x480 / 2048-node workload gives METRIC itself)."""
    return f"ED Gauss-Newton iters/s @{W}x{H}, {nodes} nodes; fraction of HBM roofline"



@contextlib.contextmanager
def gc_paused():
    """A timed region runs with Python's garbage collector off (collected just
    before), as timeit does: the host loop issues work between its waits for
    the GPU, and a collection pass of a few milliseconds there would show up as
    GPU idle time in a region of some tens of milliseconds."""
    gc.collect()
    gc.disable()
    try:
        yield
    finally:
        gc.enable()

def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--workload", default="single", choices=["single", "batch16", "push_sequence", "grad"],
                    help="batch16: 16 independent problems (320x240 / 640x480 / 1280x720, 200-4096 nodes) "
                         "as one batched, graph-captured GN iteration vs 16 sequential solves; push_sequence: "
                         "the frame loop (registration, fusion, downsampling, node regeneration) over a "
                         "synthetic 640x480 push sequence, one frame per step; grad: the differentiable "
                         "energy, forward (ed_energy) and hand-written backward (ed_energy_grad), per step")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed", "mixed_fp64"],
                    help="mixed: float-float PCG dot products; mixed_fp64: FP64 PCG dot products (both with "
                         "compensated block reductions and FP64 master parameters)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--keypoints", type=int, default=0,
                    help="sparse key correspondences (E_corr, w_corr = 10): this many seeded key points")
    ap.add_argument("--weights", default="gaussian", choices=["gaussian", "eq2"],
                    help="skinning weights: Gaussian (the workload's) or the paper's Eq. (2)")
    ap.add_argument("--lm", type=float, default=None, metavar="LAMBDA0",
                    help="Levenberg-Marquardt acceptance on the device from this damping (Sec. II.F); "
                         "default: plain Gauss-Newton (lambda = 0)")
    ap.add_argument("--radius", type=float, default=0.0,
                    help="Poisson radius (mm); 0 = calibrate to the workload's node count")
    ap.add_argument("--oracle-leg", default=None, help=argparse.SUPPRESS)   # child process of the OpenMP CPU leg
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank):
    """Every rank registers its own frame: independent problems, no data-path
    collective (weak scaling)."""
    return 1 + rank


def max_over_ranks(seconds, dist=None, device="cpu"):
    """The job's time is the slowest rank's; `dist` is torch.distributed or None."""
    if dist is None:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, gn_per_step, seconds):
    """GN iterations per second summed over all ranks (each rank did steps x gn_per_step)."""
    return world * steps * gn_per_step / seconds


class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, its maximum, clock
    event reasons) on the GPU with the given UUID."""

    def __init__(self, uuid):
        import ctypes
        self.C = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.lib.nvmlDeviceGetHandleByUUID(("GPU-" + uuid).encode(), ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        self._reasons = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sm_mhz(self):
        v = self.C.c_uint(0)
        return float(v.value) if self.lib.nvmlDeviceGetClockInfo(self.h, 1, self.C.byref(v)) == 0 else None

    def sm_max_mhz(self):
        v = self.C.c_uint(0)
        return float(v.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, self.C.byref(v)) == 0 else None

    def reasons(self):
        v = self.C.c_ulonglong(0)
        return int(v.value) if self._reasons(self.h, self.C.byref(v)) == 0 else 0


class ClockSampler:
    """SM clocks and clock event reasons sampled every 20 ms during the timed
    region (read-only NVML queries); nvidia-smi is the fallback.  (Every 2 ms,
    the sampler's driver calls held back the host loop's launches and waits
    often enough to take 10-20% off the end-to-end figure on some runs.)"""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index):
        self.cuda_index = cuda_index
        self.sm, self.reasons, self.smax = [], set(), None
        self.stop_ev = threading.Event()
        self.thread = None
        self.mode = None
        self.proc = None

    def _poll_nvml(self, nv):
        while not self.stop_ev.is_set():
            v = nv.sm_mhz()
            if v is not None:
                self.sm.append(v)
            bits = nv.reasons()
            for bit, name in self.REASONS.items():
                if bits & bit:
                    self.reasons.add(name)
            self.stop_ev.wait(0.02)

    def _poll_smi(self):
        fields = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.cuda_index}", f"--query-gpu={fields}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 6:
                continue
            try:
                self.sm.append(float(parts[0]))
                self.smax = max(self.smax or 0.0, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:6]):
                if v.lower() == "active":
                    self.reasons.add(nm)

    def start(self):
        try:
            import torch
            nv = _Nvml(str(torch.cuda.get_device_properties(self.cuda_index).uuid))
            self.smax = nv.sm_max_mhz()
            self.mode = "nvml"
            self.thread = threading.Thread(target=self._poll_nvml, args=(nv,), daemon=True)
        except Exception:
            self.mode = "nvidia-smi"
            self.thread = threading.Thread(target=self._poll_smi, daemon=True)
        self.thread.start()
        if self.mode == "nvidia-smi":
            time.sleep(0.5)   # nvidia-smi needs a moment before its first line

    def stop(self):
        if self.mode is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock query unavailable"]}
        self.stop_ev.set()
        if self.proc is not None:
            self.proc.terminate()
        self.thread.join(timeout=5)
        return {"sm_mhz": statistics.median(self.sm) if self.sm else None, "sm_max_mhz": self.smax,
                "reasons": sorted(self.reasons), "samples": len(self.sm), "source": self.mode}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def pcg_bytes_per_launch(m, n_upper, n_pcg):
    """Algorithmic bytes of one PCG launch (n_pcg iterations): per iteration the
    upper 12x12 blocks (576 B each), the block inverses (576 B per node) and 8
    FP32 vector passes over the P = 12m + 6 unknowns."""
    P = 12 * m + 6
    return n_pcg * (n_upper * 576 + m * 576 + 8 * P * 4)


def gn_bytes_per_iteration(n_points, n_valid, m, n_upper, n_pcg):
    """Algorithmic bytes of one Gauss-Newton iteration: the point pass (60 B per
    associated point: position, normal, node indices, depth, target normal;
    40 B per other point), writing the upper blocks and pose-node blocks, and
    the PCG launch."""
    return (n_valid * 60 + (n_points - n_valid) * 40 + n_upper * 576 + m * 288
            + pcg_bytes_per_launch(m, n_upper, n_pcg))


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def run_ours(args, rank, world, local):
    import torch
    import paper_1803_02009_b300 as E
    import synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    s = synth.make_scene(args.config, seed=rank_seed(rank))
    cfg = s.cfg
    fx, fy, cx, cy, W, H = s.intr
    dev = "cuda"
    cap_pts = s.N + W * H
    ctx = E.Context(max_points=cap_pts + 3 * args.keypoints, max_nodes=max(cfg.node_count, 64), max_width=W,
                    max_height=H, max_cells=1 << 24)
    pos = torch.from_numpy(s.model_pos).to(dev)
    nrm = torch.from_numpy(s.model_nrm).to(dev)
    col = torch.from_numpy(s.model_col).to(dev)
    tst = torch.from_numpy(s.model_t).to(dev)
    depth = torch.from_numpy(s.tgt_depth).to(dev)
    color = torch.from_numpy(np.ascontiguousarray(s.tgt_color)).to(dev)
    nmap = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    frame = E.make_frame(depth, nmap, s.intr, color)
    # the grid-node workload (160x120, an 8x8 node grid) keeps its given nodes;
    # the others sample Poisson nodes at the radius that yields the node count
    nodes_t = torch.from_numpy(s.nodes).to(dev) if s.nodes is not None else None
    radius = (0.0 if nodes_t is not None else
              args.radius if args.radius > 0 else E.calibrate_radius(ctx, pos, nrm, cfg.node_count))
    wmode = E.ED_WEIGHT_EQ2 if args.weights == "eq2" else E.ED_WEIGHT_GAUSSIAN
    kp_keep = None
    if args.keypoints > 0:
        kp, kp_tgt, _ = synth.make_keypoints(s, args.keypoints, seed=rank_seed(rank))
        kp_keep = (torch.from_numpy(kp).to(dev), torch.from_numpy(kp_tgt).to(dev))
        ctx.set_keypoints(kp_keep[0], kp_keep[1], 10.0)
    prm = E.SolverParams(n_pcg=cfg.n_pcg, prior=tuple(float(v) for v in s.pose_prior),
                         precision={"fp32": E.ED_PRECISION_FP32, "mixed": E.ED_PRECISION_MIXED,
                                    "mixed_fp64": E.ED_PRECISION_MIXED_FP64}[args.precision],
                         lm_accept=args.lm is not None)
    prm_c = prm.c()
    F = E.FuseParams(frame=1)
    x = torch.empty((cfg.node_count, 12), dtype=torch.float32, device=dev)
    xm = torch.empty((cfg.node_count, 12), dtype=torch.float64, device=dev)
    pose = torch.empty(6, dtype=torch.float64, device=dev)
    stats = E.new_stats(cfg.n_gn)
    wpos = torch.empty_like(pos)
    wnrm = torch.empty_like(nrm)
    fout = dict(pos=torch.empty((cap_pts, 4), dtype=torch.float32, device=dev),
                nrm=torch.empty((cap_pts, 4), dtype=torch.float32, device=dev),
                col=torch.empty((cap_pts, 4), dtype=torch.float32, device=dev),
                t=torch.empty(cap_pts, dtype=torch.int32, device=dev),
                counts=torch.zeros(2, dtype=torch.int32, device=dev))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2

    gn_ev = []
    ph_ev = []

    def ev_now():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    def step(record_gn=False, depth=depth, color=color, frame=frame, while_solving=None):
        if record_gn:
            p0 = ev_now()
        ctx.compute_normals(depth, s.intr, cfg.normal_half_width, out=nmap)
        if nodes_t is not None:
            g = ctx.build_graph(pos, nrm, nodes=nodes_t, sigma=s.sigma, weight_mode=wmode, reuse=True)
        else:
            g = ctx.build_graph(pos, nrm, node_radius=radius, max_nodes=cfg.node_count, sigma=radius,
                                weight_mode=wmode, reuse=True)
        m = g.m
        ctx.reset_params(x[:m], pose, x_master=xm[:m], prior=s.pose_prior)
        if args.lm is not None:
            ctx.lm_reset(args.lm)
        if record_gn:
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record()
        for it in range(cfg.n_gn):
            ctx.gn_step(frame, prm_c, x[:m], pose, x_master=xm[:m], stats=stats[it:it + 1])
            if it == 0 and while_solving is not None:
                while_solving()              # (host work while the GPU has the solve queued)
        if record_gn:
            e1 = torch.cuda.Event(enable_timing=True)
            e1.record()
            gn_ev.append((e0, e1))
        ctx.warp(x[:m], pose, pos, nrm, wpos, wnrm)
        ctx.fuse(pos, nrm, col, tst, wpos, wnrm, frame, F, cap_pts, out=fout)
        if record_gn:
            ph_ev.append((p0, e0, e1, ev_now()))
        return g

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g = ctx.graph
    st_last = E.read_stats(stats)

    # timed region.  The roofline's PCG duration comes from events around the
    # last PCG solve of every timed step (one pair per step: an event between
    # two kernels ends their programmatic overlap, so the other launches of the
    # step carry none); the phase breakdown comes from a separate pass below.
    K = args.steps
    tm_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
    ctx.set_timing(E.ED_KERNEL_PCG, tm_ev, every=cfg.n_gn)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = E.launch_count()
    step_ms = []
    barrier()
    torch.cuda.synchronize()
    with gc_paused():
        for k in range(K):
            flush.fill_(k & 0xff)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record()
            step()
            ev1.record()
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    barrier()
    launches = E.launch_count() - l0
    clk = clocks.stop()
    n_rec = ctx.timing_count()
    ctx.set_timing(E.ED_KERNEL_PCG, [])
    pcg_ms = [tm_ev[2 * i].elapsed_time(tm_ev[2 * i + 1]) for i in range(n_rec)]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    value = whole_job_rate(world, K, cfg.n_gn, total_s)

    # end to end through the public API with host buffers: every step copies
    # its frame (depth, colour) in from pinned host memory and reads its result
    # (node parameters, statistics) back; the next frame's copy runs on a copy
    # stream into the other of two input buffers while this frame's solve runs
    # (issued after the first Gauss-Newton step: during the graph build, whose
    # host reads wait for the GPU, the copy held the build back)
    h_depth = torch.from_numpy(s.tgt_depth).pin_memory()
    h_color = torch.from_numpy(np.ascontiguousarray(s.tgt_color)).pin_memory()
    h_x = torch.empty((cfg.node_count, 12), dtype=torch.float32).pin_memory()
    h_stats = torch.empty(stats.shape, dtype=torch.uint8).pin_memory()
    h2d = h_depth.numel() * 4 + h_color.numel() * 4
    d2h = h_x.numel() * 4 + h_stats.numel()
    d_in = [torch.empty_like(depth) for _ in range(2)]
    c_in = [torch.empty_like(color) for _ in range(2)]
    f_in = [E.make_frame(d_in[i], nmap, s.intr, c_in[i]) for i in range(2)]
    copy_stream = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    released = [torch.cuda.Event() for _ in range(2)]
    compute = torch.cuda.current_stream()
    def fetch(k):
        b = k & 1
        copy_stream.wait_stream(compute) if k == 0 else copy_stream.wait_event(released[b])
        with torch.cuda.stream(copy_stream):
            d_in[b].copy_(h_depth, non_blocking=True)
            c_in[b].copy_(h_color, non_blocking=True)
            copied[b].record()

    flush_ev = []

    def e2e_run(n, timed=False):
        fetch(0)
        for k in range(n):
            b = k & 1
            nxt = (lambda kk=k + 1: fetch(kk)) if k + 1 < n else None
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record()
            flush.fill_(k & 0xff)            # L2 flushed before every step; its time is taken out below
            f1.record()
            if timed:
                flush_ev.append((f0, f1))
            compute.wait_event(copied[b])
            gg = step(depth=d_in[b], color=c_in[b], frame=f_in[b], while_solving=nxt)
            released[b].record()
            h_x[:gg.m].copy_(x[:gg.m], non_blocking=True)
            h_stats.copy_(stats, non_blocking=True)

    e2e_run(args.warmup)                     # untimed: first use of the copy stream and buffers
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    e2e_clocks = ClockSampler(local)
    e2e_clocks.start()
    with gc_paused():
        t_host = time.perf_counter()
        ev0.record()
        e2e_run(K, timed=True)
        ev1.record()
        ev1.synchronize()
        e2e_wall_ms = (time.perf_counter() - t_host) * 1e3
    e2e_clk = e2e_clocks.stop()
    flush_ms = sum(a.elapsed_time(b) for a, b in flush_ev)
    e2e_s = max_over_ranks((ev0.elapsed_time(ev1) - flush_ms) / 1e3, dist, dev)
    e2e_value = whole_job_rate(world, K, cfg.n_gn, e2e_s)

    # the step's phases: K more steps, the same as the timed ones, with events
    # between the phases (outside the timed region: the events end the
    # programmatic overlap of the kernels on either side)
    for k in range(K):
        flush.fill_(k & 0xff)
        step(record_gn=True)
    torch.cuda.synchronize()
    gn_ms = [a.elapsed_time(b) for a, b in gn_ev[-K:]]
    phases_us = {
        "normals_and_graph_build": statistics.median(a.elapsed_time(b) * 1e3 for a, b, _, _ in ph_ev[-K:]),
        "gauss_newton": statistics.median(b.elapsed_time(c) * 1e3 for _, b, c, _ in ph_ev[-K:]),
        "warp_and_fuse": statistics.median(c.elapsed_time(d) * 1e3 for _, _, c, d in ph_ev[-K:]),
        "note": "median over K steps run after the timed region with CUDA events between the step's phases "
                "(the build's parameter reset included in the first)"}

    # per-kernel device time of a Gauss-Newton iteration (events recorded by
    # the library around each launch of one kernel; two extra steps per
    # kernel, outside the timed region)
    kern_us = {}
    for kid, name in ((E.ED_KERNEL_POINTS, "k_points"), (E.ED_KERNEL_ASSEMBLE, "k_assemble"),
                      (E.ED_KERNEL_FINALIZE, "k_fin_totals"), (E.ED_KERNEL_PCG, "k_pcg")):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4 * cfg.n_gn)]
        ctx.set_timing(kid, ev)
        for k in range(2):
            flush.fill_(k & 0xff)
            step()
        torch.cuda.synchronize()
        n_r = ctx.timing_count()
        ctx.set_timing(kid, [])
        t = [ev[2 * i].elapsed_time(ev[2 * i + 1]) * 1e3 for i in range(n_r)]
        kern_us[name] = statistics.median(t) if t else None

    peak, peak_kind = measured_peaks()
    n_upper = (g.nnzb + g.m) // 2          # symmetric pattern, every diagonal block present
    n_pcg_last = int(st_last[-1]["pcg_iters"])   # (the timed launches: the last solve of a step)
    byt = pcg_bytes_per_launch(g.m, n_upper, n_pcg_last)
    n_valid_last = int(st_last[-1]["n_valid"])
    gn_byt = gn_bytes_per_iteration(s.N, n_valid_last, g.m, n_upper, cfg.n_pcg)
    gn_rate = whole_job_rate(world, K, cfg.n_gn, max_over_ranks(sum(gn_ms) / 1e3, dist, dev)) if gn_ms else None
    avg_pcg_s = (sum(pcg_ms) / len(pcg_ms)) / 1e3 if pcg_ms else float("nan")
    achieved = byt / avg_pcg_s / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "pcg_traffic.json")
    if os.path.exists(tr_path):
        with open(tr_path) as f:
            tr = json.load(f)
        if tr.get("workload") == args.config and tr.get("kernel_rev") == kernel_rev():
            traffic = tr.get("bytes_per_launch")

    out = {
        "metric": metric_for(W, H, cfg.node_count), "value": value, "unit": "GN iters/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f32+f64",
        "data": "synthetic (seeded stereo-scope tissue scene, no dataset)",
        "config": {"workload": args.config, "width": W, "height": H, "model_points": s.N, "nodes": g.m,
                   "nnz_blocks": g.nnzb, "gn_iters_per_step": cfg.n_gn, "pcg_iters": cfg.n_pcg,
                   "node_radius_mm": radius, "precision": args.precision, "keypoints": args.keypoints,
                   "weights": args.weights,
                   "solver": "gauss-newton" if args.lm is None else f"levenberg-marquardt, lambda0 = {args.lm:g}",
                   "l2": "flushed between steps (512 MB write)",
                   "step": "normals + build_graph + 10 x gn_step + warp + fuse"},
        "gn_only_iters_per_s": gn_rate,
        "step_phases_us": phases_us,
        "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms),
                    "note": "this rank's timed steps one by one (CUDA events)"},
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "GN iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "K steps end to end: each frame copied in from pinned host memory (the next frame's copy "
                        "overlapping this frame's compute on a copy stream), results read back; the L2 flush "
                        "before every step is timed by events and taken out",
                "host_wall_ms_per_step": e2e_wall_ms / K, "clocks": e2e_clk},
        "roofline": {"kernel": "k_pcg (persistent block-Jacobi PCG)", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes_per_launch": byt,
                     "avg_launch_us": avg_pcg_s * 1e6, "launches_timed": len(pcg_ms),
                     "pcg_iters_per_launch": n_pcg_last,
                     "note": "CUDA events around the last PCG solve of every timed step (one launch per step; "
                             "the step's other launches carry no events)"},
        "gn_kernels_us": dict(kern_us, note="median device time per launch (library events on the launching "
                                             "stream, 2 extra steps outside the timed region)"),
        "gn_iteration_roofline": {"bound": "hbm", "algorithmic_bytes": gn_byt,
                                  "achieved": gn_byt * gn_rate / world / 1e9 if gn_rate else None,
                                  "peak": peak, "unit": "GB/s",
                                  "frac": gn_byt * gn_rate / world / 1e9 / peak if gn_rate else None,
                                  "note": "per GPU, over the GN iterations alone (no graph build, warp, fuse)"},
        "final_stats": {k: st_last[-1][k] for k in ("energy", "n_valid", "pcg_iters", "status")},
    }
    return out, s


def kernel_rev():
    """Content hash of the PCG kernel sources (ties an ncu traffic figure to a build)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1803_02009_b300", "csrc")
    for fn in ("pcg.cu", "ed_internal.cuh"):
        with open(os.path.join(d, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------
# differentiation: forward energy + hand-written backward
# ----------------------------------------------------------------------------

def grad_bytes(n_points, n_valid, m):
    """Algorithmic bytes of one evaluation: the forward point pass (position,
    normal, node indices: 40 B per point, + depth and target normal 20 B per
    associated point, association 4 B out), the backward point pass (the same
    40 B + association 4 B in, two 16 B records out) and the per-node gradient
    kernel (every point once for each of its 4 nodes: sorted position 4 B,
    record 16 B, position 16 B, node indices 8 B; 48 B of parameters and 48 B
    of gradient per node)."""
    fwd = n_points * 44 + n_valid * 20
    bwd = n_points * (44 + 32) + n_valid * 20
    nodes = 4 * n_points * 44 + m * 96
    return fwd, bwd, nodes


def run_grad(args, rank, world, local):
    import torch
    import paper_1803_02009_b300 as E
    import synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    s = synth.make_scene(args.config, seed=rank_seed(rank))
    cfg = s.cfg
    fx, fy, cx, cy, W, H = s.intr
    dev = "cuda"
    ctx = E.Context(max_points=s.N, max_nodes=max(cfg.node_count, 64), max_width=W, max_height=H,
                    max_cells=1 << 24)
    pos = torch.from_numpy(s.model_pos).to(dev)
    nrm = torch.from_numpy(s.model_nrm).to(dev)
    depth = torch.from_numpy(s.tgt_depth).to(dev)
    nmap = ctx.compute_normals(depth, s.intr, cfg.normal_half_width)
    frame = E.make_frame(depth, nmap, s.intr)
    radius = E.calibrate_radius(ctx, pos, nrm, cfg.node_count)
    g = ctx.build_graph(pos, nrm, node_radius=radius, max_nodes=cfg.node_count, sigma=radius)
    prm = E.SolverParams(n_pcg=cfg.n_pcg, prior=tuple(float(v) for v in s.pose_prior))
    # the evaluation point: three Gauss-Newton steps from the identity (a
    # representative association), then fixed
    x = ctx.identity_x()
    pose = torch.tensor(s.pose_prior, dtype=torch.float64, device=dev)
    for _ in range(3):
        ctx.gn_step(frame, prm, x, pose)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    e_out = torch.empty(6, dtype=torch.float64, device=dev)

    def step():
        ctx.energy(frame, prm, x, pose, out=e_out)
        return ctx.energy_grad(frame, prm, x, pose)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    K = args.steps
    tm_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
    ctx.set_timing(E.ED_KERNEL_GRAD, tm_ev)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = E.launch_count()
    step_ms = []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with gc_paused():
        for k in range(K):
            flush.fill_(k & 0xff)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            step()
            ev1.record()
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
    torch.cuda.synchronize()
    launches = E.launch_count() - l0
    clk = clocks.stop()
    n_rec = ctx.timing_count()
    ctx.set_timing(E.ED_KERNEL_GRAD, [])

    # end to end: the node parameters and the pose come from pinned host
    # memory every step, the energy and both gradients go back to it
    h_x = x.cpu().pin_memory()
    h_pose = pose.cpu().pin_memory()
    h_e = torch.empty(6, dtype=torch.float64).pin_memory()
    h_gx = torch.empty(x.shape, dtype=torch.float32).pin_memory()
    h_gp = torch.empty(6, dtype=torch.float32).pin_memory()
    d_x, d_pose = torch.empty_like(x), torch.empty_like(pose)

    def e2e_step():
        d_x.copy_(h_x, non_blocking=True)
        d_pose.copy_(h_pose, non_blocking=True)
        ctx.energy(frame, prm, d_x, d_pose, out=e_out)
        gx, gp = ctx.energy_grad(frame, prm, d_x, d_pose)
        h_e.copy_(e_out, non_blocking=True)
        h_gx.copy_(gx, non_blocking=True)
        h_gp.copy_(gp, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    with gc_paused():
        for k in range(K):
            flush.fill_(k & 0xff)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            e2e_step()
            ev1.record()
            ev1.synchronize()
            e2e_ms.append(ev0.elapsed_time(ev1))
    e2e_value = world * K / max_over_ranks(sum(e2e_ms) / 1e3, dist, dev)
    h2d = h_x.numel() * 4 + h_pose.numel() * 8
    d2h = h_e.numel() * 8 + h_gx.numel() * 4 + h_gp.numel() * 4
    kern_us = statistics.median([tm_ev[2 * i].elapsed_time(tm_ev[2 * i + 1]) * 1e3 for i in range(n_rec)])
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    value = world * K / total_s
    st = E.new_stats()
    ctx.gn_step(frame, prm, x.clone(), pose.clone(), stats=st)   # (only to read the association's size)
    n_valid = E.read_stats(st)[0]["n_valid"]
    fwd, bwd, nodes_b = grad_bytes(s.N, n_valid, g.m)
    peak, peak_kind = measured_peaks()
    achieved = nodes_b / (kern_us * 1e-6) / 1e9
    return {
        "metric": f"ED energy + gradient evaluations/s @{W}x{H}, {cfg.node_count} nodes "
                  "(forward + hand-written backward)",
        "value": value, "unit": "evaluations/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_s * 1e3 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded stereo-scope tissue scene, no dataset)",
        "config": {"workload": args.config, "model_points": s.N, "nodes": g.m, "unknowns": 12 * g.m + 6,
                   "evaluation_point": "after 3 Gauss-Newton steps from the identity",
                   "skinning_weights": "recomputed from the node indices in both passes (not stored)",
                   "l2": "flushed between steps (512 MB write)"},
        "gpu_launches": launches, "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "evaluations/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "node parameters and pose copied in from pinned host memory every step, energy and "
                        "gradients copied back; L2 flushed before every step (outside the events)"},
        "algorithmic_bytes": {"forward": fwd, "backward_points": bwd, "backward_nodes": nodes_b,
                              "valid_points": n_valid},
        "roofline": {"kernel": "k_grad_nodes (per-node gradient)", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "avg_launch_us": kern_us, "launches_timed": n_rec, "traffic": None},
        "evaluation_roofline": {"bound": "hbm", "algorithmic_bytes": fwd + bwd + nodes_b,
                                "achieved": (fwd + bwd + nodes_b) * value / world / 1e9, "peak": peak,
                                "frac": (fwd + bwd + nodes_b) * value / world / 1e9 / peak, "unit": "GB/s"},
    }


# ----------------------------------------------------------------------------
# batched workload: many independent problems per GN iteration
# ----------------------------------------------------------------------------

def run_batch(args, rank, world, local):
    import torch
    import paper_1803_02009_b300 as E
    import synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    members = synth.batch_scenes(16, seed0=1 + 16 * rank)
    n_gn, n_pcg = members[0][0].cfg.n_gn, members[0][0].cfg.n_pcg
    probs = []
    for s, m in members:
        fx, fy, cx, cy, W, H = s.intr
        ctx = E.Context(max_points=s.N, max_nodes=m, max_width=W, max_height=H, max_cells=1 << 24)
        pos = torch.from_numpy(s.model_pos).cuda()
        nrm = torch.from_numpy(s.model_nrm).cuda()
        depth = torch.from_numpy(s.tgt_depth).cuda()
        nmap = ctx.compute_normals(depth, s.intr, s.cfg.normal_half_width)
        r = E.calibrate_radius(ctx, pos, nrm, m)
        g = ctx.build_graph(pos, nrm, node_radius=r, max_nodes=m, sigma=r)
        x0 = torch.zeros((g.m, 12), dtype=torch.float32, device="cuda")
        x0[:, 0] = 1.0
        x0[:, 5] = 1.0
        x0[:, 10] = 1.0
        probs.append(dict(s=s, ctx=ctx, keep=(pos, nrm, depth, nmap), g=g, frame=E.make_frame(depth, nmap, s.intr),
                          prm=E.SolverParams(n_pcg=n_pcg, prior=tuple(float(v) for v in s.pose_prior)),
                          x0=x0, pose0=torch.tensor(s.pose_prior, dtype=torch.float64, device="cuda")))
    xs = [p["x0"].clone() for p in probs]
    poses = [p["pose0"].clone() for p in probs]

    def reset():
        for p, x, q in zip(probs, xs, poses):
            x.copy_(p["x0"])
            q.copy_(p["pose0"])

    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    K = args.steps

    # 16 sequential single-problem solves (ed_gn_step, no graph)
    def sequential():
        for p, x, q in zip(probs, xs, poses):
            for _ in range(n_gn):
                p["ctx"].gn_step(p["frame"], p["prm"], x, q)

    for _ in range(args.warmup):
        reset()
        sequential()
    torch.cuda.synchronize()
    seq_ms = []
    with gc_paused():
        for k in range(K):
            reset()
            flush.fill_(k & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sequential()
            e1.record()
            e1.synchronize()
            seq_ms.append(e0.elapsed_time(e1))
    seq_x = [x.cpu().numpy() for x in xs]
    reset()
    for p, x, q in zip(probs, xs, poses):
        p["ctx"].gn_step(p["frame"], p["prm"], x, q)
    seq_x1 = [x.cpu().numpy() for x in xs]

    # batched: autotuned schedule, n_gn iterations captured as one CUDA graph
    B = E.Batch([p["ctx"] for p in probs])
    stats = [E.new_stats(n_gn) for _ in probs]
    B.bind([p["frame"] for p in probs], [p["prm"] for p in probs], xs, poses, stats=stats)
    reset()
    sched, tune_ms = B.autotune()
    reset()
    B.gn_step()
    torch.cuda.synchronize()
    diff1 = max(float(np.max(np.abs(x.cpu().numpy() - xr) / np.maximum(1.0, np.abs(xr)))) for x, xr in zip(xs, seq_x1))
    B.capture(n_iters=n_gn)
    for _ in range(args.warmup):
        reset()
        B.launch()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = E.launch_count()
    bat_ms = []
    with gc_paused():
        for k in range(K):
            reset()
            flush.fill_(k & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            B.stream.wait_stream(torch.cuda.current_stream())   # reset and flush done before the clock starts
            e0.record(B.stream)
            B.launch(stream=B.stream)
            e1.record(B.stream)
            e1.synchronize()
            bat_ms.append(e0.elapsed_time(e1))
    launches = E.launch_count() - l0
    clk = clocks.stop()
    torch.cuda.synchronize()
    diff = max(float(np.max(np.abs(x.cpu().numpy() - xr) / np.maximum(1.0, np.abs(xr)))) for x, xr in zip(xs, seq_x))
    st = [E.read_stats(b)[-1] for b in stats]
    units = len(probs) * n_gn
    bat_s = max_over_ranks(sum(bat_ms) / 1e3, dist, "cuda")
    seq_s = max_over_ranks(sum(seq_ms) / 1e3, dist, "cuda")
    value = whole_job_rate(world, K, units, bat_s)
    seq_value = whole_job_rate(world, K, units, seq_s)
    peak, peak_kind = measured_peaks()
    gn_bytes = sum(gn_bytes_per_iteration(p["s"].N, int(q["n_valid"]), p["g"].m, (p["g"].nnzb + p["g"].m) // 2, n_pcg)
                   for p, q in zip(probs, st))
    achieved = gn_bytes * (value / len(probs)) / world / 1e9    # batched iterations per second per GPU

    # the batched PCG launches (one per group of problems) timed by the
    # library's events in two uncaptured batched iterations
    evs = []
    for p in probs:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        p["ctx"].set_timing(E.ED_KERNEL_PCG, ev)
        evs.append(ev)
    for k in range(2):
        reset()
        flush.fill_(k & 0xff)
        B.gn_step()
    torch.cuda.synchronize()
    pcg_us = 0.0
    for p, ev in zip(probs, evs):
        n_r = p["ctx"].timing_count()
        p["ctx"].set_timing(E.ED_KERNEL_PCG, [])
        if n_r:
            pcg_us += statistics.median(ev[2 * i].elapsed_time(ev[2 * i + 1]) * 1e3 for i in range(n_r))
    pcg_byt = sum(pcg_bytes_per_launch(p["g"].m, (p["g"].nnzb + p["g"].m) // 2, n_pcg) for p in probs)
    pcg_achieved = pcg_byt / (pcg_us * 1e-6) / 1e9

    # end to end: every member's depth map copied in from pinned host memory
    # and its normal map recomputed, the parameters reset from host copies,
    # the captured iterations replayed, the parameters and statistics read back
    h_depth = [torch.from_numpy(p["s"].tgt_depth).pin_memory() for p in probs]
    h_x0 = [p["x0"].cpu().pin_memory() for p in probs]
    h_p0 = [p["pose0"].cpu().pin_memory() for p in probs]
    h_x = [torch.empty(p["x0"].shape, dtype=torch.float32).pin_memory() for p in probs]
    h_st = [torch.empty(b.shape, dtype=b.dtype).pin_memory() for b in stats]

    def e2e_step():
        for p, hd, hx, hp, x, q in zip(probs, h_depth, h_x0, h_p0, xs, poses):
            depth, nmap = p["keep"][2], p["keep"][3]
            depth.copy_(hd, non_blocking=True)
            p["ctx"].compute_normals(depth, p["s"].intr, p["s"].cfg.normal_half_width, out=nmap)
            x.copy_(hx, non_blocking=True)
            q.copy_(hp, non_blocking=True)
        B.launch()
        for x, hx, b, hb in zip(xs, h_x, stats, h_st):
            hx.copy_(x, non_blocking=True)
            hb.copy_(b, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    with gc_paused():
        for k in range(K):
            flush.fill_(k & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            e2e_step()
            e1.record()
            e1.synchronize()
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = whole_job_rate(world, K, units, max_over_ranks(sum(e2e_ms) / 1e3, dist, "cuda"))
    h2d = sum(t.numel() * t.element_size() for t in h_depth + h_x0 + h_p0)
    d2h = sum(t.numel() * t.element_size() for t in h_x + h_st)
    return {
        "metric": "batched ED GN iters/s (16 independent problems, one CUDA graph per frame)",
        "value": value, "unit": "GN iters/s (summed over problems)", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": bat_s * 1e3 / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded stereo-scope tissue scenes)",
        "config": {"workload": "batch16", "problems": [{"W": p["s"].cfg.W, "H": p["s"].cfg.H, "points": p["s"].N,
                                                         "nodes": p["g"].m} for p in probs],
                   "gn_iters": n_gn, "pcg_iters": n_pcg, "schedule": sched, "autotune_best_ms": tune_ms,
                   "l2": "flushed between steps (512 MB write)",
                   "step": "16 problems x n_gn GN iterations (graph build excluded)"},
        "sequential": {"value": seq_value, "unit": "GN iters/s", "ms_per_step": seq_s * 1e3 / K,
                       "what": "the same 16 problems solved one after another through ed_gn_step"},
        "speedup_vs_sequential": value / seq_value,
        "max_rel_diff_vs_sequential": {"after_1_gn_iter": diff1, f"after_{n_gn}_gn_iters": diff,
                                        "note": "different PCG reduction partitions; later iterations re-associate"},
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "GN iters/s (summed over problems)", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "note": "per step: 16 depth maps in from pinned host memory, normal maps recomputed, parameters "
                        "reset from host copies, the captured iterations replayed, parameters and statistics "
                        "back; L2 flushed before every step (outside the events)"},
        "roofline": {"kernel": "k_pcg_batch (batched persistent block-Jacobi PCG, one launch per group)",
                     "bound": "hbm", "achieved": pcg_achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": pcg_achieved / peak, "traffic": None, "algorithmic_bytes_per_iteration": pcg_byt,
                     "launch_us_per_iteration": pcg_us,
                     "note": "sum over the 16 problems of the single-problem PCG bytes, over the summed device "
                             "time of the batched launches of one iteration"},
        "gn_iteration_roofline": {"bound": "hbm", "algorithmic_bytes_per_batched_iteration": gn_bytes,
                                  "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                                  "frac": achieved / peak},
        "final_status": [int(q["status"]) for q in st],
    }


# ----------------------------------------------------------------------------
# push sequence: the frame loop of Algorithm 2 with Algorithm 3
# ----------------------------------------------------------------------------

SEQ_WORKLOAD = "push_640x480_n2048"
SEQ_BOX_MM = 0.2        # point-cloud density of Sec. III.A (dataset 6)


def run_sequence(args, rank, world, local):
    import torch
    import paper_1803_02009_b300 as E
    import synth

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = "cuda"
    W0, K = args.warmup, args.steps
    S = synth.make_push_sequence(SEQ_WORKLOAD, W0 + K, seed=rank_seed(rank))
    cfg = S.cfg
    fx, fy, cx, cy, W, H = S.intr
    cap = S.model_pos.shape[0] + 2 * W * H
    ctx = E.Context(max_points=cap, max_nodes=cfg.node_count, max_width=W, max_height=H, max_cells=1 << 24)
    pos0 = torch.from_numpy(S.model_pos).to(dev)
    nrm0 = torch.from_numpy(S.model_nrm).to(dev)
    radius = E.calibrate_radius(ctx, pos0, nrm0, cfg.node_count)
    tc = E.TrackerConfig(node_radius=radius, max_nodes=cfg.node_count, box=SEQ_BOX_MM, n_gn=cfg.n_gn,
                         normal_half_width=cfg.normal_half_width, solver=E.SolverParams(n_pcg=cfg.n_pcg),
                         fuse=E.FuseParams())
    T = E.Tracker(pos0, nrm0, torch.from_numpy(S.model_col).to(dev), torch.from_numpy(S.model_t).to(dev), S.intr,
                  tc, cap, ctx=ctx)
    # observations in pinned host memory; each step copies its frame in (e2e)
    h_depth = [torch.from_numpy(f.depth).pin_memory() for f in S.frames]
    h_color = [torch.from_numpy(np.ascontiguousarray(f.color)).pin_memory() for f in S.frames]
    truth = [torch.from_numpy(f.depth_clean).to(dev) for f in S.frames]
    depth = torch.empty((H, W), dtype=torch.float32, device=dev)
    color = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    infos = []
    for k in range(W0):
        depth.copy_(h_depth[k])
        color.copy_(h_color[k])
        infos.append(T.process(depth, color, k + 1, truth_depth=truth[k]))
    # (events around the last PCG solve of every frame only: an event between
    # two kernels ends their programmatic overlap)
    tm_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
    ctx.set_timing(E.ED_KERNEL_PCG, tm_ev, every=cfg.n_gn)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = E.launch_count()
    step_ms = []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with gc_paused():
        t_wall = time.perf_counter()
        for k in range(W0, W0 + K):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record()
            depth.copy_(h_depth[k], non_blocking=True)
            color.copy_(h_color[k], non_blocking=True)
            infos.append(T.process(depth, color, k + 1, truth_depth=truth[k]))
            ev1.record()
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
        torch.cuda.synchronize()
        wall_s = time.perf_counter() - t_wall
    if dist is not None:
        dist.barrier()
    launches = E.launch_count() - l0
    clk = clocks.stop()
    n_rec = ctx.timing_count()
    ctx.set_timing(E.ED_KERNEL_PCG, [])
    pcg_ms = [tm_ev[2 * i].elapsed_time(tm_ev[2 * i + 1]) for i in range(n_rec)]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    value = whole_job_rate(world, K, cfg.n_gn, total_s)
    e2e_value = whole_job_rate(world, K, cfg.n_gn, max_over_ranks(wall_s, dist, dev))
    timed = infos[W0:]
    g = ctx.graph
    n_upper = (g.nnzb + g.m) // 2
    byt = pcg_bytes_per_launch(g.m, n_upper, cfg.n_pcg)
    avg_pcg_s = (sum(pcg_ms) / len(pcg_ms)) / 1e3 if pcg_ms else float("nan")
    peak, peak_kind = measured_peaks()
    achieved = byt / avg_pcg_s / 1e9
    h2d = h_depth[0].numel() * 4 + h_color[0].numel() * 4
    d2h = 4 * 8 + 4 + 2 * 4 + E.STATS_BYTES        # error sums, fused count, model count + status, the last step's statistics
    return {
        "metric": METRIC, "value": value, "unit": "GN iters/s", "n_gpus": world, "steps": K, "warmup": W0,
        "ms_per_step": total_s * 1e3 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded push sequence: static camera, one 2-3 mm push per frame)",
        "config": {"workload": SEQ_WORKLOAD, "width": W, "height": H, "frames_timed": K, "nodes": cfg.node_count,
                   "node_radius_mm": radius, "box_mm": SEQ_BOX_MM, "gn_iters_per_step": cfg.n_gn,
                   "pcg_iters": cfg.n_pcg,
                   "step": "normals + node regeneration + 10 x gn_step + warp + error + fuse + downsample (one frame)",
                   "l2": "inputs of every step differ (a new frame); model 0.3-0.6 M points"},
        "frames_per_s": K / total_s,
        "accuracy": {"metric": "back-projection error vs the noise-free depth (Sec. III)", "unit": "mm",
                     "mean": float(np.mean([i["error_mean_mm"] for i in timed])),
                     "rms": float(np.sqrt(np.mean([i["error_rms_mm"] ** 2 for i in timed]))),
                     "max": float(max(i["error_max_mm"] for i in timed)),
                     "per_frame_mean": [round(i["error_mean_mm"], 4) for i in infos]},
        "model_points": [i["model"] for i in infos],
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "GN iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "wall clock of the timed loop: pinned host frames copied in, results read back"},
        "roofline": {"kernel": "k_pcg (persistent block-Jacobi PCG)", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": byt, "avg_launch_us": avg_pcg_s * 1e6,
                     "launches_timed": len(pcg_ms),
                     "note": "CUDA events around the last PCG solve of every timed frame (bytes: the last "
                             "frame's graph)"},
    }, S, radius


def sequence_cpu_baseline(S, radius, budget_s):
    import oracle
    cfg = S.cfg
    model = (S.model_pos, S.model_nrm, S.model_col, S.model_t)
    times = []
    t_start = time.perf_counter()
    for f in S.frames:
        if times and (time.perf_counter() - t_start > budget_s or len(times) >= 3):
            break
        t0 = time.perf_counter()
        model, _ = oracle.track_frame(model, f.depth, f.color, S.intr, radius, cfg.node_count, SEQ_BOX_MM, cfg.n_gn,
                                      cfg.n_pcg, f.index, cfg.normal_half_width, truth_depth=f.depth_clean)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    return {"value": len(times) * cfg.n_gn / tot, "unit": "GN iters/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {len(times)} frame(s) of the same push sequence (normals, nodes, {cfg.n_gn} GN x "
                      f"{cfg.n_pcg} PCG, warp, error, fuse, downsample) in the single-threaded FP64 oracle, "
                      f"{tot:.1f} s"}


# ----------------------------------------------------------------------------
# oracle (CPU) leg
# ----------------------------------------------------------------------------

def oracle_frame(s, radius, keypoints=0, weights="gaussian", seed=1, lm=None):
    """One frame of the whole path in the FP64 oracle; returns seconds."""
    import oracle
    import synth
    cfg = s.cfg
    mode = 1 if weights == "eq2" else 0
    t0 = time.perf_counter()
    nm = oracle.normals(s.tgt_depth, s.intr, cfg.normal_half_width)
    if s.nodes is not None:   # the grid-node workload
        G = oracle.build_graph(s.model_pos, nodes=s.nodes, K=4, KG=4, mode=mode, sigma=s.sigma)
    else:
        G = oracle.build_graph(s.model_pos, radius=radius, max_nodes=cfg.node_count, K=4, KG=4, mode=mode,
                               sigma=radius)
    K = None
    if keypoints > 0:
        kp, kp_tgt, _ = synth.make_keypoints(s, keypoints, seed=seed)
        K = oracle.keypoints(kp, kp_tgt[:, :3].astype(np.float64), G.g, K=4, mode=mode, sigma=radius)
    P = oracle.Problem(s.model_pos, s.model_nrm, G, s.tgt_depth, nm, s.intr, s.pose_prior, keypoints=K)
    x, pose, hist, st = oracle.gn_solve(P, P.identity_x(), s.pose_prior, cfg.n_gn, cfg.n_pcg,
                                        lam=0.0 if lm is None else lm, lm_accept=lm is not None)
    wp, wn, _ = oracle.warp(P, x, pose)
    wp4 = np.concatenate([wp, s.model_pos[:, 3:4]], 1).astype(np.float32)
    wn4 = np.concatenate([wn, s.model_nrm[:, 3:4]], 1).astype(np.float32)
    oracle.fuse(s.model_pos, s.model_nrm, s.model_col, s.model_t, wp4, wn4, s.tgt_depth, nm, s.tgt_color, s.intr,
                oracle.FuseParams(frame=1), s.N + cfg.W * cfg.H)
    return time.perf_counter() - t0


def oracle_frames(s, budget_s, max_frames, keypoints=0, weights="gaussian", lm=None):
    """Whole frames of the workload in the oracle (as many as fit the budget,
    at least one, at most max_frames); GN iters/s from the median frame."""
    import oracle
    radius = None if s.nodes is not None else oracle.calibrate_radius(s.model_pos, s.cfg.node_count)
    times = []
    t_start = time.perf_counter()
    while not times or (time.perf_counter() - t_start < budget_s and len(times) < max_frames):
        times.append(oracle_frame(s, radius, keypoints, weights, lm=lm))
    return times


def cpu_baseline(s, budget_s, keypoints=0, weights="gaussian", lm=None, config=WORKLOAD):
    """The oracle as it stands (single-threaded), and beside it the OpenMP
    build of the same source over every host core (os.cpu_count()), each on
    whole frames of the same workload, the figure from the median frame."""
    times = oracle_frames(s, budget_s, 3, keypoints, weights, lm)
    med = statistics.median(times)
    out = {"value": s.cfg.n_gn / med, "unit": "GN iters/s", "cores": 1, "kind": "oracle",
           "sample": f"{len(times)} whole frame(s) of the same workload (normals, graph, {s.cfg.n_gn} GN x "
                     f"{s.cfg.n_pcg} PCG, warp, fuse) in the single-threaded FP64 oracle, median of "
                     f"{len(times)} frames ({sum(times):.1f} s)"}
    out["openmp"] = cpu_baseline_openmp(config, budget_s, keypoints, weights, lm)
    return out


def cpu_baseline_openmp(config, budget_s, keypoints, weights, lm):
    """The OpenMP build of the oracle (liboracle_omp.so, chosen by the
    library loader of a fresh process: a child that never touches CUDA) on
    os.cpu_count() threads, median of up to 5 whole frames."""
    cores = os.cpu_count() or 1
    spec = json.dumps({"config": config, "budget_s": budget_s, "keypoints": keypoints, "weights": weights, "lm": lm})
    env = dict(os.environ, ED_ORACLE_OPENMP="1", OMP_NUM_THREADS=str(cores), OMP_PROC_BIND="false",
               CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg", spec], env=env,
                           capture_output=True, text=True, timeout=max(120.0, 6 * budget_s))
        times = json.loads(r.stdout.strip().splitlines()[-1])["times"]
    except Exception as e:   # reported, not fatal: the GPU figures stand without it
        return {"value": None, "cores": cores, "kind": "oracle (OpenMP build)", "error": str(e)[:200]}
    med = statistics.median(times)
    s_cfg = _scene_cfg(config)
    return {"value": s_cfg.n_gn / med, "unit": "GN iters/s", "cores": cores, "kind": "oracle (OpenMP build)",
            "sample": f"{len(times)} whole frame(s) of the same workload in the OpenMP build of the FP64 oracle on "
                      f"{cores} threads, median of {len(times)} frames ({sum(times):.1f} s)"}


def _scene_cfg(config):
    import synth
    return synth.CONFIGS[config] if config in synth.CONFIGS else synth.make_scene(config, seed=1).cfg


def oracle_leg_main(spec):
    """--oracle-leg: whole oracle frames only (no GPU), times as JSON."""
    import synth
    d = json.loads(spec)
    s = synth.make_scene(d["config"], seed=1)
    times = oracle_frames(s, d["budget_s"], 5, d["keypoints"], d["weights"], d["lm"])
    print(json.dumps({"times": times}))


def run_reference_sequence(args, world):
    import synth
    import oracle
    S = synth.make_push_sequence(SEQ_WORKLOAD, args.warmup + args.steps, seed=1)
    cfg = S.cfg
    radius = oracle.calibrate_radius(S.model_pos, cfg.node_count)
    model = (S.model_pos, S.model_nrm, S.model_col, S.model_t)
    times, errs = [], []
    for k, f in enumerate(S.frames):
        t0 = time.perf_counter()
        model, info = oracle.track_frame(model, f.depth, f.color, S.intr, radius, cfg.node_count, SEQ_BOX_MM, cfg.n_gn,
                                         cfg.n_pcg, f.index, cfg.normal_half_width, truth_depth=f.depth_clean)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
            errs.append(info["error_mean_mm"])
    tot = sum(times)
    value = args.steps * cfg.n_gn / tot
    return {"metric": METRIC, "value": value, "unit": "GN iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": SEQ_WORKLOAD, "width": cfg.W, "height": cfg.H, "frames_timed": args.steps,
                       "nodes": cfg.node_count, "box_mm": SEQ_BOX_MM},
            "accuracy": {"metric": "back-projection error vs the noise-free depth (Sec. III)", "unit": "mm",
                         "mean": float(np.mean(errs))},
            "cpu_baseline": {"value": value, "unit": "GN iters/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} frames of the push sequence, single-threaded FP64 oracle"},
            "e2e": {"value": value, "unit": "GN iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference(args, rank, world):
    import synth
    import oracle
    if rank != 0:
        return None
    if args.workload == "push_sequence":
        return run_reference_sequence(args, world)
    s = synth.make_scene(args.config, seed=1)
    radius = None if s.nodes is not None else oracle.calibrate_radius(s.model_pos, s.cfg.node_count)
    for _ in range(args.warmup):
        oracle_frame(s, radius, args.keypoints, args.weights, lm=args.lm)
    times = [oracle_frame(s, radius, args.keypoints, args.weights, lm=args.lm)
             for _ in range(args.steps)]
    tot = sum(times)
    value = args.steps * s.cfg.n_gn / tot
    return {"metric": metric_for(s.cfg.W, s.cfg.H, s.cfg.node_count), "value": value, "unit": "GN iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.config, "width": s.cfg.W, "height": s.cfg.H, "model_points": s.N,
                       "nodes": s.cfg.node_count, "keypoints": getattr(args, "keypoints", 0),
                       "weights": getattr(args, "weights", "gaussian"),
                       "solver": "gauss-newton" if args.lm is None else f"levenberg-marquardt, lambda0 = {args.lm:g}"},
            "cpu_baseline": {"value": value, "unit": "GN iters/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} whole frames, single-threaded FP64 oracle"},
            "e2e": {"value": value, "unit": "GN iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.oracle_leg is not None:
        oracle_leg_main(args.oracle_leg)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if args.workload == "batch16":
        out = run_batch(args, rank, world, local)
        if rank == 0:
            print(json.dumps(out))
        return
    if args.workload == "grad":
        out = run_grad(args, rank, world, local)
        if rank == 0:
            print(json.dumps(out))
        return
    if args.workload == "push_sequence":
        out, S, radius = run_sequence(args, rank, world, local)
        if rank == 0:
            out["cpu_baseline"] = (sequence_cpu_baseline(S, radius, args.cpu_budget_s)
                                   if world == 1 and not args.no_cpu_baseline else None)
            print(json.dumps(out))
        return
    out, s = run_ours(args, rank, world, local)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(s, args.cpu_budget_s, args.keypoints, args.weights, args.lm,
                                               config=args.config)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))


if __name__ == "__main__":
    main()
