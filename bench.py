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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=20.0)
    ap.add_argument("--radius", type=float, default=0.0,
                    help="Poisson radius (mm); 0 = calibrate to the workload's node count")
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


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def pcg_bytes_per_launch(m, nnzb, n_pcg):
    """Algorithmic bytes of one PCG launch: per iteration the 12x12 blocks,
    pose-node blocks, block inverses and 11 vector passes of 12m+6 floats; plus
    the set-up pass (inverses and 4 vector passes)."""
    P = 12 * m + 6
    per_iter = nnzb * 576 + m * 288 + m * 576 + 11 * P * 4
    return n_pcg * per_iter + m * 576 + 4 * P * 4


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
    ctx = E.Context(max_points=cap_pts, max_nodes=max(cfg.node_count, 64), max_width=W, max_height=H,
                    max_cells=1 << 24)
    pos = torch.from_numpy(s.model_pos).to(dev)
    nrm = torch.from_numpy(s.model_nrm).to(dev)
    col = torch.from_numpy(s.model_col).to(dev)
    tst = torch.from_numpy(s.model_t).to(dev)
    depth = torch.from_numpy(s.tgt_depth).to(dev)
    color = torch.from_numpy(np.ascontiguousarray(s.tgt_color)).to(dev)
    nmap = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
    frame = E.make_frame(depth, nmap, s.intr, color)
    radius = args.radius if args.radius > 0 else E.calibrate_radius(ctx, pos, nrm, cfg.node_count)
    prm = E.SolverParams(n_pcg=cfg.n_pcg, prior=tuple(float(v) for v in s.pose_prior),
                         precision=E.ED_PRECISION_MIXED if args.precision == "mixed" else E.ED_PRECISION_FP32)
    F = E.FuseParams(frame=1)
    x = torch.empty((cfg.node_count, 12), dtype=torch.float32, device=dev)
    xm = torch.empty((cfg.node_count, 12), dtype=torch.float64, device=dev)
    pose = torch.empty(6, dtype=torch.float64, device=dev)
    prior = torch.tensor(s.pose_prior, dtype=torch.float64, device=dev)
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

    def step(record_gn=False):
        ctx.compute_normals(depth, s.intr, cfg.normal_half_width, out=nmap)
        g = ctx.build_graph(pos, nrm, node_radius=radius, max_nodes=cfg.node_count, sigma=radius)
        m = g.m
        x[:m].zero_()
        x[:m, 0] = 1.0
        x[:m, 5] = 1.0
        x[:m, 10] = 1.0
        xm[:m].copy_(x[:m])
        pose.copy_(prior)
        if record_gn:
            e0 = torch.cuda.Event(enable_timing=True)
            e0.record()
        for it in range(cfg.n_gn):
            ctx.gn_step(frame, prm, x[:m], pose, x_master=xm[:m], stats=stats[it:it + 1])
        if record_gn:
            e1 = torch.cuda.Event(enable_timing=True)
            e1.record()
            gn_ev.append((e0, e1))
        ctx.warp(x[:m], pose, pos, nrm, wpos, wnrm)
        ctx.fuse(pos, nrm, col, tst, wpos, wnrm, frame, F, cap_pts, out=fout)
        return g

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g = ctx.graph
    st_last = E.read_stats(stats)

    # timed region
    K = args.steps
    n_events = K * cfg.n_gn
    tm_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n_events)]
    ctx.set_timing(E.ED_KERNEL_PCG, tm_ev)
    clocks = ClockSampler(local)
    clocks.start()
    l0 = E.launch_count()
    step_ms = []
    barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_(k & 0xff)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        step(record_gn=True)
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
    gn_ms = [a.elapsed_time(b) for a, b in gn_ev[-K:]]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    value = whole_job_rate(world, K, cfg.n_gn, total_s)

    # end to end through the public API with host buffers
    h_depth = torch.from_numpy(s.tgt_depth).pin_memory()
    h_color = torch.from_numpy(np.ascontiguousarray(s.tgt_color)).pin_memory()
    h_x = torch.empty((cfg.node_count, 12), dtype=torch.float32).pin_memory()
    h_stats = torch.empty(stats.shape, dtype=torch.uint8).pin_memory()
    h2d = h_depth.numel() * 4 + h_color.numel() * 4
    d2h = h_x.numel() * 4 + h_stats.numel()
    e2e_ms = []
    barrier()
    torch.cuda.synchronize()
    for k in range(K):
        flush.fill_(k & 0xff)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        depth.copy_(h_depth, non_blocking=True)
        color.copy_(h_color, non_blocking=True)
        gg = step()
        h_x[:gg.m].copy_(x[:gg.m], non_blocking=True)
        h_stats.copy_(stats, non_blocking=True)
        ev1.record()
        ev1.synchronize()
        e2e_ms.append(ev0.elapsed_time(ev1))
    e2e_s = max_over_ranks(sum(e2e_ms) / 1e3, dist, dev)
    e2e_value = whole_job_rate(world, K, cfg.n_gn, e2e_s)

    peak, peak_kind = measured_peaks()
    byt = pcg_bytes_per_launch(g.m, g.nnzb, cfg.n_pcg)
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
        "metric": METRIC, "value": value, "unit": "GN iters/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_s * 1e3 / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f32+f64",
        "data": "synthetic (seeded stereo-scope tissue scene, no dataset)",
        "config": {"workload": args.config, "width": W, "height": H, "model_points": s.N, "nodes": g.m,
                   "nnz_blocks": g.nnzb, "gn_iters_per_step": cfg.n_gn, "pcg_iters": cfg.n_pcg,
                   "node_radius_mm": radius, "precision": args.precision,
                   "l2": "flushed between steps (512 MB write)",
                   "step": "normals + build_graph + 10 x gn_step + warp + fuse"},
        "gn_only_iters_per_s": whole_job_rate(world, K, cfg.n_gn, max_over_ranks(sum(gn_ms) / 1e3, dist, dev))
        if gn_ms else None,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": "GN iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": {"kernel": "k_pcg (persistent block-Jacobi PCG)", "bound": "hbm", "achieved": achieved,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "algorithmic_bytes_per_launch": byt,
                     "avg_launch_us": avg_pcg_s * 1e6, "launches_timed": len(pcg_ms)},
        "final_stats": {k: st_last[-1][k] for k in ("energy", "n_valid", "pcg_iters", "status")},
    }
    return out, s


def kernel_rev():
    """Content hash of the CUDA sources (ties an ncu traffic figure to a build)."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1803_02009_b300", "csrc")
    for fn in sorted(os.listdir(d)):
        with open(os.path.join(d, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ----------------------------------------------------------------------------
# oracle (CPU) leg
# ----------------------------------------------------------------------------

def oracle_frame(s, radius):
    """One frame of the whole path in the FP64 oracle; returns seconds."""
    import oracle
    cfg = s.cfg
    t0 = time.perf_counter()
    nm = oracle.normals(s.tgt_depth, s.intr, cfg.normal_half_width)
    G = oracle.build_graph(s.model_pos, radius=radius, max_nodes=cfg.node_count, K=4, KG=4, mode=0, sigma=radius)
    P = oracle.Problem(s.model_pos, s.model_nrm, G, s.tgt_depth, nm, s.intr, s.pose_prior)
    x, pose, hist, st = oracle.gn_solve(P, P.identity_x(), s.pose_prior, cfg.n_gn, cfg.n_pcg)
    wp, wn, _ = oracle.warp(P, x, pose)
    wp4 = np.concatenate([wp, s.model_pos[:, 3:4]], 1).astype(np.float32)
    wn4 = np.concatenate([wn, s.model_nrm[:, 3:4]], 1).astype(np.float32)
    oracle.fuse(s.model_pos, s.model_nrm, s.model_col, s.model_t, wp4, wn4, s.tgt_depth, nm, s.tgt_color, s.intr,
                oracle.FuseParams(frame=1), s.N + cfg.W * cfg.H)
    return time.perf_counter() - t0


def cpu_baseline(s, budget_s):
    import oracle
    radius = oracle.calibrate_radius(s.model_pos, s.cfg.node_count)
    times = []
    t_start = time.perf_counter()
    while not times or (time.perf_counter() - t_start < budget_s and len(times) < 3):
        times.append(oracle_frame(s, radius))
    tot = sum(times)
    return {"value": len(times) * s.cfg.n_gn / tot, "unit": "GN iters/s", "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} whole frame(s) of the same workload (normals, graph, {s.cfg.n_gn} GN x "
                      f"{s.cfg.n_pcg} PCG, warp, fuse) in the single-threaded FP64 oracle, {tot:.1f} s"}


def run_reference(args, rank, world):
    import synth
    import oracle
    if rank != 0:
        return None
    s = synth.make_scene(args.config, seed=1)
    radius = oracle.calibrate_radius(s.model_pos, s.cfg.node_count)
    for _ in range(args.warmup):
        oracle_frame(s, radius)
    times = [oracle_frame(s, radius) for _ in range(args.steps)]
    tot = sum(times)
    value = args.steps * s.cfg.n_gn / tot
    return {"metric": METRIC, "value": value, "unit": "GN iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.config, "width": s.cfg.W, "height": s.cfg.H, "model_points": s.N,
                       "nodes": s.cfg.node_count},
            "cpu_baseline": {"value": value, "unit": "GN iters/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} whole frames, single-threaded FP64 oracle"},
            "e2e": {"value": value, "unit": "GN iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    out, s = run_ours(args, rank, world, local)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(s, args.cpu_budget_s)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))


if __name__ == "__main__":
    main()
