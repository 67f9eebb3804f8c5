"""Frame-by-frame registration and model maintenance (Sec. II.G, Algorithm 2
with Algorithm 3).

Per frame: the target normal map, node regeneration on the current model
(Alg. 2 step 5), Gauss-Newton steps of Eq. (3) from the identity warp, the
final warp of every model point, fusion with the new depth (registration,
Eqs. fusion1-4, lifting of unregistered pixels, deletion of unstable points)
and box downsampling (Sec. III.A).  The fused model lives in the camera
frame of the frame just fused, so the next frame's warp again starts from
the identity and its nodes are sampled afresh.  Every step runs in the
library's kernels; this class holds the buffers and the call order only.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import torch

from . import (Context, FuseParams, SolverParams, make_frame, new_stats, read_stats, ED_WEIGHT_GAUSSIAN)


@dataclasses.dataclass
class TrackerConfig:
    node_radius: float                 # Poisson-disk radius of the regenerated nodes (mm)
    max_nodes: int                     # nodes kept per frame (selection order)
    box: float                         # downsampling box edge (mm)
    n_gn: int = 10                     # Gauss-Newton steps per frame
    normal_half_width: int = 16        # target normal stencil half width (pixels)
    sigma: Optional[float] = None      # skinning width (default: the node radius)
    solver: SolverParams = dataclasses.field(default_factory=SolverParams)
    fuse: FuseParams = dataclasses.field(default_factory=FuseParams)


class Tracker:
    """Holds the model (pos with omega in w, nrm with the stability flag in w,
    colour, time stamps) in two device buffers of `capacity` points and
    processes one frame per call of `process`."""

    def __init__(self, pos, nrm, col, tstamp, intr, cfg: TrackerConfig, capacity: int, ctx: Context = None):
        fx, fy, cx, cy, W, H = intr
        self.intr = intr
        self.cfg = cfg
        self.capacity = int(capacity)
        n = int(pos.shape[0])
        if n + W * H > self.capacity:
            raise ValueError("capacity must hold the model plus one frame of lifted pixels")
        self.ctx = ctx if ctx is not None else Context(max_points=self.capacity, max_nodes=cfg.max_nodes,
                                                       max_width=W, max_height=H, max_cells=1 << 24)
        dev = "cuda"

        def model():
            return dict(pos=torch.zeros((self.capacity, 4), dtype=torch.float32, device=dev),
                        nrm=torch.zeros((self.capacity, 4), dtype=torch.float32, device=dev),
                        col=torch.zeros((self.capacity, 4), dtype=torch.float32, device=dev),
                        t=torch.zeros(self.capacity, dtype=torch.int32, device=dev),
                        counts=torch.zeros(2, dtype=torch.int32, device=dev))
        self.A, self.B = model(), model()
        self.A["pos"][:n].copy_(pos)
        self.A["nrm"][:n].copy_(nrm)
        self.A["col"][:n].copy_(col)
        self.A["t"][:n].copy_(tstamp)
        self.n = n
        self.nmap = torch.empty((H, W, 4), dtype=torch.float32, device=dev)
        self.wpos = torch.empty((self.capacity, 4), dtype=torch.float32, device=dev)
        self.wnrm = torch.empty_like(self.wpos)
        self.x = torch.empty((cfg.max_nodes, 12), dtype=torch.float32, device=dev)
        self.xm = torch.empty((cfg.max_nodes, 12), dtype=torch.float64, device=dev)
        self.pose = torch.zeros(6, dtype=torch.float64, device=dev)
        self.stats = new_stats(cfg.n_gn)
        self.err = torch.zeros(4, dtype=torch.float64, device=dev)

    def process(self, depth, color, frame_index: int, truth_depth=None):
        """One frame: register the model to `depth` (float32 [H, W] mm), fuse
        and downsample.  Returns the Gauss-Newton statistics of the last step,
        the model size and the back-projection error of the registered model
        against `truth_depth` (default: the observation) in mm."""
        c, ctx, n = self.cfg, self.ctx, self.n
        ctx.compute_normals(depth, self.intr, c.normal_half_width, out=self.nmap)
        frame = make_frame(depth, self.nmap, self.intr, color)
        pos, nrm = self.A["pos"][:n], self.A["nrm"][:n]
        sigma = c.sigma if c.sigma is not None else c.node_radius
        g = ctx.build_graph(pos, nrm, node_radius=c.node_radius, max_nodes=c.max_nodes, sigma=sigma,
                            weight_mode=ED_WEIGHT_GAUSSIAN, reuse=True)
        m = g.m
        x, xm = self.x[:m], self.xm[:m]
        ctx.reset_params(x, self.pose, x_master=xm, prior=c.solver.prior)
        if c.solver.lm_accept:
            ctx.lm_reset(c.solver.lam)
        prm = c.solver.c()
        for it in range(c.n_gn):
            ctx.gn_step(frame, prm, x, self.pose, x_master=xm, stats=self.stats[it:it + 1])
        wpos, wnrm = self.wpos[:n], self.wnrm[:n]
        ctx.warp(x, self.pose, pos, nrm, wpos, wnrm)
        ctx.depth_error(wpos, truth_depth if truth_depth is not None else depth, self.intr, out=self.err)
        fp = dataclasses.replace(c.fuse, frame=int(frame_index))
        ctx.fuse(pos, nrm, self.A["col"][:n], self.A["t"][:n], wpos, wnrm, frame, fp, self.capacity, out=self.B)
        nf = int(self.B["counts"][0].item())
        ctx.downsample(self.B["pos"][:nf], self.B["nrm"][:nf], self.B["col"][:nf], self.B["t"][:nf], c.box,
                       omega_max=c.fuse.omega_max, tau_weight=c.fuse.tau_weight, capacity=self.capacity, out=self.A)
        cnt = self.A["counts"].cpu()
        self.n = int(cnt[0])
        st = read_stats(self.stats[c.n_gn - 1:c.n_gn])[0]
        e = self.err.cpu().tolist()
        return dict(frame=int(frame_index), nodes=m, fused=nf, model=self.n, status=int(cnt[1]), gn=st,
                    error_mean_mm=e[0] / e[1] if e[1] else 0.0, error_max_mm=e[2],
                    error_rms_mm=(e[3] / e[1]) ** 0.5 if e[1] else 0.0, error_pixels=int(e[1]))

    def model(self):
        """The current model (views of the first n points)."""
        n = self.n
        return {k: self.A[k][:n] for k in ("pos", "nrm", "col", "t")}
