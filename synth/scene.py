"""Seeded synthetic stereo-scope scenes for the ED registration hot path.

This module only *renders inputs*: a smooth tissue height field seen by a
pinhole camera, a deformed and rigidly moved copy of it, depth noise, holes,
colours and the ED node grid of the small workload.  It contains none of the
registration method's arithmetic (no warp, association, residual, Jacobian,
solver or fusion step); both the CUDA path and the FP64 oracle consume the
arrays it returns.

Scene recipe (the paper's data is in vivo stereo video at 640x480, 40-70 mm
from the tissue, Sec. III; none of it is used here):

* tissue surface in the source camera frame, millimetres:
  z = h(x, y) = 60 + 4 sin(x/12) cos(y/15);
* target surface: h'(x, y) = h(x, y) + sum of Gaussian bumps
  a exp(-((x-xc)^2 + (y-yc)^2) / (2 s^2)), then a rigid motion
  M(p) = R_M (p - c) + c + t_M with c = (0, 0, 60);
* depth maps by FP64 ray casting of every pixel ray
  r = ((u - cx)/fx, (v - cy)/fy, 1) (Newton on the ray parameter), plus
  N(0, sigma_noise) depth noise and Bernoulli(p_hole) holes (depth 0);
* model points: the valid source pixels placed at their noisy depth along
  their ray, with the analytic (noise-free) surface normal, oriented to the
  camera (n_z < 0);
* the rigid motion is drawn as a small Euler-angle vector of the given
  magnitude (R_M = Rz(gamma) Ry(beta) Rx(alpha)) plus a translation of the
  given length; the pose prior handed to the solver is that motion plus small
  seeded noise, standing in for the ORB-SLAM pose of Sec. II.C.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

# ----------------------------------------------------------------------------
# workload presets (sizes follow the stereo-scope scope of Sec. III)
# ----------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class SceneConfig:
    name: str
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    n_bumps: int
    bump_amp: Tuple[float, float]        # mm, uniform range
    bump_width: Tuple[float, float]      # mm, uniform range
    rot_deg: float = 2.0                 # rigid offset magnitude
    trans_mm: float = 3.0
    noise_mm: float = 0.2
    p_hole: float = 0.02
    node_mode: str = "poisson"           # "grid8" or "poisson"
    node_count: int = 2048
    k: int = 4
    kg: int = 4
    n_gn: int = 10
    n_pcg: int = 20
    normal_half_width: int = 16          # target-normal stencil half width (pixels)
    model_weight: float = 5.0            # fusion weight of the existing model points
    prior_noise_rad: float = 0.002
    prior_noise_mm: float = 0.1


CONFIGS = {
    # 160x120, 64 nodes on an 8x8 grid, one bump: the small workload
    "tissue_160x120_n64": SceneConfig(
        name="tissue_160x120_n64", W=160, H=120, fx=131.25, fy=131.25, cx=80.0, cy=60.0,
        n_bumps=1, bump_amp=(2.0, 2.0), bump_width=(10.0, 10.0), node_mode="grid8",
        node_count=64, n_gn=5, n_pcg=10, normal_half_width=4),
    # 640x480, 2048 Poisson-disk nodes, eight bumps: the metric workload
    "tissue_640x480_n2048": SceneConfig(
        name="tissue_640x480_n2048", W=640, H=480, fx=525.0, fy=525.0, cx=320.0, cy=240.0,
        n_bumps=8, bump_amp=(1.0, 3.0), bump_width=(5.0, 15.0), node_mode="poisson",
        node_count=2048, n_gn=10, n_pcg=20, normal_half_width=16),
    # 1280x720, 4096 Poisson-disk nodes: the large mixed-precision workload
    "tissue_1280x720_n4096": SceneConfig(
        name="tissue_1280x720_n4096", W=1280, H=720, fx=1050.0, fy=1050.0, cx=640.0, cy=360.0,
        n_bumps=8, bump_amp=(1.0, 3.0), bump_width=(5.0, 15.0), node_mode="poisson",
        node_count=4096, n_gn=10, n_pcg=20, normal_half_width=32),
    # push sequences (static camera, one 2-3 mm push per frame): 160x120 for the
    # oracle's lock-step tests, 640x480 / 2048 nodes for the benchmark
    "push_160x120": SceneConfig(
        name="push_160x120", W=160, H=120, fx=131.25, fy=131.25, cx=80.0, cy=60.0,
        n_bumps=0, bump_amp=(0.0, 0.0), bump_width=(10.0, 10.0), rot_deg=0.0, trans_mm=0.0,
        node_mode="poisson", node_count=128, n_gn=5, n_pcg=10, normal_half_width=4),
    "push_640x480_n2048": SceneConfig(
        name="push_640x480_n2048", W=640, H=480, fx=525.0, fy=525.0, cx=320.0, cy=240.0,
        n_bumps=0, bump_amp=(0.0, 0.0), bump_width=(10.0, 10.0), rot_deg=0.0, trans_mm=0.0,
        node_mode="poisson", node_count=2048, n_gn=10, n_pcg=20, normal_half_width=16),
    # 320x240 member size of the batched workload
    "tissue_320x240": SceneConfig(
        name="tissue_320x240", W=320, H=240, fx=262.5, fy=262.5, cx=160.0, cy=120.0,
        n_bumps=1, bump_amp=(2.0, 2.0), bump_width=(10.0, 10.0), node_mode="poisson",
        node_count=1024, n_gn=5, n_pcg=10, normal_half_width=8),
}

Z0 = 60.0
CENTER = np.array([0.0, 0.0, Z0])


# ----------------------------------------------------------------------------
# surface
# ----------------------------------------------------------------------------


def h_base(x, y):
    return Z0 + 4.0 * np.sin(x / 12.0) * np.cos(y / 15.0)


def h_base_grad(x, y):
    hx = (4.0 / 12.0) * np.cos(x / 12.0) * np.cos(y / 15.0)
    hy = -(4.0 / 15.0) * np.sin(x / 12.0) * np.sin(y / 15.0)
    return hx, hy


@dataclasses.dataclass
class Bumps:
    amp: np.ndarray
    xc: np.ndarray
    yc: np.ndarray
    s: np.ndarray

    def value(self, x, y):
        out = np.zeros(np.broadcast(x, y).shape)
        for a, xc, yc, s in zip(self.amp, self.xc, self.yc, self.s):
            out = out + a * np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (2.0 * s * s))
        return out

    def grad(self, x, y):
        gx = np.zeros(np.broadcast(x, y).shape)
        gy = np.zeros_like(gx)
        for a, xc, yc, s in zip(self.amp, self.xc, self.yc, self.s):
            e = a * np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (2.0 * s * s))
            gx = gx - e * (x - xc) / (s * s)
            gy = gy - e * (y - yc) / (s * s)
        return gx, gy


def euler_matrix(alpha, beta, gamma):
    """Rz(gamma) Ry(beta) Rx(alpha): builds the synthetic rigid motion."""
    ca, sa = math.cos(alpha), math.sin(alpha)
    cb, sb = math.cos(beta), math.sin(beta)
    cg, sg = math.cos(gamma), math.sin(gamma)
    rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
    ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    rz = np.array([[cg, -sg, 0], [sg, cg, 0], [0, 0, 1]])
    return rz @ ry @ rx


def _rays(cfg: SceneConfig):
    u = np.arange(cfg.W, dtype=np.float64)
    v = np.arange(cfg.H, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    a = (uu - cfg.cx) / cfg.fx
    b = (vv - cfg.cy) / cfg.fy
    return a, b


def raycast(cfg: SceneConfig, bumps: Optional[Bumps], R: np.ndarray, t: np.ndarray):
    """FP64 ray cast of every pixel ray against M(graph of h + bumps).

    Returns (depth t, surface-frame hit coordinates qx, qy) per pixel.
    """
    a, b = _rays(cfg)
    Rt = R.T
    # q(t) = M^-1(t r) = R^T (t r - c - t_M) + c ; dq/dt = R^T r
    dqx = Rt[0, 0] * a + Rt[0, 1] * b + Rt[0, 2]
    dqy = Rt[1, 0] * a + Rt[1, 1] * b + Rt[1, 2]
    dqz = Rt[2, 0] * a + Rt[2, 1] * b + Rt[2, 2]
    off = Rt @ (-CENTER - t) + CENTER
    tt = np.full(a.shape, Z0)
    for _ in range(60):
        qx = tt * dqx + off[0]
        qy = tt * dqy + off[1]
        qz = tt * dqz + off[2]
        hv = h_base(qx, qy)
        gx, gy = h_base_grad(qx, qy)
        if bumps is not None:
            hv = hv + bumps.value(qx, qy)
            bx, by = bumps.grad(qx, qy)
            gx, gy = gx + bx, gy + by
        f = qz - hv
        fp = dqz - gx * dqx - gy * dqy
        step = f / fp
        tt = np.clip(tt - step, 30.0, 100.0)
        if np.max(np.abs(step)) < 1e-12:
            break
    qx = tt * dqx + off[0]
    qy = tt * dqy + off[1]
    return tt, qx, qy


def texture(qx, qy):
    r = 0.5 + 0.5 * np.sin(qx / 3.0)
    g = 0.5 + 0.5 * np.cos(qy / 4.0)
    b = 0.5 + 0.5 * np.sin((qx + qy) / 5.0)
    return np.stack([r, g, b, np.ones_like(r)], axis=-1)


@dataclasses.dataclass
class Scene:
    cfg: SceneConfig
    seed: int
    intr: Tuple[float, float, float, float, int, int]      # fx, fy, cx, cy, W, H
    src_depth: np.ndarray      # float32 [H, W] (0 = hole)
    tgt_depth: np.ndarray      # float32 [H, W]
    tgt_color: np.ndarray      # float32 [H, W, 4]
    model_pos: np.ndarray      # float32 [N, 4]  xyz mm, w = fusion weight
    model_nrm: np.ndarray      # float32 [N, 4]  xyz unit normal, w = stability flag
    model_col: np.ndarray      # float32 [N, 4]
    model_t: np.ndarray        # int32 [N] time stamps
    model_pix: np.ndarray      # int32 [N] source pixel of each model point
    nodes: Optional[np.ndarray]  # float32 [m, 4] for grid nodes, else None
    sigma: Optional[float]     # skinning width for grid nodes
    pose_true: np.ndarray      # float64 [6] (alpha, beta, gamma, Tx, Ty, Tz)
    pose_prior: np.ndarray     # float64 [6]
    bumps: Bumps
    R_true: np.ndarray
    T_true: np.ndarray
    model_q: np.ndarray        # float64 [N, 2] noise-free surface coordinates

    @property
    def N(self):
        return int(self.model_pos.shape[0])

    def gt_positions(self):
        """Ground-truth target positions of the model points (noise-free)."""
        qx, qy = self.model_q[:, 0], self.model_q[:, 1]
        z = h_base(qx, qy) + self.bumps.value(qx, qy)
        p = np.stack([qx, qy, z], axis=1)
        return p @ self.R_true.T + self.T_true


def make_scene(cfg: SceneConfig | str, seed: int = 1) -> Scene:
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    ss = np.random.SeedSequence([seed, cfg.W, cfg.H])
    rng_bump, rng_rigid, rng_noise, rng_hole, rng_prior = [np.random.default_rng(s) for s in ss.spawn(5)]

    ext_x = (0.0 - cfg.cx) / cfg.fx * Z0, (cfg.W - cfg.cx) / cfg.fx * Z0
    ext_y = (0.0 - cfg.cy) / cfg.fy * Z0, (cfg.H - cfg.cy) / cfg.fy * Z0

    # deformation: bumps with centres in the central 60% of the extent
    nb = cfg.n_bumps
    amp = rng_bump.uniform(cfg.bump_amp[0], cfg.bump_amp[1], nb)
    wid = rng_bump.uniform(cfg.bump_width[0], cfg.bump_width[1], nb)
    cxs = rng_bump.uniform(0.2, 0.8, nb) * (ext_x[1] - ext_x[0]) + ext_x[0]
    cys = rng_bump.uniform(0.2, 0.8, nb) * (ext_y[1] - ext_y[0]) + ext_y[0]
    bumps = Bumps(amp, cxs, cys, wid)

    # rigid offset drawn as Euler angles of the stated magnitude
    d = rng_rigid.normal(size=3)
    d /= np.linalg.norm(d)
    ang = d * math.radians(cfg.rot_deg)
    R = euler_matrix(*ang)
    tv = rng_rigid.normal(size=3)
    tv = tv / np.linalg.norm(tv) * cfg.trans_mm
    T = CENTER + tv - R @ CENTER
    pose_true = np.concatenate([ang, T])
    prior = pose_true + np.concatenate([rng_prior.normal(0, cfg.prior_noise_rad, 3),
                                        rng_prior.normal(0, cfg.prior_noise_mm, 3)])

    # source (undeformed, identity) and target depth maps
    I3 = np.eye(3)
    z_src, qx_s, qy_s = raycast(cfg, None, I3, np.zeros(3))
    z_tgt, qx_t, qy_t = raycast(cfg, bumps, R, tv)

    src = z_src + rng_noise.normal(0.0, cfg.noise_mm, z_src.shape)
    tgt = z_tgt + rng_noise.normal(0.0, cfg.noise_mm, z_tgt.shape)
    src[rng_hole.random(src.shape) < cfg.p_hole] = 0.0
    tgt[rng_hole.random(tgt.shape) < cfg.p_hole] = 0.0
    src32 = src.astype(np.float32)
    tgt32 = tgt.astype(np.float32)
    tcol = texture(qx_t, qy_t).astype(np.float32)

    # model = valid source pixels at their noisy depth along their ray
    a, b = _rays(cfg)
    valid = src32 > 0
    pix = np.nonzero(valid.reshape(-1))[0].astype(np.int32)
    dval = src32.reshape(-1)[pix].astype(np.float64)
    ar, br = a.reshape(-1)[pix], b.reshape(-1)[pix]
    pos = np.stack([ar * dval, br * dval, dval, np.full_like(dval, cfg.model_weight)], axis=1)
    qx, qy = qx_s.reshape(-1)[pix], qy_s.reshape(-1)[pix]
    gx, gy = h_base_grad(qx, qy)
    nrm = np.stack([gx, gy, -np.ones_like(gx)], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    nrm4 = np.concatenate([nrm, np.ones((nrm.shape[0], 1))], axis=1)
    col = texture(qx, qy)

    nodes = None
    sigma = None
    if cfg.node_mode == "grid8":
        sx = (ext_x[1] - ext_x[0]) / 8.0
        sy = (ext_y[1] - ext_y[0]) / 8.0
        gxs = ext_x[0] + (np.arange(8) + 0.5) * sx
        gys = ext_y[0] + (np.arange(8) + 0.5) * sy
        GX, GY = np.meshgrid(gxs, gys)
        GZ = h_base(GX, GY)
        nodes = np.stack([GX.ravel(), GY.ravel(), GZ.ravel(), np.zeros(64)], axis=1).astype(np.float32)
        sigma = float((ext_x[1] - ext_x[0] + ext_y[1] - ext_y[0]) / 16.0)

    return Scene(cfg=cfg, seed=seed, intr=(cfg.fx, cfg.fy, cfg.cx, cfg.cy, cfg.W, cfg.H),
                 src_depth=src32, tgt_depth=tgt32, tgt_color=tcol,
                 model_pos=pos.astype(np.float32), model_nrm=nrm4.astype(np.float32),
                 model_col=col.astype(np.float32), model_t=np.zeros(pix.shape[0], np.int32),
                 model_pix=pix, nodes=nodes, sigma=sigma, pose_true=pose_true, pose_prior=prior,
                 bumps=bumps, R_true=R, T_true=T, model_q=np.stack([qx, qy], axis=1))


def batch_scenes(count: int = 16, seed0: int = 1) -> List[Tuple[Scene, int]]:
    """Member problems of the batched workload: sizes drawn from 320x240,
    640x480 and 1280x720, node counts uniform in 200..4096, one bump each.
    Returns (scene, node_count) pairs."""
    rng = np.random.default_rng(seed0 + 1000)
    out = []
    sizes = ["tissue_320x240", "tissue_640x480_n2048", "tissue_1280x720_n4096"]
    for i in range(count):
        base = CONFIGS[sizes[int(rng.integers(0, 3))]]
        m = int(rng.integers(200, 4097))
        cfg = dataclasses.replace(base, name=f"{base.name}_b{i}", n_bumps=1,
                                  bump_amp=(2.0, 2.0), bump_width=(10.0, 10.0),
                                  node_count=m, n_gn=5, n_pcg=10)
        out.append((make_scene(cfg, seed=seed0 + i), m))
    return out


def make_keypoints(scene: Scene, count: int = 500, seed: int = 1, noise_mm: float = 0.2):
    """Synthetic sparse key correspondences standing in for matched ORB
    features: `count` seeded model points (float4, model frame) and their
    ground-truth positions in the new frame plus N(0, noise_mm) localisation
    noise (float4, w = 1).  Returns (kp_pos [count][4], kp_target [count][4],
    indices into the model)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7, count]))
    sel = np.sort(rng.choice(scene.N, size=min(count, scene.N), replace=False))
    kp = scene.model_pos[sel].astype(np.float32).copy()
    kp[:, 3] = 0.0
    tgt = scene.gt_positions()[sel] + rng.normal(0.0, noise_mm, (len(sel), 3))
    tgt4 = np.concatenate([tgt, np.ones((len(sel), 1))], axis=1).astype(np.float32)
    return kp, tgt4, sel


# ----------------------------------------------------------------------------
# push sequence (a synthetic analogue of the simulation experiment, Sec. III.D)
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class PushFrame:
    index: int                 # frame number (1, 2, ...)
    depth: np.ndarray          # float32 [H, W] noisy observation, 0 = hole
    depth_clean: np.ndarray    # float32 [H, W] noise-free ray cast (ground truth)
    color: np.ndarray          # float32 [H, W, 4]
    bumps: Bumps               # cumulative deformation of the rest surface up to this frame


@dataclasses.dataclass
class PushSequence:
    cfg: SceneConfig
    seed: int
    intr: Tuple[float, float, float, float, int, int]
    model_pos: np.ndarray      # float32 [N, 4] frame-0 model, w = fusion weight
    model_nrm: np.ndarray      # float32 [N, 4] w = stability flag
    model_col: np.ndarray      # float32 [N, 4]
    model_t: np.ndarray        # int32 [N] time stamps (0)
    frames: List[PushFrame]


def make_push_sequence(cfg: SceneConfig | str, n_frames: int, seed: int = 1, push_amp=(2.0, 3.0),
                       push_width=(5.0, 15.0)) -> PushSequence:
    """A tissue surface seen by a static camera and pushed once per frame.

    Frame 0 is the rest surface h (its valid pixels, at their noisy depth,
    make the initial model, as in make_scene).  Frame k adds one push to the
    deformation of frame k-1: a Gaussian dent or bulge of amplitude
    U(push_amp) mm with a random sign, width U(push_width) mm, centred in the
    central 60% of the field of view.  Every frame is ray cast in FP64 (noise
    N(0, noise_mm) and Bernoulli(p_hole) holes on the observation; the clean
    depth is kept as ground truth)."""
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    ss = np.random.SeedSequence([seed, cfg.W, cfg.H, 77])
    rng_push, rng_noise, rng_hole = [np.random.default_rng(s) for s in ss.spawn(3)]
    ext_x = (0.0 - cfg.cx) / cfg.fx * Z0, (cfg.W - cfg.cx) / cfg.fx * Z0
    ext_y = (0.0 - cfg.cy) / cfg.fy * Z0, (cfg.H - cfg.cy) / cfg.fy * Z0
    I3, t0 = np.eye(3), np.zeros(3)

    z0, qx0, qy0 = raycast(cfg, None, I3, t0)
    src = z0 + rng_noise.normal(0.0, cfg.noise_mm, z0.shape)
    src[rng_hole.random(src.shape) < cfg.p_hole] = 0.0
    src32 = src.astype(np.float32)
    a, b = _rays(cfg)
    pix = np.nonzero(src32.reshape(-1) > 0)[0]
    dval = src32.reshape(-1)[pix].astype(np.float64)
    ar, br = a.reshape(-1)[pix], b.reshape(-1)[pix]
    pos = np.stack([ar * dval, br * dval, dval, np.full_like(dval, cfg.model_weight)], axis=1)
    qx, qy = qx0.reshape(-1)[pix], qy0.reshape(-1)[pix]
    gx, gy = h_base_grad(qx, qy)
    nrm = np.stack([gx, gy, -np.ones_like(gx)], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    nrm4 = np.concatenate([nrm, np.ones((nrm.shape[0], 1))], axis=1)
    col = texture(qx, qy)

    amp, xc, yc, wid = [], [], [], []
    frames = []
    for k in range(1, n_frames + 1):
        sgn = 1.0 if rng_push.random() < 0.5 else -1.0
        amp.append(sgn * rng_push.uniform(push_amp[0], push_amp[1]))
        wid.append(rng_push.uniform(push_width[0], push_width[1]))
        xc.append(rng_push.uniform(0.2, 0.8) * (ext_x[1] - ext_x[0]) + ext_x[0])
        yc.append(rng_push.uniform(0.2, 0.8) * (ext_y[1] - ext_y[0]) + ext_y[0])
        bumps = Bumps(np.array(amp), np.array(xc), np.array(yc), np.array(wid))
        zk, qxk, qyk = raycast(cfg, bumps, I3, t0)
        obs = zk + rng_noise.normal(0.0, cfg.noise_mm, zk.shape)
        obs[rng_hole.random(obs.shape) < cfg.p_hole] = 0.0
        frames.append(PushFrame(index=k, depth=obs.astype(np.float32), depth_clean=zk.astype(np.float32),
                                color=texture(qxk, qyk).astype(np.float32), bumps=bumps))
    return PushSequence(cfg=cfg, seed=seed, intr=(cfg.fx, cfg.fy, cfg.cx, cfg.cy, cfg.W, cfg.H),
                        model_pos=pos.astype(np.float32), model_nrm=nrm4.astype(np.float32),
                        model_col=col.astype(np.float32), model_t=np.zeros(pix.shape[0], np.int32), frames=frames)
