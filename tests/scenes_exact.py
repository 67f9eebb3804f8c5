"""Small hand-built inputs whose exact answers are known (used by the pins).

* exact_plane(): a tilted plane seen by a camera with power-of-two focal
  length, so back-projection, projection and the FP32 gates are exact and
  the model is self-registered with its own depth map.
* rigid_problem(): a noise-free tissue surface seen after a rigid motion
  M; the model is M^-1 of the back-projected target pixels, so the energy
  vanishes exactly at (x = identity, pose = M).
"""
import math

import numpy as np

from synth import scene as S


def exact_plane(W=32, H=24, f=32.0):
    cx, cy = W / 2.0, H / 2.0
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    depth = 64.0 + (u - cx) / 8.0 + (v - cy) / 16.0          # multiples of 1/16: exact in FP32
    intr = (f, f, cx, cy, W, H)
    return depth.astype(np.float32), intr


def backproject64(depth, intr):
    fx, fy, cx, cy, W, H = intr
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    D = depth.astype(np.float64)
    return np.stack([(u - cx) * D / fx, (v - cy) * D / fy, D], axis=-1)


def grid_nodes(pos3, nx, ny):
    lo = pos3.min(0)
    hi = pos3.max(0)
    xs = lo[0] + (np.arange(nx) + 0.5) * (hi[0] - lo[0]) / nx
    ys = lo[1] + (np.arange(ny) + 0.5) * (hi[1] - lo[1]) / ny
    X, Y = np.meshgrid(xs, ys)
    g = np.zeros((nx * ny, 4), np.float32)
    g[:, 0] = X.ravel()
    g[:, 1] = Y.ravel()
    # z from the nearest model point (nodes sit on the surface)
    for j in range(g.shape[0]):
        d = (pos3[:, 0] - g[j, 0]) ** 2 + (pos3[:, 1] - g[j, 1]) ** 2
        g[j, 2] = pos3[np.argmin(d), 2]
    spacing = float(((hi[0] - lo[0]) / nx + (hi[1] - lo[1]) / ny) / 2.0)
    return g, spacing


def rigid_problem(W=80, H=60, pose=(0.01, -0.015, 0.02, 1.5, -1.0, 2.0)):
    """Noise-free, hole-free height field rendered after the rigid motion
    `pose` (Euler angles + T in the solver's convention v~ = R v + T)."""
    import oracle

    f = 131.25 * W / 160.0
    cfg = S.SceneConfig(name="rigid", W=W, H=H, fx=f, fy=f, cx=W / 2.0, cy=H / 2.0, n_bumps=0,
                        bump_amp=(0, 0), bump_width=(1, 1), noise_mm=0.0, p_hole=0.0)
    R = S.euler_matrix(*pose[:3])
    T = np.asarray(pose[3:], dtype=np.float64)
    # M(p) = R p + T  ==  R (p - c) + c + t_M with t_M = T + R c - c
    tM = T + R @ S.CENTER - S.CENTER
    z, _, _ = S.raycast(cfg, None, R, tM)
    depth = z.astype(np.float32)
    intr = (f, f, W / 2.0, H / 2.0, W, H)
    nmap = oracle.normals(depth, intr, 2)
    V = backproject64(depth, intr).reshape(-1, 3)
    ok = nmap.reshape(-1, 4)[:, 3] > 0
    pix = np.nonzero(ok)[0]
    model = (V[pix] - T) @ R          # R^T (p - T)
    nrm = nmap.reshape(-1, 4)[pix, :3].astype(np.float64) @ R
    pos4 = np.concatenate([model, np.ones((len(pix), 1))], axis=1)
    nrm4 = np.concatenate([nrm, np.ones((len(pix), 1))], axis=1)
    return dict(depth=depth, nmap=nmap, intr=intr, pos=pos4, nrm=nrm4, pix=pix,
                pose=np.asarray(pose, dtype=np.float64), target=V[pix])
