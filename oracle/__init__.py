"""FP64 CPU oracle of the ED registration hot path (ctypes binding of ed_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark.  It shares no code with the CUDA path (it
never imports the package that holds it) and is never a fallback for it.

Conventions (the same ones the C file documents):
* node parameters x[j] = the 3x4 affine [A_j | t_j] row-major (12 values);
* pose = (alpha, beta, gamma, Tx, Ty, Tz), R = Rz(gamma) Ry(beta) Rx(alpha);
* unknown vector = 12 m node parameters followed by the 6 pose parameters;
* association pix[i] = v*W + u, or -1 when the point fails the gate.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
from typing import Optional

import numpy as np

from . import build as _build

_lib = None


def lib():
    """The oracle library.  With ED_ORACLE_OPENMP=1 in the environment of the
    process (set before the first call), the OpenMP build of the same source
    is loaded instead: the multi-core timing baseline of the benchmark, not
    the oracle of the tests."""
    global _lib
    if _lib is None:
        omp = os.environ.get("ED_ORACLE_OPENMP", "0") == "1"
        _lib = C.CDLL(_build.build_openmp() if omp else _build.build())
        _declare(_lib)
    return _lib


def variant():
    """'openmp' or 'serial': which build lib() loads in this process."""
    return "openmp" if os.environ.get("ED_ORACLE_OPENMP", "0") == "1" else "serial"


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int)


class _Problem(C.Structure):
    _fields_ = [("N", C.c_int), ("m", C.c_int), ("K", C.c_int), ("KG", C.c_int),
                ("pos", _dp), ("nrm", _dp), ("idx", _ip), ("w", _dp), ("g", _dp), ("nbr", _ip),
                ("depth", _fp), ("nmap", _fp),
                ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("W", C.c_int), ("H", C.c_int),
                ("w_data", C.c_double), ("w_rot", C.c_double), ("w_reg", C.c_double),
                ("w_r", C.c_double), ("w_p", C.c_double),
                ("eps_d", C.c_float), ("cos_eps_n", C.c_float), ("prior", C.c_double * 6),
                ("NK", C.c_int), ("kp_pos", _dp), ("kp_idx", _ip), ("kp_w", _dp), ("kp_tgt", _dp),
                ("w_corr", C.c_double)]


class _Solver(C.Structure):
    _fields_ = [("n_gn", C.c_int), ("n_pcg", C.c_int), ("pcg_tol", C.c_double), ("jitter", C.c_double),
                ("lam", C.c_double), ("lm_accept", C.c_int), ("dense", C.c_int)]


class _FuseParams(C.Structure):
    _fields_ = [("tau_d", C.c_float), ("cos_delta", C.c_float), ("omega_max", C.c_double),
                ("tau_time", C.c_int), ("tau_weight", C.c_double), ("frame", C.c_int)]


def _declare(L):
    L.or_associate_f32.argtypes = [_fp, _fp, C.c_int, _fp, _fp, C.c_float, C.c_float, C.c_float, C.c_float,
                                   C.c_int, C.c_int, C.c_float, C.c_float, _ip]
    L.or_normals.argtypes = [_fp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, _fp]
    L.or_poisson_nodes.argtypes = [_fp, C.c_int, C.c_float, C.c_int, C.c_long, _ip, _ip]
    L.or_poisson_nodes.restype = C.c_int
    L.or_knn.argtypes = [_fp, C.c_int, _ip, C.c_int, _fp, C.c_int, C.c_int, _ip, _fp]
    L.or_node_graph.argtypes = [_fp, C.c_int, C.c_int, _ip]
    L.or_skin_weights.argtypes = [_fp, C.c_int, _fp, _ip, C.c_int, C.c_int, C.c_double, _dp]
    L.or_rotation.argtypes = [_dp, _dp, _dp]
    L.or_warp.argtypes = [C.POINTER(_Problem), _dp, _dp, _dp, _dp, _dp]
    L.or_linearize.argtypes = [C.POINTER(_Problem), _dp, _dp, _ip, _ip, C.c_void_p]
    L.or_linearize.restype = C.c_int
    L.or_energy.argtypes = [C.POINTER(_Problem), _dp, _dp, _ip, _dp, _ip]
    L.or_energy.restype = C.c_double
    L.or_residual_count.argtypes = [C.POINTER(_Problem), _ip]
    L.or_residual_count.restype = C.c_int
    L.or_residuals.argtypes = [C.POINTER(_Problem), _dp, _dp, _ip, _dp, _dp]
    L.or_normal_eq_new.restype = C.c_void_p
    L.or_normal_eq_delete.argtypes = [C.c_void_p]
    L.or_normal_eq_nnzb.argtypes = [C.c_void_p]
    L.or_normal_eq_nnzb.restype = C.c_int
    L.or_normal_eq_export.argtypes = [C.c_void_p, _ip, _ip, _dp, _dp, _dp, _dp, _dp, _ip]
    L.or_normal_eq_dense.argtypes = [C.c_void_p, _dp]
    L.or_pcg_eq.argtypes = [C.c_void_p, _dp, C.c_int, C.c_double, C.c_double, _dp, _ip, _dp]
    L.or_pcg_eq.restype = C.c_int
    L.or_dense_solve.argtypes = [C.c_void_p, _dp, _dp]
    L.or_dense_solve.restype = C.c_int
    L.or_damp.argtypes = [C.c_void_p, C.c_double]
    L.or_gn_solve.argtypes = [C.POINTER(_Problem), C.POINTER(_Solver), _dp, _dp, _dp]
    L.or_gn_solve.restype = C.c_int
    L.or_fuse.argtypes = [_fp, _fp, _fp, _ip, C.c_int, _fp, _fp, _fp, _fp, _fp, C.c_float, C.c_float, C.c_float,
                          C.c_float, C.c_int, C.c_int, C.POINTER(_FuseParams), C.c_int, _fp, _fp, _fp, _ip, _ip]
    L.or_fuse.restype = C.c_int
    L.or_downsample.argtypes = [_fp, _fp, _fp, _ip, C.c_int, C.c_float, C.c_double, C.c_double, C.c_int, _fp, _fp,
                                _fp, _ip, C.POINTER(C.c_uint32)]
    L.or_downsample.restype = C.c_int
    L.or_depth_error.argtypes = [_fp, C.c_int, _fp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int, C.c_int, _dp]
    L.or_depth_error.restype = None


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


# ----------------------------------------------------------------------------
# constants of the method (Sec. III.B) and the readings of the paper
# ----------------------------------------------------------------------------

W_DATA, W_ROT, W_REG, W_R, W_P = 1.0, 1000.0, 10000.0, 1.0e6, 1000.0
EPS_D_MM, EPS_N_DEG = 15.0, 10.0


def cos_deg_f32(deg: float) -> np.float32:
    """cos of an angle threshold, rounded once to FP32 (the gate's constant)."""
    return np.float32(math.cos(math.radians(deg)))


# ----------------------------------------------------------------------------
# per-step functions
# ----------------------------------------------------------------------------


def normals(depth, intr, h):
    fx, fy, cx, cy, W, H = intr
    depth = _f(depth)
    out = np.zeros((H, W, 4), np.float32)
    lib().or_normals(_p(depth, _fp), W, H, fx, fy, cx, cy, int(h), _p(out, _fp))
    return out


def poisson_nodes(pos, r, max_nodes, max_cells=1 << 25):
    pos = _f(pos)
    out = np.zeros(max(1, max_nodes), np.int32)
    mt = C.c_int(0)
    st = lib().or_poisson_nodes(_p(pos, _fp), pos.shape[0], C.c_float(r), int(max_nodes), int(max_cells),
                                _p(out, _ip), C.byref(mt))
    if st != 0:
        raise RuntimeError("poisson grid too large")
    m = min(mt.value, max_nodes)
    return out[:m].copy(), mt.value


def knn(pos, g, K, sel=None):
    pos, g = _f(pos), _f(g)
    cnt = pos.shape[0] if sel is None else len(sel)
    sel_a = None if sel is None else _i(sel)
    idx = np.zeros((cnt, K), np.int32)
    key = np.zeros((cnt, K), np.float32)
    lib().or_knn(_p(pos, _fp), pos.shape[0], _p(sel_a, _ip), cnt, _p(g, _fp), g.shape[0], K, _p(idx, _ip),
                 _p(key, _fp))
    return idx, key


def node_graph(g, KG):
    g = _f(g)
    nbr = np.zeros((g.shape[0], KG), np.int32)
    lib().or_node_graph(_p(g, _fp), g.shape[0], KG, _p(nbr, _ip))
    return nbr


def skin_weights(pos, g, idx_k1, K, mode, sigma):
    pos, g, idx_k1 = _f(pos), _f(g), _i(idx_k1)
    w = np.zeros((pos.shape[0], K), np.float64)
    lib().or_skin_weights(_p(pos, _fp), pos.shape[0], _p(g, _fp), _p(idx_k1, _ip), K, int(mode), float(sigma),
                          _p(w, _dp))
    return w


def rotation(pose):
    pose = _d(pose)
    R = np.zeros(9)
    dR = np.zeros(27)
    lib().or_rotation(_p(pose, _dp), _p(R, _dp), _p(dR, _dp))
    return R.reshape(3, 3), dR.reshape(3, 3, 3)


def associate_f32(wpos4, wnrm4, depth, nmap, intr, eps_d=EPS_D_MM, cos_eps_n=None):
    fx, fy, cx, cy, W, H = intr
    if cos_eps_n is None:
        cos_eps_n = cos_deg_f32(EPS_N_DEG)
    wpos4, wnrm4, depth, nmap = _f(wpos4), _f(wnrm4), _f(depth), _f(nmap)
    pix = np.zeros(wpos4.shape[0], np.int32)
    lib().or_associate_f32(_p(wpos4, _fp), _p(wnrm4, _fp), wpos4.shape[0], _p(depth, _fp), _p(nmap, _fp),
                           fx, fy, cx, cy, W, H, C.c_float(eps_d), C.c_float(cos_eps_n), _p(pix, _ip))
    return pix


@dataclasses.dataclass
class Graph:
    g: np.ndarray          # float32 [m, 4]
    idx: np.ndarray        # int32 [N, K]  (first K of the K+1 nearest)
    idx_k1: np.ndarray     # int32 [N, K+1]
    key: np.ndarray        # float32 [N, K+1]
    w: np.ndarray          # float64 [N, K]
    nbr: np.ndarray        # int32 [m, KG]
    node_pt: Optional[np.ndarray]
    m_total: int


def build_graph(pos, nodes=None, radius=None, max_nodes=None, K=4, KG=4, mode=0, sigma=None):
    """Node sampling (given nodes or Poisson radius), K(+1) nearest nodes,
    weights and node graph (Sec. II.D / II.E)."""
    pos = _f(pos)
    node_pt = None
    m_total = 0
    if nodes is None:
        node_pt, m_total = poisson_nodes(pos, radius, max_nodes)
        g = pos[node_pt].copy()
        g[:, 3] = 0.0
    else:
        g = _f(nodes).copy()
        m_total = g.shape[0]
    idx_k1, key = knn(pos, g, K + 1)
    w = skin_weights(pos, g, idx_k1, K, mode, sigma if sigma is not None else 1.0)
    nbr = node_graph(g, KG)
    return Graph(g=g, idx=np.ascontiguousarray(idx_k1[:, :K]), idx_k1=idx_k1, key=key, w=w, nbr=nbr,
                 node_pt=node_pt, m_total=m_total)


def calibrate_radius(pos, count, lo=None, hi=None, iters=40):
    """Largest Poisson radius (FP32) whose node set has at least `count` nodes,
    by bisection; the node set is then truncated to `count`."""
    pos = _f(pos)
    ext = pos[:, :3].max(0) - pos[:, :3].min(0)
    area = float(ext[0] * ext[1])
    guess = math.sqrt(area / count)
    lo = lo if lo is not None else 0.5 * guess
    hi = hi if hi is not None else 4.0 * guess
    _, m_lo = poisson_nodes(pos, lo, 0)
    if m_lo < count:
        raise RuntimeError("lower radius bound yields too few nodes")
    for _ in range(iters):
        mid = float(np.float32(0.5 * (lo + hi)))
        if mid == lo or mid == hi:
            break
        _, mm = poisson_nodes(pos, mid, 0)
        if mm >= count:
            lo = mid
        else:
            hi = mid
    return float(np.float32(lo))


W_CORR = 10.0   # weight of the sparse correspondence term (Sec. III.B, reading R18)


@dataclasses.dataclass
class Keypoints:
    """Sparse key correspondences (E_corr, Sec. II.E): model key points
    pos [NK][4] (mm, model frame), their K nearest nodes and normalised
    weights (the same rule as the model points), and 3D targets [NK][3] in the
    camera frame of the new frame."""
    pos: np.ndarray
    idx: np.ndarray
    w: np.ndarray
    target: np.ndarray
    w_corr: float = W_CORR


def keypoints(pos, target, g, K=4, mode=0, sigma=1.0, w_corr=W_CORR) -> Keypoints:
    """Key points skinned by the oracle's own nearest-node rule and weights."""
    pos = _f(pos)
    idx_k1, _ = knn(pos, g, K + 1)
    w = skin_weights(pos, g, idx_k1, K, mode, sigma)
    return Keypoints(pos=pos, idx=np.ascontiguousarray(idx_k1[:, :K]), w=w, target=_d(target), w_corr=w_corr)


class Problem:
    """Holds the arrays of one registration problem (double geometry)."""

    def __init__(self, pos, nrm, graph: Graph, depth, nmap, intr, prior,
                 weights=(W_DATA, W_ROT, W_REG, W_R, W_P), eps_d=EPS_D_MM, eps_n_deg=EPS_N_DEG, cos_eps_n=None,
                 keypoints: Optional["Keypoints"] = None):
        self.pos = _d(pos)
        self.nrm = _d(nrm)
        self.idx = _i(graph.idx)
        self.w = _d(graph.w)
        self.g = _d(graph.g)
        self.nbr = _i(graph.nbr)
        self.depth = _f(depth)
        self.nmap = _f(nmap)
        self.intr = intr
        self.N = self.pos.shape[0]
        self.m = self.g.shape[0]
        self.K = self.idx.shape[1]
        self.KG = self.nbr.shape[1]
        fx, fy, cx, cy, W, H = intr
        s = _Problem()
        s.N, s.m, s.K, s.KG = self.N, self.m, self.K, self.KG
        s.pos, s.nrm, s.idx, s.w = _p(self.pos, _dp), _p(self.nrm, _dp), _p(self.idx, _ip), _p(self.w, _dp)
        s.g, s.nbr = _p(self.g, _dp), _p(self.nbr, _ip)
        s.depth, s.nmap = _p(self.depth, _fp), _p(self.nmap, _fp)
        s.fx, s.fy, s.cx, s.cy, s.W, s.H = fx, fy, cx, cy, W, H
        s.w_data, s.w_rot, s.w_reg, s.w_r, s.w_p = weights
        s.eps_d = float(np.float32(eps_d))
        s.cos_eps_n = float(cos_eps_n if cos_eps_n is not None else cos_deg_f32(eps_n_deg))
        for t in range(6):
            s.prior[t] = float(prior[t])
        self.kp = keypoints
        if keypoints is not None and keypoints.pos.shape[0] > 0:
            self.kp_pos = _d(keypoints.pos)
            self.kp_idx = _i(keypoints.idx)
            self.kp_w = _d(keypoints.w)
            self.kp_tgt = _d(keypoints.target)
            s.NK = self.kp_pos.shape[0]
            s.kp_pos, s.kp_idx = _p(self.kp_pos, _dp), _p(self.kp_idx, _ip)
            s.kp_w, s.kp_tgt = _p(self.kp_w, _dp), _p(self.kp_tgt, _dp)
            s.w_corr = float(keypoints.w_corr)
        self.s = s

    @property
    def n_unknowns(self):
        return 12 * self.m + 6

    def identity_x(self):
        x = np.zeros((self.m, 12))
        x[:, 0] = x[:, 5] = x[:, 10] = 1.0
        return x


def warp(P: Problem, x, pose):
    x, pose = _d(x), _d(pose)
    wpos = np.zeros((P.N, 3))
    wnrm = np.zeros((P.N, 3))
    spre = np.zeros((P.N, 3))
    lib().or_warp(C.byref(P.s), _p(x, _dp), _p(pose, _dp), _p(wpos, _dp), _p(wnrm, _dp), _p(spre, _dp))
    return wpos, wnrm, spre


class NormalEq:
    """J^T J (block-sparse, full symmetric pattern) and J^T r at one point."""

    def __init__(self, P: Problem, x, pose, pix_in=None):
        self.P = P
        self.h = lib().or_normal_eq_new()
        x, pose = _d(x), _d(pose)
        pin = None if pix_in is None else _i(pix_in)
        self.pix = np.zeros(P.N, np.int32)
        lib().or_linearize(C.byref(P.s), _p(x, _dp), _p(pose, _dp), _p(pin, _ip), _p(self.pix, _ip), self.h)
        m = P.m
        nnzb = lib().or_normal_eq_nnzb(self.h)
        self.row_ptr = np.zeros(m + 1, np.int32)
        self.col = np.zeros(nnzb, np.int32)
        self.blk = np.zeros((nnzb, 12, 12))
        self.C = np.zeros((m, 6, 12))
        self.Hpp = np.zeros((6, 6))
        self.g = np.zeros(12 * m + 6)
        self.E = np.zeros(6)   # data, rot, reg, rot prior, pos prior, correspondence
        nv = C.c_int(0)
        lib().or_normal_eq_export(self.h, _p(self.row_ptr, _ip), _p(self.col, _ip), _p(self.blk, _dp),
                                  _p(self.C, _dp), _p(self.Hpp, _dp), _p(self.g, _dp), _p(self.E, _dp),
                                  C.byref(nv))
        self.n_valid = nv.value

    def __del__(self):
        try:
            lib().or_normal_eq_delete(self.h)
        except Exception:
            pass

    @property
    def energy(self):
        return float(self.E.sum())

    def block(self, j, l):
        s, e = self.row_ptr[j], self.row_ptr[j + 1]
        k = np.searchsorted(self.col[s:e], l)
        if k < e - s and self.col[s + k] == l:
            return self.blk[s + k]
        return None

    def dense(self):
        n = self.P.n_unknowns
        H = np.zeros((n, n))
        lib().or_normal_eq_dense(self.h, _p(H, _dp))
        return H

    def damp(self, lam):
        lib().or_damp(self.h, float(lam))
        # keep the exported copy in step
        m = self.P.m
        for j in range(m):
            b = self.block(j, j)
            b[np.arange(12), np.arange(12)] *= 1.0 + lam
        self.Hpp[np.arange(6), np.arange(6)] *= 1.0 + lam

    def pcg(self, b, n_iter, tol=0.0, jitter=1e-6):
        b = _d(b)
        d = np.zeros_like(b)
        it = C.c_int(0)
        hist = np.zeros(n_iter + 1)
        st = lib().or_pcg_eq(self.h, _p(b, _dp), int(n_iter), float(tol), float(jitter), _p(d, _dp),
                             C.byref(it), _p(hist, _dp))
        return d, it.value, st, hist[:it.value + 1]

    def dense_solve(self, b):
        b = _d(b)
        d = np.zeros_like(b)
        st = lib().or_dense_solve(self.h, _p(b, _dp), _p(d, _dp))
        if st != 0:
            raise RuntimeError("dense Cholesky failed")
        return d


def energy(P: Problem, x, pose, pix_in=None):
    x, pose = _d(x), _d(pose)
    terms = np.zeros(6)   # data, rot, reg, rot prior, pos prior, correspondence
    nv = C.c_int(0)
    pin = None if pix_in is None else _i(pix_in)
    E = lib().or_energy(C.byref(P.s), _p(x, _dp), _p(pose, _dp), _p(pin, _ip), _p(terms, _dp), C.byref(nv))
    return E, terms, nv.value


def residuals(P: Problem, x, pose, pix, jacobian=False):
    x, pose, pix = _d(x), _d(pose), _i(pix)
    n = lib().or_residual_count(C.byref(P.s), _p(pix, _ip))
    r = np.zeros(n)
    J = np.zeros((n, P.n_unknowns)) if jacobian else None
    lib().or_residuals(C.byref(P.s), _p(x, _dp), _p(pose, _dp), _p(pix, _ip), _p(r, _dp), _p(J, _dp))
    return (r, J) if jacobian else r


def gn_solve(P: Problem, x, pose, n_gn, n_pcg, lam=0.0, lm_accept=False, dense=False, pcg_tol=0.0,
             jitter=1e-6):
    x = _d(x).copy()
    pose = _d(pose).copy()
    S = _Solver(n_gn=n_gn, n_pcg=n_pcg, pcg_tol=pcg_tol, jitter=jitter, lam=lam, lm_accept=int(lm_accept),
                dense=int(dense))
    hist = np.zeros((n_gn, 6))
    st = lib().or_gn_solve(C.byref(P.s), C.byref(S), _p(x, _dp), _p(pose, _dp), _p(hist, _dp))
    return x, pose, hist, st


def gradient(P: Problem, x, pose, pix_in=None):
    """dE/d(x, pose) = 2 J^T r (association frozen when pix_in is given)."""
    Q = NormalEq(P, x, pose, pix_in)
    return 2.0 * Q.g


@dataclasses.dataclass
class FuseParams:
    tau_d: float = 10.0
    delta_deg: float = 10.0
    omega_max: float = 20.0
    tau_time: int = 10
    tau_weight: float = 3.0
    frame: int = 1


def fuse(pos, nrm, col, tstamp, wpos, wnrm, depth, nmap, color, intr, F: FuseParams, capacity):
    fx, fy, cx, cy, W, H = intr
    pos, nrm, col, tstamp = _f(pos), _f(nrm), _f(col), _i(tstamp)
    wpos, wnrm, depth, nmap, color = _f(wpos), _f(wnrm), _f(depth), _f(nmap), _f(color)
    fp = _FuseParams(tau_d=float(np.float32(F.tau_d)), cos_delta=float(cos_deg_f32(F.delta_deg)),
                     omega_max=F.omega_max, tau_time=F.tau_time, tau_weight=F.tau_weight, frame=F.frame)
    po = np.zeros((capacity, 4), np.float32)
    no = np.zeros((capacity, 4), np.float32)
    co = np.zeros((capacity, 4), np.float32)
    to = np.zeros(capacity, np.int32)
    reg = np.zeros(H * W, np.int32)
    n = lib().or_fuse(_p(pos, _fp), _p(nrm, _fp), _p(col, _fp), _p(tstamp, _ip), pos.shape[0], _p(wpos, _fp),
                      _p(wnrm, _fp), _p(depth, _fp), _p(nmap, _fp), _p(color, _fp), fx, fy, cx, cy, W, H,
                      C.byref(fp), capacity, _p(po, _fp), _p(no, _fp), _p(co, _fp), _p(to, _ip), _p(reg, _ip))
    if n < 0:
        raise RuntimeError("fuse capacity exceeded")
    return po[:n], no[:n], co[:n], to[:n], reg


def downsample(pos, nrm, col, tstamp, box, omega_max=20.0, tau_weight=3.0, capacity=None):
    """Box downsampling of the model (Sec. III.A, Alg. 3): returns (pos, nrm,
    col, t, box keys) of the merged points in increasing key order."""
    pos, nrm, col, tstamp = _f(pos), _f(nrm), _f(col), _i(tstamp)
    n = pos.shape[0]
    cap = n if capacity is None else int(capacity)
    po = np.zeros((max(cap, 1), 4), np.float32)
    no = np.zeros_like(po)
    co = np.zeros_like(po)
    to = np.zeros(max(cap, 1), np.int32)
    ko = np.zeros(max(cap, 1), np.uint32)
    k = lib().or_downsample(_p(pos, _fp), _p(nrm, _fp), _p(col, _fp), _p(tstamp, _ip), n, float(np.float32(box)),
                            float(omega_max), float(tau_weight), cap, _p(po, _fp), _p(no, _fp), _p(co, _fp),
                            _p(to, _ip), ko.ctypes.data_as(C.POINTER(C.c_uint32)))
    if k == -1:
        raise RuntimeError("downsample capacity exceeded")
    if k == -2:
        raise RuntimeError("downsample box grid too large")
    return po[:k], no[:k], co[:k], to[:k], ko[:k]


def depth_error(wpos, depth, intr):
    """Back-projection error of warped model points against a depth image
    (Sec. III): (mean |z - D|, count, max |z - D|, rms) over the pixels that
    keep a point (nearest z, then lowest index) and have D > 0."""
    fx, fy, cx, cy, W, H = intr
    wpos, depth = _f(wpos), _f(depth)
    out = np.zeros(4)
    lib().or_depth_error(_p(wpos, _fp), wpos.shape[0], _p(depth, _fp), fx, fy, cx, cy, W, H, _p(out, _dp))
    cnt = out[1]
    return (out[0] / cnt if cnt else 0.0), int(cnt), out[2], (math.sqrt(out[3] / cnt) if cnt else 0.0)


def track_frame(model, depth, color, intr, radius, max_nodes, box, n_gn, n_pcg, frame_index, normal_half_width,
                truth_depth=None, prior=(0.0, 0.0, 0.0, 0.0, 0.0, 0.0), fuse_params=None, capacity=None):
    """One frame of Algorithm 2 with Algorithm 3: the target normals, nodes
    sampled afresh on the current model (Alg. 2 step 5) with identity
    parameters, n_gn Gauss-Newton steps (block-Jacobi PCG, n_pcg iterations),
    the final warp, the back-projection error against `truth_depth` (default
    the observation), fusion (Alg. 1-2, Eqs. fusion1-4) and box downsampling
    (Sec. III.A).  `model` = (pos, nrm, col, t); returns (new model, info)."""
    pos, nrm, col, t = model
    fx, fy, cx, cy, W, H = intr
    nm = normals(depth, intr, normal_half_width)
    G = build_graph(pos, radius=radius, max_nodes=max_nodes, K=4, KG=4, mode=0, sigma=radius)
    P = Problem(pos, nrm, G, depth, nm, intr, np.asarray(prior, float))
    x, pose, hist, st = gn_solve(P, P.identity_x(), np.asarray(prior, float), n_gn, n_pcg)
    wp, wn, _ = warp(P, x, pose)
    wp4 = np.concatenate([wp, pos[:, 3:4]], 1).astype(np.float32)
    wn4 = np.concatenate([wn, nrm[:, 3:4]], 1).astype(np.float32)
    err = depth_error(wp4, truth_depth if truth_depth is not None else depth, intr)
    F = dataclasses.replace(fuse_params or FuseParams(), frame=int(frame_index))
    cap = capacity if capacity is not None else pos.shape[0] + W * H
    fpos, fnrm, fcol, ft, _ = fuse(pos, nrm, col, t, wp4, wn4, depth, nm, color, intr, F, cap)
    dpos, dnrm, dcol, dt, _ = downsample(fpos, fnrm, fcol, ft, box, F.omega_max, F.tau_weight)
    info = dict(nodes=G.g.shape[0], fused=fpos.shape[0], model=dpos.shape[0], status=st, energy=hist,
                error_mean_mm=err[0], error_pixels=err[1], error_max_mm=err[2], error_rms_mm=err[3], x=x, pose=pose)
    return (dpos, dnrm, dcol, dt), info
