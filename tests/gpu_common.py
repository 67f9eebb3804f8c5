"""Shared set-up of the GPU parity tests: the same seeded scene goes to the
CUDA path (through the C ABI) and to the FP64 oracle."""
import functools
import json
import os

import numpy as np

import oracle
import synth

# tolerances (stated by the benchmark spec: node parameters 1e-4 relative, energy 1e-5
# relative, integer indices bit-exact); block-level tolerances derive from
# FP32 accumulation over <= a few thousand terms
TOL_X = 1e-4
TOL_E = 1e-5


@functools.lru_cache(maxsize=8)
def scene(name, seed=1):
    return synth.make_scene(name, seed)


@functools.lru_cache(maxsize=8)
def radius_for(name, seed=1):
    s = scene(name, seed)
    return oracle.calibrate_radius(s.model_pos, s.cfg.node_count)


def gpu_setup(s, radius=None, max_nodes=None, weight_mode=0, k_graph=4, sigma=None, extra_points=0):
    import torch
    import paper_1803_02009_b300 as E
    dev = "cuda"
    fx, fy, cx, cy, W, H = s.intr
    m_cap = max(64, max_nodes or (s.nodes.shape[0] if s.nodes is not None else 64))
    ctx = E.Context(max_points=s.N + extra_points, max_nodes=m_cap, max_width=W, max_height=H, max_cells=1 << 24)
    pos = torch.from_numpy(s.model_pos).to(dev)
    nrm = torch.from_numpy(s.model_nrm).to(dev)
    depth = torch.from_numpy(s.tgt_depth).to(dev)
    color = torch.from_numpy(np.ascontiguousarray(s.tgt_color)).to(dev)
    nmap = ctx.compute_normals(depth, s.intr, s.cfg.normal_half_width)
    if s.nodes is not None and radius is None:
        sig = s.sigma if sigma is None else sigma
        g = ctx.build_graph(pos, nrm, nodes=torch.from_numpy(s.nodes).to(dev), k_graph=k_graph,
                            weight_mode=weight_mode, sigma=sig)
    else:
        sig = radius if sigma is None else sigma
        g = ctx.build_graph(pos, nrm, node_radius=radius, max_nodes=max_nodes, k_graph=k_graph,
                            weight_mode=weight_mode, sigma=sig)
    frame = E.make_frame(depth, nmap, s.intr, color)
    torch.cuda.synchronize()
    return dict(ctx=ctx, pos=pos, nrm=nrm, depth=depth, color=color, nmap=nmap, graph=g, frame=frame, sigma=sig)


def oracle_graph_from_gpu(G):
    """The GPU-built graph as an oracle Graph (weights widened to FP64)."""
    g = G["graph"]
    m = g.m
    idx = g.idx_long().cpu().numpy().astype(np.int32)
    return oracle.Graph(g=g.nodes[:m].cpu().numpy(), idx=idx, idx_k1=None, key=None,
                        w=g.weights.cpu().numpy().astype(np.float64), nbr=g.nbr[:m].cpu().numpy(),
                        node_pt=None, m_total=m)


def oracle_problem_from_gpu(s, G, prior=None):
    og = oracle_graph_from_gpu(G)
    nmap = G["nmap"].cpu().numpy()
    return oracle.Problem(s.model_pos, s.model_nrm, og, s.tgt_depth, nmap, s.intr,
                          s.pose_prior if prior is None else prior)


def solver(s, **kw):
    import paper_1803_02009_b300 as E
    p = E.SolverParams(n_pcg=s.cfg.n_pcg, prior=tuple(float(v) for v in s.pose_prior))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def blocks_dict(row_ptr, col, blk):
    out = {}
    for j in range(len(row_ptr) - 1):
        for t in range(row_ptr[j], row_ptr[j + 1]):
            out[(j, int(col[t]))] = blk[t]
    return out


def report(name, data):
    """Prints a test's figures and, with ED_REPORT_DIR set, writes them there as JSON."""
    d = os.environ.get("ED_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, name + ".json"), "w") as f:
            json.dump(data, f, indent=1, default=float)
    print(name, json.dumps(data, default=float))


def block_errors(got, ref, floor_rel=1e-6):
    """Per 12x12 block: the largest entry error over the block's own largest
    entry (blocks of the FP32 system against the FP64 one).  A block whose
    entries are all (near) zero is measured against floor_rel times the
    largest entry of the whole system."""
    got = np.asarray(got, dtype=np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    # (an all-zero reference must be matched by zeros: any other value fails)
    scale = np.maximum(np.maximum(np.abs(ref).max(1), floor_rel * np.abs(ref).max()), 1e-30)
    return np.abs(got - ref).max(1) / scale
