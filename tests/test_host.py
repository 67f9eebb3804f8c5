"""Host-side checks that need no GPU: the C-ABI library loads and exports
every function the public header declares, the Python binding refuses to run
without it, and the multi-rank bench logic (independent problems per rank,
slowest-rank timing, whole-job rate) holds on two gloo ranks."""
import ctypes
import os
import re
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ed.h")


def declared_functions():
    """Names of every function prototype in include/ed.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(ed_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def built_library():
    sys.path.insert(0, ROOT)
    from paper_1803_02009_b300 import build_lib
    return build_lib.build(force=False)


def test_header_declares_the_path():
    names = declared_functions()
    for need in ("ed_build_graph", "ed_warp", "ed_gn_step", "ed_fuse", "ed_compute_normals", "ed_energy",
                 "ed_energy_grad", "ed_query_workspace", "ed_create", "ed_destroy", "ed_status_string"):
        assert need in names, need


def test_library_loads_and_exports_every_declared_symbol():
    lib_path = built_library()
    lib = ctypes.CDLL(lib_path)          # loads without a GPU: no CUDA call happens at load time
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in ed.h but not exported by libed.so: {missing}"
    # the exported table also matches the dynamic symbol list
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (ed_[a-z0-9_]+)\b", out))
    assert set(declared_functions()) <= exported


def test_status_strings_without_gpu():
    lib = ctypes.CDLL(built_library())
    lib.ed_status_string.restype = ctypes.c_char_p
    seen = set()
    for code in range(8):
        s = lib.ed_status_string(code)
        assert s and len(s) >= 2
        seen.add(s)
    assert len(seen) == 8


def test_query_workspace_rejects_bad_limits_without_gpu():
    sys.path.insert(0, ROOT)
    built_library()
    import paper_1803_02009_b300 as E
    lib = E.lib()
    size = ctypes.c_size_t(0)
    ED_OK, ED_ERR_ARG = 0, 1
    bad = E.Limits(0, 0, 0, 0, 0, 0)
    assert lib.ed_query_workspace(ctypes.byref(bad), ctypes.byref(size)) == ED_ERR_ARG
    ok = E.Limits(20000, 64, 160, 120, 0, 0)
    assert lib.ed_query_workspace(ctypes.byref(ok), ctypes.byref(size)) == ED_OK
    assert size.value > 0


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import paper_1803_02009_b300 as E
    monkeypatch.setattr(E, "_lib", None)
    monkeypatch.setattr(E, "LIB_PATH", str(tmp_path / "missing.so"), raising=False)
    with pytest.raises(Exception):
        E.lib()


# ---------------------------------------------------------------------------
# two gloo ranks: the bench's multi-rank logic
# ---------------------------------------------------------------------------

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.rank_seed(rank)
        s = synth.make_scene("tissue_160x120_n64", seed)
        local_seconds = 1.0 + rank          # rank 1 is the slow one
        job = bench.max_over_ranks(local_seconds, dist)
        rate = bench.whole_job_rate(world, 4, s.cfg.n_gn, job)
        q.put((rank, seed, float(s.tgt_depth.sum()), job, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_independent_problems():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (r0, seed0, d0, job0, rate0), (r1, seed1, d1, job1, rate1) = res
    assert seed0 != seed1 and d0 != d1            # each rank registers its own frame
    assert job0 == job1 == 2.0                    # the slowest rank's time, seen by both
    assert rate0 == rate1 == pytest.approx(2 * 4 * 5 / 2.0)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        config = "tissue_160x120_n64"
        steps = 1
        warmup = 0
    assert bench.run_reference(A, 1, 2) is None
