"""The bounded device waits give up, report ED_ERR_TIMEOUT and leave the
context usable.

The PCG grid barrier is made to wait for one arrival more than the launch
has CTAs (a count that no CTA ever brings), with the wait limit shortened to
1 ms: every CTA must leave the barrier after the limit, the step must report
ED_ERR_TIMEOUT in its statistics, the update must not be applied (x and the
pose unchanged), and the next step with the normal barrier must give the
same result as a context that never timed out.  No kernel faults or traps:
the waits end by their own limit."""
import numpy as np
import pytest

from tests import gpu_common as C

pytestmark = pytest.mark.gpu

SMALL = "tissue_160x120_n64"
ED_ERR_TIMEOUT = 6


def test_pcg_barrier_wait_gives_up_and_context_recovers():
    import torch
    import paper_1803_02009_b300 as E
    s = C.scene(SMALL)
    G = C.gpu_setup(s)
    ctx = G["ctx"]
    prm = C.solver(s)
    x = ctx.identity_x()
    pose = torch.tensor(s.pose_prior, dtype=torch.float64, device="cuda")
    x0, p0 = x.clone(), pose.clone()
    with pytest.raises(E.EDError):
        ctx.set_wait_limit(1000)          # below the 100 us floor
    ctx.set_wait_limit(1_000_000)         # 1 ms
    ctx.set_barrier_test(1)
    st = E.new_stats()
    ctx.gn_step(G["frame"], prm, x, pose, stats=st)
    torch.cuda.synchronize()
    r = E.read_stats(st)[0]
    assert r["status"] == ED_ERR_TIMEOUT, r
    assert torch.equal(x, x0) and torch.equal(pose, p0)
    # the context is usable afterwards: the same step with the normal barrier
    ctx.set_barrier_test(0)
    ctx.set_wait_limit(0)
    st2 = E.new_stats()
    ctx.gn_step(G["frame"], prm, x, pose, stats=st2)
    torch.cuda.synchronize()
    r2 = E.read_stats(st2)[0]
    assert r2["status"] == 0, r2
    # a context that never timed out takes the identical step
    G2 = C.gpu_setup(s)
    x2 = G2["ctx"].identity_x()
    pose2 = torch.tensor(s.pose_prior, dtype=torch.float64, device="cuda")
    st3 = E.new_stats()
    G2["ctx"].gn_step(G2["frame"], prm, x2, pose2, stats=st3)
    torch.cuda.synchronize()
    assert torch.equal(x, x2) and torch.equal(pose, pose2)
    assert E.read_stats(st3)[0]["energy"] == r2["energy"]
