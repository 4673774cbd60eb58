"""Failure detection of the kernels that wait, without a GPU fault.

The fused kernel's blocks wait on per-plane counters that other blocks set,
and the pipelined column kernel's blocks wait on an mbarrier for the TMA
copies of their next tile.  Each wait is bounded.  Here the test hook makes
the waits unsatisfiable (one producer more than exists; 16 bytes more than
the copies deliver) with a short bound: the waits run out, the kernel returns
early and raises its error flag, the host reads the flag, and the same plan
then computes correctly again (the context stays usable)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("direction", ["r2c", "c2r"])
def test_bounded_wait_reports_and_recovers(direction):
    import torch
    import paper_2202_12756_gb300 as fft3d
    shape = (6, 512, 512)
    plan = fft3d.Plan(shape, torch.float32)
    plan.set_fused(True)
    assert plan.info()["fused_plane_pass"]
    f = synth.uniform_field(shape, 41).astype(np.float32)
    x = torch.from_numpy(f).cuda()
    X = plan.r2c(x)
    torch.cuda.synchronize()
    assert plan.status() == 0

    plan.set_debug(True, spin_limit=20000)  # ~ a few ms per wait
    if direction == "r2c":
        plan.r2c(x, X)
    else:
        plan.c2r(X.clone())
    torch.cuda.synchronize()
    assert plan.status() == 1, "the stalled wait was not reported"
    assert plan.status() == 0, "the flag is cleared once read"

    plan.set_debug(False)
    X2 = plan.r2c(x)
    back = plan.c2r(X2)
    torch.cuda.synchronize()
    assert plan.status() == 0
    ref = oracle.rfft3(f.astype(np.float64))
    assert rel_l2(X2.cpu().numpy(), ref) <= TOL["f32"]
    assert rel_l2(back.cpu().numpy(), f) <= TOL["f32"]


def test_plans_without_fused_pass_report_no_error():
    import torch
    import paper_2202_12756_gb300 as fft3d
    plan = fft3d.Plan((8, 16, 32), torch.float64)
    assert not plan.info()["fused_plane_pass"]
    plan.r2c(torch.zeros((8, 16, 32), dtype=torch.float64, device="cuda"))
    assert plan.status() == 0


@pytest.mark.parametrize("shape", [(1024, 16, 32), (8, 1024, 64), (2048, 16, 32), (8, 2048, 64), (1536, 16, 32)],
                         ids=lambda s: "x".join(map(str, s)))
def test_pipelined_tile_wait_reports_and_recovers(shape):
    """The pipelined column kernel waits on an mbarrier for the TMA copies of
    each tile.  With the test hook every tile wait expects 16 bytes more than
    its copies deliver, so it runs out after a short bound: the blocks stop,
    the flag is reported once, and the same plan then computes correctly.
    (1024, 16, 32): x-pass over whole rows; (8, 1024, 64): y-pass with the
    even/odd row-pair copies of an odd row pitch; (2048, 16, 32): the x-pass
    on clusters of two CTAs, which meet at a final cluster barrier whichever
    of their waits runs out; (8, 2048, 64): the 2048-point y-pass on one SM
    per 8-column tile; (1536, 16, 32): the 1536-point x-pass on the kernel
    whose staging buffer is also its exchange buffer.)"""
    import torch
    import paper_2202_12756_gb300 as fft3d
    plan = fft3d.Plan(shape, torch.float32)
    f = synth.uniform_field(shape, 43).astype(np.float32)
    x = torch.from_numpy(f).cuda()
    X = plan.r2c(x)
    torch.cuda.synchronize()
    assert plan.status() == 0

    plan.set_debug(True, spin_limit=1 << 14)
    plan.r2c(x, X)
    torch.cuda.synchronize()
    assert plan.status() == 1, "the stalled tile wait was not reported"
    assert plan.status() == 0, "the flag is cleared once read"

    plan.set_debug(False)
    X2 = plan.r2c(x)
    back = plan.c2r(X2)
    torch.cuda.synchronize()
    assert plan.status() == 0
    assert rel_l2(X2.cpu().numpy(), oracle.rfft3(f.astype(np.float64))) <= TOL["f32"]
    assert rel_l2(back.cpu().numpy(), f) <= TOL["f32"]
