"""Batched plans: several fields per exec call (fft3d_plan_create_batched).

Each field of a batch must come out exactly as a plan of batch 1 computes it
(same kernels, same per-field arithmetic: compared bit for bit), and match
the FP64 oracle field by field.  Shapes cover the x-pass tiles of several
fields (field b's columns start at row b N0), the pipelined column kernel
with TMA staging on either axis, ragged tiles, both layouts and both dtypes."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, rel_l2, torch_dtype

pytestmark = pytest.mark.gpu

SHAPES = [
    (3, 16, 12, 24),     # small, ragged tiles, 3·2^k lengths
    (3, 64, 64, 64),     # the three velocity components of a 64^3 field
    (2, 1024, 32, 32),   # FP32 x-pass: pipelined kernel, one TMA map over both fields' rows
    (2, 8, 1024, 64),    # FP32 y-pass: pipelined kernel, even/odd row-pair TMA maps (odd pitch 33)
    (2, 2048, 16, 32),   # FP32 x-pass of 2048 points: CTA pairs, row-parity map over both fields' rows
    (2, 4, 2048, 64),    # FP32 y-pass of 2048 points: pipelined kernel on 8-column tiles over both fields' planes
    (2, 1536, 8, 16),    # FP32 x-pass of 1536 points: one-buffer kernel, TMA rows of both fields
    (4, 6, 8, 12),
    (3, 1, 16, 32),      # N0 = 1: no x-pass
    (2, 32, 1, 16),      # N1 = 1: no y-pass
]


def _fields(shape, seed):
    b = shape[0]
    return np.stack([synth.uniform_field(shape[1:], seed + i) for i in range(b)])


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", ["f64", "f32"])
def test_batched_matches_single_plans_and_oracle(shape, name):
    import torch
    import paper_2202_12756_gb300 as fft3d
    dt = torch_dtype(name)
    b, fshape = shape[0], shape[1:]
    f = _fields(shape, 70)
    if name == "f32":
        f = f.astype(np.float32).astype(np.float64)
    x = torch.from_numpy(f).to(dt).cuda()
    pb = fft3d.get_plan(fshape, dt, "cuda", batch=b)
    p1 = fft3d.get_plan(fshape, dt, "cuda")
    X = pb.r2c(x)
    back = pb.c2r(X)
    for i in range(b):
        Xi = p1.r2c(x[i].contiguous())
        assert torch.equal(X[i], Xi), i
        assert torch.equal(back[i], p1.c2r(Xi)), i
    torch.cuda.synchronize()
    Xh = X.cpu().numpy().astype(np.complex128)
    for i in range(b):
        assert rel_l2(Xh[i], oracle.rfft3(f[i])) <= TOL[name]
    assert rel_l2(back.cpu().numpy().astype(np.float64), f) <= TOL[name]


@pytest.mark.parametrize("shape", [(3, 32, 24, 48), (2, 1024, 32, 32), (2, 8, 1024, 64)],
                         ids=lambda s: "x".join(map(str, s)))
def test_batched_in_place_and_input_preserved(shape):
    import torch
    import paper_2202_12756_gb300 as fft3d
    dt = torch.float32
    b, fshape = shape[0], shape[1:]
    n2 = fshape[2]
    f = _fields(shape, 80).astype(np.float32)
    pb = fft3d.get_plan(fshape, dt, "cuda", batch=b)
    x = torch.from_numpy(f).cuda()
    X_oop = pb.r2c(x)
    X_keep = X_oop.clone()
    y = pb.c2r(X_oop)
    assert torch.equal(X_oop, X_keep)  # the out-of-place inverse keeps its input
    buf = pb.empty_padded()
    buf[..., :n2].copy_(x)
    Xin = pb.r2c_(buf)
    assert torch.equal(Xin, X_keep)    # in place = out of place, bit for bit
    pb.c2r_(buf)
    assert torch.equal(buf[..., :n2], y)


def test_batched_autograd():
    import torch
    import paper_2202_12756_gb300 as fft3d
    x = torch.from_numpy(_fields((2, 4, 6, 8), 90)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: fft3d.rfft3(t), (x,), eps=1e-6, atol=1e-8, rtol=1e-6)
    X = torch.from_numpy(np.stack([synth.random_half_spectrum((4, 6, 8), 91 + i) for i in range(2)]))
    X = X.cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: fft3d.irfft3(t, (2, 4, 6, 8)), (X,), eps=1e-6, atol=1e-8,
                                    rtol=1e-6)


def test_batched_plan_rejects_bad_batch():
    import torch
    import paper_2202_12756_gb300 as fft3d
    for bad in (0, -1, (1 << 31) // (1024 * 1024) + 1):
        with pytest.raises(fft3d.FFT3DError) as e:
            fft3d.fft3d_plan_create_batched(bad, 1024, 1024, 1024, 0)
        assert e.value.status == fft3d.FFT3D_ERR_SIZE
    # (4, 512, 512) FP32 offers the fused plane pass at batch 1, not in a batch
    plan = fft3d.Plan((4, 512, 512), torch.float32, batch=2)
    with pytest.raises(fft3d.FFT3DError) as e:
        plan.set_fused(True)
    assert e.value.status == fft3d.FFT3D_ERR_SIZE
    assert not plan.info()["fused_plane_pass"]


def test_batched_host_resident_fields():
    """A batch of three fields in pinned host memory: the first and last passes
    stream them over the CPU-GPU link on the limited, looping grid (1536 line
    groups here); the result equals the device-resident call bit for bit."""
    import torch
    import paper_2202_12756_gb300 as fft3d
    shape = (3, 64, 256, 256)
    f = _fields(shape, 99).astype(np.float32)
    pb = fft3d.get_plan(shape[1:], torch.float32, "cuda", batch=3)
    host_in = torch.from_numpy(f).pin_memory()
    host_out = torch.full(shape, float("nan"), dtype=torch.float32).pin_memory()
    X = pb.r2c(host_in)
    X_dev = pb.r2c(host_in.cuda())
    torch.cuda.synchronize()
    assert torch.equal(X, X_dev)
    y_dev = pb.c2r_overwrite(X_dev)
    pb.c2r_overwrite(X, host_out)
    torch.cuda.synchronize()
    assert torch.equal(host_out, y_dev.cpu())
    assert rel_l2(host_out.numpy().astype(np.float64), f.astype(np.float64)) <= TOL["f32"]
