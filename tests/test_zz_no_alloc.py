"""The allocation-free inverse entry point, fft3d_exec_c2r_noalloc.

It serves callers that cannot call cudaMalloc (their own pool allocator
already holds the GPU's memory, or they must not trigger the device
synchronisation cudaMalloc / cudaFree can cause), so it runs without a plan
on one static scratch array of the library.  Here it is called through the
C ABI on two calls in a row (the second call reuses the scratch the first one
left) and compared with the plan-based fft3d_exec_c2r on the same input and
with the FP64 oracle's inverse; its device error word must read 0 afterwards.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, rel_l2

pytestmark = pytest.mark.gpu


def _run(shape, name, inplace):
    import torch
    import paper_2202_12756_gb300 as fft3d
    lib = fft3d.load_library()
    dt = torch.float32 if name == "f32" else torch.float64
    cdt = fft3d.complex_of(dt)
    code = fft3d.FFT3D_F32 if name == "f32" else fft3d.FFT3D_F64
    n0, n1, n2 = shape
    G_host = synth.random_half_spectrum(shape, 31)
    if name == "f32":
        G_host = G_host.astype(np.complex64).astype(np.complex128)
    g_ref = oracle.irfft3(G_host, shape)
    G = torch.from_numpy(G_host).to(cdt).cuda()
    plan = fft3d.Plan(shape, dt)
    ref = plan.c2r(G.clone()).cpu().numpy().astype(np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):
        if inplace:
            buf = torch.empty((n0, n1, 2 * (n2 // 2 + 1)), dtype=dt, device="cuda")
            buf.view(cdt).copy_(G)
            rc = lib.fft3d_exec_c2r_noalloc(buf.data_ptr(), buf.data_ptr(), n0, n1, n2, code, stream)
            out = buf[..., :n2]
        else:
            src = G.clone()
            out = torch.full(shape, float("nan"), dtype=dt, device="cuda")
            rc = lib.fft3d_exec_c2r_noalloc(src.data_ptr(), out.data_ptr(), n0, n1, n2, code, stream)
        assert rc == fft3d.FFT3D_OK, fft3d.fft3d_strerror(rc)
        torch.cuda.synchronize()
        if not inplace:
            assert torch.equal(src, G), "input modified"
        outs.append(out.cpu().numpy().astype(np.float64))
    assert fft3d.fft3d_noalloc_status() == 0
    for o in outs:
        assert not np.isnan(o).any()
        assert rel_l2(o, ref) <= TOL[name]
        assert rel_l2(o, g_ref) <= TOL[name]


@pytest.mark.parametrize("shape", [(64, 48, 96), (16, 24, 12), (128, 128, 256), (2048, 8, 16), (4, 2048, 32),
                                   (1536, 8, 16), (512, 512, 16), (3, 3, 1024)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", ["f64", "f32"])
def test_noalloc_matches_plan_c2r(shape, name):
    _run(shape, name, inplace=False)


@pytest.mark.parametrize("name", ["f64", "f32"])
def test_noalloc_in_place(name):
    _run((32, 64, 48), name, inplace=True)


def test_noalloc_in_place_beyond_the_scratch_plane():
    """In place the scratch plane is not used, so N0 * N1 may exceed it
    (2048 * 1024 complex64 = 16 MiB > 8 MiB); the 2048-point x-pass runs on
    clusters of two blocks."""
    _run((2048, 1024, 8), "f32", inplace=True)


def test_noalloc_rejects_beyond_scratch():
    import torch
    import paper_2202_12756_gb300 as fft3d
    lib = fft3d.load_library()
    dummy = torch.empty(64, dtype=torch.float64, device="cuda")
    p, q = dummy.data_ptr(), dummy.data_ptr() + 256  # distinct: out of place
    # (the sizes are rejected before either pointer is looked at)
    # 2048 x 2048 complex64 = 32 MiB of scratch plane > the 8 MiB array
    assert lib.fft3d_exec_c2r_noalloc(p, q, 2048, 2048, 2, fft3d.FFT3D_F32, None) == fft3d.FFT3D_ERR_SIZE
    assert lib.fft3d_exec_c2r_noalloc(p, q, 1024, 1024, 2, fft3d.FFT3D_F64, None) == fft3d.FFT3D_ERR_SIZE
    assert lib.fft3d_exec_c2r_noalloc(p, p, 5, 8, 8, fft3d.FFT3D_F32, None) == fft3d.FFT3D_ERR_SIZE
    assert lib.fft3d_exec_c2r_noalloc(None, None, 8, 8, 8, fft3d.FFT3D_F32, None) == fft3d.FFT3D_ERR_NULL
