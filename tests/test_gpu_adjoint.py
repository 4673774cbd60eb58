"""Adjoint entry points and the autograd functions (the differentiation
workload: a spectrally weighted energy and a spectral x-derivative chain).

The library's adjoints (fft3d_exec_r2c_adjoint / fft3d_exec_c2r_adjoint) are
compared with the oracle's closed-form adjoints, and the gradients that the
autograd functions produce are compared with the same gradients assembled
from oracle calls and with central finite differences in FP64.
Gradients follow torch's convention for complex tensors:
G = dL/dRe + i dL/dIm."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, rel_l2, torch_dtype

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(8, 6, 12), (16, 16, 16), (4, 12, 6), (64, 32, 48), (32, 1024, 8),
                                   (4, 8, 2048), (4, 8, 1536), (3, 3, 1024)],
                         ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("name", ["f64", "f32"])
def test_adjoints_vs_oracle(shape, name):
    import torch
    import paper_2202_12756_gb300 as fft3d
    dt = torch_dtype(name)
    cdt = fft3d.complex_of(dt)
    plan = fft3d.get_plan(shape, dt, "cuda")
    G = synth.random_half_spectrum(shape, 51)
    g = synth.uniform_field(shape, 52)
    if name == "f32":
        G = G.astype(np.complex64).astype(np.complex128)
        g = g.astype(np.float32).astype(np.float64)
    out_r = plan.r2c_adjoint(torch.from_numpy(G).to(cdt).cuda())
    out_c = plan.c2r_adjoint(torch.from_numpy(g).to(dt).cuda())
    torch.cuda.synchronize()
    assert rel_l2(out_r.cpu().numpy(), oracle.rfft3_adjoint(G, shape)) <= TOL[name]
    assert rel_l2(out_c.cpu().numpy(), oracle.irfft3_adjoint(g)) <= TOL[name]


def test_adjoints_in_place():
    import torch
    import paper_2202_12756_gb300 as fft3d
    shape = (16, 24, 32)
    plan = fft3d.get_plan(shape, torch.float64, "cuda")
    G = synth.random_half_spectrum(shape, 53)
    buf = plan.empty_padded()
    buf.view(torch.complex128).copy_(torch.from_numpy(G))
    fft3d.fft3d_exec_r2c_adjoint(plan.handle, buf.data_ptr(), buf.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rel_l2(buf[..., :32].cpu().numpy(), oracle.rfft3_adjoint(G, shape)) <= TOL["f64"]


def test_autograd_gradcheck_small():
    import torch
    import paper_2202_12756_gb300 as fft3d
    x = torch.from_numpy(synth.uniform_field((4, 6, 8), 54)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: fft3d.rfft3(t), (x,), eps=1e-6, atol=1e-8, rtol=1e-6)
    X = torch.from_numpy(synth.random_half_spectrum((4, 6, 8), 55)).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: fft3d.irfft3(t, (4, 6, 8)), (X,), eps=1e-6, atol=1e-8, rtol=1e-6)


# ------------------------------------------------ the differentiation workload
def _weights(shape, device, dtype):
    """w(k) = exp(-|k|^2 / 64^2) on the stored half spectrum (signed k)."""
    import torch
    n0, n1, n2 = shape
    k0 = torch.as_tensor(synth.signed_wavenumbers(n0), dtype=dtype, device=device)
    k1 = torch.as_tensor(synth.signed_wavenumbers(n1), dtype=dtype, device=device)
    k2 = torch.arange(n2 // 2 + 1, dtype=dtype, device=device)
    ksq = k0[:, None, None] ** 2 + k1[None, :, None] ** 2 + k2[None, None, :] ** 2
    return torch.exp(-ksq / 64.0 ** 2)


def _kx(shape, device, dtype):
    """i k_x along axis 0, with k = 0 at the Nyquist index N0/2."""
    import torch
    n0 = shape[0]
    k = synth.signed_wavenumbers(n0).astype(np.float64)
    k[n0 // 2] = 0.0
    return torch.as_tensor(k, dtype=dtype, device=device)[:, None, None]


def workload_loss(f, fft3d):
    """L(f) = sum_k w(k) |F(k)|^2 / N^3 + sum_j (df/dx)_j^2 / N^3, with
    F = rfft3(f), df/dx = irfft3(i k_x F); sums over the stored half spectrum
    without Hermitian doubling."""
    shape = tuple(f.shape)
    N3 = float(np.prod(shape))
    F = fft3d.rfft3(f)
    w = _weights(shape, f.device, f.dtype)
    kx = _kx(shape, f.device, f.dtype)
    dfdx = fft3d.irfft3(1j * kx * F, shape)
    return (w * (F.real ** 2 + F.imag ** 2)).sum() / N3 + (dfdx ** 2).sum() / N3


def oracle_workload_grad(f):
    """The same gradient from oracle transforms and the closed-form adjoints."""
    shape = f.shape
    N3 = float(np.prod(shape))
    n0, n1, n2 = shape
    k0 = synth.signed_wavenumbers(n0).astype(np.float64)
    k1 = synth.signed_wavenumbers(n1).astype(np.float64)
    k2 = np.arange(n2 // 2 + 1, dtype=np.float64)
    w = np.exp(-(k0[:, None, None] ** 2 + k1[None, :, None] ** 2 + k2[None, None, :] ** 2) / 64.0 ** 2)
    kx = k0.copy()
    kx[n0 // 2] = 0.0
    kx = kx[:, None, None]
    F = oracle.rfft3(f)
    # term 1: dL/dF = 2 w F / N^3
    gF = 2.0 * w * F / N3
    # term 2: d = irfft3(i kx F); dL/dd = 2 d / N^3; dL/dX = irfft3^T(2 d / N^3);
    # X = i kx F  =>  dL/dF = conj(i kx) dL/dX
    d = oracle.irfft3(1j * kx * F, shape)
    gX = oracle.irfft3_adjoint(2.0 * d / N3)
    gF = gF + np.conj(1j * kx) * gX
    return oracle.rfft3_adjoint(gF, shape)


@pytest.mark.parametrize("name", ["f64", "f32"])
def test_workload_gradient_vs_oracle_256(name):
    """256^3 differentiation workload: autograd gradient through the library's
    adjoints against the oracle chain.  FP32 bar: four FP32 transforms in
    the chain, each within the 5e-6 transform bound -> 2e-5."""
    import torch
    import paper_2202_12756_gb300 as fft3d
    shape = (256, 256, 256)
    f = synth.uniform_field(shape, 3)
    if name == "f32":
        f = f.astype(np.float32).astype(np.float64)
    x = torch.from_numpy(f).to(torch_dtype(name)).cuda().requires_grad_(True)
    loss = workload_loss(x, fft3d)
    loss.backward()
    torch.cuda.synchronize()
    ref = oracle_workload_grad(f)
    tol = 1e-13 if name == "f64" else 2e-5
    assert rel_l2(x.grad.cpu().numpy(), ref) <= tol


def test_workload_gradient_finite_differences_256():
    """Central differences of the FP64 loss on 64 random voxels.

    The loss is a quadratic form in f, so central differences carry no
    truncation error: (L(f + h e) - L(f - h e)) / 2h equals the gradient up to
    rounding, whose size is about eps |L| log2(N^3) / h.  With the specified
    h = 1e-6 that bound (a few 1e-4 of the gradient here) is the bar; with
    h = 1e-2 the rounding term is 1e4 times smaller and the bar is 1e-6 of the
    gradient's RMS."""
    import torch
    import paper_2202_12756_gb300 as fft3d
    shape = (256, 256, 256)
    f = synth.uniform_field(shape, 3)
    x = torch.from_numpy(f).cuda().requires_grad_(True)
    loss = workload_loss(x, fft3d)
    loss.backward()
    grad = x.grad.detach()
    L = abs(loss.item())
    rms = grad.pow(2).mean().sqrt().item()
    rng = np.random.default_rng(60)
    idx = [tuple(int(rng.integers(0, n)) for n in shape) for _ in range(64)]
    eps = np.finfo(np.float64).eps
    with torch.no_grad():
        base = x.detach().clone()
        for h, bar in ((1e-6, None), (1e-2, 1e-6 * rms)):
            bound = 8 * eps * L * np.log2(np.prod(shape)) / (2 * h)
            limit = bound if bar is None else max(bar, bound)
            worst = 0.0
            for j in idx:
                base[j] += h
                lp = workload_loss(base, fft3d).item()
                base[j] -= 2 * h
                lm = workload_loss(base, fft3d).item()
                base[j] += h
                fd = (lp - lm) / (2 * h)
                worst = max(worst, abs(fd - grad[j].item()))
            print(f"FD h={h:g}: worst |fd - g| = {worst:.3e} (limit {limit:.3e}, gradient rms {rms:.3e})")
            assert worst <= limit, (h, worst, limit)
