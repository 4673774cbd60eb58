"""Seeded synthetic inputs shared by the tests and the bench.

This module holds no FFT arithmetic: it only draws random numbers and
evaluates closed-form fields on the grid.  Both the CUDA path and the FP64
oracle consume what it returns, so they see bit-identical inputs.

Every generator draws from ``numpy.random.default_rng(seed)`` (PCG64) in FP64;
FP32 runs round the FP64 field once.  Grid coordinates follow Sec. 2 of arXiv
2202.12756: the field is periodic on (2 pi)^3 with N points per axis, so
x_j = 2 pi j / N, and the last (fastest) axis is z.
"""
import numpy as np


def uniform_field(shape, seed):
    """iid uniform[-1, 1) real field in FP64."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=tuple(shape))


def eq5_field(n0, n1, n2):
    """Eq. 5 test field: 8 sin x sin 2y sin 3z + 8 sin 4x sin 5y sin 6z."""
    x = 2.0 * np.pi * np.arange(n0) / n0
    y = 2.0 * np.pi * np.arange(n1) / n1
    z = 2.0 * np.pi * np.arange(n2) / n2
    t1 = np.sin(x)[:, None, None] * np.sin(2 * y)[None, :, None] * np.sin(3 * z)[None, None, :]
    t2 = np.sin(4 * x)[:, None, None] * np.sin(5 * y)[None, :, None] * np.sin(6 * z)[None, None, :]
    return 8.0 * t1 + 8.0 * t2


def plane_wave_vectors(seed, count=8, kmax=256):
    """`count` random integer wave vectors with |k_i| < kmax (signed)."""
    rng = np.random.default_rng(seed)
    return rng.integers(-(kmax - 1), kmax, size=(count, 3))


def _cos_phase_1d(k, n):
    # exp(2 pi i k j / n) for j < n, with k j reduced mod n exactly
    p = (int(k) * np.arange(n, dtype=np.int64)) % n
    return np.exp(2j * np.pi * p / n)


def plane_waves(shape, kvecs):
    """sum over k of cos(2 pi (k0 j0/N0 + k1 j1/N1 + k2 j2/N2)), in FP64."""
    n0, n1, n2 = shape
    out = np.zeros(shape, dtype=np.float64)
    for k0, k1, k2 in kvecs:
        e0 = _cos_phase_1d(k0, n0)
        e1 = _cos_phase_1d(k1, n1)
        e2 = _cos_phase_1d(k2, n2)
        # cos(a + b + c) = Re(e^{ia} e^{ib} e^{ic}); one plane of axis 0 at a time
        e12 = e1[:, None] * e2[None, :]
        for j0 in range(n0):
            out[j0] += (e0[j0] * e12).real
    return out


def signed_wavenumbers(n):
    """k = idx for idx <= n/2, idx - n above, as integers (FFTW order)."""
    k = np.arange(n, dtype=np.int64)
    return np.where(k <= n // 2, k, k - n)


def turbulence_spectrum(n0, n1, n2, seed, kmin=1.0, kmax=None, slope=-11.0 / 6.0):
    """Half spectrum [n0][n1][n2//2+1] with random phases and |k|^slope amplitude.

    Amplitude |k|^(-11/6) on kmin <= |k| <= kmax (kmax defaults to N/2 of the
    smallest axis), zero elsewhere; phases iid uniform[0, 2 pi).  Signed
    wavenumbers on axes 0 and 1, k2 = 0..n2/2 on the halved axis.
    """
    if kmax is None:
        kmax = min(n0, n1, n2) // 2
    rng = np.random.default_rng(seed)
    m1 = n2 // 2 + 1
    k0 = signed_wavenumbers(n0).astype(np.float64)
    k1 = signed_wavenumbers(n1).astype(np.float64)
    k2 = np.arange(m1, dtype=np.float64)
    out = np.empty((n0, n1, m1), dtype=np.complex128)
    k12sq = k1[:, None] ** 2 + k2[None, :] ** 2
    chunk = max(1, (1 << 22) // (n1 * m1))
    for i in range(0, n0, chunk):
        c = min(chunk, n0 - i)
        kk = np.sqrt(k0[i:i + c, None, None] ** 2 + k12sq[None])
        inside = (kk >= kmin) & (kk <= kmax)
        amp = np.where(inside, np.power(np.where(inside, kk, 1.0), slope), 0.0)
        # phases drawn plane after plane in C order (same stream for any chunk)
        phase = rng.uniform(0.0, 2.0 * np.pi, size=(c, n1, m1))
        out[i:i + c].real = amp * np.cos(phase)
        out[i:i + c].imag = amp * np.sin(phase)
    return out


def random_half_spectrum(shape, seed):
    """iid complex normal half spectrum (not Hermitian-consistent on the edge planes)."""
    n0, n1, n2 = shape
    rng = np.random.default_rng(seed)
    m1 = n2 // 2 + 1
    return rng.standard_normal((n0, n1, m1)) + 1j * rng.standard_normal((n0, n1, m1))


def turbulence_spectrum_device(n0, n1, n2, seed, device, kmin=1.0, kmax=None, slope=-11.0 / 6.0):
    """Same recipe as ``turbulence_spectrum`` drawn on a CUDA device with
    torch's seeded generator (the values differ from the numpy stream; the
    distribution and structure are the same).  For timing runs, where a host
    draw of ~1e9 modes would dominate the set-up time."""
    import torch
    if kmax is None:
        kmax = min(n0, n1, n2) // 2
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    m1 = n2 // 2 + 1
    k0 = torch.as_tensor(signed_wavenumbers(n0), dtype=torch.float64, device=device)
    k1 = torch.as_tensor(signed_wavenumbers(n1), dtype=torch.float64, device=device)
    k2 = torch.arange(m1, dtype=torch.float64, device=device)
    out = torch.empty((n0, n1, m1), dtype=torch.complex128, device=device)
    k12sq = k1[:, None] ** 2 + k2[None, :] ** 2
    for i in range(n0):
        kk = torch.sqrt(k0[i] ** 2 + k12sq)
        inside = (kk >= kmin) & (kk <= kmax)
        amp = torch.where(inside, torch.where(inside, kk, torch.ones_like(kk)) ** slope, torch.zeros_like(kk))
        phase = torch.rand((n1, m1), generator=gen, dtype=torch.float64, device=device) * (2.0 * np.pi)
        out[i] = torch.polar(amp, phase)
    return out


def uniform_field_device(shape, seed, device, dtype=None, out=None):
    """iid uniform[-1, 1) field drawn on a CUDA device with torch's seeded
    generator (for grids too large to draw and ship from the host); `out`
    may be a strided view (e.g. the real part of a padded buffer)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    t = torch.empty(tuple(shape), dtype=dtype or torch.float64, device=device) if out is None else out
    t.uniform_(-1.0, 1.0, generator=gen)
    return t


def plane_waves_device(shape, kvecs, device, dtype=None, out=None):
    """sum over k of cos(2 pi (k0 j0/N0 + k1 j1/N1 + k2 j2/N2)) on a CUDA
    device, phases reduced mod N on integers before scaling."""
    import torch
    n0, n1, n2 = shape
    dtype = dtype or torch.float64
    out = torch.zeros(tuple(shape), dtype=dtype, device=device) if out is None else out
    j0 = torch.arange(n0, dtype=torch.int64, device=device)
    j1 = torch.arange(n1, dtype=torch.int64, device=device)
    j2 = torch.arange(n2, dtype=torch.int64, device=device)
    for k0, k1, k2 in kvecs:
        e0 = torch.exp(2j * np.pi * ((int(k0) * j0) % n0).to(torch.float64) / n0)
        e1 = torch.exp(2j * np.pi * ((int(k1) * j1) % n1).to(torch.float64) / n1)
        e2 = torch.exp(2j * np.pi * ((int(k2) * j2) % n2).to(torch.float64) / n2)
        e12 = e1[:, None] * e2[None, :]
        for i in range(n0):
            out[i] += (e0[i] * e12).real.to(dtype)
    return out
