"""Pins for the FP64 oracle: checks against facts fixed by the paper and by
mathematics, never against the oracle itself.

Each ``pin_*`` takes an oracle library handle and raises AssertionError when
the oracle disagrees.  ``test_oracle_pins.py`` runs them on the oracle;
``test_oracle_mutants.py`` runs them on copies of the oracle with a planted
mistake and requires that at least one pin fails for every mistake.

References are to arXiv 2202.12756: Eq. 1 (forward DFT), Eq. 2 (inverse DFT),
Eqs. 3-4 (Hermitian half spectrum), Eq. 5 (test field), Sec. 4 (round-trip
accuracy of 1e-14 in double precision, normalisation step).
"""
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

LD = np.longdouble


# ---------------------------------------------------------------- helpers
def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.linalg.norm((a - b).ravel())
    n = np.linalg.norm(np.asarray(b).ravel())
    return d / n if n > 0 else d


def brute_dft3(f, sign=-1):
    """Triple sum of Eq. 1 (sign -1) or Eq. 2 (sign +1, unnormalised), O(N^6),
    in long double; the phase (j.k/N) mod 1 is reduced on integers first."""
    n0, n1, n2 = f.shape
    big = n0 * n1 * n2
    j0, j1, j2 = np.meshgrid(np.arange(n0), np.arange(n1), np.arange(n2), indexing="ij")
    j0 = j0.ravel().astype(np.int64)
    j1 = j1.ravel().astype(np.int64)
    j2 = j2.ravel().astype(np.int64)
    fr = np.asarray(f).ravel()
    fre = fr.real.astype(LD)
    fim = fr.imag.astype(LD) if np.iscomplexobj(fr) else np.zeros_like(fre)
    out = np.empty((n0, n1, n2), dtype=np.complex128)
    two_pi = 2 * LD(np.pi)
    for k0 in range(n0):
        for k1 in range(n1):
            for k2 in range(n2):
                p = (j0 * k0 * n1 * n2 + j1 * k1 * n0 * n2 + j2 * k2 * n0 * n1) % big
                ang = two_pi * p.astype(LD) / LD(big)
                c = np.cos(ang)
                s = sign * np.sin(ang)
                re = np.sum(fre * c - fim * s)
                im = np.sum(fre * s + fim * c)
                out[k0, k1, k2] = complex(float(re), float(im))
    return out


def dft_matrix(n, sign=-1):
    """W[k, j] = exp(sign 2 pi i j k / n) in long double, index reduced mod n."""
    jk = (np.arange(n)[:, None] * np.arange(n)[None, :]) % n
    ang = 2 * LD(np.pi) * jk.astype(LD) / LD(n)
    return np.cos(ang), sign * np.sin(ang)


def apply_dft_axis(x_re, x_im, axis, sign=-1):
    """Apply the length-n DFT matrix along `axis` (long double)."""
    n = x_re.shape[axis]
    c, s = dft_matrix(n, sign)
    xr = np.moveaxis(x_re, axis, -1)
    xi = np.moveaxis(x_im, axis, -1)
    yr = xr @ c.T - xi @ s.T
    yi = xr @ s.T + xi @ c.T
    return np.moveaxis(yr, -1, axis), np.moveaxis(yi, -1, axis)


def separable_dft3(f, sign=-1):
    """Eq. 1 evaluated axis by axis with explicit DFT matrices (long double)."""
    fr = np.asarray(f)
    re = fr.real.astype(LD)
    im = fr.imag.astype(LD) if np.iscomplexobj(fr) else np.zeros_like(re)
    for ax in (2, 1, 0):
        re, im = apply_dft_axis(re, im, ax, sign)
    return re.astype(np.float64) + 1j * im.astype(np.float64)


def half(F):
    return F[:, :, : F.shape[2] // 2 + 1]


def hermitian_full(Fh, n2):
    """Full spectrum from a Hermitian-consistent half: F[k] = conj F[-k]."""
    n0, n1, _ = Fh.shape
    full = np.empty((n0, n1, n2), dtype=np.complex128)
    full[:, :, : n2 // 2 + 1] = Fh
    for k2 in range(n2 // 2 + 1, n2):
        src = Fh[:, :, n2 - k2]
        full[:, :, k2] = np.conj(src[(-np.arange(n0)) % n0][:, (-np.arange(n1)) % n1])
    return full


# ---------------------------------------------------------------- pins
def pin_dft4_golden(lib):
    """1D worked example: sign and (absent) forward normalisation of Eq. 1."""
    d = np.loadtxt(os.path.join(GOLDEN, "dft4_example.txt"))
    x = d[:, 1] + 1j * d[:, 2]
    X = d[:, 3] + 1j * d[:, 4]
    got = oracle.fft1d(x, -1, lib=lib)
    assert np.max(np.abs(got - X)) < 1e-14, got
    back = oracle.fft1d(X, +1, lib=lib) / 4
    assert np.max(np.abs(back - x)) < 1e-14, back


def pin_fft1d_brute(lib):
    """Oracle 1D C2C vs the DFT matrix at every supported kind of length."""
    rng = np.random.default_rng(11)
    lengths = list(range(1, 33)) + [48, 64, 96, 128, 192, 256, 384, 512, 768, 1024]
    for n in lengths:
        x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        for sign in (-1, +1):
            c, s = dft_matrix(n, sign)
            xr = x.real.astype(LD)
            xi = x.imag.astype(LD)
            ref = (c @ xr - s @ xi).astype(np.float64) + 1j * (s @ xr + c @ xi).astype(np.float64)
            got = oracle.fft1d(x, sign, lib=lib)
            assert rel(got, ref) < 1e-14, (n, sign, rel(got, ref))


def pin_rfft3_brute_triple_sum(lib):
    """Eq. 1 as a literal triple sum on tiny grids, kept half per Eqs. 3-4."""
    rng = np.random.default_rng(12)
    for shape in [(2, 2, 2), (4, 4, 4), (2, 4, 6), (3, 4, 6), (6, 6, 6), (4, 2, 8), (5, 3, 4)]:
        f = rng.uniform(-1, 1, shape)
        ref = half(brute_dft3(f, -1))
        got = oracle.rfft3(f, lib=lib)
        assert got.shape == ref.shape, (got.shape, ref.shape)
        assert rel(got, ref) < 1e-14, (shape, rel(got, ref))


def pin_rfft3_separable(lib):
    """Eq. 1 on larger non-cubic grids via per-axis DFT matrices (long double)."""
    rng = np.random.default_rng(13)
    for shape in [(8, 8, 8), (12, 12, 12), (16, 8, 24), (6, 16, 12), (24, 3, 10), (1, 5, 8)]:
        f = rng.uniform(-1, 1, shape)
        ref = half(separable_dft3(f, -1))
        got = oracle.rfft3(f, lib=lib)
        assert rel(got, ref) < 1e-14, (shape, rel(got, ref))


def pin_irfft3_brute(lib):
    """Eq. 2 on the Hermitian extension, times 1/N^3, as a literal triple sum."""
    rng = np.random.default_rng(14)
    for shape in [(4, 4, 4), (2, 4, 6), (3, 4, 6), (6, 6, 6), (4, 6, 8)]:
        f = rng.uniform(-1, 1, shape)
        Fh = half(brute_dft3(f, -1))          # a Hermitian-consistent half
        full = hermitian_full(Fh, shape[2])
        ref = brute_dft3(full, +1).real / np.prod(shape)
        got = oracle.irfft3(Fh, shape, lib=lib)
        assert rel(got, ref) < 1e-14, (shape, rel(got, ref))


def pin_irfft3_non_hermitian(lib):
    """Reading for a half spectrum that is not Hermitian-consistent: inverse
    C2C along axes 0 and 1 as is, then along axis 2 only the real parts of
    the k2 = 0 and k2 = N2/2 entries count.  Literal sums in long double."""
    rng = np.random.default_rng(15)
    for shape in [(4, 4, 4), (3, 2, 6), (2, 6, 8), (4, 4, 5)]:
        n0, n1, n2 = shape
        G = rng.standard_normal((n0, n1, n2 // 2 + 1)) + 1j * rng.standard_normal((n0, n1, n2 // 2 + 1))
        re, im = G.real.astype(LD), G.imag.astype(LD)
        re, im = apply_dft_axis(re, im, 0, +1)
        re, im = apply_dft_axis(re, im, 1, +1)
        # f[j] = Re Y0 + (-1)^j Re Y_{N/2} + 2 sum_{0<k<N/2} Re(Y_k e^{2 pi i j k / N})
        j = np.arange(n2)
        out = np.zeros((n0, n1, n2), dtype=LD)
        out += re[:, :, 0:1]
        top = (n2 - 1) // 2
        for k in range(1, top + 1):
            ang = 2 * LD(np.pi) * ((j * k) % n2).astype(LD) / LD(n2)
            out += 2 * (re[:, :, k:k + 1] * np.cos(ang) - im[:, :, k:k + 1] * np.sin(ang))
        if n2 % 2 == 0:
            out += re[:, :, n2 // 2:n2 // 2 + 1] * np.where(j % 2 == 0, 1, -1).astype(LD)
        ref = (out / LD(n0 * n1 * n2)).astype(np.float64)
        got = oracle.irfft3(G, shape, lib=lib)
        assert rel(got, ref) < 1e-14, (shape, rel(got, ref))


def pin_eq5_golden(lib):
    """Eq. 5 field at 16^3: closed-form half spectrum, and the round trip to
    1e-14 (the double-precision accuracy stated in Sec. 4)."""
    d = np.loadtxt(os.path.join(GOLDEN, "eq5_spectrum_n16.txt"))
    n = 16
    ref = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    for k0, k1, k2, re, im in d:
        ref[int(k0), int(k1), int(k2)] = re + 1j * im
    f = synth.eq5_field(n, n, n)
    got = oracle.rfft3(f, lib=lib)
    assert np.max(np.abs(got - ref)) < 1e-9, np.max(np.abs(got - ref))
    back = oracle.irfft3(got, (n, n, n), lib=lib)
    # Sec. 4 states the recovered field agrees "within 1e-14" without naming
    # a norm; read as the max-abs error relative to the field's peak (16).
    err = np.max(np.abs(back - f)) / np.max(np.abs(f))
    assert err < 1e-14, err


def pin_eq5_closed_form(lib):
    """Eq. 5 at 32^3 and 64^3: the eight coefficients i (+-1) N^3, zero elsewhere."""
    for n in (32, 64):
        f = synth.eq5_field(n, n, n)
        got = oracle.rfft3(f, lib=lib)
        ref = np.zeros_like(got)
        N3 = float(n) ** 3
        for (a0, a1, a2) in ((1, 2, 3), (4, 5, 6)):
            for s0 in (1, -1):
                for s1 in (1, -1):
                    ref[(s0 * a0) % n, (s1 * a1) % n, a2] = 1j * s0 * s1 * N3
        assert np.max(np.abs(got - ref)) < 1e-9 * N3, np.max(np.abs(got - ref))
        back = oracle.irfft3(got, (n, n, n), lib=lib)
        err = np.max(np.abs(back - f)) / np.max(np.abs(f))
        assert err < 1e-14, (n, err)


def plane_wave_spectrum(shape, kvecs):
    """Closed form: cos(2 pi k.j/N) -> N^3/2 at +k and at -k (mod N); only the
    images with k2 in the stored half appear (both when k2 = 0 or N2/2)."""
    n0, n1, n2 = shape
    N3 = float(n0 * n1 * n2)
    F = np.zeros((n0, n1, n2 // 2 + 1), dtype=np.complex128)
    for k in kvecs:
        for s in (1, -1):
            q0, q1, q2 = (s * k[0]) % n0, (s * k[1]) % n1, (s * k[2]) % n2
            if q2 <= n2 // 2:
                F[q0, q1, q2] += N3 / 2
    return F


def pin_plane_waves(lib):
    for shape, seed in (((32, 32, 32), 21), ((16, 24, 12), 22), ((64, 64, 64), 23)):
        kv = synth.plane_wave_vectors(seed, count=8, kmax=min(shape) // 2)
        kv = np.vstack([kv, [[0, 0, 0], [3, 0, 0], [0, 0, shape[2] // 2]]])
        f = synth.plane_waves(shape, kv)
        got = oracle.rfft3(f, lib=lib)
        ref = plane_wave_spectrum(shape, kv)
        scale = float(np.prod(shape))
        assert np.max(np.abs(got - ref)) < 1e-10 * scale, (shape, np.max(np.abs(got - ref)))


def pin_parseval(lib):
    """sum |f|^2 = (1/N^3) [sum_{k2 in {0, N2/2}} |F|^2 + 2 sum_{other k2} |F|^2]."""
    rng = np.random.default_rng(16)
    for shape in [(16, 16, 16), (12, 8, 6), (32, 16, 24)]:
        f = rng.uniform(-1, 1, shape)
        F = oracle.rfft3(f, lib=lib)
        n2 = shape[2]
        w = np.full(F.shape[2], 2.0)
        w[0] = 1.0
        if n2 % 2 == 0:
            w[n2 // 2] = 1.0
        lhs = np.sum(f * f)
        rhs = np.sum(w[None, None, :] * np.abs(F) ** 2) / np.prod(shape)
        assert abs(lhs - rhs) < 1e-13 * lhs, (shape, lhs, rhs)


def pin_invariants(lib):
    """Linearity, shift theorem on each axis, DC = sum f, Hermitian edge planes."""
    rng = np.random.default_rng(17)
    shape = (12, 16, 10)
    n0, n1, n2 = shape
    f = rng.uniform(-1, 1, shape)
    g = rng.uniform(-1, 1, shape)
    F = oracle.rfft3(f, lib=lib)
    G = oracle.rfft3(g, lib=lib)
    H = oracle.rfft3(2.5 * f - 0.75 * g, lib=lib)
    assert rel(H, 2.5 * F - 0.75 * G) < 1e-14
    assert abs(F[0, 0, 0] - np.sum(f)) < 1e-12
    # roll by one along axis a multiplies F by exp(-2 pi i k_a / N_a)
    for ax, n in enumerate(shape):
        Fs = oracle.rfft3(np.roll(f, 1, axis=ax), lib=lib)
        k = np.arange(F.shape[ax])
        ph = np.exp(-2j * np.pi * k / n)
        sh = [1, 1, 1]
        sh[ax] = -1
        assert rel(Fs, F * ph.reshape(sh)) < 1e-13, ax
    # k2 = 0 and k2 = N2/2 planes are Hermitian in (k0, k1)
    for k2 in (0, n2 // 2):
        P = F[:, :, k2]
        Pm = np.conj(P[(-np.arange(n0)) % n0][:, (-np.arange(n1)) % n1])
        assert rel(P, Pm) < 1e-14, k2


def pin_numpy_library(lib):
    """Library cross-check: numpy.fft (pocketfft) rfftn / irfftn in FP64."""
    rng = np.random.default_rng(18)
    for shape in [(32, 32, 32), (48, 24, 36), (64, 64, 64)]:
        f = rng.uniform(-1, 1, shape)
        F = oracle.rfft3(f, lib=lib)
        assert rel(F, np.fft.rfftn(f)) < 1e-14, shape
        G = synth.random_half_spectrum(shape, 5)
        assert rel(oracle.irfft3(G, shape, lib=lib), np.fft.irfftn(G, s=shape, axes=(0, 1, 2))) < 1e-14, shape


def pin_round_trip(lib):
    rng = np.random.default_rng(19)
    for shape in [(64, 64, 64), (96, 48, 24), (6, 12, 10)]:
        f = rng.uniform(-1, 1, shape)
        back = oracle.irfft3(oracle.rfft3(f, lib=lib), shape, lib=lib)
        assert np.max(np.abs(back - f)) < 1e-14, shape


def pin_adjoint_dot_products(lib):
    """Re<R2C x, G> = <x, R2C^T G> and <C2R X, g> = Re<X, C2R^T g> for any
    (not necessarily Hermitian) X, G; also R2C^T against a literal sum."""
    rng = np.random.default_rng(20)
    for shape in [(8, 6, 10), (16, 16, 16), (4, 12, 6)]:
        n0, n1, n2 = shape
        x = rng.uniform(-1, 1, shape)
        g = rng.uniform(-1, 1, shape)
        G = synth.random_half_spectrum(shape, 7)
        X = synth.random_half_spectrum(shape, 8)
        lhs = np.real(np.vdot(G, oracle.rfft3(x, lib=lib)))
        rhs = np.sum(x * oracle.rfft3_adjoint(G, shape, lib=lib))
        assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1), (shape, lhs, rhs)
        lhs = np.sum(g * oracle.irfft3(X, shape, lib=lib))
        rhs = np.real(np.vdot(oracle.irfft3_adjoint(g, lib=lib), X))
        assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1), (shape, lhs, rhs)
    # literal: g[j] = Re sum_{k in half} G[k] exp(+2 pi i k.j / N)
    shape = (4, 2, 6)
    G = synth.random_half_spectrum(shape, 9)
    full = np.zeros(shape, dtype=np.complex128)
    full[:, :, : shape[2] // 2 + 1] = G
    ref = brute_dft3(full, +1).real
    assert rel(oracle.rfft3_adjoint(G, shape, lib=lib), ref) < 1e-14


ALL_PINS = [
    pin_dft4_golden,
    pin_fft1d_brute,
    pin_rfft3_brute_triple_sum,
    pin_rfft3_separable,
    pin_irfft3_brute,
    pin_irfft3_non_hermitian,
    pin_eq5_golden,
    pin_eq5_closed_form,
    pin_plane_waves,
    pin_parseval,
    pin_invariants,
    pin_numpy_library,
    pin_round_trip,
    pin_adjoint_dot_products,
]
