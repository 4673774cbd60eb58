"""Host model of the two-lines-per-transform z-pass (zr2c_pairs / zc2r_pairs).

FP64 lines of N2 = N points run two real lines per complex transform of N
points: z[n] = x_l[n] + i x_{l+1}[n].  Thread j of a pair holds the slots
k = j + i NT (NT = N / E threads, E elements each) of Z = DFT_N(z), taken as
given here (numpy).  The test replays the kernels' index arithmetic slot by
slot and checks it against the definitions (Eqs. 1-4 along one axis):

* forward: for k <= M = N/2 the thread owning slot k writes
  X_l[k] = f (Z[k] + conj Z[N - k]) and X_{l+1}[k] = f (Z[k] - conj Z[N - k]) / i
  with f = scale_edge / 2 at k = 0 and M, scale_mid / 2 elsewhere (Z[N - k]
  read from its partner, Z[0] and Z[M] being their own mirrors); each output
  entry must be written exactly once and equal numpy's rfft times the scale;
* inverse: every slot k builds Z[k] = Xt_l[k] + i Xt_{l+1}[k] from the
  Hermitian extensions (X[k] for k <= M, conj X[N - k] above, only the real
  parts of the k = 0 and M entries, weighted by scale_edge), the inverse
  transform follows, and Re / Im go to the two lines times scale_mid; the
  result must equal the C2R definition on arbitrary (not Hermitian-consistent)
  half spectra, the reading the oracle takes.

An odd line count leaves the last pair's second line zero and unwritten.
Pure numpy: runs without a GPU."""
import numpy as np
import pytest


def forward_pairs(x, E, se=1.0, sm=1.0):
    """x: [lines][N] real; returns [lines][M + 1] complex as the kernel writes it."""
    lines, N = x.shape
    M, NT = N // 2, N // E
    out = np.full((lines, M + 1), np.nan + 1j * np.nan)
    written = np.zeros((lines, M + 1), dtype=int)
    for l0 in range(0, lines, 2):
        act1 = l0 + 1 < lines
        z = x[l0] + 1j * (x[l0 + 1] if act1 else 0.0)
        Z = np.fft.fft(z)
        for j in range(NT):
            for i in range(M // NT + 1):
                if not (i < M // NT or j == 0):
                    continue
                k = j + i * NT
                zk = Z[k]
                zm = zk if k in (0, M) else Z[N - k]
                f = 0.5 * (se if k in (0, M) else sm)
                out[l0, k] = f * ((zk.real + zm.real) + 1j * (zk.imag - zm.imag))
                written[l0, k] += 1
                if act1:
                    out[l0 + 1, k] = f * ((zk.imag + zm.imag) + 1j * (zm.real - zk.real))
                    written[l0 + 1, k] += 1
    return out, written


def inverse_pairs(X, N, E, we=1.0, s=1.0):
    """X: [lines][M + 1] complex half spectra; returns [lines][N] real lines."""
    lines = X.shape[0]
    M, NT = N // 2, N // E
    out = np.full((lines, N), np.nan)
    for l0 in range(0, lines, 2):
        act1 = l0 + 1 < lines
        Zs = np.zeros(N, dtype=complex)
        for j in range(NT):
            for i in range(E):
                k = j + i * NT
                idx = k if k <= M else N - k
                x0 = X[l0, idx]
                x1 = X[l0 + 1, idx] if act1 else 0.0
                if idx in (0, M):
                    x0, x1 = we * np.real(x0), we * np.real(x1)
                elif k > M:
                    x0, x1 = np.conj(x0), np.conj(x1)
                Zs[k] = x0 + 1j * x1
        z = np.fft.ifft(Zs) * N  # the unnormalised inverse the kernel computes
        out[l0] = s * z.real
        if act1:
            out[l0 + 1] = s * z.imag
    return out


def c2r_definition(X, N, we=1.0, s=1.0):
    """f[n] = s (we Re X[0] + we (-1)^n Re X[M] + 2 sum_{0<k<M} Re(X[k] e^{2 pi i k n / N}))."""
    M = N // 2
    n = np.arange(N)
    k = np.arange(1, M)
    out = []
    for row in X:
        mid = 2.0 * np.real(row[1:M][None, :] * np.exp(2j * np.pi * np.outer(n, k) / N)).sum(axis=1)
        out.append(s * (we * row[0].real + we * (-1.0) ** n * row[M].real + mid))
    return np.array(out)


@pytest.mark.parametrize("N,E,lines", [(1024, 16, 4), (1024, 16, 3), (1024, 16, 1), (64, 8, 5)])
@pytest.mark.parametrize("se,sm", [(1.0, 1.0), (0.25, 0.5)])
def test_forward_pairs_match_rfft(N, E, lines, se, sm):
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, size=(lines, N))
    out, written = forward_pairs(x, E, se, sm)
    assert (written == 1).all()  # every half-spectrum entry of every line exactly once
    ref = np.fft.rfft(x, axis=1)
    M = N // 2
    ref[:, 1:M] *= sm
    ref[:, [0, M]] *= se
    assert np.allclose(out, ref, rtol=0, atol=1e-11 * N)


@pytest.mark.parametrize("N,E,lines", [(1024, 16, 4), (1024, 16, 3), (64, 8, 5)])
@pytest.mark.parametrize("we,s", [(1.0, 1.0), (2.0, 0.5)])
def test_inverse_pairs_match_c2r_definition(N, E, lines, we, s):
    """Arbitrary half spectra: the imaginary parts of the k = 0 and M entries
    must not enter, and the rest follows the Hermitian extension."""
    rng = np.random.default_rng(8)
    M = N // 2
    X = rng.uniform(-1, 1, size=(lines, M + 1)) + 1j * rng.uniform(-1, 1, size=(lines, M + 1))
    out = inverse_pairs(X, N, E, we, s)
    assert not np.isnan(out).any()
    ref = c2r_definition(X, N, we, s)
    assert np.allclose(out, ref, rtol=0, atol=1e-10 * N)


def test_round_trip_of_paired_scheme():
    rng = np.random.default_rng(9)
    N, E = 1024, 16
    x = rng.uniform(-1, 1, size=(3, N))
    X, _ = forward_pairs(x, E)
    y = inverse_pairs(X, N, E, s=1.0 / N)
    assert np.allclose(y, x, rtol=0, atol=1e-12)
