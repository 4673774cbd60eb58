"""Host model of the two-CTA column transform (colpass_pair_kernel).

A column of L points is split by row parity: CTA r holds x[2n + r], n < L/2,
and its thread j holds slots i with n = j + i NT (NT = L/2 / E threads per
column, E elements each).  Each CTA's L/2-point transform Y_r is taken as
given here (numpy); the test then replays the kernel's data flow slot by slot
and checks the result against the DFT of the column (radix-2 decimation in
time, Sec. 2's Cooley-Tukey splitting applied once):

* CTA 1 multiplies the slots it keeps (i >= H = E/2) by W_L^k, k = j + i NT,
  with W_L^k formed as the kernel forms it: the table value W_L^j times the
  constant exp(-pi i * slot / E);
* the CTAs swap halves thread to thread: CTA 0 sends slots i >= H, CTA 1
  slots i < H, into the partner's receive slot i - H or i;
* CTA 0 multiplies what it receives by W_L^k, k = j + i NT;
* each writes lo = y0 + y1 to row k and hi = y0 - y1 to row k + L/2, CTA 0 for
  k = j + i NT (i < H), CTA 1 for k = j + (H + i) NT.

The inverse runs the same flow on re/im-swapped data and swaps the result
back (the unnormalised inverse DFT).  Every output row must be written
exactly once.  Pure numpy: runs without a GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def pair_transform(x, E):
    L = x.shape[0]
    LH = L // 2
    NT = LH // E
    H = E // 2
    Y = [np.fft.fft(x[r::2]) for r in (0, 1)]  # each CTA's LH-point transform, slot (j, i) = Y[j + i NT]
    rot = np.exp(-2j * np.pi * np.arange(NT) / L)  # the table value W_L^j
    slot_tw = np.exp(-1j * np.pi * np.arange(E) / E)  # the compile-time constant of slot i
    out = np.full(L, np.nan + 1j * np.nan)
    written = np.zeros(L, dtype=int)
    for j in range(NT):
        v0 = np.array([Y[0][j + i * NT] for i in range(E)])
        v1 = np.array([Y[1][j + i * NT] for i in range(E)])
        v1[H:] = v1[H:] * (rot[j] * slot_tw[H:])  # CTA 1: its kept half times W_L^k
        rx0 = v1[:H].copy()   # CTA 1 -> CTA 0: slots i < H (untwiddled)
        rx1 = v0[H:].copy()   # CTA 0 -> CTA 1: slots i >= H, into receive slot i - H
        rx0 = rx0 * (rot[j] * slot_tw[:H])  # CTA 0: received half times W_L^k
        for i in range(H):
            for rank, (y0, y1) in enumerate(((v0[i], rx0[i]), (rx1[i], v1[H + i]))):
                k = j + (i + rank * H) * NT
                out[k] = y0 + y1
                out[k + LH] = y0 - y1
                written[k] += 1
                written[k + LH] += 1
    assert (written == 1).all(), "every row written exactly once"
    return out


def swap(z):
    return z.imag + 1j * z.real


@pytest.mark.parametrize("L,E", [(2048, 32), (1536, 24), (256, 8)])
def test_pair_flow_equals_dft(L, E):
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    ref = np.fft.fft(x)
    got = pair_transform(x, E)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    # inverse through swapped re / im on input and output
    inv = swap(pair_transform(swap(ref), E))
    assert np.linalg.norm(inv - L * x) <= 1e-12 * np.linalg.norm(L * x)


def test_pair_receive_buffer_fits_exchange_buffer():
    # the partner's half (H slots x W columns x NT threads of complex float)
    # lands in the split exchange buffer of the L/2-point transform, whose
    # rows are padded one in 32 plus one: (L/2 + L/64 + 1) rows x W floats
    for L, E in [(2048, 32), (1536, 24)]:
        W, LH = 16, L // 2
        NT, H = LH // E, E // 2
        rx_bytes = H * W * NT * 8
        ex_bytes = (LH + (LH >> 5) + 1) * W * 4
        assert rx_bytes <= ex_bytes, (L, rx_bytes, ex_bytes)
