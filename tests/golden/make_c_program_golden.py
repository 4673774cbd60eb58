"""Writes c_program_spectrum.txt: FP64 oracle values for the plain C program
of tests/test_gpu_c_program.py.

The program draws its 64 x 48 x 32 field with a 32-bit linear congruential
generator (s <- 1664525 s + 1013904223 mod 2^32, f = (s >> 8) / 2^24 - 0.5);
this script draws the same field (every value is a 24-bit integer over 2^24
minus 1/2, so FP32 holds it exactly and both of the program's runs see it),
transforms it with the oracle's R2C (Eq. 1, half spectrum per Eqs. 3-4) and
stores the energy sum |X|^2 of the whole half spectrum and 80 sampled entries
(every combination of a few k0, k1 and k2, including DC and the k2 = N2/2
plane).  It calls nothing but oracle/.

    python tests/golden/make_c_program_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle  # noqa: E402

N0, N1, N2 = 64, 48, 32
K0 = (0, 1, 31, 32, 63)
K1 = (0, 5, 24, 47)
K2 = (0, 1, 7, 16)


def lcg_field():
    n = N0 * N1 * N2
    out = np.empty(n, dtype=np.float64)
    s = 12345
    for i in range(n):
        s = (s * 1664525 + 1013904223) & 0xFFFFFFFF
        out[i] = (s >> 8) / 16777216.0 - 0.5
    return out.reshape(N0, N1, N2)


def main():
    f = lcg_field()
    assert np.array_equal(f.astype(np.float32).astype(np.float64), f)
    X = oracle.rfft3(f)
    lines = ["# FP64 oracle half spectrum of the C program's LCG field (see make_c_program_golden.py)",
             "# E sum|X|^2 over the half spectrum; then: k0 k1 k2 re im",
             f"E {float(np.sum(np.abs(X) ** 2)):.17g}"]
    for k0 in K0:
        for k1 in K1:
            for k2 in K2:
                x = X[k0, k1, k2]
                lines.append(f"{k0} {k1} {k2} {x.real:.17g} {x.imag:.17g}")
    with open(os.path.join(HERE, "c_program_spectrum.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
