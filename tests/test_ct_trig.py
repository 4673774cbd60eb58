"""Compile-time twiddle constants (`ct_cossin_pi` in csrc/line_plan.cuh).

The FP32 kernels multiply table twiddles by constants cos(pi p/q), sin(pi p/q)
that the compiler evaluates.  This host-only check compares them with the
long-double libm values for every angle pi p/q, |p| <= 2q, over the
denominators the kernels use and a few more: absolute error below 1e-15, and
the same float after rounding (the values the kernels actually use), except
at exact zeros where libm's long double leaves a residue of order 1e-20."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2202_12756_gb300", "csrc")

PROGRAM = r"""
#include "line_plan.cuh"
#include <cmath>
#include <cstdio>
int main()
{
    const long long qs[] = {1, 2, 3, 4, 5, 6, 7, 8, 12, 16, 24, 32, 48, 64, 96, 128, 256, 384, 512, 768,
                            1024, 1536, 2048, 3072, 4096};
    const long double pi = 3.14159265358979323846264338327950288L;
    double worst = 0.0;
    long long checked = 0, float_mismatch = 0;
    for (long long q : qs)
        for (long long p = -2 * q; p <= 2 * q; ++p) {
            const fft3d::CtCosSin r = fft3d::ct_cossin_pi(p, q);
            const long double th = pi * (long double)p / (long double)q;
            const long double c = cosl(th), s = sinl(th);
            const double e = fmax(fabs((double)(r.c - c)), fabs((double)(r.s - s)));
            if (e > worst) worst = e;
            if (((float)r.c != (float)c && fabsl(c) > 1e-12L) || ((float)r.s != (float)s && fabsl(s) > 1e-12L))
                ++float_mismatch;
            ++checked;
        }
    constexpr fft3d::CtCosSin k = fft3d::ct_cossin_pi(-3, 16);  // a constant expression
    static_assert(k.c > 0.8314 && k.c < 0.8315 && k.s < -0.5555 && k.s > -0.5556, "cos/sin(-3 pi / 16)");
    printf("%lld %.6e %lld\n", checked, worst, float_mismatch);
    return 0;
}
"""


def test_ct_cossin_pi_against_long_double(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "ct.cu"
    exe = tmp_path / "ct"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split()
    checked, worst, mismatch = int(out[0]), float(out[1]), int(out[2])
    assert checked > 40000
    assert worst < 1e-15, worst
    assert mismatch == 0
