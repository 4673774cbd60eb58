"""The C ABI from a plain C program (no Python, no torch): include/fft3d.h,
libfft3d.so and the CUDA runtime only.

The program plans a 64 x 48 x 32 transform in both dtypes, runs the forward
transform out of place and in place and the normalised inverse on cudaMalloc'd
buffers, and checks on the host: the spectrum against FP64 oracle values
(tests/golden/c_program_spectrum.txt, written by make_c_program_golden.py
beside it from the same generator: 80 sampled entries to relative L2 FP64
1e-13 / FP32 5e-6, and the energy of the whole half spectrum), the DC term
equals the sum of the field, the in-place spectrum equals the out-of-place
one bit for bit, and the round trip returns the field (FP64 1e-13, FP32 5e-6
relative L2).  It also checks the status codes of a few invalid calls."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <cuda_runtime.h>
#include "fft3d.h"

#define N0 64
#define N1 48
#define N2 32
#define M1 (N2 / 2 + 1)

static const char *golden_path;

/* relative L2 error of the sampled entries against the oracle values, and
 * the relative error of the energy sum |X|^2 of the whole half spectrum */
static int check_golden(const void *hX, int dtype, double tol)
{
    FILE *g = fopen(golden_path, "r");
    if (!g) return 30;
    char line[512];
    double e_ref = -1.0, num = 0.0, den = 0.0;
    int count = 0;
    while (fgets(line, sizeof line, g)) {
        if (line[0] == '#') continue;
        if (line[0] == 'E') {
            e_ref = strtod(line + 1, NULL);
            continue;
        }
        int k0, k1, k2;
        double re, im;
        if (sscanf(line, "%d %d %d %lf %lf", &k0, &k1, &k2, &re, &im) != 5) continue;
        const size_t i = ((size_t)k0 * N1 + k1) * M1 + k2;
        const double xr = dtype == FFT3D_F32 ? ((const float *)hX)[2 * i] : ((const double *)hX)[2 * i];
        const double xi = dtype == FFT3D_F32 ? ((const float *)hX)[2 * i + 1] : ((const double *)hX)[2 * i + 1];
        num += (xr - re) * (xr - re) + (xi - im) * (xi - im);
        den += re * re + im * im;
        ++count;
    }
    fclose(g);
    if (count != 80 || e_ref <= 0.0) return 31;
    double e = 0.0;
    for (size_t i = 0; i < 2 * (size_t)N0 * N1 * M1; ++i) {
        const double v = dtype == FFT3D_F32 ? ((const float *)hX)[i] : ((const double *)hX)[i];
        e += v * v;
    }
    const double rel = sqrt(num / den), erel = fabs(e - e_ref) / e_ref;
    printf("dtype %d vs oracle: sampled rel-L2 %.3e, energy %.3e\n", dtype, rel, erel);
    if (!(rel <= tol)) return 32;
    if (!(erel <= 4.0 * tol)) return 33;
    return 0;
}

static int run(int dtype, double tol)
{
    const size_t es = dtype == FFT3D_F32 ? 4 : 8, n = (size_t)N0 * N1 * N2, nc = (size_t)N0 * N1 * M1;
    double *f = (double *)malloc(n * sizeof(double));
    unsigned s = 12345u;
    double sum = 0.0;
    for (size_t i = 0; i < n; ++i) {
        s = s * 1664525u + 1013904223u;
        f[i] = (double)(s >> 8) / 16777216.0 - 0.5;
        if (dtype == FFT3D_F32) f[i] = (double)(float)f[i];
        sum += f[i];
    }
    void *h = malloc(2 * nc * es);
    for (size_t i = 0; i < n; ++i) {
        if (dtype == FFT3D_F32) ((float *)h)[i] = (float)f[i];
        else ((double *)h)[i] = f[i];
    }
    void *x, *X, *buf;
    if (cudaMalloc(&x, n * es) || cudaMalloc(&X, 2 * nc * es) || cudaMalloc(&buf, 2 * nc * es)) return 10;
    cudaMemcpy(x, h, n * es, cudaMemcpyHostToDevice);
    /* padded copy for the in-place transform */
    cudaMemcpy2D(buf, 2 * M1 * es, x, N2 * es, N2 * es, (size_t)N0 * N1, cudaMemcpyDeviceToDevice);

    fft3d_plan p = NULL;
    if (fft3d_plan_create(&p, N0, N1, N2, dtype) != FFT3D_OK) return 11;
    if (fft3d_exec_r2c(p, x, X, NULL) != FFT3D_OK) return 12;
    if (fft3d_exec_r2c(p, buf, buf, NULL) != FFT3D_OK) return 13;
    void *hX = malloc(2 * nc * es), *hB = malloc(2 * nc * es);
    cudaMemcpy(hX, X, 2 * nc * es, cudaMemcpyDeviceToHost);
    cudaMemcpy(hB, buf, 2 * nc * es, cudaMemcpyDeviceToHost);
    if (memcmp(hX, hB, 2 * nc * es) != 0) return 14;  /* in place == out of place */
    const int gr = check_golden(hX, dtype, tol);
    if (gr) return gr;
    const double dc = dtype == FFT3D_F32 ? (double)((float *)hX)[0] : ((double *)hX)[0];
    if (fabs(dc - sum) > tol * 100.0 * sqrt((double)n)) return 15;

    if (fft3d_exec_c2r(p, X, x, NULL) != FFT3D_OK) return 16;
    if (cudaDeviceSynchronize() != cudaSuccess) return 17;
    cudaMemcpy(h, x, n * es, cudaMemcpyDeviceToHost);
    double e2 = 0.0, r2 = 0.0;
    for (size_t i = 0; i < n; ++i) {
        const double y = dtype == FFT3D_F32 ? (double)((float *)h)[i] : ((double *)h)[i];
        e2 += (y - f[i]) * (y - f[i]);
        r2 += f[i] * f[i];
    }
    const double rel = sqrt(e2 / r2);
    printf("dtype %d round trip rel-L2 %.3e\n", dtype, rel);
    if (!(rel <= tol)) return 18;

    /* invalid calls return status codes */
    if (fft3d_exec_r2c(NULL, x, X, NULL) != FFT3D_ERR_NULL) return 19;
    if (fft3d_exec_r2c(p, (char *)x + 1, X, NULL) != FFT3D_ERR_ALIGN) return 20;
    if (fft3d_exec_c2r(p, X, (char *)X + es * 2, NULL) != FFT3D_ERR_LAYOUT) return 21;
    fft3d_plan q = NULL;
    if (fft3d_plan_create(&q, 5, N1, N2, dtype) != FFT3D_ERR_SIZE || q != NULL) return 22;

    fft3d_plan_destroy(p);
    cudaFree(x);
    cudaFree(X);
    cudaFree(buf);
    free(f);
    free(h);
    free(hX);
    free(hB);
    return 0;
}

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    golden_path = argv[1];
    int rc = run(FFT3D_F64, 1e-13);
    if (rc) {
        printf("f64 failed: %d\n", rc);
        return rc;
    }
    rc = run(FFT3D_F32, 5e-6);
    if (rc) printf("f32 failed: %d\n", rc);
    return rc;
}
"""


def test_c_program_through_the_abi(tmp_path):
    import paper_2202_12756_gb300 as fft3d
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lib = fft3d.LIB_PATH
    assert os.path.exists(lib), "build the library first"
    src = tmp_path / "prog.c"
    exe = tmp_path / "prog"
    src.write_text(PROGRAM)
    libdir = os.path.dirname(lib)
    subprocess.run([nvcc, "-x", "cu", "-O1", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lfft3d", f"-Xlinker=-rpath={libdir}"], check=True, capture_output=True,
                   timeout=300)
    golden = os.path.join(ROOT, "tests", "golden", "c_program_spectrum.txt")
    r = subprocess.run([str(exe), golden], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "dtype 1 round trip" in r.stdout and "dtype 0 round trip" in r.stdout
    assert "dtype 1 vs oracle" in r.stdout and "dtype 0 vs oracle" in r.stdout
