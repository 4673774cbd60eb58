/*
 * FP64 CPU oracle for the 3D real-to-complex / complex-to-real FFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the tests, the smoke check and the bench's CPU-baseline leg
 * do.  It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (Sec. 2 of "Scalable Multi-node Fast Fourier Transform on
 * GPUs", arXiv 2202.12756):
 *
 *   forward  (Eq. 1):  F[k0][k1][k2] = sum_{j} f[j0][j1][j2]
 *                        * exp(-2 pi i (j0 k0/N0 + j1 k1/N1 + j2 k2/N2)),
 *                      unnormalised, kept for k2 = 0 .. N2/2 only (Eqs. 3-4:
 *                      a real field has a Hermitian spectrum, so half of it
 *                      is stored; the last, fastest axis is the halved one).
 *   inverse  (Eq. 2):  f[j] = (1/(N0 N1 N2)) sum_{k, all k2} Ft[k] exp(+2 pi i ...)
 *                      where Ft is the Hermitian extension of the stored half,
 *                      Ft[k0][k1][k2] = conj F[-k0][-k1][N2-k2] for k2 > N2/2.
 *                      The 1/N^3 factor is the separate normalisation step of
 *                      Sec. 4 (timing breakdown); the paper's Eq. 2 itself is
 *                      unnormalised.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - Inverse on a half spectrum that is not Hermitian-consistent: the inverse
 *     C2C transforms along axes 0 and 1 run as they are; along axis 2 only the
 *     real parts of the k2 = 0 and k2 = N2/2 entries are used.
 *   - The 3D transform is evaluated one axis at a time (axis 2, then 1, then
 *     0 for the forward; 0, 1, then 2 for the inverse), as in the paper's
 *     Sec. 3 steps; the triple sum factorises exactly this way.
 *
 * Algorithm for each 1D line: a plain recursive mixed-radix (2, 3, otherwise
 * direct) decimation-in-time Cooley-Tukey FFT.  Roots of unity are taken from
 * a table filled with cos/sin(2 pi p / n) after reducing p mod n exactly.
 * Lines along an axis are independent; OpenMP runs them in parallel.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORACLE_PI 3.14159265358979323846264338327950288

/* table[p] = exp(sign * 2 pi i p / n), p = 0 .. n-1 */
static cplx *root_table(long n, int sign)
{
    cplx *t = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!t) return NULL;
    for (long p = 0; p < n; ++p) {
        double a = 2.0 * ORACLE_PI * (double)p / (double)n;
        t[p] = cos(a) + (double)sign * I * sin(a);
    }
    return t;
}

/*
 * y[k] = sum_{j<n} x[j*stride] * W^(j k),  W = exp(sign 2 pi i / n), k < n.
 * `roots` is the root table of the top-level length `ntop`; this level's root
 * W^p is roots[(p * (ntop / n)) mod ntop].  `scratch` holds n entries.
 *
 * Cooley-Tukey split with radix r (the smallest of 2, 3 dividing n, else a
 * direct sum): with m = n / r and S_q the length-m transform of the
 * subsequence x[r j + q],
 *     y[k + s m] = sum_{q<r} W^(q (k + s m)) S_q[k],   k < m, s < r.
 */
static void fft_rec(const cplx *x, long stride, cplx *y, long n,
                    const cplx *roots, long ntop, cplx *scratch)
{
    long step = ntop / n;
    if (n == 1) {
        y[0] = x[0];
        return;
    }
    long r = (n % 2 == 0) ? 2 : ((n % 3 == 0) ? 3 : n);
    if (r == n) {
        /* direct DFT of a prime length (2 and 3 land here too) */
        for (long k = 0; k < n; ++k) {
            cplx acc = 0;
            for (long j = 0; j < n; ++j)
                acc += x[j * stride] * roots[((j * k) % n) * step];
            scratch[k] = acc;
        }
        memcpy(y, scratch, sizeof(cplx) * (size_t)n);
        return;
    }
    long m = n / r;
    for (long q = 0; q < r; ++q)
        fft_rec(x + q * stride, stride * r, y + q * m, m, roots, ntop, scratch);
    for (long k = 0; k < m; ++k) {
        for (long s = 0; s < r; ++s) {
            cplx acc = 0;
            for (long q = 0; q < r; ++q)
                acc += roots[((q * (k + s * m)) % n) * step] * y[q * m + k];
            scratch[k + s * m] = acc;
        }
    }
    memcpy(y, scratch, sizeof(cplx) * (size_t)n);
}

/*
 * In place C2C along one axis of a strided array:
 *   line l (l < howmany) starts at data[base(l)], element i at + i*stride,
 *   where base(l) = (l / inner) * outer_dist + (l % inner).
 * sign = -1 forward, +1 inverse (unnormalised).
 */
static int c2c_axis(cplx *data, long n, long howmany, long inner,
                    long outer_dist, long stride, int sign)
{
    cplx *roots = root_table(n, sign);
    if (!roots) return -1;
    int err = 0;
#pragma omp parallel
    {
        cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *scratch = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        if (!line || !out || !scratch) {
#pragma omp atomic write
            err = -1;
        } else {
#pragma omp for schedule(static)
            for (long l = 0; l < howmany; ++l) {
                cplx *p = data + (l / inner) * outer_dist + (l % inner);
                for (long i = 0; i < n; ++i) line[i] = p[i * stride];
                fft_rec(line, 1, out, n, roots, n, scratch);
                for (long i = 0; i < n; ++i) p[i * stride] = out[i];
            }
        }
        free(line);
        free(out);
        free(scratch);
    }
    free(roots);
    return err;
}

/* 1D C2C of `howmany` contiguous lines of length n (unnormalised). */
int oracle_fft1d(cplx *data, long n, long howmany, int sign)
{
    if (n < 1 || howmany < 0 || (sign != 1 && sign != -1)) return -2;
    return c2c_axis(data, n, howmany, 1, n, 1, sign);
}

/*
 * Forward 3D R2C (Eq. 1, half spectrum per Eqs. 3-4).
 *   f: real [n0][n1][n2], dense.   F: complex [n0][n1][n2/2+1].
 */
int oracle_rfft3(const double *f, long n0, long n1, long n2, cplx *F)
{
    if (n0 < 1 || n1 < 1 || n2 < 1) return -2;
    long m1 = n2 / 2 + 1;
    long lines = n0 * n1;
    cplx *roots = root_table(n2, -1);
    if (!roots) return -1;
    int err = 0;
    /* axis 2: real input line -> full complex DFT, keep k2 = 0 .. n2/2 */
#pragma omp parallel
    {
        cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)n2);
        cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)n2);
        cplx *scratch = (cplx *)malloc(sizeof(cplx) * (size_t)n2);
        if (!line || !out || !scratch) {
#pragma omp atomic write
            err = -1;
        } else {
#pragma omp for schedule(static)
            for (long l = 0; l < lines; ++l) {
                for (long i = 0; i < n2; ++i) line[i] = f[l * n2 + i];
                fft_rec(line, 1, out, n2, roots, n2, scratch);
                for (long k = 0; k < m1; ++k) F[l * m1 + k] = out[k];
            }
        }
        free(line);
        free(out);
        free(scratch);
    }
    free(roots);
    if (err) return err;
    /* axis 1: columns (j0, k2), rows k1 at stride m1 */
    if (c2c_axis(F, n1, n0 * m1, m1, n1 * m1, m1, -1)) return -1;
    /* axis 0: columns (k1, k2), rows k0 at stride n1*m1 */
    if (c2c_axis(F, n0, n1 * m1, n1 * m1, 0, n1 * m1, -1)) return -1;
    return 0;
}

/*
 * Inverse 3D C2R (Eq. 2 with the Hermitian extension, then x 1/(n0 n1 n2)).
 *   F: complex [n0][n1][n2/2+1] (read only).   f: real [n0][n1][n2], dense.
 */
int oracle_irfft3(const cplx *F, long n0, long n1, long n2, double *f)
{
    if (n0 < 1 || n1 < 1 || n2 < 1) return -2;
    long m1 = n2 / 2 + 1;
    long lines = n0 * n1;
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)(lines * m1));
    if (!work) return -1;
    memcpy(work, F, sizeof(cplx) * (size_t)(lines * m1));
    /* axis 0, then axis 1: inverse C2C */
    if (c2c_axis(work, n0, n1 * m1, n1 * m1, 0, n1 * m1, +1) ||
        c2c_axis(work, n1, n0 * m1, m1, n1 * m1, m1, +1)) {
        free(work);
        return -1;
    }
    cplx *roots = root_table(n2, +1);
    if (!roots) {
        free(work);
        return -1;
    }
    double scale = 1.0 / ((double)n0 * (double)n1 * (double)n2);
    int err = 0;
    /* axis 2: Hermitian extension of each line, inverse DFT, real part */
#pragma omp parallel
    {
        cplx *line = (cplx *)malloc(sizeof(cplx) * (size_t)n2);
        cplx *out = (cplx *)malloc(sizeof(cplx) * (size_t)n2);
        cplx *scratch = (cplx *)malloc(sizeof(cplx) * (size_t)n2);
        if (!line || !out || !scratch) {
#pragma omp atomic write
            err = -1;
        } else {
#pragma omp for schedule(static)
            for (long l = 0; l < lines; ++l) {
                const cplx *y = work + l * m1;
                line[0] = creal(y[0]);
                for (long k = 1; k < n2; ++k)
                    line[k] = (k <= n2 / 2) ? y[k] : conj(y[n2 - k]);
                if (n2 % 2 == 0) line[n2 / 2] = creal(y[n2 / 2]);
                fft_rec(line, 1, out, n2, roots, n2, scratch);
                for (long i = 0; i < n2; ++i) f[l * n2 + i] = creal(out[i]) * scale;
            }
        }
        free(line);
        free(out);
        free(scratch);
    }
    free(roots);
    free(work);
    return err;
}

/*
 * Adjoint of the forward R2C: for a cotangent G on the half spectrum (torch
 * convention G = dL/dRe F + i dL/dIm F),
 *     g[j] = Re sum_{k in half spectrum} G[k] exp(+2 pi i k.j/N).
 * Evaluated from that formula directly: G is placed in a full complex
 * spectrum (zero for k2 > n2/2), inverse 3D C2C (unnormalised), real part.
 */
int oracle_rfft3_adjoint(const cplx *G, long n0, long n1, long n2, double *g)
{
    if (n0 < 1 || n1 < 1 || n2 < 1) return -2;
    long m1 = n2 / 2 + 1;
    long total = n0 * n1 * n2;
    cplx *full = (cplx *)calloc((size_t)total, sizeof(cplx));
    if (!full) return -1;
    for (long l = 0; l < n0 * n1; ++l)
        for (long k = 0; k < m1; ++k) full[l * n2 + k] = G[l * m1 + k];
    if (c2c_axis(full, n2, n0 * n1, 1, n2, 1, +1) ||       /* axis 2 */
        c2c_axis(full, n1, n0 * n2, n2, n1 * n2, n2, +1) || /* axis 1 */
        c2c_axis(full, n0, n1 * n2, n1 * n2, 0, n1 * n2, +1)) { /* axis 0 */
        free(full);
        return -1;
    }
    for (long i = 0; i < total; ++i) g[i] = creal(full[i]);
    free(full);
    return 0;
}

/*
 * Adjoint of the normalised inverse C2R: for a real cotangent g,
 *     G[k] = (c(k2) / (n0 n1 n2)) * sum_j g[j] exp(-2 pi i k.j/N),
 * with c = 1 on the k2 = 0 plane (and on k2 = n2/2 when n2 is even) and
 * c = 2 elsewhere: every other stored entry stands for itself and its
 * Hermitian mirror in the inverse sum.
 */
int oracle_irfft3_adjoint(const double *g, long n0, long n1, long n2, cplx *G)
{
    long m1 = n2 / 2 + 1;
    int rc = oracle_rfft3(g, n0, n1, n2, G);
    if (rc) return rc;
    double scale = 1.0 / ((double)n0 * (double)n1 * (double)n2);
    for (long l = 0; l < n0 * n1; ++l)
        for (long k = 0; k < m1; ++k) {
            int edge = (k == 0) || (n2 % 2 == 0 && k == n2 / 2);
            G[l * m1 + k] *= (edge ? 1.0 : 2.0) * scale;
        }
    return 0;
}

/* number of OpenMP threads the oracle runs with */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
