// Compile-time plan of one length-L complex line FFT, shared by the host
// (twiddle-table layout) and the kernels (stage structure).
//
// A line is transformed by NT = L / E cooperating threads that each hold E
// elements in registers: thread j holds x[j + i*NT], i < E.  The radix
// sequence R_0 .. R_{S-1} (product L, every R_s dividing E) is run as a
// Stockham autosort FFT: stage s combines R_s sub-transforms of length
// Ns = R_0 * .. * R_{s-1}, so the output comes out in natural order with no
// bit reversal.  Power-of-two lengths use radix min(E, 32) (then one smaller
// radix); 3 * 2^k lengths start with one radix-24 (3 x 8) or radix-3 stage,
// followed by radix 8 (then smaller).
#pragma once

#include <stdint.h>

namespace fft3d {

__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

__host__ __device__ constexpr bool line_supported(int L)
{
    return L >= 1 && L <= 2048 && (is_pow2(L) || (L % 3 == 0 && is_pow2(L / 3) && L / 3 <= 512));
}

// default elements per thread: 16 for powers of two, 24 for 3 * 2^k
__host__ __device__ constexpr int line_E(int L)
{
    return is_pow2(L) ? (L < 16 ? L : 16) : 3 * ((L / 3) < 8 ? (L / 3) : 8);
}

__host__ __device__ constexpr int line_NT(int L) { return L / line_E(L); }

// First stage of a 3 * 2^k length: radix 24 (a 3 x 8 butterfly, one stage and
// one exchange fewer) when E and L allow it, else radix 3.
#ifndef FFT3D_RADIX24
#define FFT3D_RADIX24 1
#endif
__host__ __device__ constexpr int line_first3(int L, int E)
{
    return (FFT3D_RADIX24 && E % 24 == 0 && (L / 3) % 8 == 0) ? 24 : 3;
}

// largest power-of-two radix used with E elements per thread
__host__ __device__ constexpr int line_cap(int L, int E)
{
    return is_pow2(L) ? (E < 32 ? E : 32) : 8;
}

__host__ __device__ constexpr int line_nstages(int L, int E)
{
    int rem = L, s = 0;
    if (!is_pow2(L)) {
        rem /= line_first3(L, E);
        s = 1;
    }
    const int cap = line_cap(L, E);
    while (rem > 1) {
        const int r = rem < cap ? rem : cap;
        rem /= r;
        ++s;
    }
    return s;
}

__host__ __device__ constexpr int line_radix(int L, int E, int s)
{
    int rem = L, i = 0;
    if (!is_pow2(L)) {
        if (s == 0) return line_first3(L, E);
        rem /= line_first3(L, E);
        i = 1;
    }
    const int cap = line_cap(L, E);
    while (rem > 1) {
        const int r = rem < cap ? rem : cap;
        if (i == s) return r;
        rem /= r;
        ++i;
    }
    return 1;
}

// Ns of stage s: product of the radices before it
__host__ __device__ constexpr int line_ns(int L, int E, int s)
{
    int p = 1;
    for (int i = 0; i < s; ++i) p *= line_radix(L, E, i);
    return p;
}

// cos(pi p / q) and sin(pi p / q) evaluated by the compiler, for twiddle
// factors that are the same in every thread: the angle is reduced exactly
// (integer arithmetic) to [0, pi/4] by the symmetries of sin and cos, then
// both Maclaurin series are summed to the x^27 term in double (the remainder
// is below 1e-30 there).  Used only in constant expressions.
struct CtCosSin {
    double c, s;
};

__host__ __device__ constexpr CtCosSin ct_maclaurin(double x)
{
    const double x2 = x * x;
    double s = x, ts = x, c = 1.0, tc = 1.0;
    for (int k = 1; k <= 13; ++k) {
        ts *= -x2 / (double)((2 * k) * (2 * k + 1));
        tc *= -x2 / (double)((2 * k - 1) * (2 * k));
        s += ts;
        c += tc;
    }
    return CtCosSin{c, s};
}

__host__ __device__ constexpr CtCosSin ct_cossin_pi(long long p, long long q)
{
    long long n = p % (2 * q), d = q;
    if (n < 0) n += 2 * q;
    bool neg_c = false, neg_s = false, swap = false;
    if (n >= d) {  // theta - pi
        n -= d;
        neg_c = !neg_c;
        neg_s = !neg_s;
    }
    if (2 * n > d) {  // pi - theta
        n = d - n;
        neg_c = !neg_c;
    }
    if (4 * n > d) {  // pi/2 - theta = pi (d - 2n) / 2d
        n = d - 2 * n;
        d = 2 * d;
        swap = true;
    }
    const CtCosSin r = ct_maclaurin(3.141592653589793238 * (double)n / (double)d);
    const double c = swap ? r.s : r.c, s = swap ? r.c : r.s;
    return CtCosSin{neg_c ? -c : c, neg_s ? -s : s};
}

// Stage s > 0 reads twiddles W_{Ns R}^{m k} (m = 1..R-1, k < Ns) from
// table[offset(s) + (m - 1) * Ns + k]; stage 0 needs none (all k = 0).
__host__ __device__ constexpr int line_tw_offset(int L, int E, int s)
{
    int o = 0;
    for (int i = 1; i < s; ++i) o += (line_radix(L, E, i) - 1) * line_ns(L, E, i);
    return o;
}

__host__ __device__ constexpr int line_tw_size(int L, int E) { return line_tw_offset(L, E, line_nstages(L, E)); }

// every radix divides E (so each thread runs whole butterflies)
__host__ __device__ constexpr bool line_plan_valid(int L, int E)
{
    if (E < 1 || L % E != 0) return false;
    for (int s = 0; s < line_nstages(L, E); ++s)
        if (E % line_radix(L, E, s) != 0) return false;
    return true;
}

}  // namespace fft3d
