// Compile-time plan of one length-L complex line FFT, shared by the host
// (twiddle-table layout) and the kernels (stage structure).
//
// A line is transformed by NT = L / E cooperating threads that each hold E
// elements in registers: thread j holds x[j + i*NT], i < E.  The radix
// sequence R_0 .. R_{S-1} (product L, every R_s dividing E) is run as a
// Stockham autosort FFT: stage s combines R_s sub-transforms of length
// Ns = R_0 * .. * R_{s-1}, so the output comes out in natural order with no
// bit reversal.  Power-of-two lengths use radix min(E, 32) (then one smaller
// radix); 3 * 2^k lengths use one radix-3 stage followed by radix 8 (then
// smaller).
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

// largest power-of-two radix used with E elements per thread
__host__ __device__ constexpr int line_cap(int L, int E)
{
    return is_pow2(L) ? (E < 32 ? E : 32) : 8;
}

__host__ __device__ constexpr int line_nstages(int L, int E)
{
    int rem = L, s = 0;
    if (!is_pow2(L)) {
        rem /= 3;
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
        if (s == 0) return 3;
        rem /= 3;
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
