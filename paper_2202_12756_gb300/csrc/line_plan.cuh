// Compile-time plan of one length-L complex line FFT, shared by the host
// (twiddle-table layout) and the kernels (stage structure).
//
// A line is transformed by NT = L / E cooperating threads that each hold E
// elements in registers: thread j holds x[j + i*NT], i < E.  The radix
// sequence R_0 .. R_{S-1} (product L, every R_s dividing E) is run as a
// Stockham autosort FFT: stage s combines R_s sub-transforms of length
// Ns = R_0 * .. * R_{s-1}, so the output comes out in natural order with no
// bit reversal.  Power-of-two lengths use radix 16 (then one smaller radix);
// 3 * 2^k lengths use one radix-3 stage followed by radix 8 (then smaller).
#pragma once

#include <stdint.h>

namespace fft3d {

__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

__host__ __device__ constexpr bool line_supported(int L)
{
    return L >= 1 && L <= 2048 && (is_pow2(L) || (L % 3 == 0 && is_pow2(L / 3) && L / 3 <= 512));
}

// elements per thread
__host__ __device__ constexpr int line_E(int L)
{
    return is_pow2(L) ? (L < 16 ? L : 16) : 3 * ((L / 3) < 8 ? (L / 3) : 8);
}

__host__ __device__ constexpr int line_NT(int L) { return L / line_E(L); }

__host__ __device__ constexpr int line_nstages(int L)
{
    int rem = L, s = 0;
    if (!is_pow2(L)) {
        rem /= 3;
        s = 1;
    }
    const int cap = is_pow2(L) ? 16 : 8;
    while (rem > 1) {
        const int r = rem < cap ? rem : cap;
        rem /= r;
        ++s;
    }
    return s;
}

__host__ __device__ constexpr int line_radix(int L, int s)
{
    int rem = L, i = 0;
    if (!is_pow2(L)) {
        if (s == 0) return 3;
        rem /= 3;
        i = 1;
    }
    const int cap = is_pow2(L) ? 16 : 8;
    while (rem > 1) {
        const int r = rem < cap ? rem : cap;
        if (i == s) return r;
        rem /= r;
        ++i;
    }
    return 1;
}

// Ns of stage s: product of the radices before it
__host__ __device__ constexpr int line_ns(int L, int s)
{
    int p = 1;
    for (int i = 0; i < s; ++i) p *= line_radix(L, i);
    return p;
}

// Stage s > 0 reads twiddles W_{Ns R}^{m k} (m = 1..R-1, k < Ns) from
// table[offset(s) + (m - 1) * Ns + k]; stage 0 needs none (all k = 0).
__host__ __device__ constexpr int line_tw_offset(int L, int s)
{
    int o = 0;
    for (int i = 1; i < s; ++i) o += (line_radix(L, i) - 1) * line_ns(L, i);
    return o;
}

__host__ __device__ constexpr int line_tw_size(int L) { return line_tw_offset(L, line_nstages(L)); }

}  // namespace fft3d
