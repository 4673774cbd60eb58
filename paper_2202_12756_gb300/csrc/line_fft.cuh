// Register-resident Stockham line FFT: complex helpers, radix-2/3/4/8/16
// butterflies and the stage engine used by every pass kernel.
//
// All butterflies compute the forward DFT y[k] = sum_n a[n] exp(-2 pi i n k / R)
// (Eq. 1's sign).  Inverse transforms reuse them through
// IDFT(x) = conj(DFT(conj(x))) = swap(DFT(swap(x))), swap exchanging the real
// and imaginary parts, applied when a pass loads and stores.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "line_plan.cuh"

namespace fft3d {

template <typename R> struct cvec;
template <> struct cvec<float> { typedef float2 T; };
template <> struct cvec<double> { typedef double2 T; };

template <typename C> __device__ __forceinline__ C cmake(decltype(C::x) x, decltype(C::x) y)
{
    C r;
    r.x = x;
    r.y = y;
    return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b)
{
    return cmake<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// -i * a
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { return cmake<C>(a.y, -a.x); }
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmake<C>(a.x, -a.y); }
// (re, im) -> (im, re); swap(DFT(swap(x))) is the unnormalised inverse DFT
template <typename C> __device__ __forceinline__ C cswap(C a) { return cmake<C>(a.y, a.x); }
template <typename C> __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return cmake<C>(a.x * s, a.y * s); }

// cos(pi/8), sin(pi/8), sqrt(1/2), sqrt(3)/2
#define FFT3D_C8 0.923879532511286756128183189396788933
#define FFT3D_S8 0.382683432365089771728459984030398866
#define FFT3D_R2 0.707106781186547524400844362104849039
#define FFT3D_S3 0.866025403784438646763723170752936183

template <int R, typename C> struct Dft;

template <typename C> struct Dft<1, C> {
    __device__ __forceinline__ static void run(C *) {}
};

template <typename C> struct Dft<2, C> {
    __device__ __forceinline__ static void run(C *a)
    {
        const C t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    }
};

template <typename C> struct Dft<3, C> {
    __device__ __forceinline__ static void run(C *a)
    {
        typedef decltype(C::x) R;
        const C t = cadd(a[1], a[2]);
        const C u = csub(a[1], a[2]);
        const C m = cmake<C>(a[0].x - R(0.5) * t.x, a[0].y - R(0.5) * t.y);
        // -i * (sqrt(3)/2) * u
        const C v = cmake<C>(R(FFT3D_S3) * u.y, -R(FFT3D_S3) * u.x);
        a[0] = cadd(a[0], t);
        a[1] = cadd(m, v);
        a[2] = csub(m, v);
    }
};

template <typename C> __device__ __forceinline__ void dft4(C &a0, C &a1, C &a2, C &a3)
{
    const C t0 = cadd(a0, a2);
    const C t1 = csub(a0, a2);
    const C t2 = cadd(a1, a3);
    const C t3 = cmul_mi(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

template <typename C> struct Dft<4, C> {
    __device__ __forceinline__ static void run(C *a) { dft4(a[0], a[1], a[2], a[3]); }
};

// z * exp(-2 pi i / 8) = z (1 - i) / sqrt 2
template <typename C> __device__ __forceinline__ C w8_1(C z)
{
    typedef decltype(C::x) R;
    return cmake<C>(R(FFT3D_R2) * (z.x + z.y), R(FFT3D_R2) * (z.y - z.x));
}
// z * exp(-2 pi i 3 / 8) = z (-1 - i) / sqrt 2
template <typename C> __device__ __forceinline__ C w8_3(C z)
{
    typedef decltype(C::x) R;
    return cmake<C>(R(FFT3D_R2) * (z.y - z.x), -R(FFT3D_R2) * (z.x + z.y));
}

template <typename C> struct Dft<8, C> {
    // radix 2 x 4: even and odd halves, then one layer of radix-2
    __device__ __forceinline__ static void run(C *a)
    {
        C e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
        C o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
        dft4(e0, e1, e2, e3);
        dft4(o0, o1, o2, o3);
        o1 = w8_1(o1);
        o2 = cmul_mi(o2);
        o3 = w8_3(o3);
        a[0] = cadd(e0, o0);
        a[4] = csub(e0, o0);
        a[1] = cadd(e1, o1);
        a[5] = csub(e1, o1);
        a[2] = cadd(e2, o2);
        a[6] = csub(e2, o2);
        a[3] = cadd(e3, o3);
        a[7] = csub(e3, o3);
    }
};

template <typename C> struct Dft<16, C> {
    // radix 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2;
    // y[k1 + 4 k2] = sum_{n2} W16^{n2 k1} W4^{n2 k2} sum_{n1} a[4 n1 + n2] W4^{n1 k1}
    __device__ __forceinline__ static void run(C *a)
    {
        typedef decltype(C::x) R;
        dft4(a[0], a[4], a[8], a[12]);
        dft4(a[1], a[5], a[9], a[13]);
        dft4(a[2], a[6], a[10], a[14]);
        dft4(a[3], a[7], a[11], a[15]);
        // a[n2 + 4 k1] now holds the inner sum for (n2, k1); twiddle by W16^{n2 k1}
        const C w1 = cmake<C>(R(FFT3D_C8), -R(FFT3D_S8));
        const C w3 = cmake<C>(R(FFT3D_S8), -R(FFT3D_C8));
        const C w9 = cmake<C>(-R(FFT3D_C8), R(FFT3D_S8));
        a[5] = cmul(a[5], w1);     // n2=1, k1=1
        a[9] = w8_1(a[9]);         // n2=1, k1=2 : W16^2
        a[13] = cmul(a[13], w3);   // n2=1, k1=3
        a[6] = w8_1(a[6]);         // n2=2, k1=1 : W16^2
        a[10] = cmul_mi(a[10]);    // n2=2, k1=2 : W16^4
        a[14] = w8_3(a[14]);       // n2=2, k1=3 : W16^6
        a[7] = cmul(a[7], w3);     // n2=3, k1=1
        a[11] = w8_3(a[11]);       // n2=3, k1=2 : W16^6
        a[15] = cmul(a[15], w9);   // n2=3, k1=3
        dft4(a[0], a[1], a[2], a[3]);
        dft4(a[4], a[5], a[6], a[7]);
        dft4(a[8], a[9], a[10], a[11]);
        dft4(a[12], a[13], a[14], a[15]);
        // a[4 k1 + k2] holds y[k1 + 4 k2]: transpose the 4x4 index
        C t;
        t = a[1]; a[1] = a[4]; a[4] = t;
        t = a[2]; a[2] = a[8]; a[8] = t;
        t = a[3]; a[3] = a[12]; a[12] = t;
        t = a[6]; a[6] = a[9]; a[9] = t;
        t = a[7]; a[7] = a[13]; a[13] = t;
        t = a[11]; a[11] = a[14]; a[14] = t;
    }
};

// z * (cr + i ci) for a compile-time constant root of unity
template <typename C> __device__ __forceinline__ C cmulk(C z, double cr, double ci)
{
    typedef decltype(C::x) R;
    return cmake<C>(z.x * R(cr) - z.y * R(ci), z.x * R(ci) + z.y * R(cr));
}

// cos(pi/16), sin(pi/16), cos(3 pi/16), sin(3 pi/16)
#define FFT3D_C16 0.980785280403230449126182236134239037
#define FFT3D_S16 0.195090322016128267848284868477022240
#define FFT3D_C316 0.831469612302545237078788377617905756
#define FFT3D_S316 0.555570233019602224742830813948532874

template <typename C> struct Dft<32, C> {
    // radix 2 x 16: y[k] = E[k] + W32^k O[k], y[k + 16] = E[k] - W32^k O[k]
    __device__ __forceinline__ static void run(C *a)
    {
        C e[16], o[16];
#pragma unroll
        for (int n = 0; n < 16; ++n) {
            e[n] = a[2 * n];
            o[n] = a[2 * n + 1];
        }
        Dft<16, C>::run(e);
        Dft<16, C>::run(o);
        // W32^k = exp(-2 pi i k / 32), k = 1..15
        o[1] = cmulk(o[1], FFT3D_C16, -FFT3D_S16);
        o[2] = cmulk(o[2], FFT3D_C8, -FFT3D_S8);
        o[3] = cmulk(o[3], FFT3D_C316, -FFT3D_S316);
        o[4] = w8_1(o[4]);
        o[5] = cmulk(o[5], FFT3D_S316, -FFT3D_C316);
        o[6] = cmulk(o[6], FFT3D_S8, -FFT3D_C8);
        o[7] = cmulk(o[7], FFT3D_S16, -FFT3D_C16);
        o[8] = cmul_mi(o[8]);
        o[9] = cmulk(o[9], -FFT3D_S16, -FFT3D_C16);
        o[10] = cmulk(o[10], -FFT3D_S8, -FFT3D_C8);
        o[11] = cmulk(o[11], -FFT3D_S316, -FFT3D_C316);
        o[12] = w8_3(o[12]);
        o[13] = cmulk(o[13], -FFT3D_C316, -FFT3D_S316);
        o[14] = cmulk(o[14], -FFT3D_C8, -FFT3D_S8);
        o[15] = cmulk(o[15], -FFT3D_C16, -FFT3D_S16);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            a[k] = cadd(e[k], o[k]);
            a[k + 16] = csub(e[k], o[k]);
        }
    }
};

// z * exp(-2 pi i p / 24) for a compile-time p; the multiples of 3 are
// cheaper (W8 rotations, -i, -1).
template <int P, typename C> __device__ __forceinline__ C w24(C z)
{
    constexpr int p = P % 24;
    if constexpr (p == 0) {
        return z;
    } else if constexpr (p == 3) {
        return w8_1(z);
    } else if constexpr (p == 6) {
        return cmul_mi(z);
    } else if constexpr (p == 9) {
        return w8_3(z);
    } else if constexpr (p == 12) {
        return cmake<C>(-z.x, -z.y);
    } else {
        constexpr CtCosSin w = ct_cossin_pi(-2LL * p, 24);
        return cmulk(z, w.c, w.s);
    }
}

template <typename C> struct Dft<24, C> {
    // radix 8 x 3: n = 3 n1 + n2, k = k1 + 8 k2;
    // y[k1 + 8 k2] = sum_{n2} W3^{n2 k2} W24^{n2 k1} sum_{n1} a[3 n1 + n2] W8^{n1 k1}
    __device__ __forceinline__ static void run(C *a)
    {
        C b0[8], b1[8], b2[8];
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) {
            b0[n1] = a[3 * n1];
            b1[n1] = a[3 * n1 + 1];
            b2[n1] = a[3 * n1 + 2];
        }
        Dft<8, C>::run(b0);
        Dft<8, C>::run(b1);
        Dft<8, C>::run(b2);
        b1[1] = w24<1>(b1[1]);
        b1[2] = w24<2>(b1[2]);
        b1[3] = w24<3>(b1[3]);
        b1[4] = w24<4>(b1[4]);
        b1[5] = w24<5>(b1[5]);
        b1[6] = w24<6>(b1[6]);
        b1[7] = w24<7>(b1[7]);
        b2[1] = w24<2>(b2[1]);
        b2[2] = w24<4>(b2[2]);
        b2[3] = w24<6>(b2[3]);
        b2[4] = w24<8>(b2[4]);
        b2[5] = w24<10>(b2[5]);
        b2[6] = w24<12>(b2[6]);
        b2[7] = w24<14>(b2[7]);
#pragma unroll
        for (int k1 = 0; k1 < 8; ++k1) {
            C t[3] = {b0[k1], b1[k1], b2[k1]};
            Dft<3, C>::run(t);
            a[k1] = t[0];
            a[k1 + 8] = t[1];
            a[k1 + 16] = t[2];
        }
    }
};

// Stockham stage s of a length-L line, E elements per thread.  Thread j holds
// v[i] = x[j + i NT].  Butterfly b = j + q NT (q < E / R) combines
// x[b + m L/R], m < R, which are v[q + m E/R]; with k = b mod Ns it applies
// W_{Ns R}^{m k} and a radix-R DFT.  Its outputs belong at
// y[(b / Ns) Ns R + k + m Ns]; they are left in the input slots and the
// exchange (for every stage but the last) moves them to their owners.  The
// last stage's output slots coincide with its input slots (natural order).
// Twiddle read: read-only global path, or a plain load when the table was
// copied to shared memory (TWS).
template <bool TWS, typename C> __device__ __forceinline__ C tw_read(const C *__restrict__ tw, int i)
{
    if constexpr (TWS) return tw[i];
    else return __ldg(tw + i);
}

// Compile-time loop: f(IntC<I>()) for I = B .. N-1.
template <int I> struct IntC {
    static constexpr int value = I;
};
template <int B, int N, class F> __device__ __forceinline__ void static_for(const F &f)
{
    if constexpr (B < N) {
        f(IntC<B>());
        static_for<B + 1, N>(f);
    }
}

#ifndef FFT3D_TWCONST
#define FFT3D_TWCONST 1
#endif

template <typename R, int L, int E, int S, bool TWS = false>
__device__ __forceinline__ void line_stage_compute(typename cvec<R>::T *v, int j,
                                                   const typename cvec<R>::T *__restrict__ tw)
{
    typedef typename cvec<R>::T C;
    constexpr int NT = L / E;
    constexpr int RS = line_radix(L, E, S);
    constexpr int NS = line_ns(L, E, S);
    constexpr int Q = E / RS;
    constexpr int TWO = line_tw_offset(L, E, S);
    static_assert(E % RS == 0, "radix must divide the elements per thread");
    if constexpr (FFT3D_TWCONST && sizeof(R) == 4 && S > 0 && Q > 1 && NS % NT == 0) {
        // Butterfly q of this thread has k = j + c_q, c_q = (q NT) mod Ns, so
        // W^{m k} = W^{m j} W^{m c_q}: the R - 1 factors W^{m j} come from the
        // table once, the W^{m c_q} (W = exp(-2 pi i / (Ns R))) are constants.
        C base[RS];
#pragma unroll
        for (int m = 1; m < RS; ++m) base[m] = tw_read<TWS>(tw, TWO + (m - 1) * NS + j);
        static_for<0, Q>([&](auto QI) {
            constexpr int q = decltype(QI)::value;
            constexpr int cq = (q * NT) % NS;
            C t[RS];
#pragma unroll
            for (int m = 0; m < RS; ++m) t[m] = v[q + m * Q];
            static_for<1, RS>([&](auto MI) {
                constexpr int m = decltype(MI)::value;
                if constexpr (cq == 0) {
                    t[m] = cmul(t[m], base[m]);
                } else {
                    constexpr CtCosSin w = ct_cossin_pi(-2LL * m * cq, (long long)NS * RS);
                    t[m] = cmul(t[m], cmul(base[m], cmake<C>(R(w.c), R(w.s))));
                }
            });
            Dft<RS, C>::run(t);
#pragma unroll
            for (int m = 0; m < RS; ++m) v[q + m * Q] = t[m];
        });
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int b = j + q * NT;
            const int k = b % NS;
            C t[RS];
#pragma unroll
            for (int m = 0; m < RS; ++m) t[m] = v[q + m * Q];
            if (S > 0) {
#pragma unroll
                for (int m = 1; m < RS; ++m) t[m] = cmul(t[m], tw_read<TWS>(tw, TWO + (m - 1) * NS + k));
            }
            Dft<RS, C>::run(t);
#pragma unroll
            for (int m = 0; m < RS; ++m) v[q + m * Q] = t[m];
        }
    }
}

struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Exchange objects address a line's (or column's) buffer by row.  A padded
// buffer (kPadShift = P >= 0) stores row r at r + (r >> P); the padding keeps
// strided writes free of bank conflicts.  A row is passed as base + off with
// `off` known at compile time; when (base mod 2^P) + (off mod 2^P) < 2^P for
// every use (LIN), pad(base + off) = pad(base) + off + (off >> P), so the
// per-element address is a constant offset from a per-thread base.
template <int P> __host__ __device__ constexpr bool pad_linear(int ns, int rs)
{
    return P < 0 || ns % (1 << P) == 0 || (ns == 1 && rs % (1 << P) == 0);
}
template <int P> __host__ __device__ constexpr bool pad_linear_reads(int nt)
{
    return P < 0 || nt % (1 << P) == 0 || (1 << P) % nt == 0;
}
template <int P, bool LIN> __device__ __forceinline__ int pad_row(int base, int off)
{
    if constexpr (P < 0) return base + off;
    else if constexpr (LIN) return base + (base >> P) + off + (off >> P);
    else return base + off + ((base + off) >> P);
}

// Exchange after stage S: slot q + m Q (butterfly b = j + q NT, output m)
// goes to row (b / Ns) Ns R + (b mod Ns) + m Ns; thread j then reads rows
// j + i NT.  `hook` runs once, right after the first barrier (when every
// thread's earlier shared-memory reads have completed).
template <typename R, int L, int E, int S, class Ex, class Hook>
__device__ __forceinline__ void line_exchange(typename cvec<R>::T *v, int j, Ex &ex, const Hook &hook)
{
    constexpr int NT = L / E;
    constexpr int RS = line_radix(L, E, S);
    constexpr int NS = line_ns(L, E, S);
    constexpr int Q = E / RS;
    constexpr int P = Ex::kPadShift;
    constexpr bool LW = pad_linear<P>(NS, RS);
    constexpr bool LR = pad_linear_reads<P>(NT);
    int base[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = j + q * NT;
        base[q] = (b / NS) * NS * RS + (b % NS);
    }
    if constexpr (Ex::kSplit) {
        // real parts, then imaginary parts, through a buffer of half the size
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int m = 0; m < RS; ++m) ex.put_real(pad_row<P, LW>(base[q], m * NS), v[q + m * Q].x);
        ex.sync();
        hook();
#pragma unroll
        for (int i = 0; i < E; ++i) v[i].x = ex.get_real(pad_row<P, LR>(j, i * NT));
        ex.sync();
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int m = 0; m < RS; ++m) ex.put_real(pad_row<P, LW>(base[q], m * NS), v[q + m * Q].y);
        ex.sync();
#pragma unroll
        for (int i = 0; i < E; ++i) v[i].y = ex.get_real(pad_row<P, LR>(j, i * NT));
        ex.sync();
    } else {
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int m = 0; m < RS; ++m) ex.put(pad_row<P, LW>(base[q], m * NS), v[q + m * Q]);
        ex.sync();
        hook();
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = ex.get(pad_row<P, LR>(j, i * NT));
        ex.sync();
    }
}

template <typename R, int L, int E, int S, bool TWS, class Ex, class Hook, class Tail>
__device__ __forceinline__ void line_stages_from(typename cvec<R>::T *v, int j,
                                                 const typename cvec<R>::T *__restrict__ tw, Ex &ex,
                                                 const Hook &hook, const Tail &tail)
{
    if constexpr (S < line_nstages(L, E)) {
        line_stage_compute<R, L, E, S, TWS>(v, j, tw);
        if constexpr (S + 1 < line_nstages(L, E)) {
            if constexpr (S == 0) line_exchange<R, L, E, S>(v, j, ex, hook);
            else line_exchange<R, L, E, S>(v, j, ex, NoHook());
            if constexpr (S + 2 == line_nstages(L, E)) tail();  // the last exchange is done with `ex`
        } else if constexpr (S == 0) {
            hook();
            tail();
        }
        line_stages_from<R, L, E, S + 1, TWS>(v, j, tw, ex, hook, tail);
    }
}

// Forward FFT of a line held as v[i] = x[j + i NT]; result in the same slots.
// `hook` runs once after the first exchange barrier (or after the only
// stage); `tail` runs once after the last exchange has ended on a barrier, so
// that every thread's reads of the exchange buffer are complete (or after the
// only stage).  TWS: `tw` points to a copy of the twiddle table in shared
// memory.
template <typename R, int L, int E, bool TWS = false, class Ex, class Hook = NoHook, class Tail = NoHook>
__device__ __forceinline__ void line_fft(typename cvec<R>::T *v, int j,
                                         const typename cvec<R>::T *__restrict__ tw, Ex &ex,
                                         const Hook &hook = Hook(), const Tail &tail = Tail())
{
    static_assert(line_plan_valid(L, E), "invalid line plan");
    if constexpr (line_nstages(L, E) == 0) {
        hook();
        tail();
    }
    line_stages_from<R, L, E, 0, TWS>(v, j, tw, ex, hook, tail);
}

}  // namespace fft3d
