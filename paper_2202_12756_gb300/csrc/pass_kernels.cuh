// Pass kernels of the 3D R2C / C2R transform.
//
//   zpass_r2c : forward, contiguous axis 2.  Each real line of N2 = 2M values
//               is read as M complex pairs z[n] = x[2n] + i x[2n+1], given an
//               M-point FFT Z, and turned into the N2/2 + 1 = M + 1 Hermitian
//               half-spectrum entries X[k] = E[k] + W_N2^k O[k] with
//               E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / 2i.
//               (Step 1 of Sec. 3 along the first of the two plane axes.)
//               Double lines of N2 = 1024 points instead run two lines per
//               N2-point complex transform (zr2c_pairs / zc2r_pairs).
//   zpass_c2r : inverse, contiguous axis 2: the same relation run backwards,
//               then the M-point inverse FFT, the unpacking into 2M reals and
//               the 1/(N0 N1 N2) normalisation (the paper's separate
//               normalisation step, fused here).
//   colpass   : C2C along a strided axis (axis 1, the second plane axis of
//               Step 1; or axis 0, the slowest axis of Step 5).  A tile of W
//               adjacent columns is read with the lanes of a warp across the
//               columns, so every row of the tile is one coalesced segment of
//               W * sizeof(complex) = 128 bytes (64 where the tile is
//               narrowed: 2048-point float columns on one SM, FP64 columns
//               of 1024 points); the column FFTs exchange through shared
//               memory.  The x-pass does in one read and one
//               write what the paper does with two transposes and an
//               all-to-all (Steps 2-5): no transposed copy of the array exists.
#pragma once

#include <cuda.h>  // CUtensorMap (type only)

#include "line_fft.cuh"

namespace fft3d {

// ------------------------------------------------------------ layouts
// Complex half-spectrum array, logically [N0][N1][M + 1].
//   standard: main[(k0 N1 + k1) (M + 1) + k2]
//   split:    k2 < M  -> main[(k0 N1 + k1) M + k2]
//             k2 == M -> nyq[k0 N1 + k1]
// The split form lets an out-of-place inverse run in a dense real output
// buffer (which has room for exactly M complex values per line) plus one
// N0 x N1 plane of scratch for the k2 = M column.
struct CLayout {
    void *main;
    void *nyq;
    int split;
};

struct ColArgs {
    CLayout src, dst;
    int64_t n0, n1, m;        // N0 (x-pass: column length; y-pass: planes of all fields, B N0), N1, M = N2 / 2
    int axis;                 // 0: rows are k0 (x-pass); 1: rows are k1 (y-pass)
    int inverse;              // 1: exp(+...) via swapped re / im in and out
    int64_t tiles_main;       // tiles of the main column set
    int64_t tiles_per_plane;  // y-pass: main tiles per k0 plane
    int nyq_in_plane;         // y-pass: tiles cover k2 = 0..M of one plane (last one ragged)
    int bulk;                 // pipelined pass, tiles t < tiles_main: 0 cp.async, 1 TMA (dense rows),
                              // 2 TMA (y-pass rows of odd complex pitch, even / odd row maps)
    unsigned *err;            // pipelined pass: device error flag (a stage-fill wait ran out)
    int64_t tiles_per_field;  // x-pass: tiles of one field; field b's columns start at row k0 = b n0
    int early;                // pipelined pass: stage the next tile before the current one's first stage
                              // (selects the kernel instance)
    unsigned stall_tx;        // pipelined pass, test hook: bytes a tile wait expects beyond its copies
    long long stage_polls;    // pipelined pass: polls of a tile wait before it gives up
    int64_t pf_stride;        // one-tile pass: > 0 prefetch tile blockIdx + pf_stride into L2 (the next wave)
    unsigned *tickets;        // pipelined pass: zeroed tile counter (dynamic tile order), or null (static order)
};

template <typename C>
__device__ __forceinline__ void layout_column(const CLayout &l, int64_t n1, int64_t m, int axis,
                                              int64_t k0, int64_t k1, int64_t k2, C *&ptr,
                                              int64_t &stride)
{
    if (!l.split) {
        ptr = (C *)l.main + ((k0 * n1 + k1) * (m + 1) + k2);
        stride = axis == 0 ? n1 * (m + 1) : (m + 1);
    } else if (k2 < m) {
        ptr = (C *)l.main + ((k0 * n1 + k1) * m + k2);
        stride = axis == 0 ? n1 * m : m;
    } else {
        ptr = (C *)l.nyq + (k0 * n1 + k1);
        stride = axis == 0 ? n1 : 1;
    }
}

// Column-tile exchange: element (row, column c) at sm[row * W + c].  With
// W * sizeof(complex) = 128 bytes, each half/quarter-warp access is one row:
// conflict-free without padding.
template <typename C, int W> struct ColEx {
    static constexpr bool kSplit = false;
    static constexpr int kPadShift = -1;
    C *sm;
    int c;
    __device__ __forceinline__ void put(int row, C v) { sm[row * W + c] = v; }
    __device__ __forceinline__ C get(int row) const { return sm[row * W + c]; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// Which column lane c of tile t owns, and where it lives in the source and
// destination layouts.  Lanes past the last column get the last column's
// address (so every load is in bounds) and `false`: they compute on a copy
// and store nothing.  Columns never mix, so this is harmless.
template <typename C, int W>
__device__ __forceinline__ bool col_decode(const ColArgs &a, int64_t t, int c, C *&sp, int64_t &ss, C *&dp,
                                           int64_t &ds)
{
    int64_t k0 = 0, k1 = 0, k2 = 0;
    bool valid;
    if (a.axis == 0) {
        const int64_t total = a.n1 * (a.m + 1);
        const int64_t b = (uint32_t)t / (uint32_t)a.tiles_per_field;  // field of a batched plan (t < 2^32)
        int64_t f = (t - b * a.tiles_per_field) * W + c;  // flat (k1, k2) index
        valid = f < total;
        f = valid ? f : total - 1;
        k0 = b * a.n0;
        k1 = f / (a.m + 1);
        k2 = f - k1 * (a.m + 1);
    } else if (a.nyq_in_plane) {
        k0 = t / a.tiles_per_plane;
        k2 = (t - k0 * a.tiles_per_plane) * W + c;
        valid = k2 <= a.m;
        k2 = valid ? k2 : a.m;
    } else if (t < a.tiles_main) {
        k0 = t / a.tiles_per_plane;
        k2 = (t - k0 * a.tiles_per_plane) * W + c;
        valid = k2 < a.m;
        k2 = valid ? k2 : a.m - 1;
    } else {  // k2 = M column of W consecutive planes
        k0 = (t - a.tiles_main) * W + c;
        k2 = a.m;
        valid = k0 < a.n0;
        k0 = valid ? k0 : a.n0 - 1;
    }
    layout_column<C>(a.src, a.n1, a.m, a.axis, k0, k1, k2, sp, ss);
    layout_column<C>(a.dst, a.n1, a.m, a.axis, k0, k1, k2, dp, ds);
    return valid;
}

// Split exchange of a column tile: real parts, then imaginary parts, through
// an [L][W] buffer of reals (half the size of a complex one).  One padding
// row every 32 rows keeps the stride-32-row writes of a radix-32 stage free of
// bank conflicts (W reals = 64 bytes per row).
template <typename R, int W> struct ColSplitEx {
    static constexpr bool kSplit = true;
    static constexpr int kPadShift = 5;  // rows arrive padded: r + (r >> 5)
    R *sm;
    int c;
    __device__ __forceinline__ void put_real(int prow, R v) { sm[prow * W + c] = v; }
    __device__ __forceinline__ R get_real(int prow) const { return sm[prow * W + c]; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// Stores of pass outputs: the next pass reads them back from HBM (an array
// far larger than L2), so they are marked evict-first (st.global.cs).
// Measured on GB300 at 1024^3 FP32: the R2C z-pass 3.4% and the whole pair
// 0.8% faster; at 1536^3 the pair is 0.5% slower.
#ifndef FFT3D_STORE_CS
#define FFT3D_STORE_CS 1
#endif
template <typename C> __device__ __forceinline__ void store_out(C *p, C v)
{
    if constexpr (FFT3D_STORE_CS) __stcs(p, v);
    else *p = v;
}

// Loads that bypass L1: a tile written earlier in the same kernel by another
// block is read from L2, never from a stale L1 line.
template <typename C> __device__ __forceinline__ C load_cg(const C *p) { return __ldcg(p); }

// One column tile (W columns x L rows) with the block's threads; the tile is
// loaded straight into registers.  CG selects L2-only loads.
template <typename R, int L, int E, int W, bool CG, bool INV>
__device__ __forceinline__ void col_tile(const ColArgs &a, int64_t tile, unsigned char *smem,
                                         const typename cvec<R>::T *__restrict__ tw, int64_t pf_tile = -1)
{
    typedef typename cvec<R>::T C;
    constexpr int NT = L / E;
    const int c = threadIdx.x % W;
    const int j = threadIdx.x / W;
    C *sp = nullptr, *dp = nullptr;
    int64_t ss = 0, ds = 0;
    const bool valid = col_decode<C, W>(a, tile, c, sp, ss, dp, ds);

    const C *sj = sp + (int64_t)j * ss;
    const int64_t sstep = (int64_t)NT * ss;
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        v[i] = CG ? load_cg(sj + i * sstep) : sj[i * sstep];
        if (INV) v[i] = cswap(v[i]);
    }
    if (pf_tile >= 0) {
        // the tile this SM is likely to run next: its rows into L2 while this one is transformed
        C *psp = nullptr, *pdp = nullptr;
        int64_t pss = 0, pds = 0;
        col_decode<C, W>(a, pf_tile, c, psp, pss, pdp, pds);
        const C *pj = psp + (int64_t)j * pss;
        const int64_t pstep = (int64_t)NT * pss;
#pragma unroll
        for (int i = 0; i < E; ++i) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(pj + i * pstep));
    }
    ColEx<C, W> ex{(C *)smem, c};
    line_fft<R, L, E>(v, j, tw, ex);
    if (valid) {
        C *dj = dp + (int64_t)j * ds;
        const int64_t dstep = (int64_t)NT * ds;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            C o = v[i];
            if (INV) o = cswap(o);
            dj[i * dstep] = o;
        }
    }
}

// One tile per block.
template <typename R, int L, int E, int W, bool INV>
__global__ void __launch_bounds__(W *(L / E))
colpass_kernel(ColArgs a, const typename cvec<R>::T *__restrict__ tw)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t pf = a.pf_stride > 0 && blockIdx.x + a.pf_stride < gridDim.x ? blockIdx.x + a.pf_stride : -1;
    col_tile<R, L, E, W, false, INV>(a, blockIdx.x, smem_raw, tw, pf);
}

template <int L> __host__ __device__ constexpr int split_rows() { return L + (L >> 5) + 1; }

__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t mb, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mb), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mb, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mb), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity; false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mb, uint32_t parity, long long limit)
{
    for (long long n = 0; n < limit; ++n) {
        if (mbar_try_wait(mb, parity)) return true;
        __nanosleep(32);
    }
    return false;
}
// TMA: copy the 2D box at (x, y) of the tensor map into this CTA's shared
// memory (x counts reals of the innermost dimension), completing on `mb`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mb)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(mb)
        : "memory");
}

// rows of one TMA box of the column-tile tensor map
constexpr int kTmaBoxRows = 256;

// Staging row: W complex values (one 128-byte segment for float); in mode 2
// the odd rows are fetched 2 complex wider, from one column before the tile.
template <typename C, int W> __host__ __device__ constexpr int stage_row_elems() { return W; }
template <typename C, int W, int L> __host__ __device__ constexpr int stage_elems() { return L / 2 * W + L / 2 * (W + 2); }

// polls of a stage-fill wait before the kernel gives up (about 0.1 s)
constexpr long long kStageWaitPolls = 1LL << 22;

// Shared memory of the pipelined column pass: staging (L/2 W + L/2 (W + 2)
// complex), the split exchange buffer, the mbarrier and two tile slots (32
// bytes), then the twiddle table.
template <typename R, int L, int E, int W> __host__ __device__ constexpr size_t pipe_smem_bytes()
{
    return (size_t)stage_elems<typename cvec<R>::T, W, L>() * sizeof(typename cvec<R>::T) +
           (size_t)split_rows<L>() * W * sizeof(R) + 32 + (size_t)line_tw_size(L, E) * sizeof(typename cvec<R>::T);
}

// Persistent, software-pipelined column pass.  Each block walks the tiles
// t = blockIdx.x, blockIdx.x + gridDim.x, ...  While a tile is transformed in
// registers, the next tile is already streaming from HBM into a shared-memory
// staging buffer.  Full tiles of the standard layout are fetched by one
// thread with TMA tensor copies of 256 rows x W columns, completing on an
// mbarrier (tensor maps over 8-byte elements, coordinates in complex units):
//   a.bulk = 1: rows 16-byte aligned (x-pass; y-pass with an even row pitch):
//               one map, rows (tile row 0) + b 256, dense [L][W] staging;
//   a.bulk = 2: y-pass with an odd row pitch (N2/2 + 1 odd): every other row
//               starts 8 bytes past a 16-byte boundary, but a pair of rows is
//               a multiple of 16 bytes, so the plane is a [N1/2][2 (M+1)]
//               tensor: even rows come from column c0 (W wide), odd rows from
//               column c0 + M of the pair (W + 2 wide, i.e. one column early),
//               into [L/2][W] + [L/2][W+2] staging.
// Other tiles are staged element by element with cp.async, each thread
// copying exactly the elements it will own.  The next tile's copies are
// issued after the first exchange barrier, when every thread's reads of the
// staging buffer have completed.  The stage exchange uses a separate split
// (real / imaginary) buffer.  A tile wait that runs out raises *a.err and the
// block leaves after a second bounded wait.  The twiddle table is copied to
// shared memory once per block (a thread's twiddles are the same in every
// tile).  The tile is W = 16 float2 columns (8 at 2048 points, where 16
// would not fit beside the staging buffer): 128-byte row segments, which
// HBM serves at about twice the rate of 64-byte ones at large row strides.
// With EARLY the next tile is staged as soon as the current one is in
// registers (one barrier more per tile) rather than after the first exchange
// barrier; which is faster depends on the access pattern (ColArgs::early,
// set by the host, selects the instance).
// Measured on GB300, two alternatives were slower: exchanging through the
// staging buffer itself (so the next tile's copies start only after the
// exchange) by 35-40%, and waiting for the next tile before storing this one
// (stores interleaved with the next tile's staging reads) by 9-25%.
template <typename R, int L, int E, int W, bool INV, bool EARLY>
__global__ void __launch_bounds__(W *(L / E), (W * (L / E) >= 512 ? 1 : 512 / (W * (L / E))))
colpass_pipe_kernel(ColArgs a, const typename cvec<R>::T *__restrict__ tw, int64_t ntiles,
                    const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap2)
{
    typedef typename cvec<R>::T C;
    constexpr int NT = L / E;
    constexpr int RSE = stage_row_elems<C, W>();
    static_assert(L % (2 * kTmaBoxRows) == 0 && NT % 2 == 0 && (RSE * sizeof(C)) % 16 == 0, "staging layout");
    extern __shared__ __align__(1024) unsigned char pipe_smem_raw[];
    C *stage = (C *)pipe_smem_raw;
    C *stage_odd = stage + L / 2 * W;  // mode 2: odd rows, W + 2 wide
    R *exbuf = (R *)(stage + stage_elems<C, W, L>());
    uint64_t *mbar = (uint64_t *)(exbuf + split_rows<L>() * W);
    int64_t *tslot = (int64_t *)(mbar + 2);  // dynamic order: tiles drawn one iteration ahead
    C *tws = (C *)(mbar + 4);                // the block's copy of the twiddle table
    constexpr int NTW = line_tw_size(L, E);
    for (int i = threadIdx.x; i < NTW; i += blockDim.x) tws[i] = __ldg(tw + i);
    const int c = threadIdx.x % W;
    const int j = threadIdx.x / W;
    ColSplitEx<R, W> ex{exbuf, c};
    const uint32_t mb = smem_u32(mbar);
    if (threadIdx.x == 0) {
        mbar_init(mb, 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t phase = 0;

    // Start staging tile tt; returns its mode (0 cp.async, 1 or 2 TMA).
    auto fill = [&](int64_t tt, const C *sp, int64_t ss) -> int {
        const int mode = tt < a.tiles_main ? a.bulk : 0;
        if (mode) {
            if (threadIdx.x == 0) {
                // order the block's earlier reads of the buffer before the async-proxy writes
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                if (mode == 1) {
                    mbar_arrive_expect_tx(mb, (unsigned)(L * W * sizeof(C)) + a.stall_tx);
                    int x, y0;
                    if (a.axis == 0) {  // [B N0][N1 (M+1)]: the tile's flat columns, its field's rows
                        const int64_t b = (uint32_t)tt / (uint32_t)a.tiles_per_field;
                        x = (int)((tt - b * a.tiles_per_field) * W);
                        y0 = (int)(b * a.n0);
                    } else {            // [N0 N1][M+1]: plane k0, columns c0..
                        const int64_t k0 = tt / a.tiles_per_plane;
                        x = (int)((tt - k0 * a.tiles_per_plane) * W);
                        y0 = (int)(k0 * a.n1);
                    }
#pragma unroll
                    for (int b = 0; b < L / kTmaBoxRows; ++b)
                        tma_load_2d(smem_u32(stage + b * kTmaBoxRows * W), &tmap, x, y0 + b * kTmaBoxRows, mb);
                } else {
                    mbar_arrive_expect_tx(mb, (unsigned)(L / 2 * (2 * W + 2) * sizeof(C)) + a.stall_tx);
                    const int64_t k0 = tt / a.tiles_per_plane;
                    const int c0 = (int)((tt - k0 * a.tiles_per_plane) * W);
                    const int y0 = (int)(k0 * (a.n1 / 2));
#pragma unroll
                    for (int b = 0; b < L / 2 / kTmaBoxRows; ++b) {
                        tma_load_2d(smem_u32(stage + b * kTmaBoxRows * W), &tmap, c0, y0 + b * kTmaBoxRows, mb);
                        tma_load_2d(smem_u32(stage_odd + b * kTmaBoxRows * (W + 2)), &tmap2, c0 + (int)a.m,
                                    y0 + b * kTmaBoxRows, mb);
                    }
                }
            }
        } else {
            const C *sj = sp + (int64_t)j * ss;
            const int64_t sstep = (int64_t)NT * ss;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                C *dst = stage + (j + i * NT) * RSE + c;
                if (sizeof(C) == 8) cp_async_8(dst, sj + i * sstep);
                else cp_async_16(dst, sj + i * sstep);
            }
            cp_async_commit();
        }
        return mode;
    };

    // Tile order.  Static: t = blockIdx.x + q gridDim.x, so that at any moment
    // the blocks work on neighbouring tiles, whose rows share DRAM pages
    // (measured on GB300: giving each block runs of 2, 4 or 8 consecutive
    // tiles instead slows the y-pass by 15, 27 and 45%, and runs of 2 to all
    // of a block's tiles gain nothing in the x-pass).  Dynamic (a.tickets):
    // a block's first two tiles are blockIdx.x and blockIdx.x + gridDim.x,
    // and each later one is 2 gridDim.x + a ticket drawn from *a.tickets
    // (zeroed before the launch), one iteration ahead so that the atomic's
    // latency stays off the tile's path: slots tslot[q & 1] alternate, each
    // written after one staging barrier and read after the next.  Tickets go
    // out in time order, so a block whose next tile is past the end has no
    // later tile pending.  Blocks that run faster take more tiles, and the
    // pass no longer waits for the slowest SM's share.
    const bool dyn = a.tickets != nullptr;
    int64_t t = blockIdx.x;
    C *sp = nullptr, *dp = nullptr;
    int64_t ss = 0, ds = 0;
    bool valid = t < ntiles && col_decode<C, W>(a, t, c, sp, ss, dp, ds);
    int mode = t < ntiles ? fill(t, sp, ss) : 0;
    for (int q = 0; t < ntiles; ++q) {
        if (mode) {
            const bool ok = mbar_wait_bounded(mb, phase, a.stage_polls);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(a.err, 1u);
                mbar_wait_bounded(mb, phase, a.stage_polls);  // copies still in flight
                return;
            }
            phase ^= 1u;
        } else {
            cp_async_wait_all();  // this thread's copies of tile t have landed
            if (dyn) __syncthreads();  // orders the tile slots (written after the previous barrier)
        }
        const int64_t tn = (dyn && q > 0) ? tslot[(q - 1) & 1] : t + gridDim.x;
        if (dyn && threadIdx.x == 0) tslot[q & 1] = 2 * (int64_t)gridDim.x + atomicAdd(a.tickets, 1u);
        C *spn = nullptr, *dpn = nullptr;
        int64_t ssn = 0, dsn = 0;
        const bool validn = tn < ntiles && col_decode<C, W>(a, tn, c, spn, ssn, dpn, dsn);
        C v[E];
        if (mode == 2) {
            // rows j + i NT (NT even) share the parity of j
            const C *base = (j & 1) ? stage_odd + (j >> 1) * (W + 2) + c + 1 : stage + (j >> 1) * W + c;
            const int step = (j & 1) ? (NT / 2) * (W + 2) : (NT / 2) * W;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                v[i] = base[i * step];
                if (INV) v[i] = cswap(v[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                v[i] = stage[(j + i * NT) * RSE + c];
                if (INV) v[i] = cswap(v[i]);
            }
        }
        int moden = 0;
        auto next = [&]() {
            if (tn < ntiles) moden = fill(tn, spn, ssn);
        };
        if constexpr (EARLY) {
            // every thread has its elements of tile t in registers: stage tile tn now
            __syncthreads();
            next();
            line_fft<R, L, E, true>(v, j, tws, ex);
        } else {
            line_fft<R, L, E, true>(v, j, tws, ex, next);
        }
        if (valid) {
            C *dj = dp + (int64_t)j * ds;
            const int64_t dstep = (int64_t)NT * ds;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                C o = v[i];
                if (INV) o = cswap(o);
                store_out(dj + i * dstep, o);
            }
        }
        t = tn;
        valid = validn;
        mode = moden;
        sp = spn;
        ss = ssn;
        dp = dpn;
        ds = dsn;
    }
    cp_async_wait_all();
}

// ------------------------------------------------------------ one-buffer pipelined column pass
// Columns whose 16-column tile fills shared memory on its own (float L = 1536:
// 192 KB, no room for a staging buffer beside a separate exchange buffer) run
// a persistent kernel whose staging buffer is also the transform's exchange
// buffer ([L][W] complex, as in colpass_kernel).  The next tile's copies can
// start only once the last exchange is done with the buffer, so they overlap
// the last radix stage and the stores of the current tile; the one-tile
// kernel overlaps nothing of its own tile (one block per SM, each loading its
// tile when it starts).  Staging (TMA modes 1 and 2, per-element cp.async
// otherwise), tile order (static, or dynamic with a.tickets) and the bounded
// tile waits are those of colpass_pipe_kernel.
template <typename R, int L, int E, int W> __host__ __device__ constexpr size_t xstage_smem_bytes()
{
    return (size_t)stage_elems<typename cvec<R>::T, W, L>() * sizeof(typename cvec<R>::T) + 32 +
           (size_t)line_tw_size(L, E) * sizeof(typename cvec<R>::T);
}

template <typename R, int L, int E, int W, bool INV>
__global__ void __launch_bounds__(W *(L / E), 1)
colpass_xstage_kernel(ColArgs a, const typename cvec<R>::T *__restrict__ tw, int64_t ntiles,
                    const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap2)
{
    typedef typename cvec<R>::T C;
    constexpr int NT = L / E;
    constexpr int RSE = stage_row_elems<C, W>();
    static_assert(L % (2 * kTmaBoxRows) == 0 && NT % 2 == 0 && (RSE * sizeof(C)) % 16 == 0, "staging layout");
    static_assert(line_nstages(L, E) >= 2 && L * W <= stage_elems<C, W, L>(), "the exchange reuses the staging buffer");
    extern __shared__ __align__(1024) unsigned char xstage_smem_raw[];
    C *stage = (C *)xstage_smem_raw;
    C *stage_odd = stage + L / 2 * W;  // mode 2: odd rows, W + 2 wide
    uint64_t *mbar = (uint64_t *)(stage + stage_elems<C, W, L>());
    int64_t *tslot = (int64_t *)(mbar + 2);  // dynamic order: tiles drawn one iteration ahead
    C *tws = (C *)(mbar + 4);                // the block's copy of the twiddle table
    constexpr int NTW = line_tw_size(L, E);
    for (int i = threadIdx.x; i < NTW; i += blockDim.x) tws[i] = __ldg(tw + i);
    const int c = threadIdx.x % W;
    const int j = threadIdx.x / W;
    ColEx<C, W> ex{stage, c};  // [L][W] over the staging buffer, once the tile is in registers
    const uint32_t mb = smem_u32(mbar);
    if (threadIdx.x == 0) {
        mbar_init(mb, 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t phase = 0;

    // Start staging tile tt; returns its mode (0 cp.async, 1 or 2 TMA).
    auto fill = [&](int64_t tt, const C *sp, int64_t ss) -> int {
        const int mode = tt < a.tiles_main ? a.bulk : 0;
        if (mode) {
            if (threadIdx.x == 0) {
                // order the block's earlier reads of the buffer before the async-proxy writes
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                if (mode == 1) {
                    mbar_arrive_expect_tx(mb, (unsigned)(L * W * sizeof(C)) + a.stall_tx);
                    int x, y0;
                    if (a.axis == 0) {  // [B N0][N1 (M+1)]: the tile's flat columns, its field's rows
                        const int64_t b = (uint32_t)tt / (uint32_t)a.tiles_per_field;
                        x = (int)((tt - b * a.tiles_per_field) * W);
                        y0 = (int)(b * a.n0);
                    } else {            // [N0 N1][M+1]: plane k0, columns c0..
                        const int64_t k0 = tt / a.tiles_per_plane;
                        x = (int)((tt - k0 * a.tiles_per_plane) * W);
                        y0 = (int)(k0 * a.n1);
                    }
#pragma unroll
                    for (int b = 0; b < L / kTmaBoxRows; ++b)
                        tma_load_2d(smem_u32(stage + b * kTmaBoxRows * W), &tmap, x, y0 + b * kTmaBoxRows, mb);
                } else {
                    mbar_arrive_expect_tx(mb, (unsigned)(L / 2 * (2 * W + 2) * sizeof(C)) + a.stall_tx);
                    const int64_t k0 = tt / a.tiles_per_plane;
                    const int c0 = (int)((tt - k0 * a.tiles_per_plane) * W);
                    const int y0 = (int)(k0 * (a.n1 / 2));
#pragma unroll
                    for (int b = 0; b < L / 2 / kTmaBoxRows; ++b) {
                        tma_load_2d(smem_u32(stage + b * kTmaBoxRows * W), &tmap, c0, y0 + b * kTmaBoxRows, mb);
                        tma_load_2d(smem_u32(stage_odd + b * kTmaBoxRows * (W + 2)), &tmap2, c0 + (int)a.m,
                                    y0 + b * kTmaBoxRows, mb);
                    }
                }
            }
        } else {
            const C *sj = sp + (int64_t)j * ss;
            const int64_t sstep = (int64_t)NT * ss;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                C *dst = stage + (j + i * NT) * RSE + c;
                if (sizeof(C) == 8) cp_async_8(dst, sj + i * sstep);
                else cp_async_16(dst, sj + i * sstep);
            }
            cp_async_commit();
        }
        return mode;
    };

    // Tile order.  Static: t = blockIdx.x + q gridDim.x, so that at any moment
    // the blocks work on neighbouring tiles, whose rows share DRAM pages
    // (measured on GB300: giving each block runs of 2, 4 or 8 consecutive
    // tiles instead slows the y-pass by 15, 27 and 45%, and runs of 2 to all
    // of a block's tiles gain nothing in the x-pass).  Dynamic (a.tickets):
    // a block's first two tiles are blockIdx.x and blockIdx.x + gridDim.x,
    // and each later one is 2 gridDim.x + a ticket drawn from *a.tickets
    // (zeroed before the launch), one iteration ahead so that the atomic's
    // latency stays off the tile's path: slots tslot[q & 1] alternate, each
    // written after one staging barrier and read after the next.  Tickets go
    // out in time order, so a block whose next tile is past the end has no
    // later tile pending.  Blocks that run faster take more tiles, and the
    // pass no longer waits for the slowest SM's share.
    const bool dyn = a.tickets != nullptr;
    // Registers are tight here (1024 threads), so a tile's source and
    // destination are decoded where they are used, not held across the transform.
    int64_t t = blockIdx.x;
    int mode = 0;
    if (t < ntiles) {
        C *sp = nullptr, *dp = nullptr;
        int64_t ss = 0, ds = 0;
        col_decode<C, W>(a, t, c, sp, ss, dp, ds);
        mode = fill(t, sp, ss);
    }
    for (int q = 0; t < ntiles; ++q) {
        if (mode) {
            const bool ok = mbar_wait_bounded(mb, phase, a.stage_polls);
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0) atomicOr(a.err, 1u);
                mbar_wait_bounded(mb, phase, a.stage_polls);  // copies still in flight
                return;
            }
            phase ^= 1u;
        } else {
            cp_async_wait_all();  // this thread's copies of tile t have landed
            if (dyn) __syncthreads();  // orders the tile slots (written after the previous barrier)
        }
        const int64_t tn = (dyn && q > 0) ? tslot[(q - 1) & 1] : t + gridDim.x;
        if (dyn && threadIdx.x == 0) tslot[q & 1] = 2 * (int64_t)gridDim.x + atomicAdd(a.tickets, 1u);
        C v[E];
        if (mode == 2) {
            // rows j + i NT (NT even) share the parity of j
            const C *base = (j & 1) ? stage_odd + (j >> 1) * (W + 2) + c + 1 : stage + (j >> 1) * W + c;
            const int step = (j & 1) ? (NT / 2) * (W + 2) : (NT / 2) * W;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                v[i] = base[i * step];
                if (INV) v[i] = cswap(v[i]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                v[i] = stage[(j + i * NT) * RSE + c];
                if (INV) v[i] = cswap(v[i]);
            }
        }
        int moden = 0;
        auto next = [&]() {
            if (tn < ntiles) {
                C *spn = nullptr, *dpn = nullptr;
                int64_t ssn = 0, dsn = 0;
                col_decode<C, W>(a, tn, c, spn, ssn, dpn, dsn);
                moden = fill(tn, spn, ssn);
            }
        };
        // every thread has its elements of tile t in registers before the exchanges
        // overwrite the buffer; tile tn is staged once the last exchange is done with it
        __syncthreads();
        line_fft<R, L, E, true>(v, j, tws, ex, NoHook(), next);
        {
            C *sp = nullptr, *dp = nullptr;
            int64_t ss = 0, ds = 0;
            if (col_decode<C, W>(a, t, c, sp, ss, dp, ds)) {
                C *dj = dp + (int64_t)j * ds;
                const int64_t dstep = (int64_t)NT * ds;
#pragma unroll
                for (int i = 0; i < E; ++i) {
                    C o = v[i];
                    if (INV) o = cswap(o);
                    store_out(dj + i * dstep, o);
                }
            }
        }
        t = tn;
        mode = moden;
    }
    cp_async_wait_all();
}


// ------------------------------------------------------------ column pairs
// Columns too long for one SM to hold W = 16 of them (L = 2048 float: a
// 256 KB tile) run on a cluster of two CTAs.  CTA r of the pair holds the
// rows 2n + r (n < L/2) of the tile's 16 columns and computes their L/2-point
// FFT Y_r (radix-2 decimation in time); the two halves meet in one radix-2
// step, X[k] = Y_0[k] + W_L^k Y_1[k] and X[k + L/2] = Y_0[k] - W_L^k Y_1[k].
// CTA 0 finishes k < L/4 and CTA 1 the rest, so each sends the other half of
// its Y into the partner's exchange buffer through distributed shared memory
// (a thread's slots k = j + i NT are the same in both CTAs: thread (j, c)
// writes to thread (j, c) of the partner); each CTA applies W_L^k to the half
// of Y_1 it ends up with.  Every row an SM reads or writes is thus a 128-byte
// segment of 16 columns; at W = 8 (one SM per tile) rows are 64-byte
// segments, which HBM serves at about half the rate at large row pitches.
// The exchange runs on mbarriers, not cluster barriers: once its transform
// is done with the exchange buffer, a CTA arms its receive barrier for the
// partner's 64 KB and tells the partner, by one remote arrival on the
// partner's "free" barrier, that it may write; the partner's st.async stores
// complete on the receive barrier.  (Two cluster barriers per tile instead,
// each a release by every thread, measured 2% slower.)  Every wait is
// bounded: a CTA whose wait runs out raises *a.err and leaves its loop, its
// partner's next wait then runs out as well, and both wait (bounded) for the
// copies and stores still in flight into their shared memory and meet at a
// final cluster barrier, so no CTA leaves while the other may address it.
// Staging as in colpass_pipe_kernel, with the row parity taking the place of
// the row pair: a.bulk = 1 reads rows 2n + r through a map over row pairs
// ([rows / 2][2 P], P the row pitch) at column x + r P; a.bulk = 2 (odd P) is
// the even / odd map pair of that kernel, one per CTA.
template <int L, int E, int W> __host__ __device__ constexpr size_t pair_smem_bytes()
{
    return (size_t)(L / 2) * (W + 2) * 8 + (size_t)split_rows<L / 2>() * W * 4 + 32 +
           (size_t)(line_tw_size(L / 2, E) + L / 2 / E) * 8;
}

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;\n" : "=r"(r));
    return r;
}
// Address of this CTA's shared variable `a` in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_map(uint32_t a, uint32_t rank)
{
    uint32_t d;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(d) : "r"(a), "r"(rank));
    return d;
}
// All threads of both CTAs: shared-memory writes before it (local or remote)
// are visible to every thread after it.
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// One arrival on an mbarrier of another CTA of the cluster (cluster address),
// ordered after this thread's earlier memory accesses.
__device__ __forceinline__ void mbar_remote_arrive(uint32_t a)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];\n" ::"r"(a) : "memory");
}
// Asynchronous 8-byte store into another CTA's shared memory, completing
// (8 bytes of transaction count) on that CTA's mbarrier `mb`.
__device__ __forceinline__ void st_async_f2(uint32_t a, float2 v, uint32_t mb)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];\n" ::"r"(a),
                 "f"(v.x), "f"(v.y), "r"(mb)
                 : "memory");
}
// Bounded wait for a phase completed from another CTA of the cluster.
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint32_t mb, uint32_t parity, long long limit)
{
    for (long long n = 0; n < limit; ++n) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mb), "r"(parity)
            : "memory");
        if (ok) return true;
        __nanosleep(32);
    }
    return false;
}

template <typename R, int L, int E, int W, bool INV, bool EARLY>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(W *(L / 2 / E), 1)
colpass_pair_kernel(ColArgs a, const typename cvec<R>::T *__restrict__ tw, int64_t ntiles,
                    const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap2)
{
    typedef typename cvec<R>::T C;
    constexpr int LH = L / 2;  // rows per CTA
    constexpr int NT = LH / E;
    constexpr int H = E / 2;   // slots sent to / received from the partner
    constexpr int NTW = line_tw_size(LH, E);
    static_assert(sizeof(R) == 4 && W * sizeof(C) == 128, "float tiles of 128-byte rows");
    static_assert(LH % kTmaBoxRows == 0 && E % 2 == 0, "staging layout");
    static_assert(H * W * NT * sizeof(C) <= (size_t)split_rows<LH>() * W * sizeof(R), "receive buffer");
    static_assert(line_nstages(LH, E) >= 2, "the transform must end its exchange-buffer use on a barrier");
    extern __shared__ __align__(1024) unsigned char pair_smem_raw[];
    C *stage = (C *)pair_smem_raw;  // [LH][W] or, odd rows of a.bulk = 2, [LH][W + 2]
    R *exbuf = (R *)(stage + LH * (W + 2));
    // mbarriers: the tile's staging copies, the partner's data, the partner's exchange buffer free
    uint64_t *mbar = (uint64_t *)(exbuf + split_rows<LH>() * W);
    C *tws = (C *)(mbar + 4);  // line table of LH points, then W_L^j for j < NT
    for (int i = threadIdx.x; i < NTW + NT; i += blockDim.x) tws[i] = __ldg(tw + i);
    const uint32_t rank = cluster_ctarank();
    const uint32_t peer = rank ^ 1u;
    const int c = threadIdx.x % W;
    const int j = threadIdx.x / W;
    ColSplitEx<R, W> ex{exbuf, c};
    const uint32_t mb = smem_u32(mbar), mb_rx = smem_u32(mbar + 1), mb_free = smem_u32(mbar + 2);
    if (threadIdx.x == 0) {
        mbar_init(mb, 1);
        mbar_init(mb_rx, 1);
        mbar_init(mb_free, 1);
        mbar_fence_init();
    }
    // both CTAs have started (and initialised) before either addresses the other's shared memory
    cluster_sync_all();
    // the partner's receive slots for this thread and its mbarriers
    const uint32_t peer_rx = cluster_map(smem_u32(exbuf), peer) + (uint32_t)threadIdx.x * (uint32_t)sizeof(C);
    const uint32_t peer_mb_rx = cluster_map(mb_rx, peer), peer_mb_free = cluster_map(mb_free, peer);
    const C *rx = (const C *)exbuf + threadIdx.x;
    constexpr uint32_t kRxStep = W * NT * sizeof(C);  // bytes between a thread's receive slots
    uint32_t phase = 0;  // staging barrier
    uint32_t xph = 0;    // receive and free barriers (one phase per tile)
    bool failed = false, stage_pending = false, rx_pending = false;

    // row pitch of the source tensor (elements) for a.bulk = 1
    const int64_t P = a.axis == 0 ? a.n1 * (a.m + 1) : (a.src.split ? a.m : a.m + 1);
    const bool odd_wide = a.bulk == 2 && rank == 1;  // staging rows W + 2 wide, column c at c + 1

    auto fill = [&](int64_t tt, const C *sp, int64_t ss) -> int {
        const int mode = tt < a.tiles_main ? a.bulk : 0;
        if (mode) {
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                int x, y0;  // y0: first row pair of the tile
                if (a.axis == 0) {
                    const int64_t b = (uint32_t)tt / (uint32_t)a.tiles_per_field;
                    x = (int)((tt - b * a.tiles_per_field) * W);
                    y0 = (int)(b * (a.n0 / 2));
                } else {
                    const int64_t k0 = tt / a.tiles_per_plane;
                    x = (int)((tt - k0 * a.tiles_per_plane) * W);
                    y0 = (int)(k0 * (a.n1 / 2));
                }
                if (mode == 1) {
                    mbar_arrive_expect_tx(mb, (unsigned)(LH * W * sizeof(C)) + a.stall_tx);
                    x += (int)(rank * P);
#pragma unroll
                    for (int b = 0; b < LH / kTmaBoxRows; ++b)
                        tma_load_2d(smem_u32(stage + b * kTmaBoxRows * W), &tmap, x, y0 + b * kTmaBoxRows, mb);
                } else if (rank == 0) {
                    mbar_arrive_expect_tx(mb, (unsigned)(LH * W * sizeof(C)) + a.stall_tx);
#pragma unroll
                    for (int b = 0; b < LH / kTmaBoxRows; ++b)
                        tma_load_2d(smem_u32(stage + b * kTmaBoxRows * W), &tmap, x, y0 + b * kTmaBoxRows, mb);
                } else {
                    mbar_arrive_expect_tx(mb, (unsigned)(LH * (W + 2) * sizeof(C)) + a.stall_tx);
#pragma unroll
                    for (int b = 0; b < LH / kTmaBoxRows; ++b)
                        tma_load_2d(smem_u32(stage + b * kTmaBoxRows * (W + 2)), &tmap2, x + (int)a.m,
                                    y0 + b * kTmaBoxRows, mb);
                }
            }
        } else {
            const C *sj = sp + (int64_t)(2 * j + (int)rank) * ss;
            const int64_t sstep = (int64_t)2 * NT * ss;
#pragma unroll
            for (int i = 0; i < E; ++i) cp_async_8(stage + (j + i * NT) * W + c, sj + i * sstep);
            cp_async_commit();
        }
        return mode;
    };

    int64_t t = cluster_id_x();
    const int64_t tstep = cluster_count_x();
    C *sp = nullptr, *dp = nullptr;
    int64_t ss = 0, ds = 0;
    bool valid = t < ntiles && col_decode<C, W>(a, t, c, sp, ss, dp, ds);
    int mode = t < ntiles ? fill(t, sp, ss) : 0;
    while (t < ntiles) {
        const int64_t tn = t + tstep;
        C *spn = nullptr, *dpn = nullptr;
        int64_t ssn = 0, dsn = 0;
        const bool validn = tn < ntiles && col_decode<C, W>(a, tn, c, spn, ssn, dpn, dsn);

        bool ok = true;
        if (mode) ok = mbar_wait_bounded(mb, phase, a.stage_polls);
        else cp_async_wait_all();
        const int bad = __syncthreads_or(!ok);
        int moden = 0;
        C v[E];
        if (!bad) {
            if (mode) phase ^= 1u;
            const int rs = (mode && odd_wide) ? W + 2 : W;
            const C *base = stage + j * rs + c + ((mode && odd_wide) ? 1 : 0);
#pragma unroll
            for (int i = 0; i < E; ++i) {
                v[i] = base[i * NT * rs];
                if (INV) v[i] = cswap(v[i]);
            }
            auto next = [&]() {
                if (tn < ntiles) moden = fill(tn, spn, ssn);
            };
            if constexpr (EARLY) {
                __syncthreads();
                next();
                line_fft<R, LH, E, true>(v, j, tws, ex);
            } else {
                line_fft<R, LH, E, true>(v, j, tws, ex, next);
            }
            if (rank == 1) {  // W_L^k on the half of Y_1 this CTA keeps (k = j + (H + i) NT)
                const C rot_j = tws[NTW + j];  // W_L^j
                static_for<0, H>([&](auto II) {
                    constexpr int i = decltype(II)::value;
                    constexpr CtCosSin w = ct_cossin_pi(-(long long)(H + i), E);
                    v[H + i] = cmul(v[H + i], cmul(rot_j, cmake<C>(R(w.c), R(w.s))));
                });
            }
        }
        // A wait that runs out ends this CTA's loop; the partner's next
        // wait then runs out too, and both meet at the final barrier.
        if (bad) {
            failed = true;
            stage_pending = mode != 0;
            break;
        }
        stage_pending = moden != 0;
        // every thread is past its last read of the exchange buffer (the
        // transform ended on a barrier): arm the receive barrier, then
        // let the partner write
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(mb_rx, (unsigned)(H * W * NT * sizeof(C)));
            mbar_remote_arrive(peer_mb_free);
        }
        rx_pending = true;
        if (__syncthreads_or(!mbar_wait_cluster_bounded(mb_free, xph, a.stage_polls))) {
            failed = true;
            break;
        }
        if (rank == 0) {
#pragma unroll
            for (int i = 0; i < H; ++i) st_async_f2(peer_rx + i * kRxStep, v[H + i], peer_mb_rx);
        } else {
#pragma unroll
            for (int i = 0; i < H; ++i) st_async_f2(peer_rx + i * kRxStep, v[i], peer_mb_rx);
        }
        if (__syncthreads_or(!mbar_wait_cluster_bounded(mb_rx, xph, a.stage_polls))) {
            failed = true;
            break;
        }
        rx_pending = false;
        stage_pending = false;
        xph ^= 1u;
        if (valid) {
            const int64_t dstep = (int64_t)NT * ds;
            const int64_t dhalf = (int64_t)LH * ds;
            // rank 0: k = j + i NT (i < H), own Y_0, received Y_1 (times W_L^k here)
            // rank 1: k = j + (H + i) NT,   received Y_0, own W_L^k Y_1
            C *dj = dp + (int64_t)(j + (int)rank * H * NT) * ds;
            const C rot_j = tws[NTW + j];
            static_for<0, H>([&](auto II) {
                constexpr int i = decltype(II)::value;
                constexpr CtCosSin w = ct_cossin_pi(-(long long)i, E);
                C u = rx[i * W * NT];
                if (rank == 0) u = cmul(u, cmul(rot_j, cmake<C>(R(w.c), R(w.s))));
                const C y0 = rank == 0 ? v[i] : u;
                const C y1 = rank == 0 ? u : v[H + i];
                C lo = cadd(y0, y1), hi = csub(y0, y1);
                if (INV) {
                    lo = cswap(lo);
                    hi = cswap(hi);
                }
                store_out(dj + i * dstep, lo);
                store_out(dj + i * dstep + dhalf, hi);
            });
        }
        t = tn;
        valid = validn;
        mode = moden;
        sp = spn;
        ss = ssn;
        dp = dpn;
        ds = dsn;
    }
    if (failed) {
        if (threadIdx.x == 0) atomicOr(a.err, 1u);
        if (stage_pending) mbar_wait_bounded(mb, phase, a.stage_polls);      // staging copies in flight
        if (rx_pending) mbar_wait_cluster_bounded(mb_rx, xph, a.stage_polls);  // the partner's stores
    }
    cp_async_wait_all();
    cluster_sync_all();  // no CTA leaves while its partner may still address its shared memory
}

// ------------------------------------------------------------ z pass
struct ZArgs {
    const void *real;     // real lines (read by r2c, written by c2r)
    void *real_out;
    int64_t real_pitch;   // line pitch of the real array, in real elements
    CLayout cplx;         // half-spectrum lines (written by r2c, read by c2r)
    int64_t nlines;       // N0 * N1
    double scale_edge;    // r2c: factor on k2 = 0 and M outputs; c2r: weight of k2 = 0, M inputs
    double scale_mid;     // r2c: factor on the other outputs;    c2r: output factor
    int64_t max_blocks;   // > 0: launch at most this many blocks, each looping over line groups
    int64_t pf_lines;     // kernels with the L2 prefetch (z_l2pf): the input line this many lines ahead
                          // (one wave of resident blocks) goes into L2 while this one is transformed
};

// Elements per thread of a z-pass line: the default plan of the length (16,
// or 24 for 3 * 2^k; radix 16 first).  32 elements (radix 32 first, one
// exchange fewer, and one warp per line up to M = 1024) doubles the registers
// of a thread; measured on GB300 it halves the resident warps and runs 25%
// slower at M = 512, and at M = 1024 (150-170 registers, one block per SM)
// 45% slower.
// Double lines of N2 = 1024 points (M = 512), bound by FP64 issue, run two
// lines per complex transform of N2 points (z_paired, zr2c_pairs /
// zc2r_pairs below; 16 elements per thread, radix 16 x 16 x 4): about 33.9
// FP64 operations per element against 36.4 for the half-length scheme on
// radix 8 x 8 x 8; measured at 1024^3 the FP64 z-passes 36.1 -> 34.5 ms.
template <typename R, int M> __host__ __device__ constexpr bool z_paired() { return sizeof(R) == 8 && M == 512; }
template <typename R, int M> __host__ __device__ constexpr int z_E() { return z_paired<R, M>() ? 16 : line_E(M); }

// Per-line shared-memory exchange with one padding slot every 2^P elements:
// P = 4 makes the stride-16 writes of a radix-16 first stage conflict-free;
// 24-element lines use P = 5 (see zline_pad).  Indices arrive padded
// (i + (i >> P), see pad_row).
// A line of more than one warp (M = 1024: 64 threads) syncs only its own
// warps, on named barrier `bar` (1..15) when bar > 0, else the whole block.
// Measured on GB300 at M = 1024 against block barriers: the C2R z-pass 9%
// and the R2C one 1.5% faster.
template <typename C, int NT, int P> struct LineEx {
    static constexpr bool kSplit = false;
    static constexpr int kPadShift = P;
    C *sm;
    int bar;
    __device__ __forceinline__ void put(int pi, C v) { sm[pi] = v; }
    __device__ __forceinline__ C get(int pi) const { return sm[pi]; }
    __device__ __forceinline__ void sync() const
    {
        if (NT <= 32) {
            __syncwarp();
        } else if (bar > 0) {
            asm volatile("bar.sync %0, %1;\n" ::"r"(bar), "n"(NT) : "memory");
        } else {
            __syncthreads();
        }
    }
};
template <int NT, int LPB> __device__ __forceinline__ int line_bar(int lt)
{
    return (NT > 32 && LPB > 1 && LPB < 16) ? 1 + lt : 0;
}

// 24-element lines pad every 32 entries: against every 8, a model of the
// exchange's addresses gives 1.38x instead of 1.75x the conflict-free
// shared-memory wavefronts, and measured on GB300 the 768-point z-passes
// are 1-3% faster (the index arithmetic costs some registers, within the
// same two blocks per SM).
template <int E> __host__ __device__ constexpr int zline_pad() { return E == 24 ? 5 : (E % 3 == 0 ? 3 : 4); }
template <int M, int E> __host__ __device__ constexpr int zline_smem_elems()
{
    return (M + 1) + ((M + 1) >> zline_pad<E>()) + 1;
}

// z-pass kernels (one line group per block) that prefetch into L2, right
// after their own loads, the input lines one wave of resident blocks ahead:
// float lines of 512 points, and the C2R kernel of 768-point lines.
// Measured on GB300: at 1024^3 both z-passes 1.29 -> 1.21 ms (7.1 TB/s); at
// 1536^3 the C2R pass 6.1 -> 5.2 ms; at M = 1024 1-2% slower, and in the
// 768-point R2C kernel the prefetch code raises the registers (120 -> 156).
template <typename R, int M, bool C2R> __host__ __device__ constexpr bool z_l2pf()
{
    return sizeof(R) == 4 && (M == 512 || (C2R && M == 768));
}

#ifndef FFT3D_ROTCONST
#define FFT3D_ROTCONST 1
#endif

// Rotation factor rot[k] = exp(-2 pi i k / 2M) of slot i (k = j + i NT).
// Float lines load rot[j] once and multiply by the slot's constant
// exp(-i pi i / E) (NT / 2M = 1 / 2E); double lines load every factor.
template <typename R, int E, int I>
__device__ __forceinline__ typename cvec<R>::T z_rot(typename cvec<R>::T rot_j,
                                                     const typename cvec<R>::T *__restrict__ rot, int k)
{
    typedef typename cvec<R>::T C;
    if constexpr (FFT3D_ROTCONST && sizeof(R) == 4) {
        if constexpr (I == 0) {
            return rot_j;
        } else {
            constexpr CtCosSin w = ct_cossin_pi(-(long long)I, E);
            return cmul(rot_j, cmake<C>(R(w.c), R(w.s)));
        }
    } else {
        return __ldg(rot + k);
    }
}

// LPB lines starting at line0, NT = M / E threads per line.  R2C: load the
// real line as M complex pairs, M-point FFT, Hermitian post-process.
// Thread j holds Z[j + i NT]; the partner Z[M - k] of k = j + i NT is slot
// E - 1 - i of lane NT - j (j > 0) or this lane's slot (E - i) mod E (j = 0),
// so when a float line fits a warp the post-process takes it by shuffle
// (double lines, bound by FP64 arithmetic, keep the shared-memory exchange
// and its lower register count).
template <typename R, int M, int E, int LPB, bool PF = false>
__device__ __forceinline__ void zr2c_lines(const ZArgs &a, int64_t line0, unsigned char *smem,
                                           const typename cvec<R>::T *__restrict__ tw,
                                           const typename cvec<R>::T *__restrict__ rot)
{
    typedef typename cvec<R>::T C;
    constexpr int NT = M / E;
    constexpr int P = zline_pad<E>();
    const int lt = threadIdx.x / NT;
    const int j = threadIdx.x % NT;
    const int64_t line = line0 + lt;
    const bool active = line < a.nlines;
    LineEx<C, NT, P> ex{(C *)smem + lt * zline_smem_elems<M, E>(), line_bar<NT, LPB>(lt)};

    const C *in = (const C *)((const R *)a.real + (active ? line : 0) * a.real_pitch);
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = active ? in[j + i * NT] : cmake<C>(R(0), R(0));
    if (PF && line + a.pf_lines < a.nlines) {
        const C *ps = (const C *)((const R *)a.real + (line + a.pf_lines) * a.real_pitch);
#pragma unroll
        for (int i = 0; i < E; ++i) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(ps + j + i * NT));
    }
    C rot_j = cmake<C>(R(1), R(0));
    if constexpr (FFT3D_ROTCONST && sizeof(R) == 4) rot_j = __ldg(rot + j);

    line_fft<R, M, E>(v, j, tw, ex);

    C *out = (C *)a.cplx.main + (active ? line : 0) * (M + 1);
    const R se = R(a.scale_edge), sm = R(a.scale_mid);
    // X[k] = (s - i d) / 2 from z = Z[k] and zm = Z[(M - k) mod M]
    auto emit = [&](int k, C z, C zm, C r) {
        const C zc = cconj(zm);
        const C s = cadd(z, zc);          // 2 E[k]
        const C d = cmul(r, csub(z, zc));  // 2i W^k O[k]
        const R f = R(0.5) * (k == 0 ? se : sm);
        if (active) store_out(out + k, cmake<C>(f * (s.x + d.y), f * (s.y - d.x)));
    };
    if constexpr (NT <= 32 && sizeof(R) == 4) {
        const int src = (NT - j) & (NT - 1);
        static_for<0, E>([&](auto II) {
            constexpr int i = decltype(II)::value;
            const int k = j + i * NT;
            C zp;
            zp.x = __shfl_sync(0xffffffffu, v[E - 1 - i].x, src, NT);
            zp.y = __shfl_sync(0xffffffffu, v[E - 1 - i].y, src, NT);
            const C zm = (j == 0) ? v[(E - i) % E] : zp;
            emit(k, v[i], zm, z_rot<R, E, i>(rot_j, rot, k));
        });
    } else if constexpr (sizeof(R) == 8) {
        // Double lines (bound by FP64 issue): X[k] = A[k] Z[k] + B[k] conj(Z[M - k]),
        // A = (1 - i r) / 2, B = (1 + i r) / 2 from the coefficient table (`rot`
        // holds [A, B] pairs), 8 FP64 operations per element instead of 12; the
        // output scale is applied only when it is not 1.
        constexpr bool LR = pad_linear_reads<P>(NT);
        constexpr bool LREV = P < 0 || NT % (1 << P) == 0;
#pragma unroll
        for (int i = 0; i < E; ++i) ex.put(pad_row<P, LR>(j, i * NT), v[i]);
        ex.sync();
        const bool unit = se == R(1) && sm == R(1);
        static_for<0, E>([&](auto II) {
            constexpr int i = decltype(II)::value;
            const int k = j + i * NT;
            const C z = ex.get(pad_row<P, LR>(j, i * NT));
            const C zm = (i == 0 && j == 0) ? z : ex.get(pad_row<P, LREV>(M - j, -i * NT));
            const C A = __ldg(rot + 2 * k), B = __ldg(rot + 2 * k + 1);
            // A z + B conj(zm)
            C x = cmake<C>(fma(A.x, z.x, fma(-A.y, z.y, fma(B.x, zm.x, B.y * zm.y))),
                           fma(A.x, z.y, fma(A.y, z.x, fma(B.y, zm.x, -B.x * zm.y))));
            if (!unit) x = cscale(x, k == 0 ? se : sm);
            if (active) store_out(out + k, x);
        });
    } else {
        constexpr bool LR = pad_linear_reads<P>(NT);
        constexpr bool LREV = P < 0 || NT % (1 << P) == 0;  // M - j - i NT stays linear in i
#pragma unroll
        for (int i = 0; i < E; ++i) ex.put(pad_row<P, LR>(j, i * NT), v[i]);
        ex.sync();
        static_for<0, E>([&](auto II) {
            constexpr int i = decltype(II)::value;
            const int k = j + i * NT;
            const C z = v[i];  // this thread's own Z[k] is still in registers
            const C zm = ex.get(pad_row<P, LREV>(M - j, -i * NT));  // Z[M - k]; k = 0 reads index M
            emit(k, z, (i == 0 && j == 0) ? z : zm, z_rot<R, E, i>(rot_j, rot, k));
        });
    }
    if (active && j == 0) {
        // X[M] = E[0] - O[0] = Re Z[0] - Im Z[0]
        out[M] = cmake<C>(se * (v[0].x - v[0].y), R(0));
    }
}

// C2R of LPB lines: Hermitian pre-process, M-point inverse FFT, unpack into
// 2M reals with the output scale.  CG selects L2-only loads of the spectrum.
// The partner X[M - k] comes by shuffle as in zr2c_lines (lane 0 pairs k = 0
// with X[M], which it loads itself).
template <typename R, int M, int E, int LPB, bool CG, bool PF = false>
__device__ __forceinline__ void zc2r_lines(const ZArgs &a, int64_t line0, unsigned char *smem,
                                           const typename cvec<R>::T *__restrict__ tw,
                                           const typename cvec<R>::T *__restrict__ rot)
{
    typedef typename cvec<R>::T C;
    constexpr int NT = M / E;
    constexpr int P = zline_pad<E>();
    const int lt = threadIdx.x / NT;
    const int j = threadIdx.x % NT;
    const int64_t line = line0 + lt;
    const bool active = line < a.nlines;
    LineEx<C, NT, P> ex{(C *)smem + lt * zline_smem_elems<M, E>(), line_bar<NT, LPB>(lt)};

    const int64_t l = active ? line : 0;
    const C *src;
    const C *nyq;
    if (a.cplx.split) {
        src = (const C *)a.cplx.main + l * M;
        nyq = (const C *)a.cplx.nyq + l;
    } else {
        src = (const C *)a.cplx.main + l * (M + 1);
        nyq = src + M;
    }
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i)
        v[i] = active ? (CG ? load_cg(src + j + i * NT) : src[j + i * NT]) : cmake<C>(R(0), R(0));
    if (PF && line + a.pf_lines < a.nlines) {
        const int64_t pl = line + a.pf_lines;
        const C *ps = (const C *)a.cplx.main + pl * (a.cplx.split ? M : M + 1);
#pragma unroll
        for (int i = 0; i < E; ++i) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(ps + j + i * NT));
    }
    C rot_j = cmake<C>(R(1), R(0));
    if constexpr (FFT3D_ROTCONST && sizeof(R) == 4) rot_j = __ldg(rot + j);

    const R we = R(a.scale_edge);
    // conj(Z[k]), Z = E + i O, from x = X[k] and y = X[M - k]
    auto pre = [&](int k, C x, C y, C r) -> C {
        if (k == 0) {
            // only the real parts of the k2 = 0 and k2 = M entries enter
            x = cmake<C>(we * x.x, R(0));
            y = cmake<C>(we * y.x, R(0));
        }
        const C yc = cconj(y);
        const C e = cadd(x, yc);               // E[k] (times 2)
        const C o = cmulc(csub(x, yc), r);     // O[k] (times 2)
        return cmake<C>(e.x - o.y, -(e.y + o.x));
    };
    if constexpr (NT <= 32 && sizeof(R) == 4) {
        const C xm = (active && j == 0) ? (CG ? load_cg(nyq) : *nyq) : cmake<C>(R(0), R(0));
        const int srcl = (NT - j) & (NT - 1);
        C pv[E];
        static_for<0, E>([&](auto II) {
            constexpr int i = decltype(II)::value;
            C p;
            p.x = __shfl_sync(0xffffffffu, v[E - 1 - i].x, srcl, NT);
            p.y = __shfl_sync(0xffffffffu, v[E - 1 - i].y, srcl, NT);
            pv[i] = (j == 0) ? (i == 0 ? xm : v[(E - i) % E]) : p;
        });
        static_for<0, E>([&](auto II) {
            constexpr int i = decltype(II)::value;
            const int k = j + i * NT;
            v[i] = pre(k, v[i], pv[i], z_rot<R, E, i>(rot_j, rot, k));
        });
    } else {
        constexpr bool LR = pad_linear_reads<P>(NT);
        constexpr bool LREV = P < 0 || NT % (1 << P) == 0;
#pragma unroll
        for (int i = 0; i < E; ++i) ex.put(pad_row<P, LR>(j, i * NT), v[i]);
        if (j == 0) ex.put(pad_row<P, true>(M, 0), active ? (CG ? load_cg(nyq) : *nyq) : cmake<C>(R(0), R(0)));
        ex.sync();
        static_for<0, E>([&](auto II) {
            constexpr int i = decltype(II)::value;
            const int k = j + i * NT;
            // float lines take their own X[k] from registers (one shared-memory read
            // fewer per element for the L1-bound two-warp lines)
            C x = sizeof(R) == 4 ? v[i] : ex.get(pad_row<P, LR>(j, i * NT));
            C y = ex.get(pad_row<P, LREV>(M - j, -i * NT));  // X[M - k]; k = 0 pairs with X[M]
            if constexpr (sizeof(R) == 8) {
                // Double lines: conj Z[k] = 2 (A[k] conj(x) + B[k] y) with the
                // coefficient table of the R2C lines (8 FP64 operations instead
                // of 10); the factor 2 goes into the output scale below.
                if (k == 0) {
                    x = cmake<C>(we * x.x, R(0));
                    y = cmake<C>(we * y.x, R(0));
                }
                const C A = __ldg(rot + 2 * k), B = __ldg(rot + 2 * k + 1);
                v[i] = cmake<C>(fma(A.x, x.x, fma(A.y, x.y, fma(B.x, y.x, -B.y * y.y))),
                                fma(A.y, x.x, fma(-A.x, x.y, fma(B.x, y.y, B.y * y.x))));
            } else {
                v[i] = pre(k, x, y, z_rot<R, E, i>(rot_j, rot, k));
            }
        });
        ex.sync();
    }

    line_fft<R, M, E>(v, j, tw, ex);

    const R s = R(sizeof(R) == 8 ? 2.0 * a.scale_mid : a.scale_mid);
    C *out = (C *)((R *)a.real_out + l * a.real_pitch);
    if (active) {
#pragma unroll
        for (int i = 0; i < E; ++i) store_out(out + j + i * NT, cmake<C>(s * v[i].x, -s * v[i].y));
    }
}

// Two real lines per complex transform (double, z_paired).  Lines l and
// l + 1 (l even) are read as z[n] = x_l[n] + i x_{l+1}[n], n < N = 2M, and
// transformed once: Z = DFT_N(z).  Since both lines are real, their spectra
// follow from Z and its mirror:
//   X_l[k] = (Z[k] + conj Z[N - k]) / 2,  X_{l+1}[k] = (Z[k] - conj Z[N - k]) / 2i,
// for k <= M (4 FP64 operations per output value, the 1/2 folded into the
// output scale), against the half-length scheme's rotation post-process.  A
// pair takes N / E threads; thread j holds Z[j + i NT] and reads Z[N - k]
// of the partner thread through the line's shared-memory buffer.  With an
// odd line count the last pair's second line is zero and not written.
template <typename R, int M, int E, int LPB>
__device__ __forceinline__ void zr2c_pairs(const ZArgs &a, int64_t line0, unsigned char *smem,
                                           const typename cvec<R>::T *__restrict__ tw)
{
    typedef typename cvec<R>::T C;
    constexpr int N = 2 * M;
    constexpr int NT = N / E;
    constexpr int PPB = LPB / 2;  // pairs per block
    constexpr int P = zline_pad<E>();
    static_assert(LPB % 2 == 0 && E % 2 == 0, "pairs of lines");
    const int pt = threadIdx.x / NT;
    const int j = threadIdx.x % NT;
    const int64_t l0 = line0 + 2 * pt;
    const bool act0 = l0 < a.nlines, act1 = l0 + 1 < a.nlines;
    LineEx<C, NT, P> ex{(C *)smem + pt * zline_smem_elems<N, E>(), line_bar<NT, PPB>(pt)};

    const R *in0 = (const R *)a.real + (act0 ? l0 : 0) * a.real_pitch;
    const R *in1 = (const R *)a.real + (act1 ? l0 + 1 : 0) * a.real_pitch;
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int n = j + i * NT;
        v[i] = cmake<C>(act0 ? in0[n] : R(0), act1 ? in1[n] : R(0));
    }
    line_fft<R, N, E>(v, j, tw, ex);

    constexpr bool LR = pad_linear_reads<P>(NT);
    constexpr bool LREV = P < 0 || NT % (1 << P) == 0;
#pragma unroll
    for (int i = 0; i < E; ++i) ex.put(pad_row<P, LR>(j, i * NT), v[i]);
    ex.sync();
    C *out0 = (C *)a.cplx.main + (act0 ? l0 : 0) * (M + 1);
    C *out1 = out0 + (M + 1);
    const R he = R(0.5 * a.scale_edge), hm = R(0.5 * a.scale_mid);
    // slots with k = j + i NT <= M: i < M / NT, and k = M itself for j = 0
    static_for<0, M / NT + 1>([&](auto II) {
        constexpr int i = decltype(II)::value;
        if (i < M / NT || j == 0) {
            const int k = j + i * NT;
            const C z = v[i];
            const C zm = (k == 0 || k == M) ? z : ex.get(pad_row<P, LREV>(N - j, -i * NT));  // Z[N - k]
            const R f = (k == 0 || k == M) ? he : hm;
            if (act0) store_out(out0 + k, cmake<C>(f * (z.x + zm.x), f * (z.y - zm.y)));
            if (act1) store_out(out1 + k, cmake<C>(f * (z.y + zm.y), f * (zm.x - z.x)));
        }
    });
}

// C2R of two lines per complex transform (double, z_paired): thread j
// builds Z[k] = Xt_l[k] + i Xt_{l+1}[k] for its k = j + i NT from the
// Hermitian extensions Xt[k] = X[k] (k <= M), conj X[N - k] (k > M) of both
// stored half spectra (only the real parts of the k = 0 and M entries enter,
// weighted by scale_edge), reading each entry it needs itself (no exchange),
// runs the inverse transform, and writes Re z to line l and Im z to line l + 1
// with the output scale.  CG selects L2-only loads.
template <typename R, int M, int E, int LPB, bool CG>
__device__ __forceinline__ void zc2r_pairs(const ZArgs &a, int64_t line0, unsigned char *smem,
                                           const typename cvec<R>::T *__restrict__ tw)
{
    typedef typename cvec<R>::T C;
    constexpr int N = 2 * M;
    constexpr int NT = N / E;
    constexpr int PPB = LPB / 2;
    constexpr int P = zline_pad<E>();
    static_assert(LPB % 2 == 0, "pairs of lines");
    const int pt = threadIdx.x / NT;
    const int j = threadIdx.x % NT;
    const int64_t l0 = line0 + 2 * pt;
    const bool act0 = l0 < a.nlines, act1 = l0 + 1 < a.nlines;
    LineEx<C, NT, P> ex{(C *)smem + pt * zline_smem_elems<N, E>(), line_bar<NT, PPB>(pt)};

    const C *src0, *src1, *nyq0, *nyq1;
    const int64_t la = act0 ? l0 : 0, lb = act1 ? l0 + 1 : 0;
    if (a.cplx.split) {
        src0 = (const C *)a.cplx.main + la * M;
        src1 = (const C *)a.cplx.main + lb * M;
        nyq0 = (const C *)a.cplx.nyq + la;
        nyq1 = (const C *)a.cplx.nyq + lb;
    } else {
        src0 = (const C *)a.cplx.main + la * (M + 1);
        src1 = (const C *)a.cplx.main + lb * (M + 1);
        nyq0 = src0 + M;
        nyq1 = src1 + M;
    }
    auto fetch = [&](const C *src, const C *nyq, bool act, int idx) -> C {
        if (!act) return cmake<C>(R(0), R(0));
        const C *p = idx == M ? nyq : src + idx;
        return CG ? load_cg(p) : *p;
    };
    const R we = R(a.scale_edge);
    C v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int k = j + i * NT;
        const int idx = k <= M ? k : N - k;
        C x0 = fetch(src0, nyq0, act0, idx), x1 = fetch(src1, nyq1, act1, idx);
        if (idx == 0 || idx == M) {
            x0 = cmake<C>(we * x0.x, R(0));
            x1 = cmake<C>(we * x1.x, R(0));
        } else if (k > M) {
            x0 = cconj(x0);
            x1 = cconj(x1);
        }
        // inverse transform as swap(DFT(swap(Z))), Z = x0 + i x1
        v[i] = cswap(cmake<C>(x0.x - x1.y, x0.y + x1.x));
    }
    line_fft<R, N, E>(v, j, tw, ex);

    const R s = R(a.scale_mid);
    R *out0 = (R *)a.real_out + la * a.real_pitch;
    R *out1 = (R *)a.real_out + lb * a.real_pitch;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const C z = cswap(v[i]);  // x0 + i x1 at n = j + i NT
        if (act0) store_out(out0 + j + i * NT, s * z.x);
        if (act1) store_out(out1 + j + i * NT, s * z.y);
    }
}

// One group of LPB lines per block; with LOOP, a grid of a.max_blocks blocks
// walks the line groups (the host-memory form, bound by the CPU-GPU link).
// Two instances because the loop slows the one-pass form down (up to 20%
// measured for the C2R lines on GB300).
// Minimum resident blocks in the launch bounds of the R2C z kernel: 1 (an
// explicit floor, which changes the compiler's register budget) for float
// lines of 3 * 2^k >= 384 points, else 0 (no floor).  Measured on GB300 the
// floor cuts registers 127 -> 107 (M = 768) and 123 -> 95 (M = 384), and
// the pass time by 7-8% (1536^3: 5.77 -> 5.33 ms); for M = 96 it is 1%
// slower, and for the C2R kernel, or powers of two, it raises registers.
template <typename R, int M, int E> __host__ __device__ constexpr int zr2c_minb()
{
    return sizeof(R) == 4 && E == 24 && M >= 384 ? 1 : 0;
}

template <typename R, int M, int E, int LPB, bool LOOP>
__global__ void __launch_bounds__(LPB *(M / E), zr2c_minb<R, M, E>())
zpass_r2c_kernel(ZArgs a, const typename cvec<R>::T *__restrict__ tw,
                 const typename cvec<R>::T *__restrict__ rot)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (LOOP) {
        for (int64_t blk = blockIdx.x; blk * LPB < a.nlines; blk += gridDim.x) {
            if (blk != blockIdx.x) __syncthreads();  // shared memory free for the next line group
            if constexpr (z_paired<R, M>()) zr2c_pairs<R, M, E, LPB>(a, blk * LPB, smem_raw, tw);
            else zr2c_lines<R, M, E, LPB>(a, blk * LPB, smem_raw, tw, rot);
        }
    } else if constexpr (z_paired<R, M>()) {
        zr2c_pairs<R, M, E, LPB>(a, (int64_t)blockIdx.x * LPB, smem_raw, tw);
    } else {
        zr2c_lines<R, M, E, LPB, z_l2pf<R, M, false>()>(a, (int64_t)blockIdx.x * LPB, smem_raw, tw, rot);
    }
}

template <typename R, int M, int E, int LPB, bool LOOP>
__global__ void __launch_bounds__(LPB *(M / E))
zpass_c2r_kernel(ZArgs a, const typename cvec<R>::T *__restrict__ tw,
                 const typename cvec<R>::T *__restrict__ rot)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (LOOP) {
        for (int64_t blk = blockIdx.x; blk * LPB < a.nlines; blk += gridDim.x) {
            if (blk != blockIdx.x) __syncthreads();  // shared memory free for the next line group
            if constexpr (z_paired<R, M>()) zc2r_pairs<R, M, E, LPB, false>(a, blk * LPB, smem_raw, tw);
            else zc2r_lines<R, M, E, LPB, false>(a, blk * LPB, smem_raw, tw, rot);
        }
    } else if constexpr (z_paired<R, M>()) {
        zc2r_pairs<R, M, E, LPB, false>(a, (int64_t)blockIdx.x * LPB, smem_raw, tw);
    } else {
        zc2r_lines<R, M, E, LPB, false, z_l2pf<R, M, true>()>(a, (int64_t)blockIdx.x * LPB, smem_raw, tw, rot);
    }
}

// ------------------------------------------------------------ twiddles
// Stage table of a line plan: entry (m - 1) * ns + k = exp(-2 pi i m k / (ns r)),
// computed in FP64 with sincospi after exact integer reduction of m k, then
// rounded once to the storage type.
template <typename R>
__global__ void twiddle_stage_kernel(typename cvec<R>::T *out, int ns, int r)
{
    typedef typename cvec<R>::T C;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (r - 1) * ns) return;
    const int m = i / ns + 1;
    const int k = i - (m - 1) * ns;
    const int64_t d = (int64_t)ns * r;
    const int64_t p = ((int64_t)m * k) % d;
    double s, c;
    sincospi(2.0 * (double)p / (double)d, &s, &c);
    out[i] = cmake<C>(R(c), R(-s));
}

// Coefficients of the Hermitian post- / pre-process of double lines, for
// k <= count - 1: with r = exp(-2 pi i k / n) = (cos t, -sin t),
//   out[2k] = A = (1 - i r) / 2 = ((1 - sin t) / 2, -cos t / 2),
//   out[2k + 1] = B = (1 + i r) / 2 = ((1 + sin t) / 2, cos t / 2),
// computed in FP64 from sincospi (after exact reduction of k mod n).
template <typename R>
__global__ void twiddle_herm_kernel(typename cvec<R>::T *out, int n, int count)
{
    typedef typename cvec<R>::T C;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    double s, c;
    sincospi(2.0 * (double)(k % n) / (double)n, &s, &c);
    out[2 * k] = cmake<C>(R(0.5 - 0.5 * s), R(-0.5 * c));
    out[2 * k + 1] = cmake<C>(R(0.5 + 0.5 * s), R(0.5 * c));
}

// rot[k] = exp(-2 pi i k / n), k < count (FP64 sincospi, rounded once)
template <typename R>
__global__ void twiddle_rot_kernel(typename cvec<R>::T *out, int n, int count)
{
    typedef typename cvec<R>::T C;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)n, &s, &c);
    out[k] = cmake<C>(R(c), R(-s));
}

}  // namespace fft3d
