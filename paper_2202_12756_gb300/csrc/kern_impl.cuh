// Launch policy and length dispatch, instantiated once per dtype by the
// kern_{col,z}_{f32,f64}.cu translation units.
#pragma once

#include <cstring>
#include <mutex>

#include "launchers.h"

namespace fft3d {

#ifndef FFT3D_COL_MAXT_F32
#define FFT3D_COL_MAXT_F32 1024
#endif
#ifndef FFT3D_COL_MAXT_F64
#define FFT3D_COL_MAXT_F64 256
#endif
#ifndef FFT3D_Z_THREADS
#define FFT3D_Z_THREADS 256
#endif

// Block-size cap of a one-tile-per-block column pass: 1024 threads for float
// (so a tile row stays one 128-byte segment even at 24 elements per thread,
// at the price of a few spilled registers there), 256 for double.  Double
// passes are bound by FP64 issue, not by HBM, so narrower tiles (64-byte row
// segments of 4 columns at 1024 points) cost them nothing in DRAM terms and
// let two blocks share an SM, which hides each tile's loads and barriers:
// measured on GB300 at 1024^3, FP64 column passes 31.5-32.0 -> 30.2-30.3 ms
// (a 128-thread cap: 30.2 ms; 512 threads, one block per SM: the former).
template <typename R, int L> __host__ __device__ constexpr int col_max_threads()
{
    return sizeof(R) == 4 ? FFT3D_COL_MAXT_F32 : (line_E(L) <= 16 ? FFT3D_COL_MAXT_F64 : 256);
}

// float columns of 2^k >= 1024 points use the persistent pipelined kernel
// with 32 elements per thread (radix-32 stages: one exchange at 1024 points);
// measured on GB300 it is a few percent faster than one tile per block at
// 1024 points and slower at 512.
template <typename R, int L> __host__ __device__ constexpr bool col_pipe()
{
#ifdef FFT3D_NO_PIPE
    return false;
#else
    return sizeof(R) == 4 && is_pow2(L) && L >= 1024;
#endif
}

// float columns of 1536 points can run the persistent kernel whose staging
// buffer doubles as its exchange buffer (colpass_xstage_kernel): a tile of 16
// such columns (192 KB) leaves no room for a second buffer.  Measured on
// GB300 at 1536^3 it makes the x-pass 11% faster (7.13 -> 6.37 ms) and the
// y-pass 8% slower (7.17 -> 7.75 ms; the one-tile kernel's next-wave L2
// prefetch serves its 6 KB row pitch better), so it serves the x-pass.
template <typename R, int L> __host__ __device__ constexpr bool col_xstage()
{
    return sizeof(R) == 4 && L == 1536;
}
__host__ __device__ constexpr bool xstage_axis(int axis) { return axis == 0; }

// float columns of 2048 points can run one tile of 16 columns per CTA pair
// (colpass_pair_kernel), every row a 128-byte segment, instead of 8-column
// tiles on one SM.  Measured on GB300 the pair makes the x-pass (rows one
// N1 (N2/2+1) pitch apart, 2-17 MB) 20-37% faster and the y-pass (rows 4 KB
// apart, where 64-byte segments of neighbouring rows share DRAM pages) 15%
// slower, so it serves the axes in FFT3D_PAIR_AXES (bit 0: x-pass, bit 1:
// y-pass).
#ifndef FFT3D_PAIR_AXES
#define FFT3D_PAIR_AXES 1
#endif
// (At 1536 points the pair, with 768-point halves, measured 19% slower than
// the one-tile kernel, whose 1024-thread blocks already read 128-byte rows.)
template <typename R, int L> __host__ __device__ constexpr bool col_pair()
{
    return sizeof(R) == 4 && L == 2048 && FFT3D_PAIR_AXES != 0;
}
// elements per thread of a pair's half-length transform (radix 32 x 32)
template <int L> __host__ __device__ constexpr int pair_E() { return 32; }
__host__ __device__ constexpr bool pair_axis(int axis) { return axis >= 0 && ((FFT3D_PAIR_AXES >> axis) & 1) != 0; }
constexpr int kPairW = 16;  // columns of a CTA-pair tile (128-byte float rows)

// Elements per thread of a column pass: 32 in the pipelined kernel, else the
// default plan of the length; double columns of 512 points, bound by FP64
// issue, take 8 (radix 8 x 8 x 8: about 28 FP64 operations per point
// against 28.75 for 16 x 16 x 2; measured at 512^3 the FP64 column passes
// 3.43 -> 3.34 ms, on 4-column tiles).
template <typename R, int L> __host__ __device__ constexpr int col_E()
{
    return col_pipe<R, L>() ? 32 : ((sizeof(R) == 8 && L == 512) ? 8 : line_E(L));
}

// Columns per tile: one 128-byte segment per row (16 float2 or 8 double2),
// halved while the block would exceed its thread cap or, for the one-tile
// kernel, the tile 200 KB of shared memory.
template <typename R, int L> __host__ __device__ constexpr int col_W()
{
    int w = 128 / (int)sizeof(typename cvec<R>::T);
    if (col_pipe<R, L>()) {
        while (w > 1 && w * (L / 32) > 512) w /= 2;
        return w;
    }
    while (w > 1 && (w * (L / col_E<R, L>()) > col_max_threads<R, L>() ||
                     (size_t)L * w * sizeof(typename cvec<R>::T) > 200 * 1024))
        w /= 2;
    return w;
}

// Lines per block of a z pass: about 256 threads, and at least one warp.
template <typename R, int M> __host__ __device__ constexpr int z_LPB()
{
    return M / z_E<R, M>() >= FFT3D_Z_THREADS ? 1 : FFT3D_Z_THREADS / (M / z_E<R, M>());
}

template <typename R, int L> inline void col_geom_t(PassGeom *g, int axis)
{
    constexpr int W = col_W<R, L>();
    constexpr int E = col_E<R, L>();
    g->threads = W * (L / E);
    g->per_block = W;
    g->E = E;
    const bool xstage = col_xstage<R, L>() && xstage_axis(axis);
    g->persistent = (col_pipe<R, L>() || xstage) ? 1 : 0;
    g->pair = col_pair<R, L>() && pair_axis(axis) ? 1 : 0;
    typedef typename cvec<R>::T C;
    if constexpr (col_pair<R, L>()) {
        if (g->pair) {
            constexpr int PE = pair_E<L>();
            g->threads = kPairW * (L / 2 / PE);
            g->per_block = kPairW;
            g->E = PE;
            g->persistent = 1;
            g->smem = pair_smem_bytes<L, PE, kPairW>();
            return;
        }
    }
    if (col_pipe<R, L>())
        g->smem = pipe_smem_bytes<R, L, E, W>();
    else if (xstage)
        g->smem = xstage_smem_bytes<R, L, E, W>();
    else
        g->smem = (size_t)L * W * sizeof(C);
}

template <typename R, int M> inline void z_geom_t(PassGeom *g)
{
    constexpr int LPB = z_LPB<R, M>();
    g->threads = LPB * (M / z_E<R, M>());
    g->per_block = LPB;
    g->E = z_E<R, M>();
    g->persistent = 0;
    // paired lines: one buffer of the 2M-point transform per pair
    g->pair = z_paired<R, M>() ? 1 : 0;
    g->smem = (z_paired<R, M>() ? (size_t)(LPB / 2) * zline_smem_elems<2 * M, z_E<R, M>()>()
                                : (size_t)LPB * zline_smem_elems<M, z_E<R, M>()>()) *
              sizeof(typename cvec<R>::T);
}

template <typename R, int L> inline cudaError_t col_prepare_t()
{
    PassGeom g;
    col_geom_t<R, L>(&g, -1);  // the one-SM kernels of the length
    cudaError_t e;
    if constexpr (col_pair<R, L>()) {
        constexpr int E = pair_E<L>(), W = kPairW;
        const void *const ks[4] = {(const void *)colpass_pair_kernel<R, L, E, W, false, false>,
                                   (const void *)colpass_pair_kernel<R, L, E, W, true, false>,
                                   (const void *)colpass_pair_kernel<R, L, E, W, false, true>,
                                   (const void *)colpass_pair_kernel<R, L, E, W, true, true>};
        for (const void *k : ks) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pair_smem_bytes<L, E, W>());
            if (e != cudaSuccess) return e;
        }
    }
    if constexpr (col_pipe<R, L>()) {
        constexpr int E = col_E<R, L>(), W = col_W<R, L>();
        const void *const ks[4] = {(const void *)colpass_pipe_kernel<R, L, E, W, false, false>,
                                   (const void *)colpass_pipe_kernel<R, L, E, W, true, false>,
                                   (const void *)colpass_pipe_kernel<R, L, E, W, false, true>,
                                   (const void *)colpass_pipe_kernel<R, L, E, W, true, true>};
        for (const void *k : ks) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    } else {
        if constexpr (col_xstage<R, L>()) {
            constexpr int E = col_E<R, L>(), W = col_W<R, L>();
            const int xs = (int)xstage_smem_bytes<R, L, E, W>();
            e = cudaFuncSetAttribute(colpass_xstage_kernel<R, L, E, W, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, xs);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(colpass_xstage_kernel<R, L, E, W, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, xs);
            if (e != cudaSuccess) return e;
        }
        e = cudaFuncSetAttribute(colpass_kernel<R, L, col_E<R, L>(), col_W<R, L>(), false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(colpass_kernel<R, L, col_E<R, L>(), col_W<R, L>(), true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    }
}

template <typename R, int M> inline cudaError_t z_prepare_t()
{
    PassGeom g;
    z_geom_t<R, M>(&g);
    constexpr int E = z_E<R, M>(), LPB = z_LPB<R, M>();
    const void *const ks[4] = {(const void *)zpass_r2c_kernel<R, M, E, LPB, false>,
                               (const void *)zpass_r2c_kernel<R, M, E, LPB, true>,
                               (const void *)zpass_c2r_kernel<R, M, E, LPB, false>,
                               (const void *)zpass_c2r_kernel<R, M, E, LPB, true>};
    for (const void *k : ks) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Resident blocks of a persistent kernel on the current device, cached per
// (kernel, device), capped at the blocks that get work: `items` work items
// taken `per_block_items` at a time.
template <class K>
inline int persistent_grid(K kernel, int threads, size_t smem, int64_t items, int per_block_items = 1)
{
    struct Entry {
        const void *k;
        int dev;
        int blocks;
    };
    static Entry cache[64];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    int per_dev = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry &e : cache)
            if (e.k == (const void *)kernel && e.dev == dev) per_dev = e.blocks;
    }
    if (per_dev <= 0) {
        int sms = 0, nb = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
        per_dev = (sms > 0 ? sms : 1) * (nb > 0 ? nb : 1);
        std::lock_guard<std::mutex> lock(mu);
        for (Entry &e : cache)
            if (e.k == nullptr) {
                e = Entry{(const void *)kernel, dev, per_dev};
                break;
            }
    }
    const int64_t need = (items + per_block_items - 1) / per_block_items;
    return (int)(need < per_dev ? need : per_dev);
}

// Co-resident clusters of two CTAs of a pair kernel on the current device,
// cached per (kernel, device), capped at `items` (one tile per cluster at a time).
template <class K> inline int pair_clusters(K kernel, int threads, size_t smem, int64_t items)
{
    struct Entry {
        const void *k;
        int dev;
        int clusters;
    };
    static Entry cache[16];
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    int per_dev = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (const Entry &e : cache)
            if (e.k == (const void *)kernel && e.dev == dev) per_dev = e.clusters;
    }
    if (per_dev <= 0) {
        int sms = 0, nc = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3((unsigned)(sms > 1 ? sms / 2 * 2 : 2), 1, 1);
        cfg.blockDim = dim3((unsigned)threads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        if (cudaOccupancyMaxActiveClusters(&nc, (const void *)kernel, &cfg) != cudaSuccess || nc <= 0) {
            (void)cudaGetLastError();
            nc = sms > 1 ? sms / 2 : 1;
        }
        per_dev = nc;
        std::lock_guard<std::mutex> lock(mu);
        for (Entry &e : cache)
            if (e.k == nullptr) {
                e = Entry{(const void *)kernel, dev, per_dev};
                break;
            }
    }
    return (int)(items < per_dev ? items : per_dev);
}

// One-tile column pass (float): each block prefetches into L2 the tile one
// wave of resident blocks ahead while it transforms its own.  Measured on
// GB300: y-passes 4-11% faster (512, 768 and 1536 points), x-passes of 768
// points 3% faster and of 512 as fast, but the 1536-point x-pass (rows one
// N1 (N2/2+1) pitch apart, one block per SM) 10% slower, so it is left out.
template <typename R, int L> constexpr bool col_l2_prefetch(int axis)
{
    return sizeof(R) == 4 && !(axis == 0 && L >= 1536);
}

template <typename R, int L>
inline cudaError_t col_launch_t(const ColArgs &a, int64_t tiles, const void *tw, const CUtensorMap *tmap,
                                const CUtensorMap *tmap2, cudaStream_t st)
{
    PassGeom g;
    col_geom_t<R, L>(&g, a.axis);
    typedef const typename cvec<R>::T *TW;
    if constexpr (col_pair<R, L>()) {
        if (g.pair) {
            constexpr int E = pair_E<L>(), W = kPairW;
            auto k = a.early ? (a.inverse ? colpass_pair_kernel<R, L, E, W, true, true>
                                          : colpass_pair_kernel<R, L, E, W, false, true>)
                             : (a.inverse ? colpass_pair_kernel<R, L, E, W, true, false>
                                          : colpass_pair_kernel<R, L, E, W, false, false>);
            const int grid = 2 * pair_clusters(k, g.threads, g.smem, tiles);
            CUtensorMap map, map2;
            if (tmap) map = *tmap;
            else memset(&map, 0, sizeof(map));
            if (tmap2) map2 = *tmap2;
            else memset(&map2, 0, sizeof(map2));
            k<<<grid, g.threads, g.smem, st>>>(a, (TW)tw, tiles, map, map2);
            return cudaGetLastError();
        }
    }
    if constexpr (col_pipe<R, L>()) {
        constexpr int E = col_E<R, L>(), W = col_W<R, L>();
        auto k = a.early ? (a.inverse ? colpass_pipe_kernel<R, L, E, W, true, true>
                                      : colpass_pipe_kernel<R, L, E, W, false, true>)
                         : (a.inverse ? colpass_pipe_kernel<R, L, E, W, true, false>
                                      : colpass_pipe_kernel<R, L, E, W, false, false>);
        const int grid = persistent_grid(k, g.threads, g.smem, tiles);
        CUtensorMap map, map2;
        if (tmap) map = *tmap;
        else memset(&map, 0, sizeof(map));
        if (tmap2) map2 = *tmap2;
        else memset(&map2, 0, sizeof(map2));
        k<<<grid, g.threads, g.smem, st>>>(a, (TW)tw, tiles, map, map2);
    } else {
        if constexpr (col_xstage<R, L>()) {
            if (g.persistent) {
                constexpr int E = col_E<R, L>(), W = col_W<R, L>();
                auto k = a.inverse ? colpass_xstage_kernel<R, L, E, W, true>
                                   : colpass_xstage_kernel<R, L, E, W, false>;
                const int grid = persistent_grid(k, g.threads, g.smem, tiles);
                CUtensorMap map, map2;
                if (tmap) map = *tmap;
                else memset(&map, 0, sizeof(map));
                if (tmap2) map2 = *tmap2;
                else memset(&map2, 0, sizeof(map2));
                k<<<grid, g.threads, g.smem, st>>>(a, (TW)tw, tiles, map, map2);
                return cudaGetLastError();
            }
        }
        auto k = a.inverse ? colpass_kernel<R, L, col_E<R, L>(), col_W<R, L>(), true>
                           : colpass_kernel<R, L, col_E<R, L>(), col_W<R, L>(), false>;
        ColArgs b = a;
        b.pf_stride = col_l2_prefetch<R, L>(a.axis) ? persistent_grid(k, g.threads, g.smem, (int64_t)1 << 40) : 0;
        k<<<(unsigned)tiles, g.threads, g.smem, st>>>(b, (TW)tw);
    }
    return cudaGetLastError();
}

template <typename R, int M>
inline cudaError_t zr2c_launch_t(const ZArgs &a, const void *tw, const void *rot, cudaStream_t st)
{
    PassGeom g;
    z_geom_t<R, M>(&g);
    constexpr int E = z_E<R, M>(), LPB = z_LPB<R, M>();
    const int64_t blocks = (a.nlines + g.per_block - 1) / g.per_block;
    typedef const typename cvec<R>::T *TW;
    if (a.max_blocks > 0 && blocks > a.max_blocks)
        zpass_r2c_kernel<R, M, E, LPB, true><<<(unsigned)a.max_blocks, g.threads, g.smem, st>>>(a, (TW)tw, (TW)rot);
    else {
        auto k = zpass_r2c_kernel<R, M, E, LPB, false>;
        ZArgs b = a;
        b.pf_lines = z_l2pf<R, M, false>() ? (int64_t)persistent_grid(k, g.threads, g.smem, (int64_t)1 << 40) * LPB : 0;
        k<<<(unsigned)blocks, g.threads, g.smem, st>>>(b, (TW)tw, (TW)rot);
    }
    return cudaGetLastError();
}

template <typename R, int M>
inline cudaError_t zc2r_launch_t(const ZArgs &a, const void *tw, const void *rot, cudaStream_t st)
{
    PassGeom g;
    z_geom_t<R, M>(&g);
    constexpr int E = z_E<R, M>(), LPB = z_LPB<R, M>();
    const int64_t blocks = (a.nlines + g.per_block - 1) / g.per_block;
    typedef const typename cvec<R>::T *TW;
    if (a.max_blocks > 0 && blocks > a.max_blocks)
        zpass_c2r_kernel<R, M, E, LPB, true><<<(unsigned)a.max_blocks, g.threads, g.smem, st>>>(a, (TW)tw, (TW)rot);
    else {
        auto k = zpass_c2r_kernel<R, M, E, LPB, false>;
        ZArgs b = a;
        b.pf_lines = z_l2pf<R, M, true>() ? (int64_t)persistent_grid(k, g.threads, g.smem, (int64_t)1 << 40) * LPB : 0;
        k<<<(unsigned)blocks, g.threads, g.smem, st>>>(b, (TW)tw, (TW)rot);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fused
// 512 threads per block: Y tiles of W = 512 / (N1 / E1) columns, Z items of
// 512 / (M / E2) lines; two blocks per SM when a thread holds 16 elements.
template <int N1, int M> struct FusedShape {
    static constexpr int T = 512;
    static constexpr int W = T / (N1 / line_E(N1));
    static constexpr int LPB = T / (M / z_E<float, M>());
    static constexpr int MINB = (line_E(N1) <= 16 && z_E<float, M>() <= 16) ? 2 : 1;
};

template <typename R, int N1, int M> inline void fused_geom_t(PassGeom *g, int *z_lines)
{
    typedef FusedShape<N1, M> S;
    const size_t cs = sizeof(typename cvec<R>::T);
    const size_t y = (size_t)N1 * S::W * cs;
    const size_t z = (size_t)S::LPB * zline_smem_elems<M, z_E<float, M>()>() * cs;
    g->threads = S::T;
    g->per_block = S::W;
    g->E = line_E(N1);
    g->persistent = 1;
    g->smem = y > z ? y : z;
    *z_lines = S::LPB;
}

template <typename R, int N1, int M> inline cudaError_t fused_prepare_t()
{
    typedef FusedShape<N1, M> S;
    PassGeom g;
    int zl;
    fused_geom_t<R, N1, M>(&g, &zl);
    return cudaFuncSetAttribute(fused_plane_kernel<R, N1, M, S::W, S::LPB, S::MINB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
}

template <typename R, int N1, int M>
inline cudaError_t fused_launch_t(const FusedArgs &a, const void *tw_y, const void *tw_z, const void *rot,
                                  cudaStream_t st)
{
    typedef FusedShape<N1, M> S;
    typedef const typename cvec<R>::T *TW;
    PassGeom g;
    int zl;
    fused_geom_t<R, N1, M>(&g, &zl);
    auto k = fused_plane_kernel<R, N1, M, S::W, S::LPB, S::MINB>;
    const int grid = persistent_grid(k, g.threads, g.smem, a.n_items);
    k<<<grid, g.threads, g.smem, st>>>(a, (TW)tw_y, (TW)tw_z, (TW)rot);
    return cudaGetLastError();
}

}  // namespace fft3d

#define FFT3D_FUSED_SHAPES(X) X(512, 256) X(768, 384) X(1024, 512) X(1536, 768) X(2048, 1024)

#define FFT3D_CASE_COL_GEOM(L) case L: col_geom_t<R, L>(g, axis); return true;
#define FFT3D_CASE_Z_GEOM(M) case M: z_geom_t<R, M>(g); return true;
#define FFT3D_CASE_COL_PREP(L) case L: return col_prepare_t<R, L>();
#define FFT3D_CASE_Z_PREP(M) case M: return z_prepare_t<R, M>();
#define FFT3D_CASE_COL_LAUNCH(L) case L: return col_launch_t<R, L>(a, tiles, tw, tmap, tmap2, st);
#define FFT3D_CASE_ZR2C_LAUNCH(M) case M: return zr2c_launch_t<R, M>(a, tw, rot, st);
#define FFT3D_CASE_ZC2R_LAUNCH(M) case M: return zc2r_launch_t<R, M>(a, tw, rot, st);

#define FFT3D_DEFINE_COL(SUF)                                                                   \
    namespace fft3d {                                                                           \
    bool col_geom_##SUF(int L, int axis, PassGeom *g)                                           \
    {                                                                                           \
        switch (L) { FFT3D_COL_LENGTHS(FFT3D_CASE_COL_GEOM) }                                   \
        return false;                                                                           \
    }                                                                                           \
    cudaError_t col_prepare_##SUF(int L)                                                        \
    {                                                                                           \
        switch (L) { FFT3D_COL_LENGTHS(FFT3D_CASE_COL_PREP) }                                   \
        return cudaErrorInvalidValue;                                                           \
    }                                                                                           \
    cudaError_t col_launch_##SUF(int L, const ColArgs &a, int64_t tiles, const void *tw,       \
                                 const CUtensorMap *tmap, const CUtensorMap *tmap2,             \
                                 cudaStream_t st)                                               \
    {                                                                                           \
        switch (L) { FFT3D_COL_LENGTHS(FFT3D_CASE_COL_LAUNCH) }                                 \
        return cudaErrorInvalidValue;                                                           \
    }                                                                                           \
    }

#define FFT3D_DEFINE_Z(SUF)                                                                     \
    namespace fft3d {                                                                           \
    bool z_geom_##SUF(int M, PassGeom *g)                                                       \
    {                                                                                           \
        switch (M) { FFT3D_Z_HALF_LENGTHS(FFT3D_CASE_Z_GEOM) }                                  \
        return false;                                                                           \
    }                                                                                           \
    cudaError_t z_prepare_##SUF(int M)                                                          \
    {                                                                                           \
        switch (M) { FFT3D_Z_HALF_LENGTHS(FFT3D_CASE_Z_PREP) }                                  \
        return cudaErrorInvalidValue;                                                           \
    }                                                                                           \
    cudaError_t zr2c_launch_##SUF(int M, const ZArgs &a, const void *tw, const void *rot,      \
                                  cudaStream_t st)                                              \
    {                                                                                           \
        switch (M) { FFT3D_Z_HALF_LENGTHS(FFT3D_CASE_ZR2C_LAUNCH) }                             \
        return cudaErrorInvalidValue;                                                           \
    }                                                                                           \
    cudaError_t zc2r_launch_##SUF(int M, const ZArgs &a, const void *tw, const void *rot,      \
                                  cudaStream_t st)                                              \
    {                                                                                           \
        switch (M) { FFT3D_Z_HALF_LENGTHS(FFT3D_CASE_ZC2R_LAUNCH) }                             \
        return cudaErrorInvalidValue;                                                           \
    }                                                                                           \
    cudaError_t twiddle_stage_launch_##SUF(void *out, int ns, int r, cudaStream_t st)          \
    {                                                                                           \
        const int n = (r - 1) * ns;                                                             \
        if (n <= 0) return cudaSuccess;                                                         \
        twiddle_stage_kernel<R><<<(n + 255) / 256, 256, 0, st>>>(                              \
            (typename cvec<R>::T *)out, ns, r);                                                 \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t twiddle_rot_launch_##SUF(void *out, int n, int count, cudaStream_t st)         \
    {                                                                                           \
        if (count <= 0) return cudaSuccess;                                                     \
        twiddle_rot_kernel<R><<<(count + 255) / 256, 256, 0, st>>>(                            \
            (typename cvec<R>::T *)out, n, count);                                              \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    cudaError_t twiddle_herm_launch_##SUF(void *out, int n, int count, cudaStream_t st)        \
    {                                                                                           \
        if (count <= 0) return cudaSuccess;                                                     \
        twiddle_herm_kernel<R><<<(count + 255) / 256, 256, 0, st>>>(                           \
            (typename cvec<R>::T *)out, n, count);                                              \
        return cudaGetLastError();                                                              \
    }                                                                                           \
    }

#define FFT3D_CASE_FUSED_GEOM(N1, M) \
    if (n1 == N1 && m == M) {         \
        fused_geom_t<R, N1, M>(g, zl); \
        return true;                   \
    }
#define FFT3D_CASE_FUSED_PREP(N1, M) \
    if (n1 == N1 && m == M) return fused_prepare_t<R, N1, M>();
#define FFT3D_CASE_FUSED_LAUNCH(N1, M) \
    if (n1 == N1 && m == M) return fused_launch_t<R, N1, M>(a, tw_y, tw_z, rot, st);

#define FFT3D_DEFINE_FUSED(SUF)                                                                   \
    namespace fft3d {                                                                             \
    bool fused_geom_##SUF(int n1, int m, PassGeom *g, int *zl)                                    \
    {                                                                                             \
        FFT3D_FUSED_SHAPES(FFT3D_CASE_FUSED_GEOM)                                                 \
        return false;                                                                             \
    }                                                                                             \
    cudaError_t fused_prepare_##SUF(int n1, int m)                                                \
    {                                                                                             \
        FFT3D_FUSED_SHAPES(FFT3D_CASE_FUSED_PREP)                                                 \
        return cudaErrorInvalidValue;                                                             \
    }                                                                                             \
    cudaError_t fused_launch_##SUF(int n1, int m, const FusedArgs &a, const void *tw_y,          \
                                   const void *tw_z, const void *rot, cudaStream_t st)            \
    {                                                                                             \
        FFT3D_FUSED_SHAPES(FFT3D_CASE_FUSED_LAUNCH)                                               \
        return cudaErrorInvalidValue;                                                             \
    }                                                                                             \
    }
