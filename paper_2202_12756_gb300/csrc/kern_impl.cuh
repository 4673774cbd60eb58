// Launch policy and length dispatch, instantiated once per dtype by the
// kern_{col,z}_{f32,f64}.cu translation units.
#pragma once

#include "launchers.h"

namespace fft3d {

// Block-size cap of a column pass: 1024 threads while a thread's registers
// stay within 64 (float, at most 16 elements per thread), else fewer so that
// the larger register footprint still fits the 64K-register file.
template <typename R, int L> __host__ __device__ constexpr int col_max_threads()
{
    return sizeof(R) == 4 ? (line_E(L) <= 16 ? 1024 : 512) : (line_E(L) <= 16 ? 512 : 256);
}

// Columns per tile: one 128-byte segment per row (16 float2 or 8 double2),
// halved while the block would exceed its thread cap or the tile 200 KB of
// shared memory.
template <typename R, int L> __host__ __device__ constexpr int col_W()
{
    int w = 128 / (int)sizeof(typename cvec<R>::T);
    while (w > 1 && (w * line_NT(L) > col_max_threads<R, L>() ||
                     (size_t)L * w * sizeof(typename cvec<R>::T) > 200 * 1024))
        w /= 2;
    return w;
}

// Lines per block of a z pass: about 256 threads, and at least one warp.
template <int M> __host__ __device__ constexpr int z_LPB()
{
    return line_NT(M) >= 256 ? 1 : 256 / line_NT(M);
}

template <typename R, int L> inline void col_geom_t(PassGeom *g)
{
    constexpr int W = col_W<R, L>();
    g->threads = W * line_NT(L);
    g->per_block = W;
    g->smem = (size_t)L * W * sizeof(typename cvec<R>::T);
}

template <typename R, int M> inline void z_geom_t(PassGeom *g)
{
    constexpr int LPB = z_LPB<M>();
    g->threads = LPB * line_NT(M);
    g->per_block = LPB;
    g->smem = (size_t)LPB * zline_smem_elems<M>() * sizeof(typename cvec<R>::T);
}

template <typename R, int L> inline cudaError_t col_prepare_t()
{
    PassGeom g;
    col_geom_t<R, L>(&g);
    return cudaFuncSetAttribute(colpass_kernel<R, L, col_W<R, L>()>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
}

template <typename R, int M> inline cudaError_t z_prepare_t()
{
    PassGeom g;
    z_geom_t<R, M>(&g);
    cudaError_t e = cudaFuncSetAttribute(zpass_r2c_kernel<R, M, z_LPB<M>()>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(zpass_c2r_kernel<R, M, z_LPB<M>()>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
}

template <typename R, int L>
inline cudaError_t col_launch_t(const ColArgs &a, int64_t tiles, const void *tw, cudaStream_t st)
{
    PassGeom g;
    col_geom_t<R, L>(&g);
    colpass_kernel<R, L, col_W<R, L>()><<<(unsigned)tiles, g.threads, g.smem, st>>>(
        a, (const typename cvec<R>::T *)tw);
    return cudaGetLastError();
}

template <typename R, int M>
inline cudaError_t zr2c_launch_t(const ZArgs &a, const void *tw, const void *rot, cudaStream_t st)
{
    PassGeom g;
    z_geom_t<R, M>(&g);
    const int64_t blocks = (a.nlines + g.per_block - 1) / g.per_block;
    zpass_r2c_kernel<R, M, z_LPB<M>()><<<(unsigned)blocks, g.threads, g.smem, st>>>(
        a, (const typename cvec<R>::T *)tw, (const typename cvec<R>::T *)rot);
    return cudaGetLastError();
}

template <typename R, int M>
inline cudaError_t zc2r_launch_t(const ZArgs &a, const void *tw, const void *rot, cudaStream_t st)
{
    PassGeom g;
    z_geom_t<R, M>(&g);
    const int64_t blocks = (a.nlines + g.per_block - 1) / g.per_block;
    zpass_c2r_kernel<R, M, z_LPB<M>()><<<(unsigned)blocks, g.threads, g.smem, st>>>(
        a, (const typename cvec<R>::T *)tw, (const typename cvec<R>::T *)rot);
    return cudaGetLastError();
}

}  // namespace fft3d

#define FFT3D_CASE_COL_GEOM(L) case L: col_geom_t<R, L>(g); return true;
#define FFT3D_CASE_Z_GEOM(M) case M: z_geom_t<R, M>(g); return true;
#define FFT3D_CASE_COL_PREP(L) case L: return col_prepare_t<R, L>();
#define FFT3D_CASE_Z_PREP(M) case M: return z_prepare_t<R, M>();
#define FFT3D_CASE_COL_LAUNCH(L) case L: return col_launch_t<R, L>(a, tiles, tw, st);
#define FFT3D_CASE_ZR2C_LAUNCH(M) case M: return zr2c_launch_t<R, M>(a, tw, rot, st);
#define FFT3D_CASE_ZC2R_LAUNCH(M) case M: return zc2r_launch_t<R, M>(a, tw, rot, st);

#define FFT3D_DEFINE_COL(SUF)                                                                   \
    namespace fft3d {                                                                           \
    bool col_geom_##SUF(int L, PassGeom *g)                                                     \
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
    }
