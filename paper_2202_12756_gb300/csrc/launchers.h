// Internal host-side launchers (C++; not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fused_kernel.cuh"

namespace fft3d {

// X-macro lists of the compiled line lengths.
#define FFT3D_COL_LENGTHS(X)                                                              \
    X(1) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(3) X(6) \
        X(12) X(24) X(48) X(96) X(192) X(384) X(768) X(1536)
#define FFT3D_Z_HALF_LENGTHS(X)                                                          \
    X(1) X(2) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(3) X(6) X(12) \
        X(24) X(48) X(96) X(192) X(384) X(768)

// Launch geometry of one pass, for the plan to size grids and shared memory.
struct PassGeom {
    int threads;      // block size
    int per_block;    // columns (colpass) or lines (zpass) per block
    int E;            // elements per thread (fixes the twiddle-table layout)
    int persistent;   // 1: grid-stride persistent kernel
    size_t smem;      // dynamic shared memory bytes
    int pair = 0;     // column pass: 1 = a cluster of two CTAs per tile (colpass_pair_kernel)
};

// Twiddle table of a column pass, in complex elements: the line table of the
// length, or for a CTA pair the line table of L/2 points followed by
// W_L^j for j < L/2 / E (written by write_col_tables).
inline int col_table_elems(int L, const PassGeom &g)
{
    return g.pair ? line_tw_size(L / 2, g.E) + L / 2 / g.E : line_tw_size(L, g.E);
}

// dtype-specific entry points, defined in kern_f32.cu / kern_f64.cu.
// Each returns cudaSuccess or the launch error.  `prepare` raises the
// dynamic shared-memory limit of the kernels a plan will use on the current
// device; `geom` reports the launch geometry (of a column pass along `axis`:
// 0 x-pass, 1 y-pass).
#define FFT3D_DECLARE_LAUNCHERS(SUF, R)                                                              \
    bool col_geom_##SUF(int L, int axis, PassGeom *g);                                               \
    bool z_geom_##SUF(int M, PassGeom *g);                                                           \
    cudaError_t col_prepare_##SUF(int L);                                                            \
    cudaError_t z_prepare_##SUF(int M);                                                              \
    cudaError_t col_launch_##SUF(int L, const ColArgs &a, int64_t tiles, const void *tw,            \
                                 const CUtensorMap *tmap, const CUtensorMap *tmap2, cudaStream_t st);\
    cudaError_t zr2c_launch_##SUF(int M, const ZArgs &a, const void *tw, const void *rot,           \
                                  cudaStream_t st);                                                  \
    cudaError_t zc2r_launch_##SUF(int M, const ZArgs &a, const void *tw, const void *rot,           \
                                  cudaStream_t st);                                                  \
    cudaError_t twiddle_stage_launch_##SUF(void *out, int ns, int r, cudaStream_t st);             \
    cudaError_t twiddle_rot_launch_##SUF(void *out, int n, int count, cudaStream_t st);             \
    cudaError_t twiddle_herm_launch_##SUF(void *out, int n, int count, cudaStream_t st);

FFT3D_DECLARE_LAUNCHERS(f32, float)
FFT3D_DECLARE_LAUNCHERS(f64, double)

// Writes the stage twiddles of an L-point line plan with E elements per
// thread (FP64 sincospi, rounded once) to dst, on stream st.
inline cudaError_t write_line_tables(bool f32, int L, int E, void *dst, cudaStream_t st)
{
    for (int s = 1; s < line_nstages(L, E); ++s) {
        void *o = (char *)dst + (size_t)line_tw_offset(L, E, s) * (f32 ? 8 : 16);
        cudaError_t e = f32 ? twiddle_stage_launch_f32(o, line_ns(L, E, s), line_radix(L, E, s), st)
                            : twiddle_stage_launch_f64(o, line_ns(L, E, s), line_radix(L, E, s), st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Writes the twiddle table of an L-point column pass of geometry g
// (col_table_elems(L, g) complex elements) to dst, on stream st.
inline cudaError_t write_col_tables(bool f32, int L, const PassGeom &g, void *dst, cudaStream_t st)
{
    if (!g.pair) return write_line_tables(f32, L, g.E, dst, st);
    cudaError_t e = write_line_tables(f32, L / 2, g.E, dst, st);
    if (e != cudaSuccess) return e;
    void *rot = (char *)dst + (size_t)line_tw_size(L / 2, g.E) * (f32 ? 8 : 16);
    return f32 ? twiddle_rot_launch_f32(rot, L, L / 2 / g.E, st) : twiddle_rot_launch_f64(rot, L, L / 2 / g.E, st);
}

// Points of a z-pass line transform of half length m with geometry gz: m,
// or 2m when two real lines share one complex transform (gz.pair).
inline int z_line_points(int m, const PassGeom &gz) { return gz.pair ? 2 * m : m; }

// Table of the contiguous-axis passes of an N2 = 2M point line (`rot` of
// the z launchers): float lines take the R2C rotations exp(-2 pi i k / N2),
// k < M; double lines take the [A, B] coefficient pairs of their Hermitian
// post- / pre-process for k <= M (see twiddle_herm_kernel).
inline size_t z_table_elems(bool f32, int m) { return f32 ? (size_t)m : 2 * ((size_t)m + 1); }
inline cudaError_t write_z_table(bool f32, int n2, void *dst, cudaStream_t st)
{
    return f32 ? twiddle_rot_launch_f32(dst, n2, n2 / 2, st) : twiddle_herm_launch_f64(dst, n2, n2 / 2 + 1, st);
}

// Fused plane pass (float only): available for (N1, M) in
// {(512, 256), (768, 384), (1024, 512), (1536, 768), (2048, 1024)}.
// geom->per_block = W (columns per Y tile), geom->E = elements per thread of
// the axis-1 transform (twiddle layout), geom->threads, geom->smem;
// z_lines = lines per Z item.
bool fused_geom_f32(int n1, int m, PassGeom *geom, int *z_lines);
cudaError_t fused_prepare_f32(int n1, int m);
cudaError_t fused_launch_f32(int n1, int m, const FusedArgs &a, const void *tw_y, const void *tw_z,
                             const void *rot, cudaStream_t st);

}  // namespace fft3d
