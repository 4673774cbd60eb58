// C-ABI implementation: plans, argument checks, pass sequencing, profiling.
//
// Forward (exec_r2c):  z-pass R2C lines -> y-pass C2C columns -> x-pass C2C
// columns, all on the caller's stream; the y- and x-passes run in place on
// the output.  This is the single-GPU form of the slab algorithm of Sec. 3 of
// arXiv 2202.12756: the batched plane FFT (Step 1) is the z- and y-passes, and
// the transposes, all-to-all and strided line FFT (Steps 2-5) collapse into
// the x-pass, which reads and writes tiles of adjacent columns directly.
// Inverse (exec_c2r): the same passes in reverse order ("the above steps in a
// reverse order", Sec. 3) with the 1/N^3 normalisation fused into the last.
#include <cuda_runtime.h>

#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder comes from the driver at run time)

#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fft3d.h"
#include "launchers.h"

using namespace fft3d;

namespace {

enum PassKind { K_R2C_Z = 0, K_R2C_Y, K_R2C_X, K_C2R_X, K_C2R_Y, K_C2R_Z, K_R2C_ZY, K_C2R_YZ, K_COUNT };
const char *const kPassName[K_COUNT] = {"r2c.z", "r2c.y", "r2c.x", "c2r.x", "c2r.y", "c2r.z", "r2c.zy", "c2r.yz"};

// default bound on a fused-pass consumer's polls (each sleeps ~0.1 us): ~1 s
constexpr long long kDefaultSpinLimit = 1LL << 23;

// half length M = N2 / 2 of the contiguous axis: 2^k <= 1024 or 3 * 2^k <= 768
bool z_half_supported(int64_t m)
{
    if (m < 1) return false;
    if (m <= 1024 && is_pow2((int)m)) return true;
    return m % 3 == 0 && m <= 768 && is_pow2((int)(m / 3));
}

bool col_supported(int64_t n) { return n >= 1 && n <= 2048 && line_supported((int)n); }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct fft3d_plan_s {
    int64_t n0, n1, n2, m, m1;
    int64_t batch;        // fields per exec call, stored one after another
    int64_t nb0;          // batch * n0: planes of all fields
    int dtype;
    int device;
    size_t rsize, csize;  // bytes of one real / one complex element
    void *tw;             // device: all twiddle tables
    const void *tw0, *tw1, *twz, *rot;
    const void *tw1f;     // axis-1 twiddles laid out for the fused kernel
    void *nyq;            // device: [n0][n1] complex scratch (k2 = M column)
    PassGeom g0, g1, gz;
    int fused;            // plane pass fused (opt-in)
    int fused_ok;         // the shape and dtype allow the fused plane pass
    PassGeom gf;          // fused geometry (per_block = W of its Y tiles)
    int fz_lines;         // lines per fused Z item
    unsigned *sync;       // device: fused-pass tickets, flags, per-plane counters
    unsigned *status;     // device: sticky error flag of the plan's kernels
    long long spin_limit;
    int inject_stall;
    char err[512];
    int profiling;
    struct Rec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double acc_ms[K_COUNT];
    int64_t acc_n[K_COUNT];
    int64_t launches;
};

namespace {

int set_err(fft3d_plan p, int status, const char *what, cudaError_t e = cudaSuccess)
{
    if (p) {
        if (e != cudaSuccess)
            snprintf(p->err, sizeof(p->err), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
        else
            snprintf(p->err, sizeof(p->err), "%s", what);
    }
    return status;
}

double pass_bytes(const fft3d_plan_s *p, int kind)
{
    const double lines = (double)p->nb0 * (double)p->n1;
    const double cplx = lines * (double)p->m1 * (double)p->csize;
    const double real = lines * (double)p->n2 * (double)p->rsize;
    return (kind == K_R2C_Z || kind == K_C2R_Z || kind == K_R2C_ZY || kind == K_C2R_YZ) ? cplx + real
                                                                                        : 2.0 * cplx;
}

cudaEvent_t take_event(fft3d_plan p)
{
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch one pass, optionally bracketed by profiling events.
template <class F> int run_pass(fft3d_plan p, int kind, cudaStream_t st, F &&launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (p->profiling) {
        a = take_event(p);
        b = take_event(p);
        cudaError_t e = (a && b) ? cudaEventRecord(a, st) : cudaErrorMemoryAllocation;
        if (e != cudaSuccess) {
            // events that were taken go back to the pool
            if (a) p->pool.push_back(a);
            if (b) p->pool.push_back(b);
            return set_err(p, FFT3D_ERR_CUDA, (a && b) ? "cudaEventRecord" : "cudaEventCreate", e);
        }
    }
    auto release = [&] {
        if (p->profiling) {
            p->pool.push_back(a);
            p->pool.push_back(b);
        }
    };
    cudaError_t e = launch();
    if (e != cudaSuccess) {
        release();
        char what[64];
        snprintf(what, sizeof(what), "launch of pass %s", kPassName[kind]);
        return set_err(p, FFT3D_ERR_CUDA, what, e);
    }
    ++p->launches;
    if (p->profiling) {
        e = cudaEventRecord(b, st);
        if (e != cudaSuccess) {
            release();
            return set_err(p, FFT3D_ERR_CUDA, "cudaEventRecord", e);
        }
        p->pending.push_back({kind, a, b});
    }
    return FFT3D_OK;
}

cudaError_t col_launch(const fft3d_plan_s *p, int L, const ColArgs &a, int64_t tiles, const void *tw,
                       cudaStream_t st, const CUtensorMap *tmap = nullptr, const CUtensorMap *tmap2 = nullptr)
{
    return p->dtype == FFT3D_F32 ? col_launch_f32(L, a, tiles, tw, tmap, tmap2, st)
                                 : col_launch_f64(L, a, tiles, tw, tmap, tmap2, st);
}

// cuTensorMapEncodeTiled, fetched from the driver once (no libcuda link).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)ptr;
    });
    return fn;
}

// 2D tensor map over 8-byte elements (one float complex): `inner` elements
// per row, `rows` rows `pitch` elements apart, boxes of box_w x 256.
bool tensor_map_2d(const void *base, int64_t inner, int64_t rows, int64_t pitch, int box_w, CUtensorMap *map)
{
    EncodeTiledFn fn = encode_tiled_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * 8};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)kTmaBoxRows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tile waits of a pipelined column pass: normal, or made to run out (test hook).
void set_stage_waits(const fft3d_plan_s *p, ColArgs &a)
{
    a.stall_tx = p->inject_stall ? 16u : 0u;
    a.stage_polls = p->inject_stall ? p->spin_limit : kStageWaitPolls;
}

// TMA mode of a pipelined column pass over `src` (see colpass_pipe_kernel):
// 0 = per-element copies; 1 = one map over 16-byte aligned rows; 2 = even /
// odd row maps (y-pass rows of odd complex pitch).  Needs float, the
// pipelined kernel for this length, a 16-byte aligned base, full tiles, and
// L a multiple of 512; the split layout (rows of pitch M plus the k2 = M
// plane) takes mode 1 in the y-pass (its k2 = M tiles use per-element copies).
int bulk_mode(const fft3d_plan_s *p, const CLayout &src, int axis, int64_t w)
{
    const PassGeom &g = axis == 0 ? p->g0 : p->g1;
    const int64_t L = axis == 0 ? p->n0 : p->n1;
    if (!g.persistent || p->dtype != FFT3D_F32 || ((uintptr_t)src.main & 15) || L % (2 * kTmaBoxRows) != 0)
        return 0;
    if (axis == 0)
        return (!src.split && (p->n1 * p->m1) % 2 == 0 && (p->n1 * p->m1) % w == 0 && (!g.pair || p->n0 % 2 == 0))
                   ? 1
                   : 0;
    if (p->m % w != 0) return 0;
    if (src.split) return 1;  // main rows of pitch M (a multiple of W): 16-byte aligned
    return (p->m1 % 2 == 0) ? 1 : 2;
}

// y-pass (axis 1) tiles: per k0 plane, ceil(M / W) tiles of the k2 < M
// columns, then ceil(N0 / W) tiles of the k2 = M column (W planes each).
ColArgs ypass_args(const fft3d_plan_s *p, CLayout src, CLayout dst, int inverse, int64_t *tiles)
{
    ColArgs a;
    a.src = src;
    a.dst = dst;
    a.n0 = p->nb0;  // the planes of all fields
    a.n1 = p->n1;
    a.m = p->m;
    a.axis = 1;
    a.inverse = inverse;
    const int64_t w = p->g1.per_block;
    a.tiles_per_plane = (p->m + w - 1) / w;
    a.tiles_main = p->nb0 * a.tiles_per_plane;
    a.nyq_in_plane = 0;
    a.bulk = bulk_mode(p, src, 1, w);
    a.err = p->status;
    a.tiles_per_field = 1;
    a.pf_stride = 0;
    a.tickets = p->status + 1;
    // the next tile is staged after the first exchange barrier, not right after the registers
    // are loaded: measured on GB300 with the dynamic tile order, 1024-point y columns are 1-2%
    // faster that way (with the static order early staging was 1-15% faster for them)
    a.early = 0;
    set_stage_waits(p, a);
    *tiles = a.tiles_main + (p->nb0 + w - 1) / w;
    return a;
}

// x-pass (axis 0) tiles: W consecutive flat (k1, k2) columns of one field.
ColArgs xpass_args(const fft3d_plan_s *p, CLayout src, CLayout dst, int inverse, int64_t *tiles)
{
    ColArgs a;
    a.src = src;
    a.dst = dst;
    a.n0 = p->n0;
    a.n1 = p->n1;
    a.m = p->m;
    a.axis = 0;
    a.inverse = inverse;
    const int64_t w = p->g0.per_block;
    a.tiles_per_field = (p->n1 * p->m1 + w - 1) / w;
    *tiles = p->batch * a.tiles_per_field;
    a.tiles_main = *tiles;
    // early staging of the next tile, measured on GB300: 1.4% faster at a 4 MB
    // row pitch (N1 (N2/2+1) complex), even at 3 MB, 4-9% slower at 1-2 MB
    const int64_t pitch = src.split ? p->n1 * p->m : p->n1 * p->m1;
    a.early = pitch * (int64_t)p->csize >= ((int64_t)3 << 20);
    a.tiles_per_plane = 0;
    a.nyq_in_plane = 0;
    a.pf_stride = 0;
    a.bulk = bulk_mode(p, src, 0, w);
    a.err = p->status;
    a.tickets = p->status + 1;
    set_stage_waits(p, a);
    return a;
}

// Fused plane pass (Z and Y items of each plane through L2).  The sync words
// (tickets, launch error flag, per-plane counters) are cleared on the stream
// first; the sticky error word after them is left alone.
int run_fused(fft3d_plan p, int kind, const ZArgs &z, CLayout ylayout, int forward, cudaStream_t st)
{
    FusedArgs f;
    f.z = z;
    f.y.src = ylayout;
    f.y.dst = ylayout;
    f.y.n0 = p->n0;
    f.y.n1 = p->n1;
    f.y.m = p->m;
    f.y.axis = 1;
    f.y.inverse = forward ? 0 : 1;
    const int64_t w = p->gf.per_block;
    f.yi = (p->m1 + w - 1) / w;
    f.y.tiles_per_plane = f.yi;
    f.y.tiles_main = p->n0 * f.yi;
    f.y.nyq_in_plane = 1;
    f.y.bulk = 0;
    f.y.err = p->status;
    f.y.tiles_per_field = 1;
    f.y.early = 0;
    f.y.stall_tx = 0;
    f.y.stage_polls = kStageWaitPolls;
    f.y.pf_stride = 0;
    f.y.tickets = nullptr;
    f.n0 = p->n0;
    f.zi = p->n1 / p->fz_lines;
#ifndef FFT3D_FUSED_LAG
#define FFT3D_FUSED_LAG 2
#endif
    f.lag = FFT3D_FUSED_LAG;
    f.n_items = p->n0 * (f.zi + f.yi);
    f.sync = p->sync;
    f.spin_limit = p->spin_limit;
    f.inject_stall = p->inject_stall;
    f.forward = forward;
    cudaError_t e = cudaMemsetAsync(p->sync, 0, sizeof(unsigned) * (size_t)(kSyncDone + p->n0), st);
    if (e != cudaSuccess) return set_err(p, FFT3D_ERR_CUDA, "cudaMemsetAsync", e);
    return run_pass(p, kind, st,
                    [&] { return fused_launch_f32((int)p->n1, (int)p->m, f, p->tw1f, p->twz, p->rot, st); });
}

// Column-pass launch; full float tiles go through TMA when the layout allows it.
int run_colpass(fft3d_plan p, int kind, ColArgs a, int64_t tiles, int L, const void *tw, cudaStream_t st)
{
    CUtensorMap map, map2;
    const CUtensorMap *mp = nullptr, *mp2 = nullptr;
    const int w = (int)(a.axis == 0 ? p->g0.per_block : p->g1.per_block);
    bool ok = true;
    // a CTA pair (colpass_pair_kernel) reads rows of one parity: mode 1 maps row pairs
    const int64_t pr = (a.axis == 0 ? p->g0.pair : p->g1.pair) ? 2 : 1;
    if (a.bulk == 1 && a.axis == 0) {
        ok = tensor_map_2d(a.src.main, pr * p->n1 * p->m1, p->nb0 / pr, pr * p->n1 * p->m1, w, &map);
    } else if (a.bulk == 1) {
        const int64_t pitch = a.src.split ? p->m : p->m1;  // the split layout's k2 < M rows
        ok = tensor_map_2d(a.src.main, pr * pitch, p->nb0 * p->n1 / pr, pr * pitch, w, &map);
    } else if (a.bulk == 2) {
        ok = tensor_map_2d(a.src.main, 2 * p->m1, p->nb0 * p->n1 / 2, 2 * p->m1, w, &map) &&
             tensor_map_2d(a.src.main, 2 * p->m1, p->nb0 * p->n1 / 2, 2 * p->m1, w + 2, &map2);
    }
    if (!ok) a.bulk = 0;
    if (a.bulk) mp = &map;
    if (a.bulk == 2) mp2 = &map2;
    const PassGeom &g = a.axis == 0 ? p->g0 : p->g1;
    if (!g.persistent || g.pair) a.tickets = nullptr;  // only the pipelined kernel draws tiles
    if (a.tickets) {
        const cudaError_t e = cudaMemsetAsync(a.tickets, 0, sizeof(unsigned), st);
        if (e != cudaSuccess) return set_err(p, FFT3D_ERR_CUDA, "cudaMemsetAsync", e);
    }
    return run_pass(p, kind, st, [&] { return col_launch(p, L, a, tiles, tw, st, mp, mp2); });
}

int run_xpass(fft3d_plan p, int kind, CLayout src, CLayout dst, int inverse, cudaStream_t st)
{
    int64_t tiles;
    const ColArgs a = xpass_args(p, src, dst, inverse, &tiles);
    return run_colpass(p, kind, a, tiles, (int)p->n0, p->tw0, st);
}

int run_ypass(fft3d_plan p, int kind, CLayout src, CLayout dst, int inverse, cudaStream_t st)
{
    int64_t tiles;
    const ColArgs a = ypass_args(p, src, dst, inverse, &tiles);
    return run_colpass(p, kind, a, tiles, (int)p->n1, p->tw1, st);
}

int check_exec(fft3d_plan p, const void *in, const void *out, bool real_in)
{
    if (!p) return FFT3D_ERR_NULL;
    if (!in || !out) return set_err(p, FFT3D_ERR_NULL, "null data pointer");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_err(p, FFT3D_ERR_CUDA, "cudaGetDevice", e);
    if (dev != p->device) return set_err(p, FFT3D_ERR_DEVICE, "current device is not the plan's device");
    if (((uintptr_t)in % p->csize) != 0 || ((uintptr_t)out % p->csize) != 0)
        return set_err(p, FFT3D_ERR_ALIGN, "data pointer not aligned to one complex element");
    if (in != out) {
        const size_t lines = (size_t)p->nb0 * (size_t)p->n1;
        const size_t rbytes = lines * (size_t)p->n2 * p->rsize;
        const size_t cbytes = lines * (size_t)p->m1 * p->csize;
        const size_t ib = real_in ? rbytes : cbytes;
        const size_t ob = real_in ? cbytes : rbytes;
        const uintptr_t i0 = (uintptr_t)in, o0 = (uintptr_t)out;
        if (i0 < o0 + ob && o0 < i0 + ib)
            return set_err(p, FFT3D_ERR_LAYOUT, "input and output overlap without being identical");
    }
    return FFT3D_OK;
}

// Blocks of a z-pass that reads or writes the real field in host memory: the
// CPU-GPU link, not the SMs, bounds such a pass, so it runs on a few SMs
// (grid-stride over line groups) and leaves the others to the strided passes
// of another stream (another field in flight).
#ifndef FFT3D_HOST_Z_BLOCKS
#define FFT3D_HOST_Z_BLOCKS 384
#endif

// True for memory the GPU reaches over the CPU-GPU link (pinned, registered
// or plain system memory), false for device and managed memory.
bool host_resident(const void *ptr)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

// R2C pipeline: z (R2C with output scales) -> y -> x.
int forward_pipeline(fft3d_plan p, const void *in, void *out, cudaStream_t st, double se, double sm)
{
    const CLayout L = {out, nullptr, 0};
    ZArgs z;
    z.real = in;
    z.real_out = nullptr;
    z.real_pitch = (in == out) ? 2 * p->m1 : p->n2;
    z.cplx = L;
    z.nlines = p->nb0 * p->n1;
    z.scale_edge = se;
    z.scale_mid = sm;
    z.pf_lines = 0;
    z.max_blocks = (in != out && host_resident(in)) ? FFT3D_HOST_Z_BLOCKS : 0;
    int rc;
    if (p->fused) {
        rc = run_fused(p, K_R2C_ZY, z, L, 1, st);
        if (rc) return rc;
        if (p->n0 > 1) rc = run_xpass(p, K_R2C_X, L, L, 0, st);
        return rc;
    }
    rc = run_pass(p, K_R2C_Z, st, [&] {
        return p->dtype == FFT3D_F32 ? zr2c_launch_f32((int)p->m, z, p->twz, p->rot, st)
                                     : zr2c_launch_f64((int)p->m, z, p->twz, p->rot, st);
    });
    if (rc) return rc;
    if (p->n1 > 1) {
        rc = run_ypass(p, K_R2C_Y, L, L, 0, st);
        if (rc) return rc;
    }
    if (p->n0 > 1) rc = run_xpass(p, K_R2C_X, L, L, 0, st);
    return rc;
}

// C2R pipeline: x -> y -> z (C2R with edge weight `we` and output scale `s`).
// Out of place, the x-pass writes the split layout (k2 < M rows in the
// output buffer, k2 = M in the plan's scratch plane) so the input survives.
int inverse_pipeline(fft3d_plan p, const void *in, void *out, cudaStream_t st, double we, double s,
                     bool overwrite_input = false)
{
    const bool inplace = (in == out);
    const CLayout src = {const_cast<void *>(in), nullptr, 0};
    // Out of place, the axis-0 and axis-1 passes work either in the output
    // (split layout, input preserved) or, when the caller allows it, in the
    // input itself (standard layout; the output is then written only once,
    // by the last pass).
    const CLayout dst = (inplace || overwrite_input) ? src : CLayout{out, p->nyq, 1};
    int rc;
    if (p->n0 > 1 || dst.main != src.main) {
        rc = run_xpass(p, K_C2R_X, src, dst, 1, st);
        if (rc) return rc;
    }
    ZArgs z;
    z.real = nullptr;
    z.real_out = out;
    z.real_pitch = inplace ? 2 * p->m1 : p->n2;
    z.cplx = dst;
    z.nlines = p->nb0 * p->n1;
    z.scale_edge = we;
    z.scale_mid = s;
    z.pf_lines = 0;
    z.max_blocks = (!inplace && host_resident(out)) ? FFT3D_HOST_Z_BLOCKS : 0;
    if (p->fused) return run_fused(p, K_C2R_YZ, z, dst, 0, st);
    if (p->n1 > 1) {
        rc = run_ypass(p, K_C2R_Y, dst, dst, 1, st);
        if (rc) return rc;
    }
    return run_pass(p, K_C2R_Z, st, [&] {
        return p->dtype == FFT3D_F32 ? zc2r_launch_f32((int)p->m, z, p->twz, p->rot, st)
                                     : zc2r_launch_f64((int)p->m, z, p->twz, p->rot, st);
    });
}

}  // namespace

extern "C" {

int fft3d_supported_length(int64_t n, int axis)
{
    if (axis == 0 || axis == 1) return col_supported(n) ? 1 : 0;
    if (axis == 2) return (n >= 2 && n % 2 == 0 && z_half_supported(n / 2)) ? 1 : 0;
    return 0;
}

int fft3d_plan_create(fft3d_plan *out, int64_t n0, int64_t n1, int64_t n2, int dtype)
{
    return fft3d_plan_create_batched(out, 1, n0, n1, n2, dtype);
}

int fft3d_plan_create_batched(fft3d_plan *out, int64_t batch, int64_t n0, int64_t n1, int64_t n2, int dtype)
{
    if (!out) return FFT3D_ERR_NULL;
    *out = nullptr;
    if (dtype != FFT3D_F32 && dtype != FFT3D_F64) return FFT3D_ERR_DTYPE;
    if (!fft3d_supported_length(n0, 0) || !fft3d_supported_length(n1, 1) || !fft3d_supported_length(n2, 2))
        return FFT3D_ERR_SIZE;
    // every plane-row index (batch * n0 * n1) must fit the kernels' 32-bit TMA coordinates
    if (batch < 1 || batch > ((int64_t)1 << 31) / (n0 * n1)) return FFT3D_ERR_SIZE;
    fft3d_plan p = new (std::nothrow) fft3d_plan_s();
    if (!p) return FFT3D_ERR_ALLOC;
    p->batch = batch;
    p->nb0 = batch * n0;
    p->n0 = n0;
    p->n1 = n1;
    p->n2 = n2;
    p->m = n2 / 2;
    p->m1 = n2 / 2 + 1;
    p->dtype = dtype;
    p->rsize = dtype == FFT3D_F32 ? 4 : 8;
    p->csize = 2 * p->rsize;
    p->err[0] = 0;
    int rc = FFT3D_OK;
    cudaError_t e = cudaGetDevice(&p->device);
    const bool f32 = dtype == FFT3D_F32;
    if (e != cudaSuccess) {
        rc = FFT3D_ERR_CUDA;
        goto fail;
    }
    if (!(f32 ? col_geom_f32((int)n0, 0, &p->g0) : col_geom_f64((int)n0, 0, &p->g0)) ||
        !(f32 ? col_geom_f32((int)n1, 1, &p->g1) : col_geom_f64((int)n1, 1, &p->g1)) ||
        !(f32 ? z_geom_f32((int)p->m, &p->gz) : z_geom_f64((int)p->m, &p->gz))) {
        rc = FFT3D_ERR_SIZE;
        goto fail;
    }
    p->spin_limit = kDefaultSpinLimit;
    p->fused_ok = f32 && batch == 1 && fused_geom_f32((int)n1, (int)p->m, &p->gf, &p->fz_lines) &&
                  n1 % p->fz_lines == 0;
    p->fused = 0;  // opt-in: see fft3d_plan_set_fused

    {
        const size_t s0 = align256((size_t)col_table_elems((int)n0, p->g0) * p->csize + 16);
        const size_t s1 = align256((size_t)col_table_elems((int)n1, p->g1) * p->csize + 16);
        const size_t sz = align256((size_t)line_tw_size(z_line_points((int)p->m, p->gz), p->gz.E) * p->csize + 16);
        const size_t sr = align256(z_table_elems(f32, (int)p->m) * p->csize);
        const size_t sf = p->fused_ok ? align256((size_t)line_tw_size((int)n1, p->gf.E) * p->csize + 16) : 0;
        e = cudaMalloc(&p->tw, s0 + s1 + sz + sr + sf);
        if (e != cudaSuccess) {
            rc = FFT3D_ERR_ALLOC;
            goto fail;
        }
        char *base = (char *)p->tw;
        p->tw0 = base;
        p->tw1 = base + s0;
        p->twz = base + s0 + s1;
        p->rot = base + s0 + s1 + sz;
        p->tw1f = base + s0 + s1 + sz + sr;
        if ((e = write_col_tables(f32, (int)n0, p->g0, base, 0)) != cudaSuccess ||
            (e = write_col_tables(f32, (int)n1, p->g1, base + s0, 0)) != cudaSuccess ||
            (e = write_line_tables(f32, z_line_points((int)p->m, p->gz), p->gz.E, base + s0 + s1, 0)) != cudaSuccess ||
            (e = write_z_table(f32, (int)n2, base + s0 + s1 + sz, 0)) != cudaSuccess ||
            (p->fused_ok && (e = write_line_tables(f32, (int)n1, p->gf.E, base + s0 + s1 + sz + sr, 0)) != cudaSuccess)) {
            rc = FFT3D_ERR_CUDA;
            goto fail;
        }
        e = cudaMalloc(&p->nyq, (size_t)p->nb0 * (size_t)n1 * p->csize);
        if (e != cudaSuccess) {
            rc = FFT3D_ERR_ALLOC;
            goto fail;
        }
        e = cudaMalloc((void **)&p->status, 4 * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMemset(p->status, 0, 4 * sizeof(unsigned));
        if (e != cudaSuccess) {
            rc = FFT3D_ERR_ALLOC;
            goto fail;
        }
        if (p->fused_ok) {
            const size_t words = (size_t)(kSyncDone + n0);
            e = cudaMalloc((void **)&p->sync, words * sizeof(unsigned));
            if (e != cudaSuccess) {
                rc = FFT3D_ERR_ALLOC;
                goto fail;
            }
            if ((e = cudaMemset(p->sync, 0, words * sizeof(unsigned))) != cudaSuccess ||
                (e = fused_prepare_f32((int)n1, (int)p->m)) != cudaSuccess) {
                rc = FFT3D_ERR_CUDA;
                goto fail;
            }
        }
        if ((e = (f32 ? col_prepare_f32 : col_prepare_f64)((int)n0)) != cudaSuccess ||
            (e = (f32 ? col_prepare_f32 : col_prepare_f64)((int)n1)) != cudaSuccess ||
            (e = (f32 ? z_prepare_f32 : z_prepare_f64)((int)p->m)) != cudaSuccess) {
            rc = FFT3D_ERR_CUDA;
            goto fail;
        }
        e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) {
            rc = FFT3D_ERR_CUDA;
            goto fail;
        }
    }
    *out = p;
    return FFT3D_OK;
fail:
    if (p->tw) cudaFree(p->tw);
    if (p->nyq) cudaFree(p->nyq);
    if (p->sync) cudaFree(p->sync);
    if (p->status) cudaFree(p->status);
    delete p;
    (void)cudaGetLastError();
    return rc;
}

int fft3d_plan_destroy(fft3d_plan p)
{
    if (!p) return FFT3D_OK;
    for (auto &r : p->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto ev : p->pool) cudaEventDestroy(ev);
    cudaError_t e1 = p->tw ? cudaFree(p->tw) : cudaSuccess;
    cudaError_t e2 = p->nyq ? cudaFree(p->nyq) : cudaSuccess;
    cudaError_t e3 = p->sync ? cudaFree(p->sync) : cudaSuccess;
    cudaError_t e4 = p->status ? cudaFree(p->status) : cudaSuccess;
    delete p;
    return (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && e4 == cudaSuccess) ? FFT3D_OK
                                                                                              : FFT3D_ERR_CUDA;
}

int fft3d_exec_r2c(fft3d_plan p, const void *in_real, void *out_cplx, void *stream)
{
    int rc = check_exec(p, in_real, out_cplx, true);
    if (rc) return rc;
    return forward_pipeline(p, in_real, out_cplx, (cudaStream_t)stream, 1.0, 1.0);
}

int fft3d_exec_c2r(fft3d_plan p, const void *in_cplx, void *out_real, void *stream)
{
    int rc = check_exec(p, in_cplx, out_real, false);
    if (rc) return rc;
    const double s = 1.0 / ((double)p->n0 * (double)p->n1 * (double)p->n2);
    return inverse_pipeline(p, in_cplx, out_real, (cudaStream_t)stream, 1.0, s);
}

int fft3d_exec_c2r_overwrite(fft3d_plan p, void *inout_cplx, void *out_real, void *stream)
{
    int rc = check_exec(p, inout_cplx, out_real, false);
    if (rc) return rc;
    const double s = 1.0 / ((double)p->n0 * (double)p->n1 * (double)p->n2);
    return inverse_pipeline(p, inout_cplx, out_real, (cudaStream_t)stream, 1.0, s, true);
}

int fft3d_exec_r2c_adjoint(fft3d_plan p, const void *in_cplx, void *out_real, void *stream)
{
    int rc = check_exec(p, in_cplx, out_real, false);
    if (rc) return rc;
    return inverse_pipeline(p, in_cplx, out_real, (cudaStream_t)stream, 2.0, 0.5);
}

int fft3d_exec_c2r_adjoint(fft3d_plan p, const void *in_real, void *out_cplx, void *stream)
{
    int rc = check_exec(p, in_real, out_cplx, true);
    if (rc) return rc;
    const double s = 1.0 / ((double)p->n0 * (double)p->n1 * (double)p->n2);
    return forward_pipeline(p, in_real, out_cplx, (cudaStream_t)stream, s, 2.0 * s);
}

const char *fft3d_strerror(int status)
{
    switch (status) {
    case FFT3D_OK: return "ok";
    case FFT3D_ERR_SIZE: return "unsupported transform size";
    case FFT3D_ERR_DTYPE: return "unsupported dtype";
    case FFT3D_ERR_NULL: return "null pointer argument";
    case FFT3D_ERR_ALIGN: return "data pointer not aligned to one complex element";
    case FFT3D_ERR_ALLOC: return "allocation failed";
    case FFT3D_ERR_CUDA: return "CUDA error";
    case FFT3D_ERR_LAYOUT: return "input and output overlap without being identical";
    case FFT3D_ERR_DEVICE: return "current device is not the plan's device";
    case FFT3D_ERR_ARG: return "invalid argument";
    default: return "unknown status";
    }
}

const char *fft3d_plan_last_error(fft3d_plan p) { return p ? p->err : ""; }

int fft3d_plan_set_profiling(fft3d_plan p, int enable)
{
    if (!p) return FFT3D_ERR_NULL;
    p->profiling = enable ? 1 : 0;
    return FFT3D_OK;
}

int fft3d_plan_profile_read(fft3d_plan p, fft3d_kernel_stat *stats, int max, int *count)
{
    if (!p || !count || (max > 0 && !stats)) return FFT3D_ERR_NULL;
    int rc = FFT3D_OK;
    for (auto &r : p->pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) {
            rc = set_err(p, FFT3D_ERR_CUDA, "profile event", e);
        } else {
            p->acc_ms[r.kind] += ms;
            p->acc_n[r.kind] += 1;
        }
        p->pool.push_back(r.a);
        p->pool.push_back(r.b);
    }
    p->pending.clear();
    int n = 0;
    for (int k = 0; k < K_COUNT; ++k) {
        if (p->acc_n[k] == 0) continue;
        if (n < max) {
            fft3d_kernel_stat &s = stats[n];
            memset(&s, 0, sizeof(s));
            snprintf(s.name, sizeof(s.name), "%s", kPassName[k]);
            s.launches = p->acc_n[k];
            s.total_ms = p->acc_ms[k];
            s.bytes_per_launch = pass_bytes(p, k);
        }
        ++n;
        p->acc_ms[k] = 0;
        p->acc_n[k] = 0;
    }
    *count = n < max ? n : max;
    return rc;
}

int fft3d_plan_launch_count(fft3d_plan p, int64_t *count)
{
    if (!p || !count) return FFT3D_ERR_NULL;
    *count = p->launches;
    return FFT3D_OK;
}

int fft3d_plan_status(fft3d_plan p, int *device_error)
{
    if (!p || !device_error) return FFT3D_ERR_NULL;
    *device_error = 0;
    unsigned *sticky = p->status;
    unsigned v = 0;
    cudaError_t e = cudaMemcpy(&v, sticky, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v) e = cudaMemset(sticky, 0, sizeof(unsigned));
    if (e != cudaSuccess) return set_err(p, FFT3D_ERR_CUDA, "reading the device error flag", e);
    *device_error = v ? 1 : 0;
    return FFT3D_OK;
}

int fft3d_plan_set_debug(fft3d_plan p, int inject_stall, int64_t spin_limit)
{
    if (!p) return FFT3D_ERR_NULL;
    p->inject_stall = inject_stall ? 1 : 0;
    p->spin_limit = spin_limit > 0 ? spin_limit : kDefaultSpinLimit;
    return FFT3D_OK;
}

int fft3d_plan_info(fft3d_plan p, int *fused_plane_pass)
{
    if (!p || !fused_plane_pass) return FFT3D_ERR_NULL;
    *fused_plane_pass = p->fused;
    return FFT3D_OK;
}

int fft3d_plan_set_fused(fft3d_plan p, int enable)
{
    if (!p) return FFT3D_ERR_NULL;
    if (enable && !p->fused_ok) return set_err(p, FFT3D_ERR_SIZE, "no fused plane pass for this shape / dtype");
    p->fused = enable ? 1 : 0;
    return FFT3D_OK;
}

}  // extern "C"
