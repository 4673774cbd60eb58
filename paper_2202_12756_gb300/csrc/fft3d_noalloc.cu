// fft3d_exec_c2r_noalloc: the normalised inverse C2R without a plan and
// without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc.  One kind has handed all
// of the GPU's memory to its own pool allocator up front (a spectral solver
// sizing its fields to fill HBM, say), so any cudaMalloc made by a library
// fails or breaks the pool's budget.  Another kind runs where an implicit
// device synchronisation is not allowed; cudaMalloc and cudaFree may
// synchronise the device.  Such callers cannot create a plan
// (fft3d_plan_create allocates its twiddle tables and its scratch plane with
// cudaMalloc).
//
// Instead of plan memory, this file keeps one file-scope device array,
// g_noalloc_scratch.  Each call writes the twiddle tables for its sizes into
// it and uses the rest as the N0 x N1 scratch plane that holds the k2 = N2/2
// column during an out-of-place inverse.  The pass kernels are the same as
// for fft3d_exec_c2r.
//
// Rules, also stated in include/fft3d.h:
//  * The array is a static device allocation of the library.  Every GPU that
//    loads the library holds it until the process exits.
//  * All calls share it.  Calls that overlap on the GPU (two streams, or two
//    host threads) race on it and corrupt each other's results.
//  * Nothing in it has to start at zero: every call rewrites the tables, the
//    x-pass writes the whole scratch plane before the y-pass reads it, and
//    the call clears the device error word (below) on its stream first.
//  * The first call on a device does the set-up: it fetches the array's
//    device address with cudaGetSymbolAddress and raises the shared-memory
//    limit of every pass kernel.  Make that first call before any stream
//    capture.  The set-up belongs to the device's CUDA context: after a
//    device reset (a new primary context) the next call repeats it.
//  * The 2048-point x-pass runs each tile on a cluster of two blocks whose
//    waits for each other are bounded; a wait that runs out sets the error
//    word in the array, and fft3d_noalloc_status reads and clears it.
#include <cuda.h>  // CUcontext (type only; cuCtxGetCurrent comes from the driver at run time)
#include <cuda_runtime.h>

#include <mutex>

#include "fft3d.h"
#include "launchers.h"

using namespace fft3d;

namespace {

// Twiddle space: three line tables (axis 0, axis 1, axis 2 half length) of
// at most 32 KB each (checked per call), then the contiguous-axis table
// (at most 2 (1024 + 1) complex double entries, see z_table_elems), then
// 256 bytes for the device error word.
constexpr size_t kTableSlot = 2048 * 16;
constexpr size_t kZTableSlot = 129 * 256;  // 2 (1024 + 1) * 16 bytes, rounded up to 256
constexpr size_t kTableBytes = 3 * kTableSlot + kZTableSlot + 256;
constexpr size_t kPlaneBytes = FFT3D_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kTableBytes + kPlaneBytes];

constexpr int kMaxDevices = 128;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices];      // device address of g_noalloc_scratch, per device
CUcontext g_scratch_ctx[kMaxDevices];  // the context that address and the kernel set-up belong to

// Offset of the device error word, after the tables.
constexpr size_t kErrOffset = kTableBytes - 256;

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

CtxGetCurrentFn ctx_get_current_fn()
{
    static CtxGetCurrentFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)ptr;
    });
    return fn;
}

#define FFT3D_NA_PREP(L)                                                   \
    if ((e = col_prepare_f32(L)) != cudaSuccess) return e;                 \
    if ((e = col_prepare_f64(L)) != cudaSuccess) return e;
#define FFT3D_NA_PREP_Z(M)                                                 \
    if ((e = z_prepare_f32(M)) != cudaSuccess) return e;                   \
    if ((e = z_prepare_f64(M)) != cudaSuccess) return e;

cudaError_t prepare_all_kernels()
{
    cudaError_t e;
    FFT3D_COL_LENGTHS(FFT3D_NA_PREP)
    FFT3D_Z_HALF_LENGTHS(FFT3D_NA_PREP_Z)
    return cudaSuccess;
}

// Device address of the scratch array on the current device; the first call
// per device (and per context of that device) looks it up and prepares the
// kernels.
cudaError_t scratch_for_current_device(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    CtxGetCurrentFn get_ctx = ctx_get_current_fn();
    if (!get_ctx) return cudaErrorUnknown;
    CUcontext ctx = nullptr;  // null while no context is current in this thread yet
    if (get_ctx(&ctx) != CUDA_SUCCESS) return cudaErrorUnknown;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!ctx || !g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // also makes the device's context current
        if (e != cudaSuccess) return e;
        e = prepare_all_kernels();
        if (e != cudaSuccess) return e;
        if (get_ctx(&ctx) != CUDA_SUCCESS) return cudaErrorUnknown;
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int fft3d_exec_c2r_noalloc(const void *in_cplx, void *out_real, int64_t n0, int64_t n1,
                                      int64_t n2, int dtype, void *stream)
{
    if (dtype != FFT3D_F32 && dtype != FFT3D_F64) return FFT3D_ERR_DTYPE;
    if (!fft3d_supported_length(n0, 0) || !fft3d_supported_length(n1, 1) || !fft3d_supported_length(n2, 2))
        return FFT3D_ERR_SIZE;
    const bool f32 = dtype == FFT3D_F32;
    const size_t csize = f32 ? 8 : 16;
    if (!in_cplx || !out_real) return FFT3D_ERR_NULL;
    // only an out-of-place call uses the scratch plane (in place, the output buffer holds every column)
    if (in_cplx != out_real && (size_t)n0 * (size_t)n1 * csize > kPlaneBytes) return FFT3D_ERR_SIZE;
    if ((uintptr_t)in_cplx % csize || (uintptr_t)out_real % csize) return FFT3D_ERR_ALIGN;
    const int64_t m = n2 / 2, m1 = m + 1;
    if (in_cplx != out_real) {
        const size_t lines = (size_t)n0 * (size_t)n1;
        const size_t ib = lines * (size_t)m1 * csize, ob = lines * (size_t)n2 * (csize / 2);
        const uintptr_t i0 = (uintptr_t)in_cplx, o0 = (uintptr_t)out_real;
        if (i0 < o0 + ob && o0 < i0 + ib) return FFT3D_ERR_LAYOUT;
    }
    PassGeom g0, g1, gz;
    if (!(f32 ? col_geom_f32((int)n0, 0, &g0) : col_geom_f64((int)n0, 0, &g0)) ||
        !(f32 ? col_geom_f32((int)n1, 1, &g1) : col_geom_f64((int)n1, 1, &g1)) ||
        !(f32 ? z_geom_f32((int)(n2 / 2), &gz) : z_geom_f64((int)(n2 / 2), &gz)))
        return FFT3D_ERR_SIZE;
    // every table must fit its slot (the largest, FP64 2048-point columns, takes 32512 of 32768 bytes)
    if ((size_t)col_table_elems((int)n0, g0) * csize > kTableSlot ||
        (size_t)col_table_elems((int)n1, g1) * csize > kTableSlot ||
        (size_t)line_tw_size(z_line_points((int)m, gz), gz.E) * csize > kTableSlot ||
        z_table_elems(f32, (int)m) * csize > kZTableSlot)
        return FFT3D_ERR_SIZE;

    void *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return FFT3D_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    char *tw0 = (char *)scratch;
    char *tw1 = tw0 + kTableSlot;
    char *twz = tw1 + kTableSlot;
    char *rot = twz + kTableSlot;
    void *plane = (char *)scratch + kTableBytes;
    unsigned *err_flag = (unsigned *)((char *)scratch + kErrOffset);

    cudaError_t e;
    if ((e = cudaMemsetAsync(err_flag, 0, sizeof(unsigned), st)) != cudaSuccess ||
        (e = write_col_tables(f32, (int)n0, g0, tw0, st)) != cudaSuccess ||
        (e = write_col_tables(f32, (int)n1, g1, tw1, st)) != cudaSuccess ||
        (e = write_line_tables(f32, z_line_points((int)m, gz), gz.E, twz, st)) != cudaSuccess ||
        (e = write_z_table(f32, (int)n2, rot, st)) != cudaSuccess)
        return FFT3D_ERR_CUDA;

    const bool inplace = in_cplx == out_real;
    const CLayout src = {const_cast<void *>(in_cplx), nullptr, 0};
    const CLayout dst = inplace ? src : CLayout{out_real, plane, 1};

    if (n0 > 1 || !inplace) {  // x-pass: axis 0, W flat (k1, k2) columns per tile
        ColArgs a;
        a.src = src;
        a.dst = dst;
        a.n0 = n0;
        a.n1 = n1;
        a.m = m;
        a.axis = 0;
        a.inverse = 1;
        const int64_t tiles = (n1 * m1 + g0.per_block - 1) / g0.per_block;
        a.tiles_main = tiles;
        a.tiles_per_field = tiles;
        a.tiles_per_plane = 0;
        a.nyq_in_plane = 0;
        a.bulk = 0;
        a.err = err_flag;
        a.early = 0;
        a.pf_stride = 0;
        a.tickets = nullptr;
        a.stall_tx = 0;
        a.stage_polls = kStageWaitPolls;
        e = f32 ? col_launch_f32((int)n0, a, tiles, tw0, nullptr, nullptr, st) : col_launch_f64((int)n0, a, tiles, tw0, nullptr, nullptr, st);
        if (e != cudaSuccess) return FFT3D_ERR_CUDA;
    }
    if (n1 > 1) {  // y-pass: axis 1, k2 < M tiles per plane, then the k2 = M column
        ColArgs a;
        a.src = dst;
        a.dst = dst;
        a.n0 = n0;
        a.n1 = n1;
        a.m = m;
        a.axis = 1;
        a.inverse = 1;
        a.tiles_per_plane = (m + g1.per_block - 1) / g1.per_block;
        a.tiles_main = n0 * a.tiles_per_plane;
        a.nyq_in_plane = 0;
        a.bulk = 0;
        a.err = err_flag;
        a.early = 0;
        a.pf_stride = 0;
        a.tickets = nullptr;
        a.stall_tx = 0;
        a.stage_polls = kStageWaitPolls;
        a.tiles_per_field = 1;
        const int64_t tiles = a.tiles_main + (n0 + g1.per_block - 1) / g1.per_block;
        e = f32 ? col_launch_f32((int)n1, a, tiles, tw1, nullptr, nullptr, st) : col_launch_f64((int)n1, a, tiles, tw1, nullptr, nullptr, st);
        if (e != cudaSuccess) return FFT3D_ERR_CUDA;
    }
    ZArgs z;
    z.real = nullptr;
    z.real_out = out_real;
    z.real_pitch = inplace ? 2 * m1 : n2;
    z.cplx = dst;
    z.nlines = n0 * n1;
    z.scale_edge = 1.0;
    z.scale_mid = 1.0 / ((double)n0 * (double)n1 * (double)n2);
    z.pf_lines = 0;
    z.max_blocks = 0;
    e = f32 ? zc2r_launch_f32((int)m, z, twz, rot, st) : zc2r_launch_f64((int)m, z, twz, rot, st);
    return e == cudaSuccess ? FFT3D_OK : FFT3D_ERR_CUDA;
}

extern "C" int fft3d_noalloc_status(int *device_error)
{
    if (!device_error) return FFT3D_ERR_NULL;
    *device_error = 0;
    void *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return FFT3D_ERR_CUDA;
    unsigned *err_flag = (unsigned *)((char *)scratch + kErrOffset);
    unsigned v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, err_flag, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v) e = cudaMemset(err_flag, 0, sizeof(unsigned));
    if (e != cudaSuccess) return FFT3D_ERR_CUDA;
    *device_error = v ? 1 : 0;
    return FFT3D_OK;
}
