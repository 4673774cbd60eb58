/*
 * fft3d -- single-GPU 3D real FFT for GB300 (sm_103a).
 *
 * C ABI.  Plain pointers and sizes only; no C++ or framework types cross it.
 * Every function returns a status code (enum fft3d_status); none throws.
 *
 * Operation (arXiv 2202.12756, Sec. 2):
 *   forward  F[k0][k1][k2] = sum_j f[j0][j1][j2] exp(-2 pi i (j0 k0/N0 + j1 k1/N1 + j2 k2/N2))
 *            (Eq. 1, unnormalised), stored for k2 = 0 .. N2/2 only (Eqs. 3-4:
 *            the spectrum of a real field is Hermitian, so half is kept).
 *   inverse  f[j] = (1/(N0 N1 N2)) sum_k Ft[k] exp(+2 pi i ...)  (Eq. 2 over the
 *            Hermitian extension Ft of the stored half, followed by the
 *            normalisation step of Sec. 4).
 * The paper's slab pipeline (Sec. 3: plane FFTs, transposes, all-to-all,
 * line FFTs along the slowest axis) runs here as three passes over HBM on one
 * GPU: contiguous-axis R2C/C2R lines, then strided C2C columns along axis 1,
 * then strided C2C columns along axis 0 (reversed for the inverse).
 *
 * Arrays are C order, axis 2 fastest.  N2 is the halved axis.
 *   real array     [N0][N1][N2]       dense (out-of-place), or
 *                  [N0][N1][2(N2/2+1)] padded rows (in-place; pad values are
 *                  neither read nor preserved);
 *   complex array  [N0][N1][N2/2+1]   interleaved (re, im) pairs of the dtype.
 * In-place means in == out (the padded layout); any other overlap between
 * the input and output ranges is FFT3D_ERR_LAYOUT.
 *
 * Supported lengths: N0, N1 in {2^k : 0 <= k <= 11} U {3 * 2^k : 0 <= k <= 9};
 * N2 even with N2/2 in {2^k : 0 <= k <= 10} U {3 * 2^k : 0 <= k <= 8}
 * (so every axis is at most 2048).  Anything else is FFT3D_ERR_SIZE.
 *
 * Devices and streams: a plan belongs to the device that was current when it
 * was created; every exec call must run with that device current
 * (FFT3D_ERR_DEVICE otherwise).  `stream` is a cudaStream_t (NULL = legacy
 * default stream).  Execution is asynchronous with respect to the host; the
 * caller owns all data buffers and keeps them alive until the stream has
 * finished.  A plan may be used by one stream at a time (its scratch is
 * shared between calls); distinct plans are independent.
 *
 * Pointers must be aligned to one complex element (8 bytes for FFT3D_F32,
 * 16 bytes for FFT3D_F64), else FFT3D_ERR_ALIGN, and point to device memory,
 * except where a function says that host memory is accepted (the real input
 * of an out-of-place fft3d_exec_r2c, the real output of
 * fft3d_exec_c2r_overwrite).  A batched plan (fft3d_plan_create_batched)
 * takes `batch` such arrays stored one after another.
 */
#ifndef FFT3D_H
#define FFT3D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft3d_plan_s *fft3d_plan;

enum fft3d_dtype {
    FFT3D_F32 = 0, /* float storage and arithmetic, twiddles generated in FP64 */
    FFT3D_F64 = 1  /* double storage and arithmetic */
};

enum fft3d_status {
    FFT3D_OK = 0,
    FFT3D_ERR_SIZE = 1,   /* unsupported N0, N1 or N2 */
    FFT3D_ERR_DTYPE = 2,  /* dtype not in enum fft3d_dtype */
    FFT3D_ERR_NULL = 3,   /* a required pointer (plan, in, out, result) is NULL */
    FFT3D_ERR_ALIGN = 4,  /* a data pointer is not aligned to one complex element */
    FFT3D_ERR_ALLOC = 5,  /* device or host allocation failed */
    FFT3D_ERR_CUDA = 6,   /* a CUDA call or kernel launch failed; see fft3d_plan_last_error */
    FFT3D_ERR_LAYOUT = 7, /* input and output overlap without being identical */
    FFT3D_ERR_DEVICE = 8, /* current device differs from the plan's device */
    FFT3D_ERR_ARG = 9     /* any other invalid argument */
};

/*
 * Create a plan for an N0 x N1 x N2 real transform of the given dtype on the
 * current device.  Allocates the plan (host) and, on the device, its FP64-
 * generated twiddle tables (O(N0 + N1 + N2) entries) and an N0*N1-element
 * complex scratch plane used only by out-of-place fft3d_exec_c2r /
 * fft3d_exec_r2c_adjoint.  Synchronises the device once (table generation).
 * On success *plan is set and FFT3D_OK returned; on failure *plan is NULL.
 */
int fft3d_plan_create(fft3d_plan *plan, int64_t n0, int64_t n1, int64_t n2, int dtype);

/*
 * Batched plan: every exec call transforms `batch` fields of N0 x N1 x N2
 * stored one after another (real [batch][N0][N1][N2] dense or
 * [batch][N0][N1][2(N2/2+1)] padded; complex [batch][N0][N1][N2/2+1]), with
 * one launch per pass for all of them, e.g. the three velocity components of
 * the pseudo-spectral turbulence solvers that motivate the paper (Sec. 1),
 * or several fields in flight as in the batched GPU-FFT it compares with
 * (Sec. 5).  Each field is transformed exactly as by a plan of batch 1 (and
 * normalised by 1/(N0 N1 N2)); the fields never mix.  The scratch plane of
 * the out-of-place inverse grows to batch*N0*N1 elements.  batch must be
 * >= 1 with batch*N0*N1 <= 2^31, else FFT3D_ERR_SIZE.  The opt-in fused
 * plane pass is not offered for batch > 1.  fft3d_plan_create(p, ...) is
 * fft3d_plan_create_batched(p, 1, ...).
 */
int fft3d_plan_create_batched(fft3d_plan *plan, int64_t batch, int64_t n0, int64_t n1, int64_t n2, int dtype);

/* Release the plan and its device memory.  NULL is accepted (no-op).
 * The caller must make sure no stream still runs work of this plan. */
int fft3d_plan_destroy(fft3d_plan plan);

/*
 * Forward R2C, Eq. 1 (unnormalised, sign -).
 *   in_real:  real array (dense [N0][N1][N2], or padded when in_real == out_cplx)
 *   out_cplx: complex array [N0][N1][N2/2+1]
 * Out-of-place calls never write in_real and read it exactly once, in the
 * first (contiguous) pass, so it may be device-accessible host memory (see
 * fft3d_exec_c2r_overwrite).
 */
int fft3d_exec_r2c(fft3d_plan plan, const void *in_real, void *out_cplx, void *stream);

/*
 * Inverse C2R, Eq. 2 (sign +) followed by the 1/(N0 N1 N2) normalisation.
 *   in_cplx:  complex array [N0][N1][N2/2+1]
 *   out_real: real array (dense [N0][N1][N2], or padded when in_cplx == out_real)
 * Input that is not Hermitian-consistent is accepted: the inverse C2C along
 * axes 0 and 1 runs as is, and along axis 2 only the real parts of the
 * k2 = 0 and k2 = N2/2 entries are used.
 * Out-of-place calls never write in_cplx (the plan's scratch plane holds the
 * k2 = N2/2 column, which does not fit in the dense real output).
 */
int fft3d_exec_c2r(fft3d_plan plan, const void *in_cplx, void *out_real, void *stream);

/*
 * The same inverse as fft3d_exec_c2r, out of place, using the input array as
 * work space: the axis-0 and axis-1 passes run in place on inout_cplx (which
 * is overwritten), and out_real (dense [N0][N1][N2]) is written exactly once,
 * by the last, contiguous pass, and never read.  Needs no plan scratch.
 * Because only that pass touches them, in_real of fft3d_exec_r2c and out_real
 * here may be host memory the GPU can access directly (pinned / registered
 * host memory, or any system memory on a coherent CPU-GPU node): the first
 * and last passes then stream the field over the CPU-GPU link while the
 * strided passes stay in HBM.  Such a pass runs on a fixed, small grid (the
 * link bounds it), so the strided passes of another plan on another stream
 * can run beside it: several fields in flight on several streams overlap
 * their link traffic with each other's work in HBM.  With inout_cplx ==
 * out_real this is the in-place inverse.
 */
int fft3d_exec_c2r_overwrite(fft3d_plan plan, void *inout_cplx, void *out_real, void *stream);

/*
 * Adjoint (vector-Jacobian product) of fft3d_exec_r2c with respect to its
 * real input: for a cotangent G on the half spectrum (G = dL/dRe F + i dL/dIm F)
 *   out[j] = Re sum_{k in half spectrum} G[k] exp(+2 pi i k.j/N),
 * computed as the C2R pipeline with the k2 = 0 and k2 = N2/2 planes weighted
 * by 2, an overall factor 1/2 and no 1/N^3.  Same layouts and aliasing rules
 * as fft3d_exec_c2r.  The paper has no adjoint; it follows from Eq. 1.
 */
int fft3d_exec_r2c_adjoint(fft3d_plan plan, const void *in_cplx, void *out_real, void *stream);

/*
 * Adjoint of fft3d_exec_c2r with respect to its complex input: for a real
 * cotangent g,
 *   out[k] = (c(k2) / (N0 N1 N2)) sum_j g[j] exp(-2 pi i k.j/N),
 * c = 1 on the k2 = 0 and k2 = N2/2 planes, 2 elsewhere; computed as the R2C
 * pipeline with those weights applied in its first pass.  Same layouts and
 * aliasing rules as fft3d_exec_r2c.  Follows from Eq. 2 and the normalisation.
 */
int fft3d_exec_c2r_adjoint(fft3d_plan plan, const void *in_real, void *out_cplx, void *stream);

/* Static text for a status code ("unknown status" for anything else). */
const char *fft3d_strerror(int status);

/* Text of the last error recorded on this plan ("" if none). */
const char *fft3d_plan_last_error(fft3d_plan plan);

/* 1 if n is a supported length for `axis` (0, 1 or 2), else 0. */
int fft3d_supported_length(int64_t n, int axis);

/*
 * Per-kernel timing of the plan's launches (diagnostics).  While enabled,
 * each kernel launch is bracketed by CUDA events on the launch stream.
 * fft3d_plan_profile_read synchronises on the recorded events, writes up to
 * `max` entries (one per pass kind that ran) into `stats`, sets *count, and
 * clears the accumulated data.  Enabling costs two event records per launch.
 */
typedef struct fft3d_kernel_stat {
    char name[32];            /* pass kind, e.g. "r2c.z", "c2r.x" */
    int64_t launches;         /* launches timed */
    double total_ms;          /* summed event-to-event time */
    double bytes_per_launch;  /* algorithmic HBM bytes one launch must move */
} fft3d_kernel_stat;

int fft3d_plan_set_profiling(fft3d_plan plan, int enable);
int fft3d_plan_profile_read(fft3d_plan plan, fft3d_kernel_stat *stats, int max, int *count);

/* Kernel launches issued through this plan since creation. */
int fft3d_plan_launch_count(fft3d_plan plan, int64_t *count);

/*
 * Fused plane pass (opt-in).  For float plans with (N1, N2/2) in
 * {(512, 256), (768, 384), (1024, 512), (1536, 768), (2048, 1024)}, axes 2
 * and 1 can run as one persistent kernel that hands each k0 plane from the
 * line transforms to the column transforms through L2, so HBM sees one read
 * and one write of the array for both axes instead of two each.  Blocks in it
 * wait on per-plane counters set by other blocks.  Off by default: on GB300
 * at 1024^3 these passes are bound by instruction issue rather than HBM, and
 * the fused kernel is slower than the separate passes.  Returns
 * FFT3D_ERR_SIZE when the plan's shape or dtype has no fused kernel.
 */
int fft3d_plan_set_fused(fft3d_plan plan, int enable);

/*
 * Device-side error flag of the plan's kernels that wait: the fused plane
 * pass (see fft3d_plan_set_fused), whose blocks wait on per-plane counters,
 * and the pipelined FP32 column passes, whose blocks wait on an mbarrier for
 * the TMA copies of their next tile (2048-point x-passes run each tile on a
 * cluster of two blocks, which also wait on mbarriers for each other's half
 * of the last radix-2 step).  Each such wait is bounded; a wait that runs out
 * makes the waiting blocks (both blocks of a cluster) stop early (the output
 * is then invalid) and sets this flag.  fft3d_plan_status synchronises the device, stores the
 * flag (0 or 1) in *device_error and clears it.
 */
int fft3d_plan_status(fft3d_plan plan, int *device_error);

/*
 * Test hook for the bounded waits above: with inject_stall != 0 every
 * waiting block of the fused pass waits for one producer more than exists,
 * and every tile wait of a pipelined column pass expects 16 bytes more than
 * its copies deliver, so the waits run out after `spin_limit` polls (about
 * 0.1 us each; <= 0 restores the defaults of about one second for the fused
 * pass and 0.1 s per tile wait) and fft3d_plan_status then reports the
 * error.  Keep inject_stall = 0 outside such tests.
 */
int fft3d_plan_set_debug(fft3d_plan plan, int inject_stall, int64_t spin_limit);

/* *fused_plane_pass = 1 when the plan currently runs axes 2 and 1 as one
 * fused pass (fft3d_plan_set_fused), else 0. */
int fft3d_plan_info(fft3d_plan plan, int *fused_plane_pass);

/*
 * Normalised inverse C2R without a plan and without allocating anything.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc: a program whose own pool allocator already holds
 * the GPU's memory, or code that must not trigger the implicit device
 * synchronisation cudaMalloc / cudaFree can cause.  fft3d_plan_create
 * allocates, so these callers cannot make a plan.
 *
 * Computes exactly what fft3d_exec_c2r computes for a plan of
 * (n0, n1, n2, dtype), with the same pass kernels, layouts, aliasing and
 * alignment rules, on `stream`.  Instead of plan memory it uses one static
 * device array of the library: FFT3D_NOALLOC_SCRATCH_BYTES for the
 * N0 x N1 scratch plane plus 128.5 KiB of twiddle tables.  So:
 *   - every GPU that loads the library holds that array until the process
 *     exits;
 *   - all calls share it and it keeps the last call's contents; calls that
 *     overlap on the GPU (other streams, other host threads) race on it;
 *   - nothing in it needs clearing by the caller: each call rewrites the
 *     tables, writes the scratch plane in full before reading it, and clears
 *     the device error word (below) on `stream` before its kernels run;
 *   - the first call on a device performs set-up (cudaGetSymbolAddress of
 *     the array and the kernels' shared-memory limits); make that first call
 *     before any stream capture.  The set-up belongs to the device's current
 *     CUDA context: after a device reset the next call repeats it.
 * Out of place, sizes beyond the array's scratch plane, n0 * n1 * (8 bytes
 * for FFT3D_F32, 16 for FFT3D_F64) > FFT3D_NOALLOC_SCRATCH_BYTES, are
 * rejected with FFT3D_ERR_SIZE before any work is queued (in place,
 * in_cplx == out_real, needs no scratch plane and has no such limit), as are
 * unsupported lengths.
 * The 2048-point x-pass (n0 = 2048, FFT3D_F32) runs each tile on a cluster of
 * two blocks whose waits for each other are bounded; a wait that runs out
 * leaves the output invalid and sets the array's device error word, which
 * this call cannot report (it returns before its kernels run): read it with
 * fft3d_noalloc_status.
 */
#define FFT3D_NOALLOC_SCRATCH_BYTES (8u << 20)
int fft3d_exec_c2r_noalloc(const void *in_cplx, void *out_real, int64_t n0, int64_t n1, int64_t n2,
                           int dtype, void *stream);

/*
 * Device error word of fft3d_exec_c2r_noalloc on the current device: 1 if a
 * bounded wait in one of its calls ran out since the word was last cleared
 * (by a call, or by this function), else 0.  Synchronises the device, stores
 * the word in *device_error and clears it.  Allocates nothing.  The paper
 * has no counterpart.
 */
int fft3d_noalloc_status(int *device_error);

/*
 * FP64 throughput of the current device, measured: the roof of the FP64
 * passes, which on GB300 are bound by FP64 add / multiply issue rather than
 * by HBM (the paper compares single and double precision in Sec. 4, Table
 * 3).  Runs three short kernels (FMA, add and multiply chains that fill every
 * SM) on a private stream and synchronises; stores the best of three timed
 * launches of each in GFLOP/s (an FMA counts two flops, an add or multiply
 * one).  A diagnostic for the bench; it touches no plan or user memory.
 */
int fft3d_measure_fp64_peak(double *fma_gflops, double *add_gflops, double *mul_gflops);

#ifdef __cplusplus
}
#endif

#endif /* FFT3D_H */
