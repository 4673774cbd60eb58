// FP64 arithmetic throughput of the current GPU, measured in place: the roof
// that bounds the FP64 passes (the paper's double-precision runs, Sec. 4,
// Table 3), which on GB300 are limited by FP64 add / multiply issue rather
// than by HBM.
//
// Each thread runs 8 independent dependency chains of one FP64 operation
// (FMA, add or multiply), so the FP64 units, not latency, set the rate; the
// grid fills every SM (8 blocks of 256 threads).  The chains' results feed a
// comparison that is never true, which keeps the work without writing memory.
#include <cuda_runtime.h>

#include "fft3d.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kIters = 4096;

static __device__ double g_probe_sink[kThreads];

template <int OP>  // 0: fma(x, b, c), 1: x + b, 2: x * b
__global__ void __launch_bounds__(kThreads) fp64_probe_kernel(double b, double c, int iters)
{
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            if (OP == 0) x[k] = fma(x[k], b, c);
            else if (OP == 1) x[k] = x[k] + b;
            else x[k] = x[k] * b;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    if (s == -1.0) g_probe_sink[threadIdx.x] = s;
}

// Best of `reps` timed launches, in FP64 operations per second.
template <int OP> cudaError_t time_op(double b, double c, int blocks, cudaStream_t st, double *ops_per_s)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const double ops = (double)blocks * kThreads * kChains * (double)kIters;
    double best = 0.0;
    for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // the first launch warms up
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            fp64_probe_kernel<OP><<<blocks, kThreads, 0, st>>>(b, c, kIters);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0 && ms > 0.f && ops / (ms * 1e-3) > best) best = ops / (ms * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ops_per_s = best;
    return e;
}

}  // namespace

extern "C" int fft3d_measure_fp64_peak(double *fma_gflops, double *add_gflops, double *mul_gflops)
{
    if (!fma_gflops || !add_gflops || !mul_gflops) return FFT3D_ERR_NULL;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) return FFT3D_ERR_CUDA;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return FFT3D_ERR_CUDA;
    const int blocks = 8 * sms;
    double fma_ops = 0.0, add_ops = 0.0, mul_ops = 0.0;
    e = time_op<0>(0.999999, 1e-7, blocks, st, &fma_ops);
    if (e == cudaSuccess) e = time_op<1>(1e-9, 0.0, blocks, st, &add_ops);
    if (e == cudaSuccess) e = time_op<2>(0.9999999, 0.0, blocks, st, &mul_ops);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) return FFT3D_ERR_CUDA;
    *fma_gflops = 2.0 * fma_ops * 1e-9;  // an FMA is two flops
    *add_gflops = add_ops * 1e-9;
    *mul_gflops = mul_ops * 1e-9;
    return FFT3D_OK;
}
