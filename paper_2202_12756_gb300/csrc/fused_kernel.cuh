// Fused plane pass: the contiguous-axis line transforms and the axis-1 column
// transforms of every k0 plane in one persistent kernel, with the plane
// handed from one to the other through L2 instead of HBM.
//
// This is Step 1 of Sec. 3 (the batched 2D FFT of each plane) done so that a
// plane's intermediate never leaves the 129 MB L2: HBM sees the array read
// once and written once for both axes, instead of twice each.
//
// Work items, for plane p:
//   Z(p, g)  LPB lines of the plane (R2C forward / C2R inverse),
//   Y(p, t)  W columns k2 of the plane, all N1 rows (C2C along axis 1);
//            the last tile of a plane is ragged and holds k2 = M.
// Forward, Z items produce and Y items consume a plane; inverse, the reverse.
// Blocks take tickets from one atomic counter; tickets follow the order
//   P(0..lag-1), then for s = lag .. N0-1: P(s), C(s - lag), then C(the rest)
// where P / C are the producer / consumer items of a plane.  A consumer waits
// until all producers of its plane have finished.  Every ticket before it was
// taken by a block that is running, and producers never wait, so each wait
// ends.  The wait is nevertheless bounded: past `spin_limit` polls it raises
// the launch and sticky error flags, and every block leaves at its next
// ticket.  Producers publish with a fence per thread, a barrier, then one
// atomic increment; consumers poll with an acquire load and read the plane
// with L2-only loads.
#pragma once

#include "pass_kernels.cuh"

namespace fft3d {

struct FusedArgs {
    ZArgs z;               // line pass over all N0 * N1 lines
    ColArgs y;             // axis-1 pass, nyq_in_plane = 1
    int64_t n0;
    int64_t zi;            // Z items per plane
    int64_t yi;            // Y items per plane
    int64_t lag;           // planes between a plane's producers and its consumers
    int64_t n_items;       // n0 * (zi + yi)
    unsigned *sync;        // [0] tickets, [1] launch error, [8 + p] producers done (sticky error: y.err)
    long long spin_limit;  // polls before a consumer gives up
    int inject_stall;      // test hook: consumers wait for one producer more than exists
    int forward;           // 1: R2C (Z -> Y); 0: C2R (Y -> Z)
};

enum { kSyncTickets = 0, kSyncLaunchErr = 1, kSyncDone = 8 };

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned *p)
{
    return *(volatile const unsigned *)p;
}

// ticket -> (producer?, plane, index in the plane's item list)
__device__ __forceinline__ void fused_decode(const FusedArgs &a, int64_t t, bool &prod, int64_t &plane,
                                             int64_t &idx)
{
    const int64_t A = a.forward ? a.zi : a.yi;  // producer items per plane
    const int64_t B = a.forward ? a.yi : a.zi;  // consumer items per plane
    const int64_t lag = a.lag < a.n0 ? a.lag : a.n0;
    const int64_t head = lag * A;
    if (t < head) {
        prod = true;
        plane = t / A;
        idx = t - plane * A;
        return;
    }
    int64_t u = t - head;
    const int64_t mid = (a.n0 - lag) * (A + B);
    if (u < mid) {
        const int64_t s = u / (A + B);
        const int64_t r = u - s * (A + B);
        if (r < A) {
            prod = true;
            plane = lag + s;
            idx = r;
        } else {
            prod = false;
            plane = s;
            idx = r - A;
        }
        return;
    }
    u -= mid;
    prod = false;
    plane = (a.n0 - lag) + u / B;
    idx = u - (u / B) * B;
}

// N1: column length (axis 1), M: half line length, W: columns per Y tile,
// LPB: lines per Z item; W * N1 / E1 == LPB * M / E2 threads per block.
template <typename R, int N1, int M, int W, int LPB, int MINB>
__global__ void __launch_bounds__(W *(N1 / line_E(N1)), MINB)
fused_plane_kernel(FusedArgs a, const typename cvec<R>::T *__restrict__ tw_y,
                   const typename cvec<R>::T *__restrict__ tw_z, const typename cvec<R>::T *__restrict__ rot)
{
    static_assert(W * (N1 / line_E(N1)) == LPB * (M / z_E<R, M>()), "Y and Z items need the same block");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_ticket;
    __shared__ int s_abort;
    unsigned *sync = a.sync;
    const int64_t A = a.forward ? a.zi : a.yi;

    for (;;) {
        if (threadIdx.x == 0) {
            const bool err = ld_volatile_u32(sync + kSyncLaunchErr) != 0;
            s_ticket = err ? a.n_items : (int64_t)atomicAdd(sync + kSyncTickets, 1u);
        }
        __syncthreads();
        const int64_t t = s_ticket;
        if (t >= a.n_items) break;
        bool prod;
        int64_t plane, idx;
        fused_decode(a, t, prod, plane, idx);
        const bool z_item = (prod == (a.forward != 0));

        if (!prod) {
            // wait for the plane's producers
            if (threadIdx.x == 0) {
                const unsigned target = (unsigned)A + (a.inject_stall ? 1u : 0u);
                long long polls = 0;
                int abort = 0;
                while (ld_acquire_u32(sync + kSyncDone + plane) < target) {
                    if (ld_volatile_u32(sync + kSyncLaunchErr) != 0) {
                        abort = 1;
                        break;
                    }
                    if (++polls > a.spin_limit) {
                        atomicOr(sync + kSyncLaunchErr, 1u);
                        atomicOr(a.y.err, 1u);  // sticky: survives the next launch
                        abort = 1;
                        break;
                    }
                    __nanosleep(128);
                }
                s_abort = abort;
            }
            __syncthreads();
            if (s_abort) break;
        }

        if (z_item) {
            const int64_t line0 = plane * a.y.n1 + idx * LPB;
            if (a.forward) zr2c_lines<R, M, z_E<R, M>(), LPB>(a.z, line0, smem_raw, tw_z, rot);
            else zc2r_lines<R, M, z_E<R, M>(), LPB, true>(a.z, line0, smem_raw, tw_z, rot);
        } else {
            const int64_t tile = plane * a.yi + idx;
            if (a.forward) col_tile<R, N1, line_E(N1), W, true, false>(a.y, tile, smem_raw, tw_y);
            else col_tile<R, N1, line_E(N1), W, false, true>(a.y, tile, smem_raw, tw_y);
        }

        if (prod) {
            __threadfence();  // this thread's stores of the item are visible GPU-wide
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(sync + kSyncDone + plane, 1u);
        } else {
            __syncthreads();  // shared memory free before the next item
        }
    }
}

}  // namespace fft3d
