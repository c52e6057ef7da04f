// sg_common.cuh -- small device helpers shared by the libsgrid kernels.
#pragma once
#include <cstdint>
#include "sg_device.h"

namespace sg {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Mark the grid's structure as changed (an activation set a new bit or
// allocated a leaf); the next list generation will not be skipped.
__device__ __forceinline__ void mark_dirty(const DevGrid &g) { *(volatile int32_t *)&g.ctrl->dirty = 1; }

__device__ __forceinline__ void raise_error(const DevGrid &g, int bits) { atomicOr(&g.ctrl->err, bits); }

// Block-wide FP64 reduction of one value per thread; result valid in thread 0.
template <int THREADS>
__device__ __forceinline__ double block_sum_f64(double v, double *smem)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) smem[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = (threadIdx.x < THREADS / 32) ? smem[threadIdx.x] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// Last-CTA reduction: every CTA stores its FP64 partial; the CTA that finishes
// last sums all partials in index order (deterministic) into sums[slot] and
// resets the ticket.  Called by all threads; `part` valid in thread 0.
__device__ __forceinline__ void finish_reduction(const DevGrid &g, double part, int slot)
{
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        g.partials[blockIdx.x] = part;
        __threadfence();
        unsigned t = atomicAdd(&g.ctrl->red_ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x < 32) {
            // fixed-order: lane handles a strided subset, then a fixed tree
            double acc = 0.0;
            for (unsigned c = threadIdx.x; c < gridDim.x; c += 32)
                acc += *(volatile double *)&g.partials[c];
            acc = warp_sum(acc);
            if (threadIdx.x == 0) {
                g.sums[slot] = acc;
                g.ctrl->red_ticket = 0;
            }
        }
    }
}

}  // namespace sg
