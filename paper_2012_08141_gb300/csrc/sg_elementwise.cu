// sg_elementwise.cu -- fused element-wise struct-fors.  A run of element-wise
// ops over the same grid (the general kernels of the paper's
// microbenchmarks: copies, increments, fills, saxpy, products; Supp. Sec. 1)
// is fused into one launch (Sec. 6.4: same list, every access at the voxel of
// the iteration): each field the run reads is loaded once, the ops run on
// values held in a per-thread register file in shared memory, and only the
// live final values are stored (Sec. 6.5).  An optional reduction of one
// field, at its place in the run, is fused as well.
#include <atomic>

#include "sg_common.cuh"

namespace sg {

__device__ __forceinline__ float4 f4_fma(float al, float4 a, float4 c)
{
    return make_float4(fmaf(al, a.x, c.x), fmaf(al, a.y, c.y), fmaf(al, a.z, c.z), fmaf(al, a.w, c.w));
}
__device__ __forceinline__ float4 f4_splat(float v) { return make_float4(v, v, v, v); }
__device__ __forceinline__ float4 f4_mask(uint32_t bits, float4 v)
{
    return make_float4((bits & 1u) ? v.x : 0.f, (bits & 2u) ? v.y : 0.f, (bits & 4u) ? v.z : 0.f,
                       (bits & 8u) ? v.w : 0.f);
}

__device__ __forceinline__ void ld8(const float *p, float4 &a, float4 &b)
{
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}
__device__ __forceinline__ void st8(float *p, float4 a, float4 b)
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x), "f"(a.y), "f"(a.z),
                 "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

constexpr int kEwThreads = 128;

// One thread handles eight consecutive voxels (a 32-byte row piece) of a
// listed leaf, as two float4 halves h = 0, 1.  The op loop is unrolled, so
// each op's fields are compile-time offsets into the kernel's parameters and
// its kind a uniform branch.  Values at inactive voxels are carried unmasked
// through the run (ops are voxel-wise, so they never reach an active voxel)
// and set to 0 where they leave it: at the stores and in the reduction.
template <int L>
__global__ void __launch_bounds__(kEwThreads, 8) k_ew(DevGrid g, EwProgram prog)
{
    constexpr int V = L * L * L, Q = V / 8, LG2 = (L == 8) ? 3 : 2;
    extern __shared__ float4 s_reg[];  // [n_slots][2][kEwThreads]
    __shared__ double s_red[kEwThreads / 32];
    const long long n = g.ctrl->list_n;
    float4 *reg = s_reg + threadIdx.x;  // slot k, half h at reg[(2k + h) * kEwThreads]
    constexpr int S = kEwThreads;
    float part = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    // the slot of the next iteration is read one iteration ahead, so the mask
    // word and the field rows of an iteration are requested together
    int slot_next = q < n * Q ? g.list_slot[q / Q] : 0;
    for (; q < n * Q; q += stride) {
        const long long e = q / Q;
        const int c = (int)(q - e * Q);
        const int slot = slot_next;
        if (q + stride < n * Q) slot_next = g.list_slot[(q + stride) / Q];
        const int l = 8 * c;
        const uint32_t bits = (g.mask[(long long)slot * g.W + (l >> 5)] >> (l & 31)) & 0xffu;
        const uint32_t b0 = bits & 0xfu, b1 = bits >> 4;
        const long long base = ((long long)slot << (3 * LG2)) + l;
#pragma unroll
        for (int k = 0; k < kMaxEwSlots; ++k)
            if (k < prog.n_slots && prog.load[k]) {
                float4 a, b;
                ld8(prog.fp[k] + base, a, b);
                reg[(2 * k) * S] = a;
                reg[(2 * k + 1) * S] = b;
            }
#pragma unroll
        for (int i = 0; i < kMaxEwOps + 1; ++i) {
            if (i >= prog.n_ops) break;
            const EwOp &o = prog.op[i];
            float4 *d = reg + 2 * o.dst * S;
            const float4 *ra = reg + 2 * o.a * S, *rb = reg + 2 * o.b * S;
            switch (o.kind) {
            case kEwFill:
                d[0] = f4_splat(o.delta);
                d[S] = f4_splat(o.delta);
                break;
            case kEwAx: {
                const float4 a0 = ra[0], a1 = ra[S];
                d[0] = f4_fma(o.alpha, a0, f4_splat(o.delta));
                d[S] = f4_fma(o.alpha, a1, f4_splat(o.delta));
                break;
            }
            case kEwAxby: {
                const float4 a0 = ra[0], a1 = ra[S], c0 = rb[0], c1 = rb[S];
                d[0] = f4_fma(o.alpha, a0, f4_fma(o.beta, c0, f4_splat(o.delta)));
                d[S] = f4_fma(o.alpha, a1, f4_fma(o.beta, c1, f4_splat(o.delta)));
                break;
            }
            case kEwSum: {
                const float4 v0 = f4_mask(b0, ra[0]), v1 = f4_mask(b1, ra[S]);
                part += ((v0.x + v0.y) + (v0.z + v0.w)) + ((v1.x + v1.y) + (v1.z + v1.w));
                break;
            }
            default: {
                const float4 a0 = ra[0], a1 = ra[S], c0 = rb[0], c1 = rb[S];
                const float4 r0 = f4_fma(o.alpha, a0, f4_fma(o.beta, c0, f4_splat(o.delta)));
                const float4 r1 = f4_fma(o.alpha, a1, f4_fma(o.beta, c1, f4_splat(o.delta)));
                d[0] = make_float4(fmaf(o.gamma * a0.x, c0.x, r0.x), fmaf(o.gamma * a0.y, c0.y, r0.y),
                                   fmaf(o.gamma * a0.z, c0.z, r0.z), fmaf(o.gamma * a0.w, c0.w, r0.w));
                d[S] = make_float4(fmaf(o.gamma * a1.x, c1.x, r1.x), fmaf(o.gamma * a1.y, c1.y, r1.y),
                                   fmaf(o.gamma * a1.z, c1.z, r1.z), fmaf(o.gamma * a1.w, c1.w, r1.w));
                break;
            }
            }
        }
#pragma unroll
        for (int k = 0; k < kMaxEwSlots; ++k)
            if (k < prog.n_slots && prog.store[k])
                st8(prog.fp[k] + base, f4_mask(b0, reg[(2 * k) * S]), f4_mask(b1, reg[(2 * k + 1) * S]));
    }
    if (prog.sum_out >= 0) {
        const double tot = block_sum_f64<kEwThreads>((double)part, s_red);
        finish_reduction(g, tot, prog.sum_out);
    }
}

// CTAs resident per SM for a program of n_slots slots (dynamic shared memory
// 4 KB per slot), all launched at once (one reduction partial each).
template <int L>
static int ew_ctas(int num_sms, int n_slots)
{
    static std::atomic<int> cache[kMaxEwSlots + 1];  // per program size; threads may race to fill it
    int per = cache[n_slots].load(std::memory_order_relaxed);
    if (!per) {
        const size_t smem = sizeof(float4) * 2 * kEwThreads * n_slots;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ew<L>, kEwThreads, smem) != cudaSuccess || per < 1)
            per = 1;
        cache[n_slots].store(per, std::memory_order_relaxed);
    }
    return per * num_sms;
}

void launch_ew(const DevGrid &g, cudaStream_t s, const EwProgram &prog, const LaunchCfg &lc)
{
    EwProgram p = prog;
    for (int k = 0; k < p.n_slots; ++k) p.fp[k] = g.field[p.field[k]];
    const int ns = p.n_slots < 1 ? 1 : p.n_slots;
    const size_t smem = sizeof(float4) * 2 * kEwThreads * ns;
    if (g.L == 8) k_ew<8><<<ew_ctas<8>(lc.num_sms, ns), kEwThreads, smem, s>>>(g, p);
    else k_ew<4><<<ew_ctas<4>(lc.num_sms, ns), kEwThreads, smem, s>>>(g, p);
}

}  // namespace sg
