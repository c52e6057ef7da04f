// sg_elementwise.cu -- fused element-wise struct-fors.  A run of element-wise
// ops over the same grid (the general kernels of the paper's
// microbenchmarks: copies, increments, fills, saxpy, products; Supp. Sec. 1)
// is fused into one launch (Sec. 6.4: same list, every access at the voxel of
// the iteration): each field the run reads is loaded once, the ops run on
// values held in a per-thread register file in shared memory, and only the
// live final values are stored (Sec. 6.5).  An optional reduction of one
// field, at its place in the run, is fused as well.
#include "sg_common.cuh"

namespace sg {

// One thread handles four consecutive voxels (a float4) of a listed leaf.
template <int L>
__global__ void __launch_bounds__(256) k_ew(DevGrid g, EwProgram prog)
{
    constexpr int V = L * L * L, Q = V / 4, LG2 = (L == 8) ? 3 : 2;
    __shared__ float4 s_reg[kMaxEwSlots][256];
    __shared__ double s_red[8];
    const long long n = g.ctrl->list_n;
    float4 *reg = &s_reg[0][threadIdx.x];  // slot k at reg[k * 256]
    float part = 0.f;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * Q;
         q += (long long)gridDim.x * blockDim.x) {
        const long long e = q / Q;
        const int c = (int)(q - e * Q);
        const int slot = g.list_slot[e];
        const int l = 4 * c;
        const uint32_t bits = (g.mask[(long long)slot * g.W + (l >> 5)] >> (l & 31)) & 0xfu;
        const long long base = ((long long)slot << (3 * LG2)) + l;
        for (int k = 0; k < prog.n_slots; ++k)
            if (prog.load[k]) reg[k * 256] = *reinterpret_cast<const float4 *>(g.field[prog.field[k]] + base);
        for (int i = 0; i < prog.n_ops; ++i) {
            const EwOp &o = prog.op[i];
            if (o.dst < 0) {  // reduction of slot o.a at this point of the run
                const float4 v = reg[o.a * 256];
                part += ((bits & 1u) ? v.x : 0.f) + ((bits & 2u) ? v.y : 0.f) + ((bits & 4u) ? v.z : 0.f) +
                        ((bits & 8u) ? v.w : 0.f);
                continue;
            }
            const float4 a = o.a >= 0 ? reg[o.a * 256] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 b = o.b >= 0 ? reg[o.b * 256] : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 r;
            r.x = (bits & 1u) ? fmaf(o.gamma * a.x, b.x, fmaf(o.alpha, a.x, fmaf(o.beta, b.x, o.delta))) : 0.f;
            r.y = (bits & 2u) ? fmaf(o.gamma * a.y, b.y, fmaf(o.alpha, a.y, fmaf(o.beta, b.y, o.delta))) : 0.f;
            r.z = (bits & 4u) ? fmaf(o.gamma * a.z, b.z, fmaf(o.alpha, a.z, fmaf(o.beta, b.z, o.delta))) : 0.f;
            r.w = (bits & 8u) ? fmaf(o.gamma * a.w, b.w, fmaf(o.alpha, a.w, fmaf(o.beta, b.w, o.delta))) : 0.f;
            reg[o.dst * 256] = r;
        }
        for (int k = 0; k < prog.n_slots; ++k)
            if (prog.store[k]) *reinterpret_cast<float4 *>(g.field[prog.field[k]] + base) = reg[k * 256];
    }
    if (prog.sum_out >= 0) {
        const double tot = block_sum_f64<256>((double)part, s_red);
        finish_reduction(g, tot, prog.sum_out);
    }
}

template <int L>
static int ew_ctas(int num_sms)
{
    static int per = 0;
    if (!per && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ew<L>, 256, 0) != cudaSuccess || per < 1))
        per = 1;
    return per * num_sms;  // all resident at once (one reduction partial each)
}

void launch_ew(const DevGrid &g, cudaStream_t s, const EwProgram &prog, const LaunchCfg &lc)
{
    if (g.L == 8) k_ew<8><<<ew_ctas<8>(lc.num_sms), 256, 0, s>>>(g, prog);
    else k_ew<4><<<ew_ctas<4>(lc.num_sms), 256, 0, s>>>(g, prog);
}

}  // namespace sg
