// sg_multigrid.cu -- transfers between a grid and its half-edge coarse grid:
// restriction with activation on write, y[i // 2] += w * x[i] over the active
// fine voxels i, and prolongation x[i] += w * y[i // 2] (the multigrid pattern
// AsyncTaichi Sec. 6.3 / Fig. 13 uses to motivate activation demotion).
//
// A fine leaf (edge L, leaf cell b) maps onto one (L/2)^3 sub-block of the
// coarse leaf b >> 1 (per axis), at offset (b & 1) * L/2: the eight children
// of a coarse voxel lie in a single fine leaf, so each coarse voxel is summed
// and written by exactly one lane, without atomics.
#include "sg_common.cuh"

namespace sg {

// Mark the coarse leaves that listed fine leaves with any active voxel map to.
__global__ void k_restrict_mark(DevGrid fine, DevGrid coarse)
{
    const int n = fine.ctrl->list_n;
    const int Rf = fine.R, Rc = coarse.R;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const uint32_t *m = fine.mask + (long long)fine.list_slot[e] * fine.W;
        uint32_t any = 0;
        for (int w = 0; w < fine.W; ++w) any |= m[w];
        if (!any) continue;
        const int b = fine.list_b[e];
        const int bi = b / (Rf * Rf), bj = (b / Rf) % Rf, bk = b % Rf;
        uint8_t *nd = &coarse.need[((long long)(bi >> 1) * Rc + (bj >> 1)) * Rc + (bk >> 1)];
        if (!__ldcg(nd)) *nd = 1;
    }
}

// One group of G = min(32, H^3) lanes per fine list entry, H = L/2; lane t of
// the group owns coarse sub-block voxels t, t + G, ...  ACTIVATE: set the bit
// of every coarse voxel with an active child (the coarse leaf is allocated);
// otherwise (activation demoted) the bits are known to be set.
template <int L, bool ACTIVATE>
__global__ void __launch_bounds__(256) k_restrict(DevGrid fine, DevGrid coarse, int f_src, int f_dst, float w)
{
    constexpr int H = L / 2, NV = H * H * H, G = NV < 32 ? NV : 32, PER = NV / G, LG2 = (L == 8) ? 3 : 2;
    const int n = fine.ctrl->list_n;
    const int Rf = fine.R, Rc = coarse.R;
    const float *x = fine.field[f_src];
    float *y = coarse.field[f_dst];
    const int gid = (blockIdx.x * blockDim.x + threadIdx.x) / G, t = threadIdx.x % G;
    const int groups = gridDim.x * blockDim.x / G;
    bool changed = false;
    for (int e = gid; e < n; e += groups) {
        const int sf = fine.list_slot[e], b = fine.list_b[e];
        const int bi = b / (Rf * Rf), bj = (b / Rf) % Rf, bk = b % Rf;
        const int sc = coarse.root[((long long)(bi >> 1) * Rc + (bj >> 1)) * Rc + (bk >> 1)];
        if (sc < 0) continue;  // no active voxel in this leaf, or the coarse pool is exhausted (latched)
        const uint32_t *mf = fine.mask + (long long)sf * fine.W;
        const float *xl = x + ((long long)sf << (3 * LG2));
        const int oi = (bi & 1) * H, oj = (bj & 1) * H, ok = (bk & 1) * H;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int v = t + u * G;
            const int ci = v / (H * H), cj = (v / H) % H, ck = v % H;
            float s = 0.f;
            bool act = false;
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int row = (2 * ci + a) * L + (2 * cj + c);  // fine row (li, lj)
                    const int l0 = row * L + 2 * ck;                  // children (.., 2ck) and (.., 2ck + 1)
                    const float2 p = __ldg(reinterpret_cast<const float2 *>(xl + l0));
                    s += p.x + p.y;  // a stored value at an inactive voxel is 0
                    act |= ((__ldg(mf + (l0 >> 5)) >> (l0 & 31)) & 3u) != 0u;
                }
            if (!act) continue;
            const int lc = ((oi + ci) * L + (oj + cj)) * L + (ok + ck);
            if (ACTIVATE) {
                uint32_t *mw = coarse.mask + (long long)sc * coarse.W + (lc >> 5);
                const uint32_t bit = 1u << (lc & 31);
                if (!(*(volatile uint32_t *)mw & bit)) changed |= !(atomicOr(mw, bit) & bit);
            }
            float *yp = y + ((long long)sc << (3 * LG2)) + lc;
            *yp = fmaf(w, s, *yp);
        }
    }
    if (ACTIVATE && changed) mark_dirty(coarse);
}

// Prolongation: one thread per voxel of the listed fine leaves.
template <int L>
__global__ void __launch_bounds__(256) k_prolong(DevGrid coarse, DevGrid fine, int f_src, int f_dst, float w)
{
    constexpr int LG2 = (L == 8) ? 3 : 2, V = L * L * L;
    const long long n = fine.ctrl->list_n;
    const int Rf = fine.R, Rc = coarse.R;
    const float *y = coarse.field[f_src];
    float *x = fine.field[f_dst];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * V;
         q += (long long)gridDim.x * blockDim.x) {
        const long long e = q >> (3 * LG2);
        const int l = (int)(q & (V - 1));
        const int sf = fine.list_slot[e];
        if (!((fine.mask[(long long)sf * fine.W + (l >> 5)] >> (l & 31)) & 1u)) continue;
        const int b = fine.list_b[e];
        const int bi = b / (Rf * Rf), bj = (b / Rf) % Rf, bk = b % Rf;
        const int sc = coarse.root[((long long)(bi >> 1) * Rc + (bj >> 1)) * Rc + (bk >> 1)];
        if (sc < 0) continue;  // the coarse voxel reads 0
        const int li = l >> (2 * LG2), lj = (l >> LG2) & (L - 1), lk = l & (L - 1);
        const int ci = ((bi & 1) * L + li) >> 1, cj = ((bj & 1) * L + lj) >> 1, ck = ((bk & 1) * L + lk) >> 1;
        // a stored value at an inactive coarse voxel is 0
        const float yv = y[((long long)sc << (3 * LG2)) + (ci * L + cj) * L + ck];
        float *xp = x + ((long long)sf << (3 * LG2)) + l;
        *xp = fmaf(w, yv, *xp);
    }
}

// Prolongation over 8^3 leaves, a warp per fine leaf: the leaf's slot, cell
// and coarse leaf are looked up once; lane t takes voxels 16t .. 16t + 15 (two
// k-rows, i = t / 4, j = 2t mod 8 and + 1), whose coarse voxels are the four
// consecutive values of one coarse row, read as one float4; the rows of x
// move as float4s.  Each active voxel takes the same fma as in k_prolong.
__global__ void __launch_bounds__(256) k_prolong8(DevGrid coarse, DevGrid fine, int f_src, int f_dst, float w)
{
    const long long n = fine.ctrl->list_n;
    const int Rf = fine.R, Rc = coarse.R;
    const float *__restrict__ y = coarse.field[f_src];
    float *__restrict__ x = fine.field[f_dst];
    const int lane = lane_id();
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long e = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < n; e += warps) {
        const int sf = fine.list_slot[e];
        const int b = fine.list_b[e];
        const int bi = b / (Rf * Rf), bj = (b / Rf) % Rf, bk = b % Rf;
        const int sc = coarse.root[((long long)(bi >> 1) * Rc + (bj >> 1)) * Rc + (bk >> 1)];
        if (sc < 0) continue;  // the coarse voxels read 0 (warp-uniform)
        const uint32_t bits = (fine.mask[(long long)sf * 16 + (lane >> 1)] >> ((lane & 1) * 16)) & 0xffffu;
        if (!bits) continue;
        const int li = lane >> 2, lj = (2 * lane) & 7;
        const int ci = ((bi & 1) * 8 + li) >> 1, cj = ((bj & 1) * 8 + lj) >> 1, ck0 = (bk & 1) * 4;
        const float4 yv = *reinterpret_cast<const float4 *>(y + ((long long)sc << 9) + (ci * 8 + cj) * 8 + ck0);
        const float yk[4] = {yv.x, yv.y, yv.z, yv.w};
        float4 *xp = reinterpret_cast<float4 *>(x + ((long long)sf << 9) + lane * 16);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float4 v = xp[h];
            float *c = reinterpret_cast<float *>(&v);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = 4 * h + u;       // voxel 16 lane + t: k = t mod 8
                if ((bits >> t) & 1u) c[u] = fmaf(w, yk[(t & 7) >> 1], c[u]);
            }
            xp[h] = v;
        }
    }
}

// Restriction from 8^3 leaves, a warp per fine leaf: the fine leaf maps onto a
// 4^3 coarse sub-block, and lane t sums the coarse voxels (ci, cj, 2h) and
// (ci, cj, 2h + 1), ci = t / 8, cj = (t / 2) mod 4, h = t mod 2.  Their
// children are the k-half h of fine rows (2ci + a, 2cj + c), one float4 each;
// both rows of one a share a mask word.  The children are added in the same
// order as in k_restrict, and the two coarse voxels move as one float2.
template <bool ACTIVATE>
__global__ void __launch_bounds__(256) k_restrict8(DevGrid fine, DevGrid coarse, int f_src, int f_dst, float w)
{
    const long long n = fine.ctrl->list_n;
    const int Rf = fine.R, Rc = coarse.R;
    const float *__restrict__ x = fine.field[f_src];
    float *y = coarse.field[f_dst];
    const int lane = lane_id();
    const int ci = lane >> 3, cj = (lane >> 1) & 3, h = lane & 1;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    bool changed = false;
    for (long long e = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < n; e += warps) {
        const int sf = fine.list_slot[e], b = fine.list_b[e];
        const int bi = b / (Rf * Rf), bj = (b / Rf) % Rf, bk = b % Rf;
        const int sc = coarse.root[((long long)(bi >> 1) * Rc + (bj >> 1)) * Rc + (bk >> 1)];
        if (sc < 0) continue;  // no active voxel in this leaf, or the coarse pool is exhausted (latched)
        const uint32_t *mf = fine.mask + (long long)sf * 16;
        const float *xl = x + ((long long)sf << 9);
        float s0 = 0.f, s1 = 0.f;
        uint32_t act = 0;  // bit kk: coarse voxel (ci, cj, 2h + kk) has an active child
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int r0 = (2 * ci + a) * 8 + 2 * cj;  // fine rows r0 and r0 + 1 (c = 0, 1)
            const uint32_t mw = __ldg(mf + (r0 >> 2));
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float4 p = __ldg(reinterpret_cast<const float4 *>(xl + (r0 + c) * 8 + 4 * h));
                s0 += p.x + p.y;  // a stored value at an inactive voxel is 0
                s1 += p.z + p.w;
                const uint32_t nib = (mw >> (((r0 + c) & 3) * 8 + 4 * h)) & 0xfu;
                act |= ((nib & 3u) != 0u) | (((nib >> 2) != 0u) << 1);
            }
        }
        if (!act) continue;
        const int lc = (((bi & 1) * 4 + ci) * 8 + ((bj & 1) * 4 + cj)) * 8 + (bk & 1) * 4 + 2 * h;
        if (ACTIVATE) {
            uint32_t *mw = coarse.mask + (long long)sc * 16 + (lc >> 5);
            const uint32_t bits = act << (lc & 31);
            if ((*(volatile uint32_t *)mw & bits) != bits) changed |= (atomicOr(mw, bits) & bits) != bits;
        }
        float2 *yp = reinterpret_cast<float2 *>(y + ((long long)sc << 9) + lc);
        float2 v = *yp;
        if (act & 1u) v.x = fmaf(w, s0, v.x);
        if (act & 2u) v.y = fmaf(w, s1, v.y);
        *yp = v;
    }
    if (ACTIVATE && changed) mark_dirty(coarse);
}

void launch_restrict_mark(const DevGrid &fine, const DevGrid &coarse, cudaStream_t s, const LaunchCfg &lc)
{
    k_restrict_mark<<<lc.num_sms * 4, 256, 0, s>>>(fine, coarse);
}

void launch_restrict(const DevGrid &fine, const DevGrid &coarse, cudaStream_t s, int f_src, int f_dst, float w,
                     bool activate, const LaunchCfg &lc)
{
    const int ctas = lc.num_sms * 8;
    if (fine.L == 8) {
        if (activate) k_restrict8<true><<<ctas, 256, 0, s>>>(fine, coarse, f_src, f_dst, w);
        else k_restrict8<false><<<ctas, 256, 0, s>>>(fine, coarse, f_src, f_dst, w);
    } else {
        if (activate) k_restrict<4, true><<<ctas, 256, 0, s>>>(fine, coarse, f_src, f_dst, w);
        else k_restrict<4, false><<<ctas, 256, 0, s>>>(fine, coarse, f_src, f_dst, w);
    }
}

void launch_prolong(const DevGrid &coarse, const DevGrid &fine, cudaStream_t s, int f_src, int f_dst, float w,
                    const LaunchCfg &lc)
{
    const int ctas = lc.num_sms * 8;
    if (fine.L == 8) k_prolong8<<<ctas, 256, 0, s>>>(coarse, fine, f_src, f_dst, w);
    else k_prolong<4><<<ctas, 256, 0, s>>>(coarse, fine, f_src, f_dst, w);
}

}  // namespace sg
