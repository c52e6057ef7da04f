// sg_stencil.cu -- struct-for kernels over the active-leaf list: clear,
// 7-point diffusion, 27-point box smoothing, their fusion, and the sum.
//
// Semantics (AsyncTaichi Sec. 3.2, Sec. 4 "States", Fig. 5 caption): every
// operation runs over the active voxels; a read of an inactive or
// out-of-domain voxel gives 0.  The inter-kernel passes of Sec. 6 decide which
// of these kernels is launched:
//   - CHECK (activation demotion off): every store first checks, in the mask
//     in global memory, that the written voxel is active, activating it if not
//     (Sec. 3.2 item 3); demoted kernels store without the check (Sec. 6.3);
//   - k_diffuse_box is the fused task of diffuse7 -> box27 (+ sum): the
//     intermediate field is recomputed on the halo instead of exchanged, and
//     is not stored unless asked (dead-store elimination, Sec. 6.5).
//
// 8^3 leaves are staged in shared memory with their halo, one k-row (8
// floats, 32 B) per load task, through the 27-neighbour table built with the
// list.  A stored value at an inactive voxel is 0 (the grid invariant), so
// staged loads need no mask; outputs are masked before they are stored, which
// keeps the invariant.  Other leaf sizes use the generic kernels at the end,
// which walk the tree for every read.
#include <atomic>
#include "sg_common.cuh"

namespace sg {

constexpr int kStageThreads = 128;
constexpr int kRow = 20;  // floats per staged row: 16-B aligned, conflict-free float4 reads

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float2 ldg2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float2 lds2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void sts4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void sts2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

__device__ __forceinline__ float sel(uint32_t bits, int k, float v) { return ((bits >> k) & 1u) ? v : 0.f; }

// Eager activation-on-write check of one 8-voxel row of the own leaf before
// it is stored: the written voxels (`bits`) must be active in the mask in
// global memory; any that is not is activated.
__device__ __forceinline__ void check_activation_row(const DevGrid &g, int slot, int row, uint32_t bits)
{
    uint32_t *w = &g.mask[(long long)slot * 16 + (row >> 2)];
    const uint32_t want = bits << ((row & 3) * 8);
    const uint32_t have = *(volatile uint32_t *)w;
    if ((have & want) != want) {
        atomicOr(w, want);
        mark_dirty(g);
    }
}

// ---------------------------------------------------------------------------
// Clear and sum: whole-leaf streams.
// ---------------------------------------------------------------------------
template <bool CHECK>
__global__ void __launch_bounds__(kStageThreads) k_clear(DevGrid g, int dst)
{
    const int n = g.ctrl->list_n;
    float *out = g.field[dst];
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const int slot = g.list_slot[e];
        if (CHECK && threadIdx.x < 64) {
            const uint32_t bits = (g.mask[(long long)slot * 16 + (threadIdx.x >> 2)] >> ((threadIdx.x & 3) * 8)) & 0xffu;
            check_activation_row(g, slot, threadIdx.x, bits);
        }
        sts4(out + (long long)slot * 512 + threadIdx.x * 4, make_float4(0.f, 0.f, 0.f, 0.f));
    }
}

__global__ void __launch_bounds__(kStageThreads) k_sum(DevGrid g, int src, int slot_out)
{
    __shared__ double s_red[kStageThreads / 32];
    const int n = g.ctrl->list_n;
    const int V4 = (g.L * g.L * g.L) >> 2;
    const float *x = g.field[src];
    double acc = 0.0;
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const long long base = (long long)g.list_slot[e] * V4 * 4;
        float part = 0.f;
        for (int q = threadIdx.x; q < V4; q += kStageThreads) {
            const float4 v = ldg4(x + base + q * 4);
            part += (v.x + v.y) + (v.z + v.w);
        }
        acc += (double)part;
    }
    const double tot = block_sum_f64<kStageThreads>(acc, s_red);
    finish_reduction(g, tot, slot_out);
}

// ---------------------------------------------------------------------------
// Single stencil over 8^3 leaves with a 1-voxel halo (10^3 staged region).
// Staged row (ri, rj), ri, rj in [0,10), region k r in [0,10) at float r + 3:
// the own leaf's 8 floats land 16-B aligned at floats 4..11.
// ---------------------------------------------------------------------------
enum { OP_DIFFUSE7 = 1, OP_BOX27 = 2 };

template <int OP, bool CHECK, bool SUM>
__global__ void __launch_bounds__(kStageThreads) k_stage1(DevGrid g, int src, int dst, float coef, int sum_slot)
{
    __shared__ __align__(16) float xs[100 * kRow];
    __shared__ int s_nb[27];
    __shared__ uint8_t s_mb[64];
    __shared__ double s_red[kStageThreads / 32];
    const int n = g.ctrl->list_n;
    const float *__restrict__ x = g.field[src];
    float *__restrict__ y = g.field[dst];
    const uint8_t *maskb = reinterpret_cast<const uint8_t *>(g.mask);
    const int tid = threadIdx.x;
    double acc = 0.0;
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        if (tid < 27) s_nb[tid] = g.nbr[(long long)e * 27 + tid];
        const int slot = g.list_slot[e];
        if (tid < 64) s_mb[tid] = maskb[(long long)slot * 64 + tid];
        __syncthreads();
        if (tid < 100) {
            const int ri = tid / 10, rj = tid - ri * 10;
            const int di = (ri == 0) ? 0 : (ri == 9 ? 2 : 1), li = (ri - 1) & 7;
            const int dj = (rj == 0) ? 0 : (rj == 9 ? 2 : 1), lj = (rj - 1) & 7;
            const int q = di * 9 + dj * 3;
            const int s0 = s_nb[q], s1 = s_nb[q + 1], s2 = s_nb[q + 2];
            const int ro = (li * 8 + lj) * 8;
            float a = 0.f, b = 0.f;
            float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0;
            if (s0 >= 0) a = __ldg(x + (long long)s0 * 512 + ro + 7);
            if (s1 >= 0) {
                c0 = ldg4(x + (long long)s1 * 512 + ro);
                c1 = ldg4(x + (long long)s1 * 512 + ro + 4);
            }
            if (s2 >= 0) b = __ldg(x + (long long)s2 * 512 + ro);
            float *row = xs + tid * kRow;
            row[3] = a;
            sts4(row + 4, c0);
            sts4(row + 8, c1);
            row[12] = b;
        }
        __syncthreads();
        if (tid < 64) {
            const int i = tid >> 3, j = tid & 7;
            const uint32_t bits = s_mb[tid];
            float o[8];
            if (OP == OP_DIFFUSE7) {
                const float *c = xs + ((i + 1) * 10 + (j + 1)) * kRow;
                const float *im = c - 10 * kRow, *ip = c + 10 * kRow, *jm = c - kRow, *jp = c + kRow;
                float cv[10];
                cv[0] = c[3];
                const float4 c0 = lds4(c + 4), c1 = lds4(c + 8);
                cv[1] = c0.x; cv[2] = c0.y; cv[3] = c0.z; cv[4] = c0.w;
                cv[5] = c1.x; cv[6] = c1.y; cv[7] = c1.z; cv[8] = c1.w;
                cv[9] = c[12];
                float nb[8];
                {
                    const float4 a0 = lds4(im + 4), a1 = lds4(im + 8), b0 = lds4(ip + 4), b1 = lds4(ip + 8);
                    const float4 d0 = lds4(jm + 4), d1 = lds4(jm + 8), e0 = lds4(jp + 4), e1 = lds4(jp + 8);
                    nb[0] = (a0.x + b0.x) + (d0.x + e0.x);
                    nb[1] = (a0.y + b0.y) + (d0.y + e0.y);
                    nb[2] = (a0.z + b0.z) + (d0.z + e0.z);
                    nb[3] = (a0.w + b0.w) + (d0.w + e0.w);
                    nb[4] = (a1.x + b1.x) + (d1.x + e1.x);
                    nb[5] = (a1.y + b1.y) + (d1.y + e1.y);
                    nb[6] = (a1.z + b1.z) + (d1.z + e1.z);
                    nb[7] = (a1.w + b1.w) + (d1.w + e1.w);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float xc = cv[k + 1];
                    const float lap = (cv[k] + cv[k + 2]) + nb[k] - 6.f * xc;
                    o[k] = sel(bits, k, xc + coef * lap);
                }
            } else {
                float col[10];
#pragma unroll
                for (int q = 0; q < 10; ++q) col[q] = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const float *r = xs + ((i + a) * 10 + (j + b)) * kRow;
                        const float4 r0 = lds4(r + 4), r1 = lds4(r + 8);
                        col[0] += r[3];
                        col[1] += r0.x; col[2] += r0.y; col[3] += r0.z; col[4] += r0.w;
                        col[5] += r1.x; col[6] += r1.y; col[7] += r1.z; col[8] += r1.w;
                        col[9] += r[12];
                    }
#pragma unroll
                for (int k = 0; k < 8; ++k) o[k] = sel(bits, k, ((col[k] + col[k + 1]) + col[k + 2]) * (1.f / 27.f));
            }
            if (CHECK) check_activation_row(g, slot, tid, bits);
            float *out = y + (long long)slot * 512 + tid * 8;
            sts4(out, make_float4(o[0], o[1], o[2], o[3]));
            sts4(out + 4, make_float4(o[4], o[5], o[6], o[7]));
            if (SUM) acc += (double)(((o[0] + o[1]) + (o[2] + o[3])) + ((o[4] + o[5]) + (o[6] + o[7])));
        }
        __syncthreads();
    }
    if (SUM) {
        const double tot = block_sum_f64<kStageThreads>(acc, s_red);
        finish_reduction(g, tot, sum_slot);
    }
}

// ---------------------------------------------------------------------------
// Fused diffuse7 -> box27 (+ sum) over 8^3 leaves with a 2-voxel halo.
// Stage x on the 12^3 region (row (ri, rj) in [0,12)^2, region k r at float
// r + 2, so the own 8 floats land at floats 4..11) and the mask bits of the
// region rows; recompute t on the 10^3 region around the leaf (t = 0 where
// the voxel is inactive, as its definition requires); box-average t onto the
// leaf.  t lives only in shared memory unless store_t.
// ---------------------------------------------------------------------------
template <bool STORE_T, bool CHECK, bool SUM>
__global__ void __launch_bounds__(kStageThreads) k_diffuse_box(DevGrid g, int src, int tmp, int dst, float coef,
                                                                  int sum_slot)
{
    __shared__ __align__(16) float xs[144 * kRow];
    __shared__ __align__(16) float ts[100 * 12];
    __shared__ uint16_t s_mrow[144];
    __shared__ int s_nb[27];
    __shared__ double s_red[kStageThreads / 32];
    const int n = g.ctrl->list_n;
    const float *__restrict__ x = g.field[src];
    float *__restrict__ y = g.field[dst];
    float *__restrict__ tout = g.field[tmp];
    const uint8_t *maskb = reinterpret_cast<const uint8_t *>(g.mask);
    const int tid = threadIdx.x;
    double acc = 0.0;
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        if (tid < 27) s_nb[tid] = g.nbr[(long long)e * 27 + tid];
        __syncthreads();
        const int slot = s_nb[13];
        for (int t = tid; t < 144; t += kStageThreads) {
            const int ri = t / 12, rj = t - ri * 12;
            const int di = (ri < 2) ? 0 : (ri < 10 ? 1 : 2), li = (ri - 2) & 7;
            const int dj = (rj < 2) ? 0 : (rj < 10 ? 1 : 2), lj = (rj - 2) & 7;
            const int q = di * 9 + dj * 3;
            const int s0 = s_nb[q], s1 = s_nb[q + 1], s2 = s_nb[q + 2];
            const int rowi = li * 8 + lj;
            const int ro = rowi * 8;
            float2 a = make_float2(0.f, 0.f), b = a;
            float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0;
            uint32_t m0 = 0, m1 = 0, m2 = 0;
            if (s0 >= 0) {
                a = ldg2(x + (long long)s0 * 512 + ro + 6);
                m0 = maskb[(long long)s0 * 64 + rowi];
            }
            if (s1 >= 0) {
                c0 = ldg4(x + (long long)s1 * 512 + ro);
                c1 = ldg4(x + (long long)s1 * 512 + ro + 4);
                m1 = maskb[(long long)s1 * 64 + rowi];
            }
            if (s2 >= 0) {
                b = ldg2(x + (long long)s2 * 512 + ro);
                m2 = maskb[(long long)s2 * 64 + rowi];
            }
            float *row = xs + t * kRow;
            sts2(row + 2, a);
            sts4(row + 4, c0);
            sts4(row + 8, c1);
            sts2(row + 12, b);
            s_mrow[t] = (uint16_t)((m0 >> 6) | (m1 << 2) | ((m2 & 3u) << 10));
        }
        __syncthreads();
        // t on the 10^3 region: rows (ri, rj) in [1,11)^2, k r in [1,11)
        if (tid < 100) {
            const int ri = 1 + tid / 10, rj = 1 + tid % 10;
            const float *c = xs + (ri * 12 + rj) * kRow;
            const float *im = c - 12 * kRow, *ip = c + 12 * kRow, *jm = c - kRow, *jp = c + kRow;
            float cv[12];
            {
                const float2 c_lo = lds2(c + 2), c_hi = lds2(c + 12);
                const float4 c0 = lds4(c + 4), c1 = lds4(c + 8);
                cv[0] = c_lo.x; cv[1] = c_lo.y;
                cv[2] = c0.x; cv[3] = c0.y; cv[4] = c0.z; cv[5] = c0.w;
                cv[6] = c1.x; cv[7] = c1.y; cv[8] = c1.z; cv[9] = c1.w;
                cv[10] = c_hi.x; cv[11] = c_hi.y;
            }
            float nb[10];
            {
                const float4 a0 = lds4(im + 4), a1 = lds4(im + 8), b0 = lds4(ip + 4), b1 = lds4(ip + 8);
                const float4 d0 = lds4(jm + 4), d1 = lds4(jm + 8), e0 = lds4(jp + 4), e1 = lds4(jp + 8);
                nb[0] = (im[3] + ip[3]) + (jm[3] + jp[3]);
                nb[1] = (a0.x + b0.x) + (d0.x + e0.x);
                nb[2] = (a0.y + b0.y) + (d0.y + e0.y);
                nb[3] = (a0.z + b0.z) + (d0.z + e0.z);
                nb[4] = (a0.w + b0.w) + (d0.w + e0.w);
                nb[5] = (a1.x + b1.x) + (d1.x + e1.x);
                nb[6] = (a1.y + b1.y) + (d1.y + e1.y);
                nb[7] = (a1.z + b1.z) + (d1.z + e1.z);
                nb[8] = (a1.w + b1.w) + (d1.w + e1.w);
                nb[9] = (im[12] + ip[12]) + (jm[12] + jp[12]);
            }
            const uint32_t mb = s_mrow[ri * 12 + rj];
            float tv[10];
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                const float xc = cv[q + 1];
                const float lap = (cv[q] + cv[q + 2]) + nb[q] - 6.f * xc;
                tv[q] = sel(mb, q + 1, xc + coef * lap);
            }
            float *trow = ts + tid * 12;
            sts4(trow, make_float4(tv[0], tv[1], tv[2], tv[3]));
            sts4(trow + 4, make_float4(tv[4], tv[5], tv[6], tv[7]));
            sts2(trow + 8, make_float2(tv[8], tv[9]));
            if (STORE_T && ri >= 2 && ri < 10 && rj >= 2 && rj < 10) {
                const int orow = (ri - 2) * 8 + (rj - 2);
                if (CHECK) check_activation_row(g, slot, orow, (mb >> 2) & 0xffu);
                float *o = tout + (long long)slot * 512 + orow * 8;
                sts4(o, make_float4(tv[1], tv[2], tv[3], tv[4]));
                sts4(o + 4, make_float4(tv[5], tv[6], tv[7], tv[8]));
            }
        }
        __syncthreads();
        if (tid < 64) {
            const int i = tid >> 3, j = tid & 7;
            float col[10];
#pragma unroll
            for (int q = 0; q < 10; ++q) col[q] = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float *r = ts + ((i + a) * 10 + (j + b)) * 12;
                    const float4 r0 = lds4(r), r1 = lds4(r + 4);
                    const float2 r2 = lds2(r + 8);
                    col[0] += r0.x; col[1] += r0.y; col[2] += r0.z; col[3] += r0.w;
                    col[4] += r1.x; col[5] += r1.y; col[6] += r1.z; col[7] += r1.w;
                    col[8] += r2.x; col[9] += r2.y;
                }
            const uint32_t bits = (s_mrow[(i + 2) * 12 + (j + 2)] >> 2) & 0xffu;
            float o[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) o[k] = sel(bits, k, ((col[k] + col[k + 1]) + col[k + 2]) * (1.f / 27.f));
            if (CHECK) check_activation_row(g, slot, tid, bits);
            float *out = y + (long long)slot * 512 + tid * 8;
            sts4(out, make_float4(o[0], o[1], o[2], o[3]));
            sts4(out + 4, make_float4(o[4], o[5], o[6], o[7]));
            if (SUM) acc += (double)(((o[0] + o[1]) + (o[2] + o[3])) + ((o[4] + o[5]) + (o[6] + o[7])));
        }
        __syncthreads();
    }
    if (SUM) {
        const double tot = block_sum_f64<kStageThreads>(acc, s_red);
        finish_reduction(g, tot, sum_slot);
    }
}

// ---------------------------------------------------------------------------
// Generic kernels for any leaf size: one thread per voxel of a listed leaf,
// every read walks root -> mask -> value (Fig. 5 caption).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tree_read(const DevGrid &g, const float *x, int i, int j, int k)
{
    if ((unsigned)i >= (unsigned)g.N || (unsigned)j >= (unsigned)g.N || (unsigned)k >= (unsigned)g.N) return 0.f;
    const int lg2 = g.lg2, L = g.L;
    const long long b = ((long long)(i >> lg2) * g.R + (j >> lg2)) * g.R + (k >> lg2);
    const int slot = g.root[b];
    if (slot < 0) return 0.f;
    const int l = (((i & (L - 1)) << lg2) + (j & (L - 1))) * L + (k & (L - 1));
    if (!((g.mask[(long long)slot * g.W + (l >> 5)] >> (l & 31)) & 1u)) return 0.f;
    return x[((long long)slot << (3 * lg2)) + l];
}

template <int OP, bool CHECK, bool SUM>
__global__ void __launch_bounds__(256) k_generic(DevGrid g, int src, int dst, float coef, int sum_slot)
{
    __shared__ double s_red[8];
    const int n = g.ctrl->list_n;
    const int L = g.L, lg2 = g.lg2, V = L * L * L, R = g.R;
    const float *x = g.field[src];
    float *y = g.field[dst];
    double acc = 0.0;
    for (int e = blockIdx.x; e < n; e += gridDim.x) {
        const int slot = g.list_slot[e], b = g.list_b[e];
        const int bi = b / (R * R), bj = (b / R) % R, bk = b % R;
        float part = 0.f;
        for (int l = threadIdx.x; l < V; l += 256) {
            uint32_t *mw = &g.mask[(long long)slot * g.W + (l >> 5)];
            if (!((*mw >> (l & 31)) & 1u)) continue;
            const int i = bi * L + (l >> (2 * lg2)), j = bj * L + ((l >> lg2) & (L - 1)), k = bk * L + (l & (L - 1));
            float v;
            if (OP == 0) {
                v = 0.f;
            } else if (OP == OP_DIFFUSE7) {
                const float c = tree_read(g, x, i, j, k);
                const float nb = (tree_read(g, x, i - 1, j, k) + tree_read(g, x, i + 1, j, k)) +
                                 (tree_read(g, x, i, j - 1, k) + tree_read(g, x, i, j + 1, k)) +
                                 (tree_read(g, x, i, j, k - 1) + tree_read(g, x, i, j, k + 1));
                v = c + coef * (nb - 6.f * c);
            } else {
                float s = 0.f;
                for (int di = -1; di <= 1; ++di)
                    for (int dj = -1; dj <= 1; ++dj)
                        for (int dk = -1; dk <= 1; ++dk) s += tree_read(g, x, i + di, j + dj, k + dk);
                v = s * (1.f / 27.f);
            }
            if (CHECK) {
                const uint32_t bit = 1u << (l & 31);
                if (!(*(volatile uint32_t *)mw & bit)) {
                    atomicOr(mw, bit);
                    mark_dirty(g);
                }
            }
            y[((long long)slot << (3 * lg2)) + l] = v;
            part += v;
        }
        acc += (double)part;
    }
    if (SUM) {
        const double tot = block_sum_f64<256>(acc, s_red);
        finish_reduction(g, tot, sum_slot);
    }
}

// ---------------------------------------------------------------------------
// Launch wrappers.  Persistent grids: CTAs resident on every SM, each walking
// the list with stride gridDim.x; the list length is read on the device.
// ---------------------------------------------------------------------------
int stencil_persistent_ctas(int num_sms, int which)
{
    static std::atomic<int> cache[8];  // threads may race to fill it
    if (cache[which].load(std::memory_order_relaxed) == 0) {
        int per = 1;
        cudaError_t err = cudaSuccess;
        switch (which) {
            case 0: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_stage1<OP_DIFFUSE7, false, false>, kStageThreads, 0); break;
            case 1: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_diffuse_box<false, false, true>, kStageThreads, 0); break;
            case 2: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sum, kStageThreads, 0); break;
            default: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_generic<OP_DIFFUSE7, false, true>, 256, 0); break;
        }
        if (err != cudaSuccess || per < 1) per = 1;
        if (per > 16) per = 16;
        cache[which].store(per, std::memory_order_relaxed);
    }
    return cache[which].load(std::memory_order_relaxed) * num_sms;
}

void launch_clear(const DevGrid &g, cudaStream_t s, int dst, int check_act, const LaunchCfg &lc)
{
    const int ctas = stencil_persistent_ctas(lc.num_sms, 2);
    if (g.L == 8) {
        if (check_act) k_clear<true><<<ctas, kStageThreads, 0, s>>>(g, dst);
        else k_clear<false><<<ctas, kStageThreads, 0, s>>>(g, dst);
    } else {
        if (check_act) k_generic<0, true, false><<<ctas, 256, 0, s>>>(g, dst, dst, 0.f, 0);
        else k_generic<0, false, false><<<ctas, 256, 0, s>>>(g, dst, dst, 0.f, 0);
    }
}

template <int OP>
static void launch_single(const DevGrid &g, cudaStream_t s, int src, int dst, float coef, int check_act,
                          int sum_slot, const LaunchCfg &lc)
{
    const bool sum = sum_slot >= 0;
    if (g.L == 8 && lc.variant != kVariantSmem) {
        launch_sweep_single(g, s, OP, src, dst, coef, check_act, sum_slot, lc);
    } else if (g.L == 8) {
        const int ctas = stencil_persistent_ctas(lc.num_sms, 0);
        if (check_act) {
            if (sum) k_stage1<OP, true, true><<<ctas, kStageThreads, 0, s>>>(g, src, dst, coef, sum_slot);
            else k_stage1<OP, true, false><<<ctas, kStageThreads, 0, s>>>(g, src, dst, coef, sum_slot);
        } else {
            if (sum) k_stage1<OP, false, true><<<ctas, kStageThreads, 0, s>>>(g, src, dst, coef, sum_slot);
            else k_stage1<OP, false, false><<<ctas, kStageThreads, 0, s>>>(g, src, dst, coef, sum_slot);
        }
    } else {
        const int ctas = stencil_persistent_ctas(lc.num_sms, 3);
        if (check_act) {
            if (sum) k_generic<OP, true, true><<<ctas, 256, 0, s>>>(g, src, dst, coef, sum_slot);
            else k_generic<OP, true, false><<<ctas, 256, 0, s>>>(g, src, dst, coef, sum_slot);
        } else {
            if (sum) k_generic<OP, false, true><<<ctas, 256, 0, s>>>(g, src, dst, coef, sum_slot);
            else k_generic<OP, false, false><<<ctas, 256, 0, s>>>(g, src, dst, coef, sum_slot);
        }
    }
}

void launch_diffuse7(const DevGrid &g, cudaStream_t s, int src, int dst, float coef, int check_act, int sum_slot,
                     const LaunchCfg &lc)
{
    launch_single<OP_DIFFUSE7>(g, s, src, dst, coef, check_act, sum_slot, lc);
}

void launch_box27(const DevGrid &g, cudaStream_t s, int src, int dst, int check_act, int sum_slot,
                  const LaunchCfg &lc)
{
    launch_single<OP_BOX27>(g, s, src, dst, 0.f, check_act, sum_slot, lc);
}

void launch_diffuse_box(const DevGrid &g, cudaStream_t s, int src, int tmp, int dst, float coef, int store_tmp,
                        int check_act, int sum_slot, const LaunchCfg &lc)
{
    if (lc.variant == kVariantSweep) {
        launch_sweep_diffuse_box(g, s, src, tmp, dst, coef, store_tmp, check_act, sum_slot, lc);
        return;
    }
    if (lc.variant == kVariantSweepColumns) {
        launch_sweep_columns(g, s, src, tmp, dst, coef, store_tmp, check_act, sum_slot, lc);
        return;
    }
    if (lc.variant == kVariantSweepJRuns || lc.variant == kVariantSweepTma) {
        launch_sweep_jruns(g, s, src, tmp, dst, coef, store_tmp, check_act, sum_slot, lc);
        return;
    }
    const int ctas = stencil_persistent_ctas(lc.num_sms, 1);
    const bool sum = sum_slot >= 0;
#define SG_DB(ST, CK, SU) k_diffuse_box<ST, CK, SU><<<ctas, kStageThreads, 0, s>>>(g, src, tmp, dst, coef, sum_slot)
    if (store_tmp) {
        if (check_act) { if (sum) SG_DB(true, true, true); else SG_DB(true, true, false); }
        else { if (sum) SG_DB(true, false, true); else SG_DB(true, false, false); }
    } else {
        if (check_act) { if (sum) SG_DB(false, true, true); else SG_DB(false, true, false); }
        else { if (sum) SG_DB(false, false, true); else SG_DB(false, false, false); }
    }
#undef SG_DB
}

void launch_sum(const DevGrid &g, cudaStream_t s, int src, int sum_slot, const LaunchCfg &lc)
{
    const int ctas = stencil_persistent_ctas(lc.num_sms, 2);
    k_sum<<<ctas, kStageThreads, 0, s>>>(g, src, sum_slot);
}

}  // namespace sg
