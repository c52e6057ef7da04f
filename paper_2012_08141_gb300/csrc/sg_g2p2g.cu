// sg_g2p2g.cu -- fused G2P2G (AsyncTaichi Sec. 8.3: the G2P of one step and
// the P2G of the next fused into one pass over the particles, with the affine
// matrix C of the MLS-MPM transfers eliminated as a dead store).
//
// One launch computes, for every particle p, exactly what
//   APIC G2P from grid `src`   (v_p, C_p, x_p += dt v_p)
//   APIC P2G into grid `dst`   (activation of the 27 stencil nodes of the new
//                               position, mass and affine momentum)
// compute one after the other, but C_p lives only in registers and shared
// memory: it is never written to or read from HBM.  x_p and v_p are written
// back (they are the particle state); the update is in place, each particle
// being visited once.
//
// Work split: one CTA per bin of the last binned P2G over these particles
// (a leaf o with the particles whose base node was in it when binned).
//   1. stage src's velocities of nodes o-2 .. o+L+1 in shared memory;
//   2. per particle: G2P from the staged block (or node by node from the grid
//      when its base has left [o-2, o+L-1]), store x', v'; a particle of the
//      bin that moved less than a cell has its new base in [o-1, o+L] (bases
//      o-2 and o-1 of the low domain face excepted); count it in its new base
//      cell and keep its P2G record (spline offsets, m, q = m v - m dx C fx
//      and m dx C) in registers;
//   3. counting sort by new base cell, records staged in shared memory;
//   4. one warp per occupied cell: lane t < 27 sums its node's contributions
//      (as in the binned P2G gather) into shared accumulators of the dst
//      nodes o-1 .. o+L+2;
//   5. flush the touched nodes: the dst leaves they fall in are allocated
//      in-kernel if null (see ensure_leaf), bits set, 4 FP32 atomics per node.
// A particle whose new base is outside [o-1, o+L], and every particle of the
// out-of-domain key, is scattered node by node straight into dst with the same
// in-kernel allocation.
#include <atomic>
#include "sg_particle.cuh"

namespace sg {

namespace {

constexpr int kRootPending = -2;  // a CTA is allocating this leaf
constexpr int kRootFailed = -3;   // allocation failed (pool exhausted)

// Self-checks of the kernel's own accesses: every vector access below first
// verifies the alignment of its address (and the shared-record loop its
// range); a failed check skips the access, latches kErrCheck on dst and
// records which check failed.  They cost a few integer operations per access.
__device__ __forceinline__ bool misaligned(const DevGrid &g, const void *p, unsigned align, int site)
{
    if (((uintptr_t)p & (uintptr_t)(align - 1)) == 0) return false;
    atomicOr(&g.ctrl->err, kErrCheck);
    g.ctrl->timeout_site = 100 + site;
    return true;
}

__device__ __forceinline__ float3 load3_checked(const DevGrid &g, const float *a, long long p, bool pair)
{
    const float *q = a + 3 * p;
    if (!pair || misaligned(g, q + (p & 1), 8, 1)) return make_float3(q[0], q[1], q[2]);
    if (p & 1) {
        const float2 hi = *reinterpret_cast<const float2 *>(q + 1);
        return make_float3(q[0], hi.x, hi.y);
    }
    const float2 lo = *reinterpret_cast<const float2 *>(q);
    return make_float3(lo.x, lo.y, q[2]);
}

__device__ __forceinline__ void store3_checked(const DevGrid &g, float *a, long long p, float3 t, bool pair)
{
    float *q = a + 3 * p;
    if (!pair || misaligned(g, q + (p & 1), 8, 2)) {
        q[0] = t.x;
        q[1] = t.y;
        q[2] = t.z;
    } else if (p & 1) {
        q[0] = t.x;
        *reinterpret_cast<float2 *>(q + 1) = make_float2(t.y, t.z);
    } else {
        *reinterpret_cast<float2 *>(q) = make_float2(t.x, t.y);
        q[2] = t.z;
    }
}

// Slot of leaf cell lb of g, allocating and zero-filling it if null.  The
// first thread to swap -1 for kRootPending takes a pool slot, zeroes its
// fields and mask, and publishes the slot; others wait for the publication
// (the allocating thread runs and waits on nothing, so the wait ends; it is
// bounded all the same and records kErrTimeout if it gives up).  Returns -1
// when the pool is exhausted (kErrPool latched).  *fresh is set when this
// thread allocated the leaf.
__device__ __forceinline__ int ensure_leaf(const DevGrid &g, long long lb, bool &fresh)
{
    volatile int32_t *r = g.root + lb;
    int s = *r;
    if (s >= 0) return s;
    if (s == -1 && atomicCAS(g.root + lb, -1, kRootPending) == -1) {
        const int slot = atomicAdd(&g.ctrl->pool_count, 1);
        if (slot >= g.cap) {
            raise_error(g, kErrPool);
            __threadfence();
            atomicExch(g.root + lb, kRootFailed);
            return -1;
        }
        const int V = g.L * g.L * g.L;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int f = 0; f < g.F; ++f) {
            float4 *p = reinterpret_cast<float4 *>(g.field[f] + (long long)slot * V);
            if (misaligned(g, p, 16, 3)) {
                for (int q = 0; q < V; ++q) g.field[f][(long long)slot * V + q] = 0.f;
                continue;
            }
            for (int q = 0; q < V / 4; ++q) p[q] = z;
        }
        for (int w = 0; w < g.W; ++w) g.mask[(long long)slot * g.W + w] = 0u;
        __threadfence();
        atomicExch(g.root + lb, slot);
        fresh = true;
        return slot;
    }
    const unsigned long long t0 = global_timer_ns();
    while ((s = *r) == kRootPending) {
        if (global_timer_ns() - t0 > 1000000000ull) {
            raise_error(g, kErrTimeout);
            g.ctrl->timeout_site = 3;
            return -1;
        }
        __nanosleep(100);
    }
    __threadfence();
    return s >= 0 ? s : -1;
}

// Activate node (i, j, k) of g and add (m, p0, p1, p2) to it; the node is in
// the domain.  Returns whether the structure changed.
__device__ __forceinline__ bool scatter_node(const DevGrid &g, int i, int j, int k, float m, float p0, float p1,
                                             float p2, int f_mass, int f_mom0)
{
    const int L = g.L, lg2 = g.lg2;
    bool fresh = false;
    const int slot = ensure_leaf(g, ((long long)(i >> lg2) * g.R + (j >> lg2)) * g.R + (k >> lg2), fresh);
    if (slot < 0) return fresh;
    const int l = (((i & (L - 1)) << lg2) + (j & (L - 1))) * L + (k & (L - 1));
    uint32_t *mw = &g.mask[(long long)slot * g.W + (l >> 5)];
    const uint32_t bit = 1u << (l & 31);
    bool changed = fresh;
    if (!(*(volatile uint32_t *)mw & bit)) changed |= !(atomicOr(mw, bit) & bit);
    const long long idx = ((long long)slot << (3 * lg2)) + l;
    atomicAdd(g.field[f_mass] + idx, m);
    atomicAdd(g.field[f_mom0] + idx, p0);
    atomicAdd(g.field[f_mom0 + 1] + idx, p1);
    atomicAdd(g.field[f_mom0 + 2] + idx, p2);
    return changed;
}

// P2G record of one particle: spline offsets and mass, q = m v - m dx C fx,
// and the 9 entries of m dx C (row-major).
struct P2GRec {
    float4 r0, r1, r2, r3;
};

__device__ __forceinline__ P2GRec make_rec(float fx, float fy, float fz, float pmass, float3 u, const float (&c)[9],
                                           float dx)
{
    float m[9];
    const float md = pmass * dx;
#pragma unroll
    for (int e = 0; e < 9; ++e) m[e] = md * c[e];
    const float q0 = pmass * u.x - (m[0] * fx + m[1] * fy + m[2] * fz);
    const float q1 = pmass * u.y - (m[3] * fx + m[4] * fy + m[5] * fz);
    const float q2 = pmass * u.z - (m[6] * fx + m[7] * fy + m[8] * fz);
    P2GRec r;
    r.r0 = make_float4(fx, fy, fz, pmass);
    r.r1 = make_float4(q0, q1, q2, m[0]);
    r.r2 = make_float4(m[1], m[2], m[3], m[4]);
    r.r3 = make_float4(m[5], m[6], m[7], m[8]);
    return r;
}

// Node-by-node APIC P2G of one particle into g (slow path).
__device__ __forceinline__ bool scatter_particle(const DevGrid &g, Spline sx, Spline sy, Spline sz, P2GRec r,
                                                 int f_mass, int f_mom0)
{
    bool changed = false;
    const int N = g.N;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = sx.base + a;
        if ((unsigned)i >= (unsigned)N) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int j = sy.base + b;
            if ((unsigned)j >= (unsigned)N) continue;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int k = sz.base + c;
                if ((unsigned)k >= (unsigned)N) continue;
                const float w = sx.w[a] * sy.w[b] * sz.w[c];
                const float ta = (float)a, tb = (float)b, tc = (float)c;
                const float u0 = fmaf(r.r1.w, ta, fmaf(r.r2.x, tb, fmaf(r.r2.y, tc, r.r1.x)));
                const float u1 = fmaf(r.r2.z, ta, fmaf(r.r2.w, tb, fmaf(r.r3.x, tc, r.r1.y)));
                const float u2 = fmaf(r.r3.y, ta, fmaf(r.r3.z, tb, fmaf(r.r3.w, tc, r.r1.z)));
                changed |= scatter_node(g, i, j, k, w * r.r0.w, w * u0, w * u1, w * u2, f_mass, f_mom0);
            }
        }
    }
    return changed;
}

// Shared-memory layout of one CTA (dynamic shared memory).
template <int L>
struct G2P2GSmem {
    static constexpr int BU = L + 4;          // staged src nodes per axis (o-2 .. o+L+1)
    static constexpr int NU = BU * BU * BU;
    static constexpr int BD = L + 4;          // dst block nodes per axis (o-1 .. o+L+2)
    static constexpr int ND = BD * BD * BD;
    static constexpr int C1 = L + 2;          // new base cells per axis (o-1 .. o+L)
    static constexpr int NC = C1 * C1 * C1;
    static constexpr int CAP = 256;           // particles per chunk (one per thread)
    static constexpr size_t off_rec = 0;                                   // float4 [4][CAP]
    static constexpr size_t off_u = off_rec + sizeof(float4) * 4 * CAP;    // float4 [NU]
    static constexpr size_t off_acc = off_u + sizeof(float4) * NU;         // float [4][ND]
    static constexpr size_t off_cnt = off_acc + sizeof(float) * 4 * ND;    // int [NC + 1]
    static constexpr size_t off_start = off_cnt + sizeof(int) * (NC + 1);  // int [NC + 1]
    static constexpr size_t off_slot = off_start + sizeof(int) * (NC + 1); // int [27]
    static constexpr size_t off_hit = off_slot + sizeof(int) * 27;         // uint8 [ND]
    static constexpr size_t bytes = (off_hit + ND + 15) / 16 * 16;
};

template <int L>
__global__ void __launch_bounds__(256, L == 4 ? 3 : 2) k_g2p2g(DevGrid src, DevGrid dst, const int32_t *__restrict__ bin_list,
                                               const int32_t *__restrict__ bin_off, const int32_t *bin_end,
                                               int32_t *perm, const int32_t *bins_used, float *__restrict__ x,
                                               float *__restrict__ v, float dt, int f_vel0, float pmass, int f_mass,
                                               int f_mom0, bool pair)
{
    using S = G2P2GSmem<L>;
    constexpr int LG2 = (L == 8) ? 3 : 2, BD = S::BD, C1 = S::C1, NC = S::NC, ND = S::ND;
    extern __shared__ __align__(16) unsigned char smem[];
    float4(*s_rec)[S::CAP] = reinterpret_cast<float4(*)[S::CAP]>(smem + S::off_rec);
    float4 *s_u = reinterpret_cast<float4 *>(smem + S::off_u);
    float(*s_acc)[ND] = reinterpret_cast<float(*)[ND]>(smem + S::off_acc);
    int *s_cnt = reinterpret_cast<int *>(smem + S::off_cnt);
    int *s_start = reinterpret_cast<int *>(smem + S::off_start);
    int *s_slot = reinterpret_cast<int *>(smem + S::off_slot);
    uint8_t *s_hit = smem + S::off_hit;
    if (threadIdx.x == 0) misaligned(dst, smem, 16, 4);

    const int N = src.N, R = src.R;
    const float dx = 1.f / (float)N;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int la = lane / 9, lc = (lane / 3) % 3, ld = lane % 3;
    const BsPoly pa = bs_poly(la), pb = bs_poly(lc), pc = bs_poly(ld);
    const float ta = (float)la, tb = (float)lc, tc = (float)ld;
    const float *u0p = src.field[f_vel0], *u1p = src.field[f_vel0 + 1], *u2p = src.field[f_vel0 + 2];
    bool changed = false;
    const int used = *bins_used;
    const long long oob_key = 8LL * R * R * R;
    for (int bl = blockIdx.x; bl <= used; bl += gridDim.x) {
        int beg, end, oi = 0, oj = 0, ok = 0;
        const bool binned = bl < used;
        if (binned) {
            const long long b = bin_list[bl];
            beg = bin_off[8 * b];
            end = bin_end[8 * b + 7];
            oi = (int)(b / ((long long)R * R)) * L;
            oj = (int)((b / R) % R) * L;
            ok = (int)(b % R) * L;
            stage_velocities<L>(src, u0p, u1p, u2p, oi, oj, ok, s_u);
            for (int q = threadIdx.x; q < ND; q += blockDim.x) {
                s_acc[0][q] = s_acc[1][q] = s_acc[2][q] = s_acc[3][q] = 0.f;
                s_hit[q] = 0;
            }
            __syncthreads();
        } else {
            beg = bin_off[oob_key];
            end = bin_end[oob_key];
        }
        for (int c0 = beg; c0 < end; c0 += S::CAP) {
            const int cnt = min(S::CAP, end - c0);
            if (binned) {
                for (int q = threadIdx.x; q <= NC; q += blockDim.x) s_cnt[q] = 0;
                __syncthreads();
            }
            // G2P of this thread's particle; its P2G record stays in registers
            int rcell = -1, rrank = 0, rp = 0;
            P2GRec rec;
            if ((int)threadIdx.x < cnt) {
                rp = perm[c0 + threadIdx.x];
                const long long p = rp;
                const float3 xp = load3_checked(dst, x, p, pair);
                const Spline ox = bspline(xp.x, N), oy = bspline(xp.y, N), oz = bspline(xp.z, N);
                const int ri = ox.base - oi + 2, rj = oy.base - oj + 2, rk = oz.base - ok + 2;
                float3 u;
                float c[9];
                if (binned && (unsigned)ri <= (unsigned)(L + 1) && (unsigned)rj <= (unsigned)(L + 1) &&
                    (unsigned)rk <= (unsigned)(L + 1))
                    g2p_from_block<L + 4, true>(s_u, ri, rj, rk, N, ox, oy, oz, u, c);
                else
                    g2p_from_grid<true>(src, u0p, u1p, u2p, ox, oy, oz, u, c);
                const float3 xn = make_float3(xp.x + dt * u.x, xp.y + dt * u.y, xp.z + dt * u.z);
                store3_checked(dst, v, p, u, pair);
                store3_checked(dst, x, p, xn, pair);
                const Spline nx = bspline(xn.x, N), ny = bspline(xn.y, N), nz = bspline(xn.z, N);
                rec = make_rec(nx.fx, ny.fx, nz.fx, pmass, u, c, dx);
                const int ci = nx.base - oi + 1, cj = ny.base - oj + 1, ck = nz.base - ok + 1;
                if (binned && (unsigned)ci < (unsigned)C1 && (unsigned)cj < (unsigned)C1 && (unsigned)ck < (unsigned)C1) {
                    rcell = (ci * C1 + cj) * C1 + ck;
                    rrank = atomicAdd(&s_cnt[rcell], 1);
                } else {
                    changed |= scatter_particle(dst, nx, ny, nz, rec, f_mass, f_mom0);
                }
            }
            if (!binned) continue;  // no shared block for the out-of-domain key
            __syncthreads();
            if (threadIdx.x < 32) {  // exclusive scan of the cell counts
                int carry = 0;
                for (int base = 0; base < NC; base += 32) {
                    const int i = base + threadIdx.x;
                    const int vv = (i < NC) ? s_cnt[i] : 0;
                    const int inc = warp_incl_scan(vv);
                    if (i < NC) s_start[i] = carry + inc - vv;
                    carry += __shfl_sync(kFull, inc, 31);
                }
                if (threadIdx.x == 0) s_start[NC] = carry;
            }
            __syncthreads();
            if (rcell >= 0 && !misaligned(dst, &s_rec[0][s_start[rcell] + rrank], 16, 5)) {
                const int pos = s_start[rcell] + rrank;
                s_rec[0][pos] = rec.r0;
                s_rec[1][pos] = rec.r1;
                s_rec[2][pos] = rec.r2;
                s_rec[3][pos] = rec.r3;
            }
            __syncthreads();
            for (int cell = warp; cell < NC; cell += blockDim.x / 32) {
                const int p0 = s_start[cell], p1 = s_start[cell + 1];
                if (p0 == p1) continue;  // uniform across the warp
                if (p0 < 0 || p1 > S::CAP || p0 > p1) {
                    if (lane == 0) {
                        atomicOr(&dst.ctrl->err, kErrCheck);
                        dst.ctrl->timeout_site = 106;
                    }
                    continue;
                }
                const int ci = cell / (C1 * C1), cj = (cell / C1) % C1, ck = cell % C1;
                float m = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
                for (int pp = p0; pp < p1; ++pp) {
                    if (misaligned(dst, &s_rec[3][pp], 16, 7)) break;
                    const float4 r0 = s_rec[0][pp];
                    const float w = bs_eval(pa, r0.x) * bs_eval(pb, r0.y) * bs_eval(pc, r0.z);
                    const float4 r1 = s_rec[1][pp], r2 = s_rec[2][pp], r3 = s_rec[3][pp];
                    const float q0 = fmaf(r1.w, ta, fmaf(r2.x, tb, fmaf(r2.y, tc, r1.x)));
                    const float q1 = fmaf(r2.z, ta, fmaf(r2.w, tb, fmaf(r3.x, tc, r1.y)));
                    const float q2 = fmaf(r3.y, ta, fmaf(r3.z, tb, fmaf(r3.w, tc, r1.z)));
                    m = fmaf(w, r0.w, m);
                    m0 = fmaf(w, q0, m0);
                    m1 = fmaf(w, q1, m1);
                    m2 = fmaf(w, q2, m2);
                }
                if (lane < 27) {  // block node (ci + la, cj + lc, ck + ld) = grid node o - 1 + that
                    const int nd = ((ci + la) * BD + (cj + lc)) * BD + (ck + ld);
                    atomicAdd(&s_acc[0][nd], m);
                    atomicAdd(&s_acc[1][nd], m0);
                    atomicAdd(&s_acc[2][nd], m1);
                    atomicAdd(&s_acc[3][nd], m2);
                    s_hit[nd] = 1;
                }
            }
            __syncthreads();
        }
        if (!binned) continue;
        // dst leaves of the block: leaf cells (o >> LG2) - 1 .. (o >> LG2) + 1 per
        // axis hold every block node; allocate the ones with a touched in-domain node
        if (threadIdx.x < 27) s_slot[threadIdx.x] = 0;
        __syncthreads();
        const int li0 = (oi >> LG2) - 1, lj0 = (oj >> LG2) - 1, lk0 = (ok >> LG2) - 1;
        for (int nd = threadIdx.x; nd < ND; nd += blockDim.x) {
            if (!s_hit[nd]) continue;
            const int i = oi - 1 + nd / (BD * BD), j = oj - 1 + (nd / BD) % BD, k = ok - 1 + nd % BD;
            if ((unsigned)i >= (unsigned)N || (unsigned)j >= (unsigned)N || (unsigned)k >= (unsigned)N) continue;
            s_slot[((i >> LG2) - li0) * 9 + ((j >> LG2) - lj0) * 3 + ((k >> LG2) - lk0)] = 1;
        }
        __syncthreads();
        if (threadIdx.x < 27) {
            const int t = threadIdx.x;
            int slot = -1;
            if (s_slot[t]) {
                bool fresh = false;
                const long long lb = ((long long)(li0 + t / 9) * R + (lj0 + (t / 3) % 3)) * R + (lk0 + t % 3);
                slot = ensure_leaf(dst, lb, fresh);
                changed |= fresh;
            }
            s_slot[t] = slot;
        }
        __syncthreads();
        for (int nd = threadIdx.x; nd < ND; nd += blockDim.x) {
            if (!s_hit[nd]) continue;
            const int i = oi - 1 + nd / (BD * BD), j = oj - 1 + (nd / BD) % BD, k = ok - 1 + nd % BD;
            if ((unsigned)i >= (unsigned)N || (unsigned)j >= (unsigned)N || (unsigned)k >= (unsigned)N) continue;
            const int slot = s_slot[((i >> LG2) - li0) * 9 + ((j >> LG2) - lj0) * 3 + ((k >> LG2) - lk0)];
            if (slot < 0) continue;  // pool exhausted; the error is latched
            const int l = (((i & (L - 1)) << LG2) + (j & (L - 1))) * L + (k & (L - 1));
            uint32_t *mw = &dst.mask[(long long)slot * dst.W + (l >> 5)];
            const uint32_t bit = 1u << (l & 31);
            if (!(*(volatile uint32_t *)mw & bit)) changed |= !(atomicOr(mw, bit) & bit);
            const long long idx = ((long long)slot << (3 * LG2)) + l;
            atomicAdd(dst.field[f_mass] + idx, s_acc[0][nd]);
            atomicAdd(dst.field[f_mom0] + idx, s_acc[1][nd]);
            atomicAdd(dst.field[f_mom0 + 1] + idx, s_acc[2][nd]);
            atomicAdd(dst.field[f_mom0 + 2] + idx, s_acc[3][nd]);
        }
        __syncthreads();  // shared state is reset for the next bin
    }
    if (changed) mark_dirty(dst);
}

template <int L>
void launch_g2p2g_L(const DevGrid &src, const DevGrid &dst, const DevGrid &bins, cudaStream_t s, float *x, float *v,
                    float dt, int f_vel0, float pmass, int f_mass, int f_mom0, bool pair, int num_sms)
{
    constexpr size_t bytes = G2P2GSmem<L>::bytes;
    static std::atomic<int> resident;  // CTAs per SM; threads may race to fill it
    int per = resident.load(std::memory_order_relaxed);
    if (!per) {
        cudaFuncSetAttribute(k_g2p2g<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_g2p2g<L>, 256, bytes) != cudaSuccess || per < 1)
            per = 1;
        resident.store(per, std::memory_order_relaxed);
    }
    const int ctas = per * num_sms;
    k_g2p2g<L><<<ctas, 256, bytes, s>>>(src, dst, bins.bin_list, bins.bin_off, bins.bin_count, bins.perm,
                                         &bins.ctrl->bins_used, x, v, dt, f_vel0, pmass, f_mass, f_mom0, pair);
}

}  // namespace

void launch_g2p2g(const DevGrid &src, const DevGrid &dst, const DevGrid &bins, cudaStream_t s, float *x, float *v,
                  long long n, float dt, int f_vel0, float pmass, int f_mass, int f_mom0, const LaunchCfg &lc)
{
    if (n <= 0) return;
    const bool pair = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(v)) & 7) == 0;
    if (dst.L == 4) launch_g2p2g_L<4>(src, dst, bins, s, x, v, dt, f_vel0, pmass, f_mass, f_mom0, pair, lc.num_sms);
    else launch_g2p2g_L<8>(src, dst, bins, s, x, v, dt, f_vel0, pmass, f_mass, f_mom0, pair, lc.num_sms);
}

}  // namespace sg
