// sg_advect.cu -- MacCormack advection with RK3 path integration over the
// sparse grid (AsyncTaichi Sec. 8.2): semi-Lagrangian advection of up to
// three channels per launch sharing one backtrace, and the backward advection
// fused with the MacCormack correction (the intermediate q~ kept in registers
// unless a later op reads it).
//
// Collocated grid: voxel (i,j,k) sits at (i+0.5, j+0.5, k+0.5) in cell units;
// velocities are in domain units per time, h = dt * N cells per unit
// velocity.  A sample between cells is trilinear over the 8 surrounding cell
// centres; each value is read from its leaf found through the list entry's
// 27-neighbour table (a null or out-of-domain neighbour is the zero leaf, and
// a stored value at an inactive voxel is 0, so every read is unconditional),
// or through the root when the sample lies more than a leaf away.  A warp's 32
// voxels lie in one leaf (L^3 is a multiple of 32), so the warp copies the
// entry's table to shared memory once and every lookup is a shared load;
// element offsets are 32-bit when the fields have fewer than 2^31 elements.
// With fusion the run's velocity is first packed as one float4 (u, v, w, 0)
// per value slot, so a velocity corner is one 16-byte load instead of three
// (the same products summed in the same order: the results are identical).
// Backtrace: Ralston's RK3, x_back = x - h (2 k1 + 3 k2 + 4 k3) / 9 with
// k1 = u(x), k2 = u(x - h/2 k1), k3 = u(x - 3h/4 k2).  Correction: q' =
// q^ + (q - q~) / 2 clamped to the 8 values of q the forward sample uses.
#include "sg_common.cuh"

namespace sg {

namespace {

constexpr int kMaxAdvectChannels = 3;

struct AdvectArgs {
    int C;                            // channels
    int dst[kMaxAdvectChannels];      // outputs
    int src[kMaxAdvectChannels];      // advect: sampled field; mac: q
    int qhat[kMaxAdvectChannels];     // mac: q^
    int qtil[kMaxAdvectChannels];     // mac: q~ (fused: its output, -1 = not stored)
    int v0;                           // velocity fields v0 .. v0+2
    float h;                          // dt * N (the forward step)
    // clamp bounds of the correction, per channel: written by an advection
    // (the min and max of the 8 values its sample reads) and read by the
    // correction of the same q, velocity and step instead of tracing again
    float *lo[kMaxAdvectChannels];
    float *hi[kMaxAdvectChannels];
    const float4 *vel4;               // packed velocity, or null (read the three fields)
};

// Slot of the leaf holding cell (ci, cj, ck), relative to the list entry's
// leaf (bi, bj, bk): through the neighbour table within one leaf, else the root.
template <int L>
__device__ __forceinline__ int leaf_slot(const DevGrid &g, const int32_t *nb, int bi, int bj, int bk, int ci, int cj,
                                         int ck)
{
    constexpr int LG2 = (L == 8) ? 3 : 2;
    const int di = (ci >> LG2) - bi, dj = (cj >> LG2) - bj, dk = (ck >> LG2) - bk;
    if ((unsigned)(di + 1) <= 2u && (unsigned)(dj + 1) <= 2u && (unsigned)(dk + 1) <= 2u)
        return __ldg(nb + (di + 1) * 9 + (dj + 1) * 3 + (dk + 1));
    if ((unsigned)ci >= (unsigned)g.N || (unsigned)cj >= (unsigned)g.N || (unsigned)ck >= (unsigned)g.N)
        return (int)g.cap;  // out of the domain: the zero leaf
    const int s = __ldg(g.root + ((long long)(ci >> LG2) * g.R + (cj >> LG2)) * g.R + (ck >> LG2));
    return s < 0 ? (int)g.cap : s;
}

// The 8 corners of a sample at p (cell units): their value offsets within a
// field and trilinear weights.
template <int L, typename Off>
struct Corners {
    Off off[8];
    float w[8];
};

// tab: the warp's copy of the list entry's neighbour table (shared memory).
template <int L, typename Off>
__device__ __forceinline__ void corners(const DevGrid &g, const int32_t *nb, const int *tab, int bi, int bj, int bk,
                                        float px, float py, float pz, Corners<L, Off> &cr)
{
    constexpr int LG2 = (L == 8) ? 3 : 2;
    const float X = px - 0.5f, Y = py - 0.5f, Z = pz - 0.5f;
    const float fx0 = floorf(X), fy0 = floorf(Y), fz0 = floorf(Z);
    const int i0 = (int)fx0, j0 = (int)fy0, k0 = (int)fz0;
    const float fx = X - fx0, fy = Y - fy0, fz = Z - fz0;
    // per axis: the leaf offsets (relative to the entry's leaf) and local indices
    // of the two corner layers
    const int di0 = (i0 >> LG2) - bi, dj0 = (j0 >> LG2) - bj, dk0 = (k0 >> LG2) - bk;
    const int di1 = ((i0 + 1) >> LG2) - bi, dj1 = ((j0 + 1) >> LG2) - bj, dk1 = ((k0 + 1) >> LG2) - bk;
    const int li[2] = {i0 & (L - 1), (i0 + 1) & (L - 1)}, lj[2] = {j0 & (L - 1), (j0 + 1) & (L - 1)},
              lk[2] = {k0 & (L - 1), (k0 + 1) & (L - 1)};
    const float wx[2] = {1.f - fx, fx}, wy[2] = {1.f - fy, fy}, wz[2] = {1.f - fz, fz};
    // within the 27-neighbourhood (the common case): the table entry; lanes
    // whose sample lies further out take the root afterwards
    const bool near = di0 >= -1 && di1 <= 1 && dj0 >= -1 && dj1 <= 1 && dk0 >= -1 && dk1 <= 1;
    const int ti[2] = {near ? (di0 + 1) * 9 : 0, near ? (di1 + 1) * 9 : 0},
              tj[2] = {near ? (dj0 + 1) * 3 : 0, near ? (dj1 + 1) * 3 : 0}, tk[2] = {near ? dk0 + 1 : 0, near ? dk1 + 1 : 0};
    int slot[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) slot[c] = tab[ti[c >> 2] + tj[(c >> 1) & 1] + tk[c & 1]];
    if (!near) {
#pragma unroll
        for (int c = 0; c < 8; ++c)
            slot[c] = leaf_slot<L>(g, nb, bi, bj, bk, i0 + (c >> 2), j0 + ((c >> 1) & 1), k0 + (c & 1));
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int a = c >> 2, b = (c >> 1) & 1, d = c & 1;
        cr.off[c] = ((Off)slot[c] << (3 * LG2)) + (Off)((((li[a] << LG2) + lj[b]) << LG2) + lk[d]);
        cr.w[c] = wx[a] * wy[b] * wz[d];
    }
}

template <int L, typename Off>
__device__ __forceinline__ float sample(const float *__restrict__ f, const Corners<L, Off> &cr)
{
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s = fmaf(cr.w[c], __ldg(f + cr.off[c]), s);
    return s;
}

template <int L, typename Off, bool PK>
__device__ __forceinline__ void velocity(const DevGrid &g, const int32_t *nb, const int *tab, int bi, int bj, int bk, int v0,
                                         const float4 *__restrict__ vel4, float px, float py, float pz, float (&u)[3])
{
    Corners<L, Off> cr;
    corners<L, Off>(g, nb, tab, bi, bj, bk, px, py, pz, cr);
    if (PK) {
        u[0] = u[1] = u[2] = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float4 w = __ldg(vel4 + cr.off[c]);
            u[0] = fmaf(cr.w[c], w.x, u[0]);
            u[1] = fmaf(cr.w[c], w.y, u[1]);
            u[2] = fmaf(cr.w[c], w.z, u[2]);
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) u[a] = sample<L, Off>(g.field[v0 + a], cr);
    }
}

// RK3 backtrace of cell centre x over h; returns the corners of the sample.
// k1 = u(x) at the cell centre itself is the voxel's stored velocity (the
// trilinear weights there are 1, 0, ..., 0), read directly at idx.
template <int L, typename Off, bool PK>
__device__ __forceinline__ void backtrace(const DevGrid &g, const int32_t *nb, const int *tab, int bi, int bj, int bk, int v0,
                                          const float4 *__restrict__ vel4, float h, const float (&x)[3], Off idx,
                                          Corners<L, Off> &cr)
{
    float k1[3], k2[3], k3[3];
    if (PK) {
        const float4 w = __ldg(vel4 + idx);
        k1[0] = w.x;
        k1[1] = w.y;
        k1[2] = w.z;
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) k1[a] = g.field[v0 + a][idx];
    }
    velocity<L, Off, PK>(g, nb, tab, bi, bj, bk, v0, vel4, x[0] - 0.5f * h * k1[0], x[1] - 0.5f * h * k1[1],
                     x[2] - 0.5f * h * k1[2], k2);
    velocity<L, Off, PK>(g, nb, tab, bi, bj, bk, v0, vel4, x[0] - 0.75f * h * k2[0], x[1] - 0.75f * h * k2[1],
                     x[2] - 0.75f * h * k2[2], k3);
    const float c = h / 9.f;
    corners<L, Off>(g, nb, tab, bi, bj, bk, x[0] - c * (2.f * k1[0] + 3.f * k2[0] + 4.f * k3[0]),
                    x[1] - c * (2.f * k1[1] + 3.f * k2[1] + 4.f * k3[1]),
                    x[2] - c * (2.f * k1[2] + 3.f * k2[2] + 4.f * k3[2]), cr);
}

// MODE 0: advect (dst = src at the backtrace over h); with BND the clamp
//         bounds of each channel's sample are stored in A.lo / A.hi;
// MODE 1: backward advect of q^ over -h fused with the correction;
// MODE 2: correction alone (q~ read from its field).
// In modes 1 and 2, BND reads the clamp bounds from A.lo / A.hi instead of
// tracing the forward path again.
// PK: the velocity is read from A.vel4 (packed).  Four CTAs per SM (at most
// 64 registers a thread): the traces are latency-bound.
template <int L, int C, int MODE, bool BND, typename Off, bool PK>
__global__ void __launch_bounds__(256, 4) k_advect(DevGrid g, AdvectArgs A)
{
    constexpr int V = L * L * L, LG2 = (L == 8) ? 3 : 2;
    const long long n = g.ctrl->list_n;
    const int R = g.R;
    __shared__ int s_nb[8][27];
    // the loop bound is a multiple of 32 and the stride a multiple of 256, so
    // a warp's lanes share one list entry per iteration and all reach the
    // __syncwarp() around the copy of its table
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * V;
         q += (long long)gridDim.x * blockDim.x) {
        const long long e = q >> (3 * LG2);
        const int l = (int)(q & (V - 1));
        const int slot = g.list_slot[e];
        const Off idx = ((Off)slot << (3 * LG2)) + (Off)l;
        const bool act = (g.mask[(long long)slot * g.W + (l >> 5)] >> (l & 31)) & 1u;
        const int32_t *nb = g.nbr + e * 27;
        int *tab = s_nb[threadIdx.x >> 5];
        __syncwarp();
        if (lane_id() < 27) tab[lane_id()] = __ldg(nb + lane_id());
        __syncwarp();
        if (!act) {  // inactive voxels keep 0
#pragma unroll
            for (int c = 0; c < C; ++c) {
                g.field[A.dst[c]][idx] = 0.f;
                if (MODE == 1 && A.qtil[c] >= 0) g.field[A.qtil[c]][idx] = 0.f;
            }
            continue;
        }
        const int b = g.list_b[e];
        const int bi = b / (R * R), bj = (b / R) % R, bk = b % R;
        const float x[3] = {(float)((bi << LG2) + (l >> (2 * LG2))) + 0.5f,
                            (float)((bj << LG2) + ((l >> LG2) & (L - 1))) + 0.5f,
                            (float)((bk << LG2) + (l & (L - 1))) + 0.5f};
        Corners<L, Off> fw;
        if (MODE == 0 || !BND) backtrace<L, Off, PK>(g, nb, tab, bi, bj, bk, A.v0, A.vel4, A.h, x, idx, fw);
        if (MODE == 0) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const float *sf = g.field[A.src[c]];
                if constexpr (!BND) {
                    g.field[A.dst[c]][idx] = sample<L, Off>(sf, fw);
                } else {
                    float v[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) v[k] = __ldg(sf + fw.off[k]);
                    float smp = 0.f, lo = v[0], hi = v[0];
#pragma unroll
                    for (int k = 0; k < 8; ++k) smp = fmaf(fw.w[k], v[k], smp);  // the order of sample()
#pragma unroll
                    for (int k = 1; k < 8; ++k) {
                        lo = fminf(lo, v[k]);
                        hi = fmaxf(hi, v[k]);
                    }
                    g.field[A.dst[c]][idx] = smp;
                    A.lo[c][idx] = lo;
                    A.hi[c][idx] = hi;
                }
            }
            continue;
        }
        float qt[C];
        if (MODE == 1) {
            Corners<L, Off> bw;
            backtrace<L, Off, PK>(g, nb, tab, bi, bj, bk, A.v0, A.vel4, -A.h, x, idx, bw);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                qt[c] = sample<L, Off>(g.field[A.qhat[c]], bw);
                if (A.qtil[c] >= 0) g.field[A.qtil[c]][idx] = qt[c];
            }
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) qt[c] = g.field[A.qtil[c]][idx];
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float *qf = g.field[A.src[c]];
            float lo, hi;
            if (BND) {
                lo = A.lo[c][idx];
                hi = A.hi[c][idx];
            } else {
                lo = __ldg(qf + fw.off[0]);
                hi = lo;
#pragma unroll
                for (int k = 1; k < 8; ++k) {
                    const float v = __ldg(qf + fw.off[k]);
                    lo = fminf(lo, v);
                    hi = fmaxf(hi, v);
                }
            }
            const float r = g.field[A.qhat[c]][idx] + 0.5f * (qf[idx] - qt[c]);
            g.field[A.dst[c]][idx] = fminf(fmaxf(r, lo), hi);
        }
    }
}

template <int L, int MODE, bool BND, typename Off, bool PK>
void launch_LBO(const DevGrid &g, cudaStream_t s, const AdvectArgs &a, int ctas)
{
    if (a.C == 1) k_advect<L, 1, MODE, BND, Off, PK><<<ctas, 256, 0, s>>>(g, a);
    else if (a.C == 2) k_advect<L, 2, MODE, BND, Off, PK><<<ctas, 256, 0, s>>>(g, a);
    else k_advect<L, 3, MODE, BND, Off, PK><<<ctas, 256, 0, s>>>(g, a);
}

template <int L, int MODE>
void launch_L(const DevGrid &g, cudaStream_t s, AdvectArgs a, int ctas)
{
    // 32-bit element offsets while every offset (the zero leaf's included)
    // fits; the packed velocity is read by the modes that trace (the fused
    // schedule's forward and backward launches) with 32-bit offsets
    const bool wide = (unsigned long long)(g.cap + 1) * (L * L * L) > 0x7fffffffull;
    if constexpr (MODE != 2) {
        if (a.vel4 && !wide) {
            if (a.lo[0]) launch_LBO<L, MODE, true, int, true>(g, s, a, ctas);
            else launch_LBO<L, MODE, false, int, true>(g, s, a, ctas);
            return;
        }
    }
    a.vel4 = nullptr;
    if (a.lo[0]) {
        if (wide) launch_LBO<L, MODE, true, long long, false>(g, s, a, ctas);
        else launch_LBO<L, MODE, true, int, false>(g, s, a, ctas);
    } else {
        if (wide) launch_LBO<L, MODE, false, long long, false>(g, s, a, ctas);
        else launch_LBO<L, MODE, false, int, false>(g, s, a, ctas);
    }
}

// Packed velocity: vel4[slot * L^3 + l] = (u, v, w, 0) of fields v0..v0+2 for
// every listed leaf (the zero leaf's block is zero from its allocation).
template <int L>
__global__ void __launch_bounds__(256) k_pack_velocity(DevGrid g, int v0, float4 *__restrict__ vel4)
{
    constexpr int V = L * L * L, LG2 = (L == 8) ? 3 : 2;
    const long long n = g.ctrl->list_n;
    const float *__restrict__ u = g.field[v0], *__restrict__ v = g.field[v0 + 1], *__restrict__ w = g.field[v0 + 2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * V;
         q += (long long)gridDim.x * blockDim.x) {
        const long long idx = ((long long)g.list_slot[q >> (3 * LG2)] << (3 * LG2)) + (q & (V - 1));
        vel4[idx] = make_float4(__ldg(u + idx), __ldg(v + idx), __ldg(w + idx), 0.f);
    }
}

}  // namespace

void launch_pack_velocity(const DevGrid &g, cudaStream_t s, int v0, float4 *vel4, const LaunchCfg &lc)
{
    const int ctas = lc.num_sms * 8;
    if (g.L == 8) k_pack_velocity<8><<<ctas, 256, 0, s>>>(g, v0, vel4);
    else k_pack_velocity<4><<<ctas, 256, 0, s>>>(g, v0, vel4);
}

void launch_advect_group(const DevGrid &g, cudaStream_t s, int mode, int C, const int *dst, const int *src,
                         const int *qhat, const int *qtil, int v0, float h, float *const *lo, float *const *hi,
                         const float4 *vel4, const LaunchCfg &lc)
{
    AdvectArgs a{};
    a.C = C;
    for (int c = 0; c < C; ++c) {
        a.dst[c] = dst[c];
        a.src[c] = src[c];
        a.qhat[c] = qhat ? qhat[c] : -1;
        a.qtil[c] = qtil ? qtil[c] : -1;
        a.lo[c] = lo ? lo[c] : nullptr;
        a.hi[c] = hi ? hi[c] : nullptr;
    }
    a.v0 = v0;
    a.h = h;
    a.vel4 = vel4;
    const int ctas = lc.num_sms * 8;
    if (g.L == 8) {
        if (mode == 0) launch_L<8, 0>(g, s, a, ctas);
        else if (mode == 1) launch_L<8, 1>(g, s, a, ctas);
        else launch_L<8, 2>(g, s, a, ctas);
    } else {
        if (mode == 0) launch_L<4, 0>(g, s, a, ctas);
        else if (mode == 1) launch_L<4, 1>(g, s, a, ctas);
        else launch_L<4, 2>(g, s, a, ctas);
    }
}

}  // namespace sg
