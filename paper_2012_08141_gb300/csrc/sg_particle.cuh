// sg_particle.cuh -- device helpers of the particle-grid transfers, shared
// by the separate (sg_particle.cu) and the fused G2P2G (sg_g2p2g.cu)
// kernels: the quadratic B-spline of a particle along one axis, G2P of one
// particle from a staged block of node velocities or node by node from the
// grid (PIC, or APIC with the matrix C), and the particle-array accessors.
#pragma once
#include "sg_common.cuh"

namespace sg {

struct Spline {
    int base;
    float fx;  // X - base, in [0.5, 1.5)
    float w[3];
};

// base = floor(X - 0.5), fx = X - base, X = x*N, all in FP32, each operation
// rounded on its own (no contraction), so that every kernel that bins a
// particle takes the same base.
__device__ __forceinline__ Spline bspline(float x, int N)
{
    Spline s;
    const float X = __fmul_rn(x, (float)N);
    const float bf = floorf(__fsub_rn(X, 0.5f));
    const float fx = __fsub_rn(X, bf);
    s.base = (int)bf;
    s.fx = fx;
    const float a = 1.5f - fx, c = fx - 1.0f, d = fx - 0.5f;
    s.w[0] = 0.5f * a * a;
    s.w[1] = 0.75f - c * c;
    s.w[2] = 0.5f * d * d;
    return s;
}

// G2P of one particle read node by node from the grid (a stored value at an
// inactive node is 0; out-of-domain and unallocated nodes are skipped).
// Returns v_p in u and, for APIC, C_p in c.
template <bool APIC>
__device__ __forceinline__ void g2p_from_grid(const DevGrid &g, const float *__restrict__ f0,
                                              const float *__restrict__ f1, const float *__restrict__ f2,
                                              const Spline &sx, const Spline &sy, const Spline &sz, float3 &u,
                                              float (&c)[9])
{
    const int L = g.L, lg2 = g.lg2, N = g.N;
    float ux = 0.f, uy = 0.f, uz = 0.f;
    float S[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};  // sum w v_e t_f
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = sx.base + a;
        if ((unsigned)i >= (unsigned)N) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int j = sy.base + b;
            if ((unsigned)j >= (unsigned)N) continue;
            const float wxy = sx.w[a] * sy.w[b];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const int k = sz.base + cc;
                if ((unsigned)k >= (unsigned)N) continue;
                const long long lb = ((long long)(i >> lg2) * g.R + (j >> lg2)) * g.R + (k >> lg2);
                const int slot = __ldg(g.root + lb);
                if (slot < 0) continue;
                const int l = (((i & (L - 1)) << lg2) + (j & (L - 1))) * L + (k & (L - 1));
                const long long idx = ((long long)slot << (3 * lg2)) + l;
                const float w = wxy * sz.w[cc];
                const float wv[3] = {w * __ldg(f0 + idx), w * __ldg(f1 + idx), w * __ldg(f2 + idx)};
                ux += wv[0];
                uy += wv[1];
                uz += wv[2];
                if (APIC) {
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        S[e][0] = fmaf((float)a, wv[e], S[e][0]);
                        S[e][1] = fmaf((float)b, wv[e], S[e][1]);
                        S[e][2] = fmaf((float)cc, wv[e], S[e][2]);
                    }
                }
            }
        }
    }
    u = make_float3(ux, uy, uz);
    if (APIC) {
        const float s4 = 4.f * (float)N, fx[3] = {sx.fx, sy.fx, sz.fx}, ue[3] = {ux, uy, uz};
#pragma unroll
        for (int e = 0; e < 3; ++e)
#pragma unroll
            for (int f = 0; f < 3; ++f) c[3 * e + f] = s4 * fmaf(-fx[f], ue[e], S[e][f]);
    }
}

// A float triple at a[3p..3p+2]; with pair set (the array is 8-byte
// aligned) in two accesses: the aligned pair (elements 0,1 for even p, 1,2
// for odd p) and the remaining single.
__device__ __forceinline__ float3 load3(const float *__restrict__ a, long long p, bool pair)
{
    const float *q = a + 3 * p;
    if (!pair) return make_float3(q[0], q[1], q[2]);
    if (p & 1) {
        const float2 hi = *reinterpret_cast<const float2 *>(q + 1);
        return make_float3(q[0], hi.x, hi.y);
    }
    const float2 lo = *reinterpret_cast<const float2 *>(q);
    return make_float3(lo.x, lo.y, q[2]);
}

__device__ __forceinline__ void store3(float *__restrict__ a, long long p, float3 t, bool pair)
{
    float *q = a + 3 * p;
    if (!pair) {
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

template <bool APIC>
__device__ __forceinline__ void g2p_store(float *__restrict__ x, float *__restrict__ v, float *__restrict__ C,
                                          long long p, float3 xp, float3 u, const float (&c)[9], float dt, bool pair)
{
    store3(v, p, u, pair);
    store3(x, p, make_float3(xp.x + dt * u.x, xp.y + dt * u.y, xp.z + dt * u.z), pair);
    if (APIC) {
#pragma unroll
        for (int q = 0; q < 9; ++q) C[9 * p + q] = c[q];
    }
}

// Stage the velocities of the (L+4)^3 nodes from o - 2 to o + L + 1 of a
// leaf with origin o as one float4 (u0, u1, u2, 0) per node: 0 outside the
// domain or the allocated leaves.
template <int L>
__device__ __forceinline__ void stage_velocities(const DevGrid &g, const float *__restrict__ f0,
                                                 const float *__restrict__ f1, const float *__restrict__ f2, int oi,
                                                 int oj, int ok, float4 *s_u)
{
    constexpr int LG2 = (L == 8) ? 3 : 2, B = L + 4, NB = B * B * B;
    const int N = g.N, R = g.R;
    for (int nd = threadIdx.x; nd < NB; nd += blockDim.x) {
        const int i = oi - 2 + nd / (B * B), j = oj - 2 + (nd / B) % B, k = ok - 2 + nd % B;
        float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((unsigned)i < (unsigned)N && (unsigned)j < (unsigned)N && (unsigned)k < (unsigned)N) {
            const int slot = __ldg(g.root + ((long long)(i >> LG2) * R + (j >> LG2)) * R + (k >> LG2));
            if (slot >= 0) {
                const long long idx =
                    ((long long)slot << (3 * LG2)) + (((i & (L - 1)) << LG2) + (j & (L - 1))) * L + (k & (L - 1));
                u = make_float4(__ldg(f0 + idx), __ldg(f1 + idx), __ldg(f2 + idx), 0.f);
            }
        }
        s_u[nd] = u;
    }
}

// The (L+2)^3 nodes from o to o + L + 1 only: every node the stencils of
// particles with base in the leaf reach (no margin for particles that moved
// since they were binned).
template <int L>
__device__ __forceinline__ void stage_velocities_tight(const DevGrid &g, const float *__restrict__ f0,
                                                       const float *__restrict__ f1, const float *__restrict__ f2,
                                                       int oi, int oj, int ok, float4 *s_u)
{
    constexpr int LG2 = (L == 8) ? 3 : 2, B = L + 2, NB = B * B * B;
    const int N = g.N, R = g.R;
    for (int nd = threadIdx.x; nd < NB; nd += blockDim.x) {
        const int i = oi + nd / (B * B), j = oj + (nd / B) % B, k = ok + nd % B;
        float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < N && j < N && k < N) {
            const int slot = __ldg(g.root + ((long long)(i >> LG2) * R + (j >> LG2)) * R + (k >> LG2));
            if (slot >= 0) {
                const long long idx =
                    ((long long)slot << (3 * LG2)) + (((i & (L - 1)) << LG2) + (j & (L - 1))) * L + (k & (L - 1));
                u = make_float4(__ldg(f0 + idx), __ldg(f1 + idx), __ldg(f2 + idx), 0.f);
            }
        }
        s_u[nd] = u;
    }
}

// G2P of one particle from a staged block of B^3 float4 node velocities (ri,
// rj, rk: its base relative to the block's first node).  APIC as in
// g2p_from_grid.
template <int B, bool APIC>
__device__ __forceinline__ void g2p_from_block(const float4 *s_u, int ri, int rj, int rk, int N, const Spline &sx,
                                               const Spline &sy, const Spline &sz, float3 &u, float (&c)[9])
{
    float ux = 0.f, uy = 0.f, uz = 0.f;
    float S[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float wxy = sx.w[a] * sy.w[b];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const float4 n = s_u[((ri + a) * B + (rj + b)) * B + (rk + cc)];
                const float w = wxy * sz.w[cc];
                const float wv[3] = {w * n.x, w * n.y, w * n.z};
                ux += wv[0];
                uy += wv[1];
                uz += wv[2];
                if (APIC) {
#pragma unroll
                    for (int e = 0; e < 3; ++e) {
                        if (a) S[e][0] = fmaf((float)a, wv[e], S[e][0]);
                        if (b) S[e][1] = fmaf((float)b, wv[e], S[e][1]);
                        if (cc) S[e][2] = fmaf((float)cc, wv[e], S[e][2]);
                    }
                }
            }
        }
    u = make_float3(ux, uy, uz);
    if (APIC) {
        const float s4 = 4.f * (float)N, fx[3] = {sx.fx, sy.fx, sz.fx}, ue[3] = {ux, uy, uz};
#pragma unroll
        for (int e = 0; e < 3; ++e)
#pragma unroll
            for (int f = 0; f < 3; ++f) c[3 * e + f] = s4 * fmaf(-fx[f], ue[e], S[e][f]);
    }
}

// Quadratic B-spline weight of stencil offset t (0, 1, 2) at spline offset f
// as a polynomial in f: 0.5(1.5-f)^2, 0.75-(f-1)^2, 0.5(f-0.5)^2.
struct BsPoly {
    float a2, a1, a0;
};
__device__ __forceinline__ BsPoly bs_poly(int t)
{
    BsPoly c;
    c.a2 = (t == 1) ? -1.f : 0.5f;
    c.a1 = (t == 0) ? -1.5f : ((t == 1) ? 2.f : -0.5f);
    c.a0 = (t == 0) ? 1.125f : ((t == 1) ? -0.25f : 0.125f);
    return c;
}
__device__ __forceinline__ float bs_eval(const BsPoly &c, float f) { return fmaf(fmaf(c.a2, f, c.a1), f, c.a0); }

}  // namespace sg
