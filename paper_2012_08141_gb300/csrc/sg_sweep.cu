// sg_sweep.cu -- register-sweep stencil kernels over 8^3 leaves.
//
// Same operations as the staged kernels in sg_stencil.cu (7-point diffusion,
// 27-point box smoothing, and their fusion with the sum; AsyncTaichi Sec. 6.4
// and Sec. 6.5 for the fusion and the dead intermediate), organised so that
// the hot loop touches no shared memory:
//   - a lane owns one k-row column of a leaf's region (all k values of one
//     (j) column) and sweeps along i, keeping the rows of consecutive i
//     planes in registers;
//   - x rows come straight from L2/HBM (read-only path), the row of plane
//     i+3 being requested while plane i is computed;
//   - the j-1 / j+1 rows are the neighbouring lanes' rows, taken by warp
//     shuffle; in the triple sweep the two edge lanes of a leaf load their
//     outer row, in the j-run sweep (the default fused kernel) lanes of a run
//     of j-adjacent leaves hold every row, the two outermost lanes x only;
//   - the 3x3x3 box sum is separable: a j-sum by shuffle, an i-sum over a
//     sliding window of the last three planes, a k-sum inside the row.
// A row of the 12^3 (fused) or 10^3 (single) region is gathered from the
// three leaves (dk = -1, 0, +1) of its column via the 27-neighbour table,
// the own leaf's 8 floats in one 256-bit load.  A null neighbour is the zero
// leaf, so every load is unconditional; an inactive voxel reads 0 because
// the stored value there is 0.
#include <atomic>
#include "sg_common.cuh"

namespace sg {

constexpr int kSweepThreads = 128;

__device__ __forceinline__ float4 ldg4s(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float2 ldg2s(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ void stg4(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ float pick(uint32_t bits, int k, float v) { return ((bits >> k) & 1u) ? v : 0.f; }

// Eager activation check of one written 8-voxel row of the own leaf.
__device__ __forceinline__ void sweep_check_row(const DevGrid &g, int slot, int row, uint32_t bits)
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
// Row gathers.
// row12: region k r = 0..11 <- k- leaf local 6,7 | own 0..7 | k+ leaf local 0,1
//        (+ 12 mask bits in the same order); used by the 2-voxel-halo fusion.
// row10: region k r = 0..9  <- k- leaf local 7 | own 0..7 | k+ leaf local 0;
//        used by the 1-voxel-halo single stencils.
// `ro` = (li*8 + lj) is the row index inside a leaf.
// ---------------------------------------------------------------------------
// One 32-byte aligned leaf row (8 floats) in a single 256-bit load.
__device__ __forceinline__ void ldg8(const float *p, float (&v)[8])
{
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
}

// Slots s0, s1, s2 are always valid: a null neighbour is the zero leaf.
__device__ __forceinline__ void row12v(const float *__restrict__ x, int s0, int s1, int s2, int ro, float (&v)[12])
{
    const float2 a = ldg2s(x + (long long)s0 * 512 + ro * 8 + 6);
    float c[8];
    ldg8(x + (long long)s1 * 512 + ro * 8, c);
    const float2 b = ldg2s(x + (long long)s2 * 512 + ro * 8);
    v[0] = a.x; v[1] = a.y;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q + 2] = c[q];
    v[10] = b.x; v[11] = b.y;
}

__device__ __forceinline__ void row12(const float *__restrict__ x, const uint8_t *__restrict__ mb, int s0, int s1,
                                      int s2, int ro, float (&v)[12], uint32_t &m)
{
    row12v(x, s0, s1, s2, ro, v);
    const uint32_t m0 = __ldg(mb + (long long)s0 * 64 + ro);
    const uint32_t m1 = __ldg(mb + (long long)s1 * 64 + ro);
    const uint32_t m2 = __ldg(mb + (long long)s2 * 64 + ro);
    m = (m0 >> 6) | (m1 << 2) | ((m2 & 3u) << 10);
}

__device__ __forceinline__ void row10(const float *__restrict__ x, int s0, int s1, int s2, int ro, float (&v)[10])
{
    v[0] = __ldg(x + (long long)s0 * 512 + ro * 8 + 7);
    float c[8];
    ldg8(x + (long long)s1 * 512 + ro * 8, c);
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q + 1] = c[q];
    v[9] = __ldg(x + (long long)s2 * 512 + ro * 8);
}

template <int N>
__device__ __forceinline__ void shfl_row(const float (&v)[N], float (&up)[N], float (&dn)[N])
{
#pragma unroll
    for (int q = 0; q < N; ++q) {
        up[q] = __shfl_up_sync(kFull, v[q], 1);
        dn[q] = __shfl_down_sync(kFull, v[q], 1);
    }
}

// Plane index -> (neighbour row di+1, local i) for a region whose own leaf
// starts at plane `h` (h = 2: 12^3 region, h = 1: 10^3 region).
template <int H>
__device__ __forceinline__ constexpr int plane_di(int ri) { return ri < H ? 0 : (ri < H + 8 ? 1 : 2); }
template <int H>
__device__ __forceinline__ constexpr int plane_li(int ri) { return (ri - H) & 7; }

// ---------------------------------------------------------------------------
// Fused diffuse7 -> box27 (+ sum).  A lane owns one t-region column tj of a
// leaf (region column rj = tj + 1); three leaves per warp.  Step s = 0..9
// computes the t plane ti = s (region plane s + 1) from x planes s, s+1, s+2,
// forms its j-sums P, and once three P planes exist writes output plane s - 2.
// ---------------------------------------------------------------------------
// One lane's part of a warp's sweep: t-region column tj (0..9) of list entry
// e, or, if !valid, zero rows that only take part in the shuffles.  For a
// lane with tj = 1..8 the lanes below and above it in the warp must hold the
// rows of the same leaf's region at j - 1 and j + 1 (a lane with tj = 0 or 9
// loads its outer row itself).  Returns this lane's FP32 sum of the outputs
// it wrote.
template <bool STORE_T, bool CHECK, bool SUM>
__device__ __forceinline__ float sweep_db_lane(const DevGrid &g, const float *__restrict__ x, float *__restrict__ y,
                                               float *__restrict__ tout, float coef, int e, int tj, bool valid)
{
    const int rj = tj + 1;
    const int djx = (rj < 2) ? 0 : (rj < 10 ? 1 : 2);
    const int lj = (rj - 2) & 7;
    const int lje = (tj == 0) ? 6 : 1;      // edge lanes' outer row: region column 0 or 11
    const bool lo_edge = (tj == 0), hi_edge = (tj == 9);
    const bool outlane = (tj >= 1 && tj <= 8);
    const float c6 = 1.f - 6.f * coef;
    const int Z = (int)g.cap;  // the zero leaf
    {
        int sl[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) sl[q] = valid ? __ldg(g.nbr + (long long)e * 27 + (q / 3) * 9 + djx * 3 + (q % 3)) : Z;
        const int own = sl[4];
        const bool edge = lo_edge || hi_edge;
        // activity bits of this lane's t-region column, 10 rows x 10 bits
        uint4 rm = make_uint4(0u, 0u, 0u, 0u);
        if (valid) rm = __ldg(reinterpret_cast<const uint4 *>(g.rmask + (long long)e * 40 + tj * 4));
        const uint32_t rmw[4] = {rm.x, rm.y, rm.z, rm.w};
        float xa[12], xb[12], xc[12], xn[12], ea[12], eb[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) xn[q] = 0.f;
        // planes 0, 1, 2 and the edge rows of plane 1
        row12v(x, sl[0], sl[1], sl[2], plane_li<2>(0) * 8 + lj, xa);
        row12v(x, sl[0], sl[1], sl[2], plane_li<2>(1) * 8 + lj, xb);
        row12v(x, sl[3], sl[4], sl[5], plane_li<2>(2) * 8 + lj, xc);
        row12v(x, edge ? sl[0] : Z, edge ? sl[1] : Z, edge ? sl[2] : Z, plane_li<2>(1) * 8 + lje, ea);
        float p1[10], p2[10];
        uint32_t mprev = 0;
        float part = 0.f;
#pragma unroll
        for (int s = 0; s < 10; ++s) {
            // prefetch plane s+3 (centre row) and the edge row of plane s+2
            if (s + 3 <= 11) {
                const int ri = s + 3, dx = plane_di<2>(ri) * 3;
                row12v(x, sl[dx], sl[dx + 1], sl[dx + 2], plane_li<2>(ri) * 8 + lj, xn);
            }
            {
                const int ri = s + 2, dx = plane_di<2>(ri) * 3;
                row12v(x, edge ? sl[dx] : Z, edge ? sl[dx + 1] : Z, edge ? sl[dx + 2] : Z, plane_li<2>(ri) * 8 + lje, eb);
            }
            const uint32_t mt = (rmw[s / 3] >> (10 * (s % 3))) & 0x3ffu;  // t row bits, bit q <-> t[q]
            // t on region plane s+1 (centre xb, i-1 xa, i+1 xc)
            float up[12], dn[12];
            shfl_row<12>(xb, up, dn);
            float t[10];
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                const float jm = lo_edge ? ea[q + 1] : up[q + 1];
                const float jp = hi_edge ? ea[q + 1] : dn[q + 1];
                const float nb = ((xb[q] + xb[q + 2]) + (xa[q + 1] + xc[q + 1])) + (jm + jp);
                t[q] = pick(mt, q, fmaf(coef, nb, c6 * xb[q + 1]));
            }
            if (STORE_T && s >= 1 && s <= 8 && outlane && valid) {
                const int orow = (s - 1) * 8 + (tj - 1);
                if (CHECK) sweep_check_row(g, own, orow, (mt >> 1) & 0xffu);
                float *o = tout + (long long)own * 512 + orow * 8;
                stg4(o, t[1], t[2], t[3], t[4]);
                stg4(o + 4, t[5], t[6], t[7], t[8]);
            }
            // j-sums of t
            float tu[10], td[10], p0[10];
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                tu[q] = __shfl_up_sync(kFull, t[q], 1);
                td[q] = __shfl_down_sync(kFull, t[q], 1);
            }
#pragma unroll
            for (int q = 0; q < 10; ++q) p0[q] = (tu[q] + t[q]) + td[q];
            if (s >= 2) {
                float S[10];
#pragma unroll
                for (int q = 0; q < 10; ++q) S[q] = (p2[q] + p1[q]) + p0[q];
                const uint32_t bits = (mprev >> 1) & 0xffu;  // own voxels of t row s-1
                float o[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) o[k] = pick(bits, k, ((S[k] + S[k + 1]) + S[k + 2]) * (1.f / 27.f));
                if (outlane && valid) {
                    const int orow = (s - 2) * 8 + (tj - 1);
                    if (CHECK) sweep_check_row(g, own, orow, bits);
                    float *op = y + (long long)own * 512 + orow * 8;
                    stg4(op, o[0], o[1], o[2], o[3]);
                    stg4(op + 4, o[4], o[5], o[6], o[7]);
                    if (SUM) part += ((o[0] + o[1]) + (o[2] + o[3])) + ((o[4] + o[5]) + (o[6] + o[7]));
                }
            }
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                p2[q] = p1[q];
                p1[q] = p0[q];
            }
            mprev = mt;
            // slide the plane window
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                xa[q] = xb[q];
                xb[q] = xc[q];
                xc[q] = xn[q];
                ea[q] = eb[q];
            }
        }
        return part;
    }
}

// One warp, one leaf triple: list entries e0, e0+1, e0+2 of grid g (entries
// >= n are skipped); lanes 10*w + tj, w = 0..2, tj = 0..9 take t-region column
// tj of leaf w, lanes 30, 31 only take part in the shuffles.
template <bool STORE_T, bool CHECK, bool SUM>
__device__ __forceinline__ float sweep_db_triple(const DevGrid &g, const float *__restrict__ x, float *__restrict__ y,
                                                 float *__restrict__ tout, float coef, int e0, int n)
{
    const int sub = lane_id() / 10;
    const int e = e0 + sub;
    return sweep_db_lane<STORE_T, CHECK, SUM>(g, x, y, tout, coef, e, lane_id() - sub * 10, sub < 3 && e < n);
}

// ---------------------------------------------------------------------------
// Column sweeps: the same fused step over a run of G leaves adjacent in i
// (G <= 3), swept in one pass, so the i-halo planes between them are loaded
// and the t planes between them computed once: 8G + 4 x planes and 8G + 2 t
// planes instead of 12G and 10G.  A warp takes three columns of the same G
// (lanes 10*w + tj as in the triple sweep); the columns come from the list by
// k_column_groups.  x plane ri of a column: ri < 2 the i-1 neighbour of its
// first leaf, ri >= 8G + 2 the i+1 neighbour of its last, else leaf
// (ri - 2) / 8; local plane (ri - 2) & 7.
// ---------------------------------------------------------------------------
// One step of the column sweep: t plane s from the x window (xa, xb, xc =
// planes s, s+1, s+2; ea = the edge row of plane s+1), its j-sums p0, and,
// from s = 2 on, output plane s - 2 into `own`.  Returns the output sum.
template <bool STORE_T, bool CHECK, bool SUM>
__device__ __forceinline__ float column_step(const DevGrid &g, float *__restrict__ y, float *__restrict__ tout,
                                             float coef, float c6, int tj, bool lo_edge, bool hi_edge, bool outlane,
                                             bool valid, uint32_t mt, uint32_t mprev, bool out, int own, int t_own,
                                             int t_plane, int o_plane, const float (&xa)[12], const float (&xb)[12],
                                             const float (&xc)[12], const float (&ea)[12], float (&p1)[10],
                                             float (&p2)[10])
{
    float up[12], dn[12];
    shfl_row<12>(xb, up, dn);
    float t[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        const float jm = lo_edge ? ea[q + 1] : up[q + 1];
        const float jp = hi_edge ? ea[q + 1] : dn[q + 1];
        const float nb = ((xb[q] + xb[q + 2]) + (xa[q + 1] + xc[q + 1])) + (jm + jp);
        t[q] = pick(mt, q, fmaf(coef, nb, c6 * xb[q + 1]));
    }
    if (STORE_T && t_plane >= 0 && outlane && valid) {
        const int orow = t_plane * 8 + (tj - 1);
        if (CHECK) sweep_check_row(g, t_own, orow, (mt >> 1) & 0xffu);
        float *o = tout + (long long)t_own * 512 + orow * 8;
        stg4(o, t[1], t[2], t[3], t[4]);
        stg4(o + 4, t[5], t[6], t[7], t[8]);
    }
    float tu[10], td[10], p0[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        tu[q] = __shfl_up_sync(kFull, t[q], 1);
        td[q] = __shfl_down_sync(kFull, t[q], 1);
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) p0[q] = (tu[q] + t[q]) + td[q];
    float part = 0.f;
    if (out) {
        float S[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) S[q] = (p2[q] + p1[q]) + p0[q];
        const uint32_t bits = (mprev >> 1) & 0xffu;
        float o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = pick(bits, k, ((S[k] + S[k + 1]) + S[k + 2]) * (1.f / 27.f));
        if (outlane && valid) {
            const int orow = o_plane * 8 + (tj - 1);
            if (CHECK) sweep_check_row(g, own, orow, bits);
            float *op = y + (long long)own * 512 + orow * 8;
            stg4(op, o[0], o[1], o[2], o[3]);
            stg4(op + 4, o[4], o[5], o[6], o[7]);
            if (SUM) part = ((o[0] + o[1]) + (o[2] + o[3])) + ((o[4] + o[5]) + (o[6] + o[7]));
        }
    }
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        p2[q] = p1[q];
        p1[q] = p0[q];
    }
    return part;
}

__device__ __forceinline__ void slide(float (&xa)[12], float (&xb)[12], float (&xc)[12], const float (&xn)[12],
                                      float (&ea)[12], const float (&eb)[12])
{
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        xa[q] = xb[q];
        xb[q] = xc[q];
        xc[q] = xn[q];
        ea[q] = eb[q];
    }
}

// The column of G <= 3 leaves (list entries rec[0 .. G-1]) for this lane's
// sub-warp.  A prologue computes t planes 0 and 1 from the i-1 halo of the
// first leaf; then a loop over the leaves m computes, in eight unrolled steps
// each, t planes 8m + 2 .. 8m + 9 and output planes 8m .. 8m + 7 of leaf m.
// The slots of leaf m ("cur") and of the next leaf, or the i+1 halo after
// the last one ("nxt"), roll along, so the code is the same for every leaf
// and every G.
template <bool STORE_T, bool CHECK, bool SUM>
__device__ __forceinline__ float sweep_db_column(const DevGrid &g, const float *__restrict__ x, float *__restrict__ y,
                                                 float *__restrict__ tout, float coef, const int32_t *rec, int G,
                                                 bool valid)
{
    const int lane = lane_id();
    const int sub = lane / 10;
    const int tj = lane - sub * 10;
    const int rj = tj + 1;
    const int djx = (rj < 2) ? 0 : (rj < 10 ? 1 : 2);
    const int lj = (rj - 2) & 7;
    const int lje = (tj == 0) ? 6 : 1;
    const bool lo_edge = (tj == 0), hi_edge = (tj == 9);
    const bool outlane = (tj >= 1 && tj <= 8);
    const float c6 = 1.f - 6.f * coef;
    const int Z = (int)g.cap;
    const bool edge = lo_edge || hi_edge;
    auto slots = [&](int e, int dirow, int (&sl)[3]) {
#pragma unroll
        for (int d = 0; d < 3; ++d) sl[d] = valid ? __ldg(g.nbr + (long long)e * 27 + dirow * 9 + djx * 3 + d) : Z;
    };
    auto row = [&](const int (&sl)[3], int local, float(&v)[12]) { row12v(x, sl[0], sl[1], sl[2], local * 8 + lj, v); };
    auto erow = [&](const int (&sl)[3], int local, float(&v)[12]) {
        row12v(x, edge ? sl[0] : Z, edge ? sl[1] : Z, edge ? sl[2] : Z, local * 8 + lje, v);
    };
    auto mword = [&](int e, int r) -> uint32_t {
        return valid ? (__ldg(g.rmask + (long long)e * 40 + tj * 4 + r / 3) >> (10 * (r % 3))) & 0x3ffu : 0u;
    };
    int e_cur = valid ? __ldg(rec) : 0;
    int e_nxt = (valid && G > 1) ? __ldg(rec + 1) : -1;
    int lo[3], cur[3], nxt[3];
    slots(e_cur, 0, lo);
    slots(e_cur, 1, cur);
    if (G > 1) slots(e_nxt, 1, nxt);
    else slots(e_cur, 2, nxt);
    float xa[12], xb[12], xc[12], xn[12], ea[12], eb[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) xn[q] = 0.f;
    row(lo, 6, xa);
    row(lo, 7, xb);
    row(cur, 0, xc);
    erow(lo, 7, ea);
    float p1[10], p2[10];
    float part = 0.f;
    // prologue: t planes 0, 1 (rows 0, 1 of leaf 0's t-region mask)
    uint32_t m0 = mword(e_cur, 0), m1 = mword(e_cur, 1);
    row(cur, 1, xn);
    erow(cur, 0, eb);
    part += column_step<STORE_T, CHECK, SUM>(g, y, tout, coef, c6, tj, lo_edge, hi_edge, outlane, valid, m0, 0u, false,
                                              0, 0, -1, 0, xa, xb, xc, ea, p1, p2);
    slide(xa, xb, xc, xn, ea, eb);
    row(cur, 2, xn);
    erow(cur, 1, eb);
    part += column_step<STORE_T, CHECK, SUM>(g, y, tout, coef, c6, tj, lo_edge, hi_edge, outlane, valid, m1, m0, false,
                                              0, cur[1], 0, 0, xa, xb, xc, ea, p1, p2);
    slide(xa, xb, xc, xn, ea, eb);
    uint32_t mprev = m1;
    for (int m = 0; m < G; ++m) {
        const bool last = m == G - 1;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            // x plane 8m + k + 5 (local (k + 3) & 7 of leaf m, or of the next
            // leaf / the i+1 halo from k = 5); none after the last halo plane
            if (k <= 4) row(cur, k + 3, xn);
            else if (!(last && k == 7)) row(nxt, k - 5, xn);
            // edge row of x plane 8m + k + 4
            if (k <= 5) erow(cur, k + 2, eb);
            else erow(nxt, k - 6, eb);
            // t plane 8m + k + 2: row k + 2 of leaf m's mask, or row 1 of the
            // next leaf's for k = 7 (row 9 of leaf m after the last leaf)
            const uint32_t mt = k < 7 ? mword(e_cur, k + 2) : (last ? mword(e_cur, 9) : mword(e_nxt, 1));
            const int t_own = k < 7 ? cur[1] : nxt[1];
            const int t_plane = k < 7 ? k + 1 : (last ? -1 : 0);
            part += column_step<STORE_T, CHECK, SUM>(g, y, tout, coef, c6, tj, lo_edge, hi_edge, outlane, valid, mt,
                                                      mprev, true, cur[1], t_own, t_plane, k, xa, xb, xc, ea, p1, p2);
            mprev = mt;
            slide(xa, xb, xc, xn, ea, eb);
        }
        // roll the slots: leaf m + 1 becomes current, the one after it (or
        // the i+1 halo of the last leaf) next
        if (!last) {
#pragma unroll
            for (int d = 0; d < 3; ++d) cur[d] = nxt[d];
            e_cur = e_nxt;
            if (m + 2 < G) {
                e_nxt = valid ? __ldg(rec + m + 2) : -1;
                slots(e_nxt, 1, nxt);
            } else {
                slots(e_cur, 2, nxt);
            }
        }
    }
    return part;
}

// Fused diffuse7 -> box27 (+ sum) over the columns of one grid: the column
// records are bucketed by length (G = 3, 2, 1 at grp + (G - 1) * cap * 3, three
// entries each, counts in cnt[G - 1]); warps stride over tasks of three
// columns of one length, the longest first.
template <bool STORE_T, bool CHECK, bool SUM>
__global__ void __launch_bounds__(kSweepThreads, 3) k_sweep_columns(DevGrid g, int src, int tmp, int dst, float coef,
                                                                   int sum_slot)
{
    __shared__ double s_red[kSweepThreads / 32];
    const long long cap3 = g.cap * 3;
    const int c3 = g.col_cnt[2], c2 = g.col_cnt[1], c1 = g.col_cnt[0];
    const int t3 = (c3 + 2) / 3, t2 = (c2 + 2) / 3, t1 = (c1 + 2) / 3;
    const int warps_total = gridDim.x * (kSweepThreads / 32);
    const int sub = lane_id() / 10;
    double acc = 0.0;
    for (int t = blockIdx.x * (kSweepThreads / 32) + (threadIdx.x >> 5); t < t3 + t2 + t1; t += warps_total) {
        const int G = t < t3 ? 3 : (t < t3 + t2 ? 2 : 1);
        const int j = 3 * (t < t3 ? t : (t < t3 + t2 ? t - t3 : t - t3 - t2)) + sub;
        const int cnt = G == 3 ? c3 : (G == 2 ? c2 : c1);
        acc += (double)sweep_db_column<STORE_T, CHECK, SUM>(g, g.field[src], g.field[dst], g.field[tmp], coef,
                                                            g.col_grp + (G - 1) * cap3 + 3LL * j, G,
                                                            sub < 3 && j < cnt);
    }
    if (SUM) {
        acc = warp_sum(acc);
        if (lane_id() == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        double tot = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < kSweepThreads / 32; ++w) tot += s_red[w];
        finish_reduction(g, tot, sum_slot);
    }
}

// ---------------------------------------------------------------------------
// j-run sweeps (the default fused kernel): the same fused step with a warp's
// leaves taken from runs of leaves adjacent in j (records built by
// k_region_masks along j, bucketed by length G = 3, 2, 1).  A run piece of G
// leaves takes 8G + 4 consecutive lanes, j = -2 .. 8G + 1 from its lowest
// leaf: the rows at the faces between its leaves are lanes' own rows, loaded
// once, and the two outer lanes only hold the x rows at j = -2 and 8G + 1
// (t-region columns tj = -1 and 10, whose t is never used), so every t lane
// takes its j - 1 / j + 1 rows by shuffle and no lane loads or holds an edge
// row.  That frees the registers for four CTAs per SM.  Tasks: one piece of
// three (28 lanes), a piece of two with a piece of one (32 lanes) or alone,
// or two pieces of one.  Every t and output value takes the same operands in
// the same order as in the triple sweep, so the results are identical.
// ---------------------------------------------------------------------------
// One lane's part: region column tj (-1 .. 10) of list entry e, or, if
// !valid, zero rows.  Returns this lane's FP32 sum of the outputs it wrote.
template <bool STORE_T, bool CHECK, bool SUM>
__device__ __forceinline__ float sweep_db_jrun_lane(const DevGrid &g, const float *__restrict__ x, float *__restrict__ y,
                                                 float *__restrict__ tout, float coef, int e, int tj, bool valid)
{
    const int rj = tj + 1;  // region column 0..11
    const int djx = (rj < 2) ? 0 : (rj < 10 ? 1 : 2);
    const int lj = (rj - 2) & 7;
    const bool tlane = valid && tj >= 0 && tj <= 9;
    const bool outlane = valid && tj >= 1 && tj <= 8;
    const float c6 = 1.f - 6.f * coef;
    const int Z = (int)g.cap;  // the zero leaf
    int sl[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) sl[q] = valid ? __ldg(g.nbr + (long long)e * 27 + (q / 3) * 9 + djx * 3 + (q % 3)) : Z;
    const int own = sl[4];
    uint4 rm = make_uint4(0u, 0u, 0u, 0u);
    if (tlane) rm = __ldg(reinterpret_cast<const uint4 *>(g.rmask + (long long)e * 40 + tj * 4));
    const uint32_t rmw[4] = {rm.x, rm.y, rm.z, rm.w};
    float xa[12], xb[12], xc[12], xn[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) xn[q] = 0.f;
    row12v(x, sl[0], sl[1], sl[2], plane_li<2>(0) * 8 + lj, xa);
    row12v(x, sl[0], sl[1], sl[2], plane_li<2>(1) * 8 + lj, xb);
    row12v(x, sl[3], sl[4], sl[5], plane_li<2>(2) * 8 + lj, xc);
    float p1[10], p2[10];
    uint32_t mprev = 0;
    float part = 0.f;
#pragma unroll
    for (int s = 0; s < 10; ++s) {
        if (s + 3 <= 11) {
            const int ri = s + 3, dx = plane_di<2>(ri) * 3;
            row12v(x, sl[dx], sl[dx + 1], sl[dx + 2], plane_li<2>(ri) * 8 + lj, xn);
        }
        const uint32_t mt = (rmw[s / 3] >> (10 * (s % 3))) & 0x3ffu;
        float up[12], dn[12];
        shfl_row<12>(xb, up, dn);
        float t[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            const float nb = ((xb[q] + xb[q + 2]) + (xa[q + 1] + xc[q + 1])) + (up[q + 1] + dn[q + 1]);
            t[q] = pick(mt, q, fmaf(coef, nb, c6 * xb[q + 1]));
        }
        if (STORE_T && s >= 1 && s <= 8 && outlane) {
            const int orow = (s - 1) * 8 + (tj - 1);
            if (CHECK) sweep_check_row(g, own, orow, (mt >> 1) & 0xffu);
            float *o = tout + (long long)own * 512 + orow * 8;
            stg4(o, t[1], t[2], t[3], t[4]);
            stg4(o + 4, t[5], t[6], t[7], t[8]);
        }
        float tu[10], td[10], p0[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            tu[q] = __shfl_up_sync(kFull, t[q], 1);
            td[q] = __shfl_down_sync(kFull, t[q], 1);
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) p0[q] = (tu[q] + t[q]) + td[q];
        if (s >= 2) {
            float S[10];
#pragma unroll
            for (int q = 0; q < 10; ++q) S[q] = (p2[q] + p1[q]) + p0[q];
            const uint32_t bits = (mprev >> 1) & 0xffu;
            float o[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) o[k] = pick(bits, k, ((S[k] + S[k + 1]) + S[k + 2]) * (1.f / 27.f));
            if (outlane) {
                const int orow = (s - 2) * 8 + (tj - 1);
                if (CHECK) sweep_check_row(g, own, orow, bits);
                float *op = y + (long long)own * 512 + orow * 8;
                stg4(op, o[0], o[1], o[2], o[3]);
                stg4(op + 4, o[4], o[5], o[6], o[7]);
                if (SUM) part += ((o[0] + o[1]) + (o[2] + o[3])) + ((o[4] + o[5]) + (o[6] + o[7]));
            }
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            p2[q] = p1[q];
            p1[q] = p0[q];
        }
        mprev = mt;
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            xa[q] = xb[q];
            xb[q] = xc[q];
            xc[q] = xn[q];
        }
    }
    return part;
}

// This lane's list entry and region column (-1 .. 10) in task t; false for
// lanes outside every piece.  c3, c2, c1: the bucket counts.
__device__ __forceinline__ bool jrun_lane(const DevGrid &g, int t, int c3, int c2, int c1, int &e, int &tj)
{
    const int lane = lane_id();
    const long long cap3 = g.cap * 3;
    const int p = c2 < c1 ? c2 : c1;
    const int32_t *rec = nullptr;
    int G = 0, start = 0;
    if (t < c3) {
        if (lane < 28) { rec = g.col_grp + 2 * cap3 + 3LL * t; G = 3; }
    } else if (t < c3 + c2) {
        const int r = t - c3;
        if (lane < 20) { rec = g.col_grp + cap3 + 3LL * r; G = 2; }
        else if (r < p) { rec = g.col_grp + 3LL * r; G = 1; start = 20; }
    } else {
        const int k = lane / 12, q = p + 2 * (t - c3 - c2) + k;
        if (k < 2 && q < c1) { rec = g.col_grp + 3LL * q; G = 1; start = 12 * k; }
    }
    if (!rec) return false;
    const int jj = lane - start - 2;                    // -2 .. 8G + 1
    const int m = jj < 0 ? 0 : min(jj >> 3, G - 1);
    tj = jj - 8 * m + 1;
    e = __ldg(rec + m);
    return true;
}

template <bool STORE_T, bool CHECK, bool SUM>
// Four CTAs of four warps per SM (at most 128 registers a thread).
__global__ void __launch_bounds__(kSweepThreads, 4) k_sweep_jruns(DevGrid g, int src, int tmp, int dst, float coef,
                                                                 int sum_slot)
{
    __shared__ double s_red[kSweepThreads / 32];
    const int c3 = g.col_cnt[2], c2 = g.col_cnt[1], c1 = g.col_cnt[0];
    const int p = c2 < c1 ? c2 : c1;
    const int tasks = c3 + c2 + (c1 - p + 1) / 2;
    const int warps_total = gridDim.x * (kSweepThreads / 32);
    double acc = 0.0;
    for (int t = blockIdx.x * (kSweepThreads / 32) + (threadIdx.x >> 5); t < tasks; t += warps_total) {
        int e = 0, tj = 0;
        const bool valid = jrun_lane(g, t, c3, c2, c1, e, tj);
        acc += (double)sweep_db_jrun_lane<STORE_T, CHECK, SUM>(g, g.field[src], g.field[dst], g.field[tmp], coef, e, tj,
                                                            valid);
    }
    if (SUM) {
        acc = warp_sum(acc);
        if (lane_id() == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        double tot = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < kSweepThreads / 32; ++w) tot += s_red[w];
        finish_reduction(g, tot, sum_slot);
    }
}


// Fused diffuse7 -> box27 (+ sum) over one grid's list: warps stride over
// leaf triples.
template <bool STORE_T, bool CHECK, bool SUM>
__global__ void __launch_bounds__(kSweepThreads, 3) k_sweep_diffuse_box(DevGrid g, int src, int tmp, int dst, float coef,
                                                                       int sum_slot)
{
    __shared__ double s_red[kSweepThreads / 32];
    const int n = g.ctrl->list_n;
    const int warps_total = gridDim.x * (kSweepThreads / 32);
    const int gw = blockIdx.x * (kSweepThreads / 32) + (threadIdx.x >> 5);
    double acc = 0.0;
    for (int e0 = gw * 3; e0 < n; e0 += warps_total * 3)
        acc += (double)sweep_db_triple<STORE_T, CHECK, SUM>(g, g.field[src], g.field[dst], g.field[tmp], coef, e0, n);
    if (SUM) {
        acc = warp_sum(acc);
        if (lane_id() == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        double tot = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < kSweepThreads / 32; ++w) tot += s_red[w];
        finish_reduction(g, tot, sum_slot);
    }
}

// ---------------------------------------------------------------------------
// Single stencils with a 1-voxel halo.  Four leaves per warp: lanes 8*w + oj
// own output column oj (region column oj + 1, always in the own leaf's j
// range); the edge lanes oj = 0 / 7 also load region column 0 / 9 from the
// j-1 / j+1 neighbour leaves.
// ---------------------------------------------------------------------------
enum { SW_DIFFUSE7 = 1, SW_BOX27 = 2 };

template <int OP, bool CHECK, bool SUM>
__global__ void __launch_bounds__(kSweepThreads, 3) k_sweep_single(DevGrid g, int src, int dst, float coef, int sum_slot)
{
    __shared__ double s_red[kSweepThreads / 32];
    const int n = g.ctrl->list_n;
    const float *__restrict__ x = g.field[src];
    float *__restrict__ y = g.field[dst];
    const uint8_t *__restrict__ mb = reinterpret_cast<const uint8_t *>(g.mask);
    const int lane = lane_id();
    const int sub = lane >> 3;
    const int oj = lane & 7;
    const bool lo_edge = (oj == 0), hi_edge = (oj == 7);
    const int edx = lo_edge ? 0 : 2;        // dj+1 of the edge lanes' outer column
    const int lje = lo_edge ? 7 : 0;
    const float c6 = 1.f - 6.f * coef;
    const int Z = (int)g.cap;  // the zero leaf
    const int warps_total = gridDim.x * (kSweepThreads / 32);
    const int gw = blockIdx.x * (kSweepThreads / 32) + (threadIdx.x >> 5);
    double acc = 0.0;

    for (int e0 = gw * 4; e0 < n; e0 += warps_total * 4) {
        const int e = e0 + sub;
        const bool valid = e < n;
        int sl[9], se[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const long long base = (long long)e * 27 + (q / 3) * 9 + (q % 3);
            sl[q] = valid ? __ldg(g.nbr + base + 3) : Z;
            se[q] = (valid && (lo_edge || hi_edge)) ? __ldg(g.nbr + base + edx * 3) : Z;
        }
        const int own = sl[4];
        float xa[10], xb[10], xc[10], xn[10], ea[10], eb[10], ec[10], en[10];
#pragma unroll
        for (int q = 0; q < 10; ++q) xn[q] = en[q] = 0.f;
        row10(x, sl[0], sl[1], sl[2], plane_li<1>(0) * 8 + oj, xa);
        row10(x, sl[3], sl[4], sl[5], plane_li<1>(1) * 8 + oj, xb);
        row10(x, sl[3], sl[4], sl[5], plane_li<1>(2) * 8 + oj, xc);
        row10(x, se[3], se[4], se[5], plane_li<1>(1) * 8 + lje, eb);
        row10(x, se[3], se[4], se[5], plane_li<1>(2) * 8 + lje, ec);
        if (OP == SW_BOX27) row10(x, se[0], se[1], se[2], plane_li<1>(0) * 8 + lje, ea);
        float p1[10], p2[10];
        float part = 0.f;
        if (OP == SW_BOX27) {
            // j-sums of planes 0 and 1
            float up[10], dn[10];
            shfl_row<10>(xa, up, dn);
#pragma unroll
            for (int q = 0; q < 10; ++q) p2[q] = ((lo_edge ? ea[q] : up[q]) + xa[q]) + (hi_edge ? ea[q] : dn[q]);
            shfl_row<10>(xb, up, dn);
#pragma unroll
            for (int q = 0; q < 10; ++q) p1[q] = ((lo_edge ? eb[q] : up[q]) + xb[q]) + (hi_edge ? eb[q] : dn[q]);
        }
#pragma unroll
        for (int oi = 0; oi < 8; ++oi) {
            const uint32_t bits = valid ? __ldg(mb + (long long)own * 64 + oi * 8 + oj) : 0u;
            float o[8];
            if (OP == SW_DIFFUSE7) {
                // prefetch plane oi+3, then t on plane oi+1 from planes oi, oi+1, oi+2
                if (oi + 3 <= 9) {
                    const int ri = oi + 3, dx = plane_di<1>(ri) * 3;
                    row10(x, sl[dx], sl[dx + 1], sl[dx + 2], plane_li<1>(ri) * 8 + oj, xn);
                    row10(x, se[dx], se[dx + 1], se[dx + 2], plane_li<1>(ri) * 8 + lje, en);
                }
                float up[10], dn[10];
                shfl_row<10>(xb, up, dn);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int q = k + 1;
                    const float jm = lo_edge ? eb[q] : up[q];
                    const float jp = hi_edge ? eb[q] : dn[q];
                    const float nb = ((xb[q - 1] + xb[q + 1]) + (xa[q] + xc[q])) + (jm + jp);
                    o[k] = pick(bits, k, fmaf(coef, nb, c6 * xb[q]));
                }
#pragma unroll
                for (int q = 0; q < 10; ++q) {
                    xa[q] = xb[q];
                    xb[q] = xc[q];
                    xc[q] = xn[q];
                    eb[q] = ec[q];
                    ec[q] = en[q];
                }
            } else {
                // prefetch plane oi+3; j-sum of plane oi+2; output plane oi
                if (oi + 3 <= 9) {
                    const int ri = oi + 3, dx = plane_di<1>(ri) * 3;
                    row10(x, sl[dx], sl[dx + 1], sl[dx + 2], plane_li<1>(ri) * 8 + oj, xn);
                    row10(x, se[dx], se[dx + 1], se[dx + 2], plane_li<1>(ri) * 8 + lje, en);
                }
                float up[10], dn[10], p0[10];
                shfl_row<10>(xc, up, dn);
#pragma unroll
                for (int q = 0; q < 10; ++q) p0[q] = ((lo_edge ? ec[q] : up[q]) + xc[q]) + (hi_edge ? ec[q] : dn[q]);
                float S[10];
#pragma unroll
                for (int q = 0; q < 10; ++q) S[q] = (p2[q] + p1[q]) + p0[q];
#pragma unroll
                for (int k = 0; k < 8; ++k) o[k] = pick(bits, k, ((S[k] + S[k + 1]) + S[k + 2]) * (1.f / 27.f));
#pragma unroll
                for (int q = 0; q < 10; ++q) {
                    p2[q] = p1[q];
                    p1[q] = p0[q];
                    xc[q] = xn[q];
                    ec[q] = en[q];
                }
            }
            if (valid) {
                const int orow = oi * 8 + oj;
                if (CHECK) sweep_check_row(g, own, orow, bits);
                float *op = y + (long long)own * 512 + orow * 8;
                stg4(op, o[0], o[1], o[2], o[3]);
                stg4(op + 4, o[4], o[5], o[6], o[7]);
                if (SUM) part += ((o[0] + o[1]) + (o[2] + o[3])) + ((o[4] + o[5]) + (o[6] + o[7]));
            }
        }
        acc += (double)part;
    }
    if (SUM) {
        acc = warp_sum(acc);
        if (lane_id() == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        double tot = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < kSweepThreads / 32; ++w) tot += s_red[w];
        finish_reduction(g, tot, sum_slot);
    }
}

// ---------------------------------------------------------------------------
// Single stencils over j-runs: the layout of the fused j-run sweep for a
// 1-voxel halo.  A run piece of G leaves takes 8G + 2 consecutive lanes, j =
// -1 .. 8G from its lowest leaf; the two outer lanes hold only the x rows of
// the j-neighbour leaves, so every output lane takes its j - 1 / j + 1 rows
// by shuffle and no lane loads an edge row.  Tasks: one piece of three (26
// lanes), a piece of two with a piece of one (28 lanes) or alone, or three
// pieces of one (30 lanes).  Every output takes the same operands in the
// same order as in k_sweep_single (an edge lane's outer row there is the
// x-only lane's row here), so the results are identical.
// ---------------------------------------------------------------------------
// This lane's list entry and column lj (-1 .. 8, relative to that entry's
// leaf) in task t; false for lanes outside every piece.
__device__ __forceinline__ bool jrun1_lane(const DevGrid &g, int t, int c3, int c2, int c1, int &e, int &lj)
{
    const int lane = lane_id();
    const long long cap3 = g.cap * 3;
    const int p = c2 < c1 ? c2 : c1;
    const int32_t *rec = nullptr;
    int G = 0, start = 0;
    if (t < c3) {
        if (lane < 26) { rec = g.col_grp + 2 * cap3 + 3LL * t; G = 3; }
    } else if (t < c3 + c2) {
        const int r = t - c3;
        if (lane < 18) { rec = g.col_grp + cap3 + 3LL * r; G = 2; }
        else if (lane < 28 && r < p) { rec = g.col_grp + 3LL * r; G = 1; start = 18; }
    } else {
        const int k = lane / 10, q = p + 3 * (t - c3 - c2) + k;
        if (k < 3 && q < c1) { rec = g.col_grp + 3LL * q; G = 1; start = 10 * k; }
    }
    if (!rec) return false;
    const int jj = lane - start - 1;                    // -1 .. 8G
    const int m = jj < 0 ? 0 : min(jj >> 3, G - 1);
    lj = jj - 8 * m;
    e = __ldg(rec + m);
    return true;
}

template <int OP, bool CHECK, bool SUM>
__device__ __forceinline__ float sweep_single_jrun_lane(const DevGrid &g, const float *__restrict__ x,
                                                        float *__restrict__ y, float coef, int e, int lj, bool valid)
{
    const uint8_t *__restrict__ mb = reinterpret_cast<const uint8_t *>(g.mask);
    const int djx = lj < 0 ? 0 : (lj < 8 ? 1 : 2);  // the row's leaf: j-1, own, j+1
    const int lr = lj & 7;                           // the row's local j there
    const bool outlane = valid && lj >= 0 && lj <= 7;
    const float c6 = 1.f - 6.f * coef;
    const int Z = (int)g.cap;  // the zero leaf
    int sl[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) sl[q] = valid ? __ldg(g.nbr + (long long)e * 27 + (q / 3) * 9 + djx * 3 + (q % 3)) : Z;
    const int own = sl[4];  // the entry's own leaf for the output lanes
    float xa[10], xb[10], xc[10], xn[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) xn[q] = 0.f;
    row10(x, sl[0], sl[1], sl[2], plane_li<1>(0) * 8 + lr, xa);
    row10(x, sl[3], sl[4], sl[5], plane_li<1>(1) * 8 + lr, xb);
    row10(x, sl[3], sl[4], sl[5], plane_li<1>(2) * 8 + lr, xc);
    float p1[10], p2[10];
    float part = 0.f;
    if (OP == SW_BOX27) {
        // j-sums of planes 0 and 1
        float up[10], dn[10];
        shfl_row<10>(xa, up, dn);
#pragma unroll
        for (int q = 0; q < 10; ++q) p2[q] = (up[q] + xa[q]) + dn[q];
        shfl_row<10>(xb, up, dn);
#pragma unroll
        for (int q = 0; q < 10; ++q) p1[q] = (up[q] + xb[q]) + dn[q];
    }
#pragma unroll
    for (int oi = 0; oi < 8; ++oi) {
        const uint32_t bits = outlane ? __ldg(mb + (long long)own * 64 + oi * 8 + lr) : 0u;
        float o[8];
        if (oi + 3 <= 9) {  // prefetch plane oi + 3
            const int ri = oi + 3, dx = plane_di<1>(ri) * 3;
            row10(x, sl[dx], sl[dx + 1], sl[dx + 2], plane_li<1>(ri) * 8 + lr, xn);
        }
        float up[10], dn[10];
        if (OP == SW_DIFFUSE7) {
            // t on plane oi + 1 from planes oi, oi + 1, oi + 2
            shfl_row<10>(xb, up, dn);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int q = k + 1;
                const float nb = ((xb[q - 1] + xb[q + 1]) + (xa[q] + xc[q])) + (up[q] + dn[q]);
                o[k] = pick(bits, k, fmaf(coef, nb, c6 * xb[q]));
            }
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                xa[q] = xb[q];
                xb[q] = xc[q];
                xc[q] = xn[q];
            }
        } else {
            // j-sum of plane oi + 2; output plane oi
            float p0[10], S[10];
            shfl_row<10>(xc, up, dn);
#pragma unroll
            for (int q = 0; q < 10; ++q) p0[q] = (up[q] + xc[q]) + dn[q];
#pragma unroll
            for (int q = 0; q < 10; ++q) S[q] = (p2[q] + p1[q]) + p0[q];
#pragma unroll
            for (int k = 0; k < 8; ++k) o[k] = pick(bits, k, ((S[k] + S[k + 1]) + S[k + 2]) * (1.f / 27.f));
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                p2[q] = p1[q];
                p1[q] = p0[q];
                xc[q] = xn[q];
            }
        }
        if (outlane) {
            const int orow = oi * 8 + lr;
            if (CHECK) sweep_check_row(g, own, orow, bits);
            float *op = y + (long long)own * 512 + orow * 8;
            stg4(op, o[0], o[1], o[2], o[3]);
            stg4(op + 4, o[4], o[5], o[6], o[7]);
            if (SUM) part += ((o[0] + o[1]) + (o[2] + o[3])) + ((o[4] + o[5]) + (o[6] + o[7]));
        }
    }
    return part;
}

template <int OP, bool CHECK, bool SUM>
__global__ void __launch_bounds__(kSweepThreads, 4) k_sweep_single_jruns(DevGrid g, int src, int dst, float coef,
                                                                        int sum_slot)
{
    __shared__ double s_red[kSweepThreads / 32];
    const int c3 = g.col_cnt[2], c2 = g.col_cnt[1], c1 = g.col_cnt[0];
    const int p = c2 < c1 ? c2 : c1;
    const int tasks = c3 + c2 + (c1 - p + 2) / 3;
    const int warps_total = gridDim.x * (kSweepThreads / 32);
    double acc = 0.0;
    for (int t = blockIdx.x * (kSweepThreads / 32) + (threadIdx.x >> 5); t < tasks; t += warps_total) {
        int e = 0, lj = 0;
        const bool valid = jrun1_lane(g, t, c3, c2, c1, e, lj);
        acc += (double)sweep_single_jrun_lane<OP, CHECK, SUM>(g, g.field[src], g.field[dst], coef, e, lj, valid);
    }
    if (SUM) {
        acc = warp_sum(acc);
        if (lane_id() == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        double tot = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < kSweepThreads / 32; ++w) tot += s_red[w];
        finish_reduction(g, tot, sum_slot);
    }
}

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
static int sweep_ctas(int num_sms, int which)
{
    static std::atomic<int> cache[5];  // threads may race to fill it
    if (cache[which].load(std::memory_order_relaxed) == 0) {
        int per = 1;
        cudaError_t err;
        if (which == 0)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_diffuse_box<false, false, true>, kSweepThreads, 0);
        else if (which == 1)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_single<SW_BOX27, false, true>, kSweepThreads, 0);
        else if (which == 2)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_columns<false, false, true>, kSweepThreads, 0);
        else if (which == 3)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_jruns<false, false, true>, kSweepThreads, 0);
        else
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_sweep_single_jruns<SW_BOX27, false, true>,
                                                                kSweepThreads, 0);
        if (err != cudaSuccess || per < 1) per = 1;
        cache[which].store(per, std::memory_order_relaxed);
    }
    return cache[which].load(std::memory_order_relaxed) * num_sms;
}

void launch_sweep_diffuse_box(const DevGrid &g, cudaStream_t s, int src, int tmp, int dst, float coef, int store_tmp,
                              int check_act, int sum_slot, const LaunchCfg &lc)
{
    const int ctas = sweep_ctas(lc.num_sms, 0);
    const bool sum = sum_slot >= 0;
#define SG_SW(ST, CK, SU) k_sweep_diffuse_box<ST, CK, SU><<<ctas, kSweepThreads, 0, s>>>(g, src, tmp, dst, coef, sum_slot)
    if (store_tmp) {
        if (check_act) { if (sum) SG_SW(true, true, true); else SG_SW(true, true, false); }
        else { if (sum) SG_SW(true, false, true); else SG_SW(true, false, false); }
    } else {
        if (check_act) { if (sum) SG_SW(false, true, true); else SG_SW(false, true, false); }
        else { if (sum) SG_SW(false, false, true); else SG_SW(false, false, false); }
    }
#undef SG_SW
}

void launch_sweep_columns(const DevGrid &g, cudaStream_t s, int src, int tmp, int dst, float coef, int store_tmp,
                          int check_act, int sum_slot, const LaunchCfg &lc)
{
    const int ctas = sweep_ctas(lc.num_sms, 2);
    const bool sum = sum_slot >= 0;
#define SG_SC(ST, CK, SU) k_sweep_columns<ST, CK, SU><<<ctas, kSweepThreads, 0, s>>>(g, src, tmp, dst, coef, sum_slot)
    if (store_tmp) {
        if (check_act) { if (sum) SG_SC(true, true, true); else SG_SC(true, true, false); }
        else { if (sum) SG_SC(true, false, true); else SG_SC(true, false, false); }
    } else {
        if (check_act) { if (sum) SG_SC(false, true, true); else SG_SC(false, true, false); }
        else { if (sum) SG_SC(false, false, true); else SG_SC(false, false, false); }
    }
#undef SG_SC
}

void launch_sweep_jruns(const DevGrid &g, cudaStream_t s, int src, int tmp, int dst, float coef, int store_tmp,
                        int check_act, int sum_slot, const LaunchCfg &lc)
{
    const int ctas = sweep_ctas(lc.num_sms, 3);
    const bool sum = sum_slot >= 0;
#define SG_SJ(ST, CK, SU) k_sweep_jruns<ST, CK, SU><<<ctas, kSweepThreads, 0, s>>>(g, src, tmp, dst, coef, sum_slot)
    if (store_tmp) {
        if (check_act) { if (sum) SG_SJ(true, true, true); else SG_SJ(true, true, false); }
        else { if (sum) SG_SJ(true, false, true); else SG_SJ(true, false, false); }
    } else {
        if (check_act) { if (sum) SG_SJ(false, true, true); else SG_SJ(false, true, false); }
        else { if (sum) SG_SJ(false, false, true); else SG_SJ(false, false, false); }
    }
#undef SG_SJ
}

void launch_sweep_single(const DevGrid &g, cudaStream_t s, int op, int src, int dst, float coef, int check_act,
                         int sum_slot, const LaunchCfg &lc)
{
    const bool sum = sum_slot >= 0;
    if (lc.single_runs) {
        const int ctas = sweep_ctas(lc.num_sms, 4);
#define SG_SR(OP, CK, SU) k_sweep_single_jruns<OP, CK, SU><<<ctas, kSweepThreads, 0, s>>>(g, src, dst, coef, sum_slot)
        if (op == SW_DIFFUSE7) {
            if (check_act) { if (sum) SG_SR(SW_DIFFUSE7, true, true); else SG_SR(SW_DIFFUSE7, true, false); }
            else { if (sum) SG_SR(SW_DIFFUSE7, false, true); else SG_SR(SW_DIFFUSE7, false, false); }
        } else {
            if (check_act) { if (sum) SG_SR(SW_BOX27, true, true); else SG_SR(SW_BOX27, true, false); }
            else { if (sum) SG_SR(SW_BOX27, false, true); else SG_SR(SW_BOX27, false, false); }
        }
#undef SG_SR
        return;
    }
    const int ctas = sweep_ctas(lc.num_sms, 1);
#define SG_SS(OP, CK, SU) k_sweep_single<OP, CK, SU><<<ctas, kSweepThreads, 0, s>>>(g, src, dst, coef, sum_slot)
    if (op == SW_DIFFUSE7) {
        if (check_act) { if (sum) SG_SS(SW_DIFFUSE7, true, true); else SG_SS(SW_DIFFUSE7, true, false); }
        else { if (sum) SG_SS(SW_DIFFUSE7, false, true); else SG_SS(SW_DIFFUSE7, false, false); }
    } else {
        if (check_act) { if (sum) SG_SS(SW_BOX27, true, true); else SG_SS(SW_BOX27, true, false); }
        else { if (sum) SG_SS(SW_BOX27, false, true); else SG_SS(SW_BOX27, false, false); }
    }
#undef SG_SS
}

// ---------------------------------------------------------------------------
// Batched fused step: one persistent launch steps many grids.  The global
// work list is the concatenation of every grid's j-run tasks; warps stride
// over it, find their grid by binary search over the tasks' prefix sums (in
// shared memory) and run the same per-lane body as the single-grid j-run
// kernel.  Each task's output sum is added to its grid's FP64 accumulator
// (zeroed before the launch).
// ---------------------------------------------------------------------------
template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 16 / WARPS) k_batch_diffuse_box(const BatchGrid *__restrict__ items,
                                                                              int n_grids, int total_tri, float coef,
                                                                              double *acc)
{
    __shared__ int s_off[kMaxBatch + 1];
    for (int i = threadIdx.x; i <= n_grids; i += WARPS * 32) s_off[i] = (i < n_grids) ? items[i].tri0 : total_tri;
    __syncthreads();
    const int warps_total = gridDim.x * WARPS;
    for (int T = blockIdx.x * WARPS + (threadIdx.x >> 5); T < total_tri; T += warps_total) {
        int lo = 0, hi = n_grids - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= T) lo = mid;
            else hi = mid - 1;
        }
        const BatchGrid &it = items[lo];
        int e = 0, tj = 0;
        const bool valid = jrun_lane(it.g, T - s_off[lo], it.c3, it.c2, it.c1, e, tj);
        const float part = sweep_db_jrun_lane<false, false, true>(it.g, it.x, it.y, it.t, coef, e, tj, valid);
        const double w = warp_sum((double)part);
        if (lane_id() == 0) atomicAdd(&acc[lo], w);
    }
}

int batch_ctas(int num_sms, int warps)
{
    static std::atomic<int> cache[9];  // threads may race to fill it
    if (warps < 1 || warps > 8) return num_sms;
    if (cache[warps].load(std::memory_order_relaxed) == 0) {
        int per = 1;
        cudaError_t err = cudaErrorInvalidValue;
        if (warps == 2) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_diffuse_box<2>, 64, 0);
        if (warps == 4) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_diffuse_box<4>, 128, 0);
        if (warps == 8) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_diffuse_box<8>, 256, 0);
        if (err != cudaSuccess || per < 1) per = 1;
        cache[warps].store(per, std::memory_order_relaxed);
    }
    return cache[warps].load(std::memory_order_relaxed) * num_sms;
}

void launch_batch_diffuse_box(const BatchGrid *items, int n_grids, int total_tri, float coef, double *acc, int warps,
                              int num_sms, cudaStream_t s)
{
    const int ctas = batch_ctas(num_sms, warps);
    if (warps == 2) k_batch_diffuse_box<2><<<ctas, 64, 0, s>>>(items, n_grids, total_tri, coef, acc);
    else if (warps == 8) k_batch_diffuse_box<8><<<ctas, 256, 0, s>>>(items, n_grids, total_tri, coef, acc);
    else k_batch_diffuse_box<4><<<ctas, 128, 0, s>>>(items, n_grids, total_tri, coef, acc);
}

}  // namespace sg
