// sg_particle.cu -- particle-grid transfers on the sparse grid (the hybrid
// Lagrangian-Eulerian workload of AsyncTaichi Sec. 8.3): P2G with activation,
// the grid velocity update, and G2P.  Quadratic B-spline weights, PIC
// transfers; the unit cube holds N^3 nodes, dx = 1/N, node (i,j,k) at
// (i,j,k)*dx, particle component a maps to grid axis a (z -> k).
#include "sg_common.cuh"

namespace sg {

struct Spline {
    int base;
    float w[3];
};

// base = floor(X - 0.5), fx = X - base, X = x*N, all in FP32.
__device__ __forceinline__ Spline bspline(float x, int N)
{
    Spline s;
    const float X = x * (float)N;
    const float bf = floorf(X - 0.5f);
    const float fx = X - bf;
    s.base = (int)bf;
    const float a = 1.5f - fx, c = fx - 1.0f, d = fx - 0.5f;
    s.w[0] = 0.5f * a * a;
    s.w[1] = 0.75f - c * c;
    s.w[2] = 0.5f * d * d;
    return s;
}

// Mark the pointer cells the particle's 27 stencil nodes fall in.
__global__ void k_p2g_mark(DevGrid g, const float *__restrict__ x, long long n)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        int lo[3], hi[3];
        bool empty = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const Spline s = bspline(__ldg(x + 3 * p + a), g.N);
            const int n0 = max(s.base, 0), n1 = min(s.base + 2, g.N - 1);
            if (n0 > n1) empty = true;
            lo[a] = n0 >> g.lg2;
            hi[a] = n1 >> g.lg2;
        }
        if (empty) continue;
        for (int bi = lo[0]; bi <= hi[0]; ++bi)
            for (int bj = lo[1]; bj <= hi[1]; ++bj)
                for (int bk = lo[2]; bk <= hi[2]; ++bk) g.need[((long long)bi * g.R + bj) * g.R + bk] = 1;
    }
}

void launch_p2g_mark(const DevGrid &g, cudaStream_t s, const float *x, long long n)
{
    if (n <= 0) return;
    long long blocks = (n + 255) / 256;
    if (blocks > 1 << 20) blocks = 1 << 20;
    k_p2g_mark<<<(unsigned)blocks, 256, 0, s>>>(g, x, n);
}

// Scatter: set the node bits and accumulate mass and momentum with FP32
// atomics (the accumulation order is unspecified).
__global__ void __launch_bounds__(256) k_p2g_scatter(DevGrid g, const float *__restrict__ x, const float *__restrict__ v,
                                                     long long n, float pmass, int f_mass, int f_mom0)
{
    const int L = g.L, lg2 = g.lg2, N = g.N;
    float *fm = g.field[f_mass];
    float *f0 = g.field[f_mom0], *f1 = g.field[f_mom0 + 1], *f2 = g.field[f_mom0 + 2];
    bool changed = false;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const Spline sx = bspline(__ldg(x + 3 * p + 0), N);
        const Spline sy = bspline(__ldg(x + 3 * p + 1), N);
        const Spline sz = bspline(__ldg(x + 3 * p + 2), N);
        const float vx = __ldg(v + 3 * p + 0), vy = __ldg(v + 3 * p + 1), vz = __ldg(v + 3 * p + 2);
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
                for (int c = 0; c < 3; ++c) {
                    const int k = sz.base + c;
                    if ((unsigned)k >= (unsigned)N) continue;
                    const long long lb = ((long long)(i >> lg2) * g.R + (j >> lg2)) * g.R + (k >> lg2);
                    const int slot = g.root[lb];
                    if (slot < 0) continue;  // pool exhausted; error latched
                    const int l = (((i & (L - 1)) << lg2) + (j & (L - 1))) * L + (k & (L - 1));
                    uint32_t *mw = &g.mask[(long long)slot * g.W + (l >> 5)];
                    const uint32_t bit = 1u << (l & 31);
                    if (!(*mw & bit)) {
                        const uint32_t old = atomicOr(mw, bit);
                        if (!(old & bit)) changed = true;
                    }
                    const long long idx = ((long long)slot << (3 * lg2)) + l;
                    const float wm = wxy * sz.w[c] * pmass;
                    atomicAdd(fm + idx, wm);
                    atomicAdd(f0 + idx, wm * vx);
                    atomicAdd(f1 + idx, wm * vy);
                    atomicAdd(f2 + idx, wm * vz);
                }
            }
        }
    }
    if (changed) mark_dirty(g);
}

void launch_p2g_scatter(const DevGrid &g, cudaStream_t s, const float *x, const float *v, long long n, float pmass,
                        int f_mass, int f_mom0)
{
    if (n <= 0) return;
    long long blocks = (n + 255) / 256;
    if (blocks > 1 << 20) blocks = 1 << 20;
    k_p2g_scatter<<<(unsigned)blocks, 256, 0, s>>>(g, x, v, n, pmass, f_mass, f_mom0);
}

// Grid update over the active nodes of the listed leaves.
__global__ void __launch_bounds__(256) k_grid_update(DevGrid g, int f_mass, int f_mom0, float dt, float gz, int bound)
{
    const long long n = g.ctrl->list_n;
    const int L = g.L, lg2 = g.lg2, R = g.R, N = g.N, V = L * L * L;
    float *fm = g.field[f_mass];
    float *fv[3] = {g.field[f_mom0], g.field[f_mom0 + 1], g.field[f_mom0 + 2]};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * V; q += (long long)gridDim.x * blockDim.x) {
        const long long e = q >> (3 * lg2);
        const int l = (int)(q - (e << (3 * lg2)));
        const int slot = g.list_slot[e];
        if (!((g.mask[(long long)slot * g.W + (l >> 5)] >> (l & 31)) & 1u)) continue;
        const int b = g.list_b[e];
        const int idx[3] = {(b / (R * R)) * L + (l >> (2 * lg2)), ((b / R) % R) * L + ((l >> lg2) & (L - 1)),
                            (b % R) * L + (l & (L - 1))};
        const long long o = (long long)slot * V + l;
        const float m = fm[o];
        float u[3] = {0.f, 0.f, 0.f};
        if (m > 0.f) {
#pragma unroll
            for (int d = 0; d < 3; ++d) u[d] = fv[d][o] / m;
            u[2] -= dt * gz;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (idx[d] < bound && u[d] < 0.f) u[d] = 0.f;
                if (idx[d] > N - bound && u[d] > 0.f) u[d] = 0.f;
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) fv[d][o] = u[d];
    }
}

void launch_grid_update(const DevGrid &g, cudaStream_t s, int f_mass, int f_mom0, float dt, float gz, int bound,
                        const LaunchCfg &lc)
{
    k_grid_update<<<lc.num_sms * 8, 256, 0, s>>>(g, f_mass, f_mom0, dt, gz, bound);
}

// G2P: gather the node velocities (a stored value at an inactive node is 0)
// and advect the particle.
__global__ void __launch_bounds__(256) k_g2p(DevGrid g, float *__restrict__ x, float *__restrict__ v, long long n, float dt,
                                             int f_mom0, const int32_t *__restrict__ order)
{
    const int L = g.L, lg2 = g.lg2, N = g.N;
    const float *f0 = g.field[f_mom0], *f1 = g.field[f_mom0 + 1], *f2 = g.field[f_mom0 + 2];
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const long long p = order ? (long long)__ldg(order + q) : q;  // any order: particles are independent
        const float px = x[3 * p], py = x[3 * p + 1], pz = x[3 * p + 2];
        const Spline sx = bspline(px, N), sy = bspline(py, N), sz = bspline(pz, N);
        float ux = 0.f, uy = 0.f, uz = 0.f;
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
                for (int c = 0; c < 3; ++c) {
                    const int k = sz.base + c;
                    if ((unsigned)k >= (unsigned)N) continue;
                    const long long lb = ((long long)(i >> lg2) * g.R + (j >> lg2)) * g.R + (k >> lg2);
                    const int slot = __ldg(g.root + lb);
                    if (slot < 0) continue;
                    const int l = (((i & (L - 1)) << lg2) + (j & (L - 1))) * L + (k & (L - 1));
                    const long long idx = ((long long)slot << (3 * lg2)) + l;
                    const float w = wxy * sz.w[c];
                    ux += w * __ldg(f0 + idx);
                    uy += w * __ldg(f1 + idx);
                    uz += w * __ldg(f2 + idx);
                }
            }
        }
        v[3 * p] = ux;
        v[3 * p + 1] = uy;
        v[3 * p + 2] = uz;
        x[3 * p] = px + dt * ux;
        x[3 * p + 1] = py + dt * uy;
        x[3 * p + 2] = pz + dt * uz;
    }
}

void launch_g2p(const DevGrid &g, cudaStream_t s, float *x, float *v, long long n, float dt, int f_mom0,
                const int32_t *order)
{
    if (n <= 0) return;
    long long blocks = (n + 255) / 256;
    if (blocks > 1 << 20) blocks = 1 << 20;
    k_g2p<<<(unsigned)blocks, 256, 0, s>>>(g, x, v, n, dt, f_mom0, order);
}

}  // namespace sg

// ===========================================================================
// Binned P2G.  Each step the particles are binned by the leaf that holds the
// lowest corner (base node) of their 3x3x3 stencil; a bin's particles
// accumulate into a shared-memory block of (L+2)^3 nodes (every node their
// stencils can reach), and each block is added to the grid once.  Global
// atomics drop from 27 x 4 per particle to 4 per touched block node, and
// inside a block no atomic is needed at all (a gather per node).
//   1. k_p2g_bin     mark the pointer cells to activate; count particles per bin
//   2. (allocation of the marked cells: k_alloc_needed)
//   3. k_bin_scan_*  exclusive scan of the counts (tile sums, top scan, apply);
//                    the count array becomes each bin's insertion cursor
//   4. k_p2g_perm    write particle indices in bin order
//   5. k_p2g_gather  per bin: sort the bin's particles by cell in shared
//                    memory, sum each block node's contributions in registers,
//                    then add the touched nodes to the grid and set their bits
// ===========================================================================
namespace sg {

constexpr int kBinTile = 1024;

__device__ __forceinline__ int p2g_bin_of(const float *__restrict__ x, long long p, int N, int lg2, int R)
{
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const Spline s = bspline(__ldg(x + 3 * p + a), N);
        c[a] = min(max(s.base, 0), N - 1) >> lg2;
    }
    return (c[0] * R + c[1]) * R + c[2];
}

__global__ void k_p2g_bin(DevGrid g, const float *__restrict__ x, long long n)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        int lo[3], hi[3], c[3];
        bool empty = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const Spline s = bspline(__ldg(x + 3 * p + a), g.N);
            const int n0 = max(s.base, 0), n1 = min(s.base + 2, g.N - 1);
            if (n0 > n1) empty = true;
            lo[a] = n0 >> g.lg2;
            hi[a] = n1 >> g.lg2;
            c[a] = min(max(s.base, 0), g.N - 1) >> g.lg2;
        }
        const long long nbins = (long long)g.R * g.R * g.R;
        if (empty) {  // no stencil node inside the domain: the extra bin nbins
            atomicAdd(&g.bin_count[nbins], 1);
            continue;
        }
        for (int bi = lo[0]; bi <= hi[0]; ++bi)
            for (int bj = lo[1]; bj <= hi[1]; ++bj)
                for (int bk = lo[2]; bk <= hi[2]; ++bk) {
                    uint8_t *nd = &g.need[((long long)bi * g.R + bj) * g.R + bk];
                    // most cells are marked already: read through L2 (coherent across SMs) and skip
                    // the same-address store
                    if (!__ldcg(nd)) *nd = 1;
                }
        atomicAdd(&g.bin_count[((long long)c[0] * g.R + c[1]) * g.R + c[2]], 1);
    }
}

// Sum of each tile of kBinTile counts.
__global__ void __launch_bounds__(256) k_bin_scan_tiles(DevGrid g, long long nbins)
{
    __shared__ int s_w[8];
    const long long base = (long long)blockIdx.x * kBinTile;
    int v = 0;
    for (int q = threadIdx.x; q < kBinTile; q += 256)
        if (base + q < nbins) v += g.bin_count[base + q];
    v = warp_sum(v);
    if (lane_id() == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        g.tile_sum[blockIdx.x] = t;
    }
}

// Exclusive scan of the tile sums by one CTA (in place).
__global__ void __launch_bounds__(1024) k_bin_scan_top(DevGrid g, int ntiles)
{
    __shared__ int s_w[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = (i < ntiles) ? g.tile_sum[i] : 0;
        const int inc = warp_incl_scan(v);
        if (lane_id() == 31) s_w[threadIdx.x >> 5] = inc;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int wv = s_w[threadIdx.x];
            s_w[threadIdx.x] = warp_incl_scan(wv) - wv;
        }
        __syncthreads();
        const int excl = s_carry + s_w[threadIdx.x >> 5] + inc - v;
        __syncthreads();
        if (i < ntiles) g.tile_sum[i] = excl;
        if (threadIdx.x == 1023) s_carry = excl + v;
        __syncthreads();
    }
}

// Per tile: exclusive offsets of the bins; the count array becomes the
// insertion cursor (= offset), bin_off keeps the offset.
__global__ void __launch_bounds__(256) k_bin_scan_apply(DevGrid g, long long nbins)
{
    __shared__ int s_w[8];
    const long long base = (long long)blockIdx.x * kBinTile + threadIdx.x * 4;
    int v[4], t = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q] = (base + q < nbins) ? g.bin_count[base + q] : 0;
        t += v[q];
    }
    const int inc = warp_incl_scan(t);
    if (lane_id() == 31) s_w[threadIdx.x >> 5] = inc;
    __syncthreads();
    int wb = 0;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) wb += s_w[w];
    int run = g.tile_sum[blockIdx.x] + wb + inc - t;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (base + q < nbins) {
            g.bin_off[base + q] = run;
            g.bin_count[base + q] = run;
        }
        run += v[q];
    }
    // list of the non-empty bins of the grid (the last, out-of-domain bin excluded)
    const long long real = nbins - 1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool want = (base + q < real) && v[q] > 0;
        const unsigned m = __ballot_sync(kFull, want);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        int first = 0;
        if (lane_id() == leader) first = atomicAdd(&g.ctrl->bins_used, __popc(m));
        first = __shfl_sync(kFull, first, leader);
        if (want) g.bin_list[first + __popc(m & lanemask_lt())] = (int32_t)(base + q);
    }
}

__global__ void k_p2g_perm(DevGrid g, const float *__restrict__ x, long long n)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        bool empty = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const Spline s = bspline(__ldg(x + 3 * p + a), g.N);
            if (max(s.base, 0) > min(s.base + 2, g.N - 1)) empty = true;
        }
        const int b = empty ? g.R * g.R * g.R : p2g_bin_of(x, p, g.N, g.lg2, g.R);
        const int pos = atomicAdd(&g.bin_count[b], 1);
        g.perm[pos] = (int)p;
    }
}

// Per bin: stage the bin's particles (stencil weights and pmass * velocity)
// in shared memory sorted by their base cell, then let one thread per block
// node sum, in registers, the contributions of the particles in the 27 cells
// whose stencils reach that node.  A node whose stencil set is non-empty is
// activated (all 27 stencil nodes of every particle are, whatever their
// weight) and its sums are added to the grid.  Bins with more particles than
// the staging capacity are processed in chunks.
template <int L>
__global__ void __launch_bounds__(256) k_p2g_gather(DevGrid g, const float *__restrict__ x, const float *__restrict__ v,
                                                    float pmass, int f_mass, int f_mom0)
{
    constexpr int B = L + 2, NB = B * B * B, LG2 = (L == 8) ? 3 : 2;
    constexpr int C1 = L + 1, NC = C1 * C1 * C1;  // base cells relative to the leaf origin, shifted by +1
    constexpr int CAP = (L == 8) ? 512 : 768;       // staged particles per chunk
    constexpr int NPER = (NB + 255) / 256;          // block nodes per thread
    __shared__ float s_w[CAP][9];                   // weights w[axis][0..2]
    __shared__ float s_mv[CAP][4];                  // pmass, pmass * v
    __shared__ uint16_t s_cell[CAP];
    __shared__ uint16_t s_sorted[CAP];
    __shared__ int s_cnt[NC + 1];
    __shared__ int s_start[NC + 1];
    const int N = g.N, R = g.R;
    float *fm = g.field[f_mass];
    float *f0 = g.field[f_mom0], *f1 = g.field[f_mom0 + 1], *f2 = g.field[f_mom0 + 2];
    bool changed = false;
    const int used = g.ctrl->bins_used;
    for (int bl = blockIdx.x; bl < used; bl += gridDim.x) {
        const long long b = g.bin_list[bl];
        const int beg = g.bin_off[b], end = g.bin_count[b];
        const int oi = (int)(b / ((long long)R * R)) * L, oj = (int)((b / R) % R) * L, ok = (int)(b % R) * L;
        float acc[NPER][4];
        bool hit[NPER];
#pragma unroll
        for (int u = 0; u < NPER; ++u) {
            acc[u][0] = acc[u][1] = acc[u][2] = acc[u][3] = 0.f;
            hit[u] = false;
        }
        for (int c0 = beg; c0 < end; c0 += CAP) {
            const int cnt = min(CAP, end - c0);
            for (int q = threadIdx.x; q <= NC; q += 256) s_cnt[q] = 0;
            __syncthreads();
            for (int q = threadIdx.x; q < cnt; q += 256) {
                const long long p = g.perm[c0 + q];
                const Spline sx = bspline(__ldg(x + 3 * p + 0), N);
                const Spline sy = bspline(__ldg(x + 3 * p + 1), N);
                const Spline sz = bspline(__ldg(x + 3 * p + 2), N);
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    s_w[q][t] = sx.w[t];
                    s_w[q][3 + t] = sy.w[t];
                    s_w[q][6 + t] = sz.w[t];
                }
                s_mv[q][0] = pmass;
                s_mv[q][1] = pmass * __ldg(v + 3 * p + 0);
                s_mv[q][2] = pmass * __ldg(v + 3 * p + 1);
                s_mv[q][3] = pmass * __ldg(v + 3 * p + 2);
                const int cell = ((sx.base - oi + 1) * C1 + (sy.base - oj + 1)) * C1 + (sz.base - ok + 1);
                s_cell[q] = (uint16_t)cell;
                atomicAdd(&s_cnt[cell], 1);
            }
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
            for (int q = threadIdx.x; q < NC; q += 256) s_cnt[q] = s_start[q];  // cursors
            __syncthreads();
            for (int q = threadIdx.x; q < cnt; q += 256) s_sorted[atomicAdd(&s_cnt[s_cell[q]], 1)] = (uint16_t)q;
            __syncthreads();
#pragma unroll
            for (int u = 0; u < NPER; ++u) {
                const int nd = threadIdx.x + u * 256;
                if (nd >= NB) break;
                const int ni = nd / (B * B), nj = (nd / B) % B, nk = nd % B;
                for (int a = 0; a < 3; ++a) {
                    const int ci = ni - a + 1;
                    if (ci < 0 || ci >= C1) continue;
                    for (int c = 0; c < 3; ++c) {
                        const int cj = nj - c + 1;
                        if (cj < 0 || cj >= C1) continue;
                        for (int d = 0; d < 3; ++d) {
                            const int ck = nk - d + 1;
                            if (ck < 0 || ck >= C1) continue;
                            const int cell = (ci * C1 + cj) * C1 + ck;
                            const int p0 = s_start[cell], p1 = s_start[cell + 1];
                            if (p0 < p1) hit[u] = true;
                            for (int pp = p0; pp < p1; ++pp) {
                                const int q = s_sorted[pp];
                                const float wt = s_w[q][a] * s_w[q][3 + c] * s_w[q][6 + d];
                                acc[u][0] += wt * s_mv[q][0];
                                acc[u][1] += wt * s_mv[q][1];
                                acc[u][2] += wt * s_mv[q][2];
                                acc[u][3] += wt * s_mv[q][3];
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int u = 0; u < NPER; ++u) {
            const int nd = threadIdx.x + u * 256;
            if (nd >= NB || !hit[u]) continue;
            const int i = oi + nd / (B * B), j = oj + (nd / B) % B, k = ok + nd % B;
            if (i >= N || j >= N || k >= N) continue;
            const long long lb = ((long long)(i >> LG2) * R + (j >> LG2)) * R + (k >> LG2);
            const int slot = g.root[lb];
            if (slot < 0) continue;  // pool exhausted; the error is latched
            const int l = (((i & (L - 1)) << LG2) + (j & (L - 1))) * L + (k & (L - 1));
            uint32_t *mw = &g.mask[(long long)slot * g.W + (l >> 5)];
            const uint32_t bit = 1u << (l & 31);
            if (!(*mw & bit)) {
                const uint32_t old = atomicOr(mw, bit);
                if (!(old & bit)) changed = true;
            }
            const long long idx = ((long long)slot << (3 * LG2)) + l;
            atomicAdd(fm + idx, acc[u][0]);
            atomicAdd(f0 + idx, acc[u][1]);
            atomicAdd(f1 + idx, acc[u][2]);
            atomicAdd(f2 + idx, acc[u][3]);
        }
    }
    if (changed) mark_dirty(g);
}

int launch_p2g_binned(const DevGrid &g, cudaStream_t s, const float *x, const float *v, long long n, float pmass,
                      int f_mass, int f_mom0, const LaunchCfg &lc)
{
    const long long nbins = (long long)g.R * g.R * g.R;
    const long long nscan = nbins + 1;  // plus the bin of particles with no stencil node in the domain
    const int ntiles = (int)((nscan + kBinTile - 1) / kBinTile);
    long long pblocks = (n + 255) / 256;
    if (pblocks > 1 << 20) pblocks = 1 << 20;
    int launches = 0;
    cudaMemsetAsync(g.bin_count, 0, sizeof(int32_t) * nscan, s);
    cudaMemsetAsync(&g.ctrl->bins_used, 0, sizeof(int32_t), s);
    k_p2g_bin<<<(unsigned)pblocks, 256, 0, s>>>(g, x, n);
    ++launches;
    launch_alloc_needed(g, s);
    ++launches;
    k_bin_scan_tiles<<<ntiles, 256, 0, s>>>(g, nscan);
    k_bin_scan_top<<<1, 1024, 0, s>>>(g, ntiles);
    k_bin_scan_apply<<<ntiles, 256, 0, s>>>(g, nscan);
    launches += 3;
    k_p2g_perm<<<(unsigned)pblocks, 256, 0, s>>>(g, x, n);
    ++launches;
    if (g.L == 4) k_p2g_gather<4><<<lc.num_sms * 4, 256, 0, s>>>(g, x, v, pmass, f_mass, f_mom0);
    else k_p2g_gather<8><<<lc.num_sms * 2, 256, 0, s>>>(g, x, v, pmass, f_mass, f_mom0);
    ++launches;
    return launches;
}

}  // namespace sg
