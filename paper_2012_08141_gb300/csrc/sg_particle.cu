// sg_particle.cu -- particle-grid transfers on the sparse grid (the hybrid
// Lagrangian-Eulerian workload of AsyncTaichi Sec. 8.3): P2G with activation,
// the grid velocity update, and G2P, as PIC transfers or as affine (APIC)
// transfers with a per-particle 3x3 matrix C (the transfers of MLS-MPM);
// quadratic B-spline weights.  The unit cube holds N^3 nodes, dx = 1/N, node
// (i,j,k) at (i,j,k)*dx, particle component a maps to grid axis a (z -> k).
// C is stored row-major, 9 floats per particle: (C d)_a = sum_b C[3a+b] d_b.
// For quadratic B-splines sum_n w d d^T = dx^2/4 I, so the APIC G2P matrix is
// C = (4/dx^2) sum_n w v_n d^T with d = node - x_p = ((a,b,c) - fx) dx.
#include "sg_particle.cuh"

namespace sg {

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

// G2P in input order, every node read from the grid.
template <bool APIC>
__global__ void __launch_bounds__(256) k_g2p(DevGrid g, float *__restrict__ x, float *__restrict__ v,
                                             float *__restrict__ C, long long n, float dt, int f_mom0)
{
    const float *f0 = g.field[f_mom0], *f1 = g.field[f_mom0 + 1], *f2 = g.field[f_mom0 + 2];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const float3 xp = load3(x, p, false);
        const Spline sx = bspline(xp.x, g.N), sy = bspline(xp.y, g.N), sz = bspline(xp.z, g.N);
        float3 u;
        float c[9];
        g2p_from_grid<APIC>(g, f0, f1, f2, sx, sy, sz, u, c);
        g2p_store<APIC>(x, v, C, p, xp, u, c, dt, false);
    }
}

// G2P over the bins of the last binned P2G: per leaf, the node velocities of
// the (L+2)^3 nodes from o to o + L + 1 (o the leaf origin; every node a
// stencil with base in [o, o + L - 1] reaches) are staged in shared memory, 0
// outside the domain or the allocated leaves, and the leaf's particles read
// their 27 nodes there.  A particle whose base lies outside that range (its
// position changed since the binning, or a base of -2 / -1 at the low domain
// face) reads the grid node by node, as do the particles whose stencil misses
// the domain (the last key).
template <int L, bool APIC>
__global__ void __launch_bounds__(256, 4) k_g2p_binned(DevGrid g, float *__restrict__ x, float *__restrict__ v,
                                                       float *__restrict__ C, float dt, int f_mom0, bool pair)
{
    constexpr int B = L + 2, NB = B * B * B;  // nodes o .. o + L + 1 of the bin's leaf o
    __shared__ float4 s_u[NB];
    const int N = g.N, R = g.R;
    const float *f0 = g.field[f_mom0], *f1 = g.field[f_mom0 + 1], *f2 = g.field[f_mom0 + 2];
    const int used = g.ctrl->bins_used;
    const long long oob_key = 8LL * R * R * R;
    for (int bl = blockIdx.x; bl <= used; bl += gridDim.x) {
        int beg, end, oi = 0, oj = 0, ok = 0;
        if (bl < used) {
            const long long b = g.bin_list[bl];
            beg = g.bin_off[8 * b];
            end = g.bin_count[8 * b + 7];
            oi = (int)(b / ((long long)R * R)) * L;
            oj = (int)((b / R) % R) * L;
            ok = (int)(b % R) * L;
            stage_velocities_tight<L>(g, f0, f1, f2, oi, oj, ok, s_u);
            __syncthreads();
        } else {
            beg = g.bin_off[oob_key];
            end = g.bin_count[oob_key];
        }
        for (int q = beg + threadIdx.x; q < end; q += blockDim.x) {
            const long long p = g.perm[q];
            const float3 xp = load3(x, p, pair);
            const Spline sx = bspline(xp.x, N), sy = bspline(xp.y, N), sz = bspline(xp.z, N);
            const int ri = sx.base - oi, rj = sy.base - oj, rk = sz.base - ok;
            float3 u;
            float c[9];
            if (bl < used && (unsigned)ri < (unsigned)L && (unsigned)rj < (unsigned)L && (unsigned)rk < (unsigned)L)
                g2p_from_block<B, APIC>(s_u, ri, rj, rk, N, sx, sy, sz, u, c);
            else
                g2p_from_grid<APIC>(g, f0, f1, f2, sx, sy, sz, u, c);
            g2p_store<APIC>(x, v, C, p, xp, u, c, dt, pair);
        }
        __syncthreads();  // s_u is restaged for the next leaf
    }
}

// CTAs of a persistent per-bin kernel: as many as fit on every SM at once.
template <typename K>
static int resident_ctas(K kernel, int num_sms)
{
    int per = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, 0) != cudaSuccess || per < 1) per = 1;
    return per * num_sms;
}

void launch_g2p(const DevGrid &g, cudaStream_t s, float *x, float *v, float *C, long long n, float dt, int f_mom0,
                int binned, const LaunchCfg &lc)
{
    if (n <= 0) return;
    if (binned) {
        const bool pair = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(v)) & 7) == 0;
#define SG_G2PB(LL, AP) k_g2p_binned<LL, AP><<<resident_ctas(k_g2p_binned<LL, AP>, lc.num_sms), 256, 0, s>>>( \
        g, x, v, C, dt, f_mom0, pair)
        if (C) {
            if (g.L == 4) SG_G2PB(4, true);
            else SG_G2PB(8, true);
        } else {
            if (g.L == 4) SG_G2PB(4, false);
            else SG_G2PB(8, false);
        }
#undef SG_G2PB
        return;
    }
    long long blocks = (n + 255) / 256;
    if (blocks > 1 << 20) blocks = 1 << 20;
    if (C) k_g2p<true><<<(unsigned)blocks, 256, 0, s>>>(g, x, v, C, n, dt, f_mom0);
    else k_g2p<false><<<(unsigned)blocks, 256, 0, s>>>(g, x, v, C, n, dt, f_mom0);
}

}  // namespace sg

// ===========================================================================
// Binned P2G.  Each step the particles are binned by the leaf that holds the
// lowest corner (base node) of their 3x3x3 stencil; a bin's particles
// accumulate into a shared-memory block of (L+2)^3 nodes (every node their
// stencils can reach), and each block is added to the grid once.  Global
// atomics drop from 27 x 4 per particle to 4 per touched block node, and
// shared-memory atomics to 27 x 4 per occupied cell.
//   1. k_p2g_bin     count particles per key (bin leaf x reach class)
//   2. k_bin_scan_tiles  tile sums of the counts; mark the leaves the occupied
//                    keys reach; k_alloc_needed allocates them
//   3. k_bin_scan_top / _apply  exclusive scan of the counts (the count array
//                    becomes each key's insertion cursor); list of occupied leaves
//   4. k_p2g_perm    write particle indices in bin order
//   5. k_p2g_gather  per bin: sort the bin's particles by cell in shared
//                    memory, sum each cell's contributions to its 27 nodes in
//                    registers (one warp per cell) into shared node sums, then
//                    add the touched nodes to the grid and set their bits
//                    (PIC, or APIC with the per-particle matrix C)
// ===========================================================================
namespace sg {

constexpr int kBinTile = 1024;

// Bin key of a particle: 8 * (leaf of its base node) + reach class, where
// bit 2 / 1 / 0 of the class says that the in-domain part of the stencil
// extends into the next leaf along i / j / k.  A particle with no stencil
// node inside the domain gets the key 8 R^3, one past the last leaf.  The
// base leaf is that of max(base, 0): base is at least -2 for a non-empty
// stencil, and -2 / -1 lie below leaf 0.
__device__ __forceinline__ long long p2g_key_of(const float *__restrict__ x, long long p, int N, int lg2, int R)
{
    long long leaf = 0;
    int cls = 0;
    bool empty = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const Spline s = bspline(__ldg(x + 3 * p + a), N);
        const int n0 = max(s.base, 0), n1 = min(s.base + 2, N - 1);
        empty |= n0 > n1;
        leaf = leaf * R + (n0 >> lg2);
        cls = (cls << 1) | ((n1 >> lg2) != (n0 >> lg2) ? 1 : 0);
    }
    return empty ? 8LL * R * R * R : leaf * 8 + cls;
}

// The count passes store each particle's key (at its position in the order
// they visit: the particle index here, the last order's slot in the rebin)
// for the order passes, which then read keys in order instead of positions.
__global__ void k_p2g_bin(DevGrid g, const float *__restrict__ x, long long n)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const long long key = p2g_key_of(x, p, g.N, g.lg2, g.R);
        g.perm_key[p] = key;
        atomicAdd(&g.bin_count[key], 1);
    }
}

// Rebinning: the particles are visited in the last binning's order, so the
// lanes of a warp mostly share a key (particles move little between steps);
// one atomic per distinct key in the warp.
__global__ void k_p2g_rebin(DevGrid g, const float *__restrict__ x, long long n)
{
    const int lane = lane_id();
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const long long key = p2g_key_of(x, g.perm[q], g.N, g.lg2, g.R);
        g.perm_key[q] = key;
        const unsigned peers = __match_any_sync(__activemask(), key);
        if (lane == __ffs(peers) - 1) atomicAdd(&g.bin_count[key], __popc(peers));
    }
}

// Sum of each tile of kBinTile counts; for every occupied key, mark the
// leaves its particles' stencils reach (the base leaf plus the neighbours in
// the directions of its reach class) for allocation.
__global__ void __launch_bounds__(256) k_bin_scan_tiles(DevGrid g, long long nkeys)
{
    __shared__ int s_w[8];
    const long long base = (long long)blockIdx.x * kBinTile;
    const long long nleaf_keys = nkeys - 1;  // the last key holds particles outside the domain
    const int R = g.R;
    int v = 0;
    for (int q = threadIdx.x; q < kBinTile; q += 256) {
        const long long key = base + q;
        const int c = (key < nkeys) ? g.bin_count[key] : 0;
        v += c;
        if (c > 0 && key < nleaf_keys) {
            const long long leaf = key >> 3;
            const int cls = (int)(key & 7);
            const int li = (int)(leaf / ((long long)R * R)), lj = (int)((leaf / R) % R), lk = (int)(leaf % R);
            for (int sub = cls;; sub = (sub - 1) & cls) {  // every subset of the class, itself and 0 included
                const long long t = ((long long)(li + (sub >> 2)) * R + (lj + ((sub >> 1) & 1))) * R + (lk + (sub & 1));
                g.need[t] = 1;
                if (sub == 0) break;
            }
        }
    }
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
    // list of the leaves with particles (the 8 keys of a leaf are held by an
    // even and the next odd thread; the out-of-domain key is excluded)
    const long long nleaves = (nbins - 1) >> 3;
    const int mine = t + __shfl_xor_sync(kFull, t, 1);
    const long long leaf = base >> 3;
    const bool want = !(threadIdx.x & 1) && mine > 0 && leaf < nleaves;
    const unsigned m = __ballot_sync(kFull, want);
    if (m) {
        const int leader = __ffs(m) - 1;
        int first = 0;
        if (lane_id() == leader) first = atomicAdd(&g.ctrl->bins_used, __popc(m));
        first = __shfl_sync(kFull, first, leader);
        if (want) g.bin_list[first + __popc(m & lanemask_lt())] = (int32_t)leaf;
    }
}

__global__ void k_p2g_perm(DevGrid g, long long n)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const int pos = atomicAdd(&g.bin_count[g.perm_key[p]], 1);
        g.perm[pos] = (int)p;
    }
}

// The new order from the last one, written to perm_alt (warp-aggregated
// cursor atomics, as in k_p2g_rebin).
__global__ void k_p2g_reperm(DevGrid g, long long n)
{
    const int lane = lane_id();
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int p = g.perm[q];
        const long long key = g.perm_key[q];
        const unsigned peers = __match_any_sync(__activemask(), key);
        const int leader = __ffs(peers) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&g.bin_count[key], __popc(peers));
        base = __shfl_sync(peers, base, leader);
        g.perm_alt[base + __popc(peers & lanemask_lt())] = p;
    }
}

// Per bin: stage the bin's particles in shared memory sorted by their base
// cell, as float4 records: (fx_i, fx_j, fx_k, m) and the momentum terms --
// PIC: m v; APIC: q = m v - m dx C fx and the 9 entries of m dx C, so that
// the momentum a particle gives stencil node base + t is w (q + m dx C t).
// One warp then takes one occupied cell at a time: lane t = (a, b, c) < 27
// owns the stencil node base + t shared by every particle of that cell and
// walks the cell's particles in step with the other lanes (each shared read
// is a broadcast), computing its own weights from fx and summing its node's
// contributions in registers; the cell's 27 sums are then added to a shared
// block of (L+2)^3 node accumulators.  A node reached by any stencil is
// activated (all 27 stencil nodes of every particle are, whatever their
// weight) and its sums are added to the grid once.  Bins with more particles
// than the staging capacity are processed in chunks.
//
// Base cells are indexed relative to the leaf origin o shifted by +2: a
// particle binned to leaf o has base in [o, o + L - 1], or base -2 / -1 at the
// low domain face (its bin is clamped to leaf 0), so the shifted index is in
// [0, L + 1].  Block node n (0 <= n < L + 2 per axis) is grid node o + n.
template <int L, bool APIC>
__global__ void __launch_bounds__(256) k_p2g_gather(DevGrid g, const float *__restrict__ x, const float *__restrict__ v,
                                                    const float *__restrict__ C, float pmass, int f_mass, int f_mom0)
{
    constexpr int B = L + 2, NB = B * B * B, LG2 = (L == 8) ? 3 : 2;
    constexpr int C1 = L + 2, NC = C1 * C1 * C1;  // shifted base cells
    constexpr int CAP = (L == 8) ? 256 : (APIC ? 512 : 1024);  // staged particles per chunk
    constexpr int PPT = CAP / 256;                  // staged particles per thread
    constexpr int NREC = APIC ? 4 : 2;              // float4 records per particle
    constexpr int NWARP = 8;
    __shared__ float4 s_rec[NREC][CAP];
    __shared__ float s_acc[4][NB];                  // block node sums
    __shared__ uint8_t s_hit[NB];
    __shared__ int s_cnt[NC + 1];
    __shared__ int s_start[NC + 1];
    __shared__ int s_occ[NC];  // the chunk's occupied cells, ascending
    __shared__ int s_nocc;
    const int N = g.N, R = g.R;
    const float dx = 1.f / (float)N;
    const int warp = threadIdx.x >> 5, lane = lane_id();
    // this lane's stencil offset (lanes 27..31 idle in the cell loop)
    const int la = lane / 9, lc = (lane / 3) % 3, ld = lane % 3;
    const BsPoly pa = bs_poly(la), pb = bs_poly(lc), pc = bs_poly(ld);
    const float ta = (float)la, tb = (float)lc, tc = (float)ld;
    float *fm = g.field[f_mass];
    float *f0 = g.field[f_mom0], *f1 = g.field[f_mom0 + 1], *f2 = g.field[f_mom0 + 2];
    bool changed = false;
    const int used = g.ctrl->bins_used;
    for (int bl = blockIdx.x; bl < used; bl += gridDim.x) {
        const long long b = g.bin_list[bl];  // a leaf; its 8 keys are contiguous in the particle order
        const int beg = g.bin_off[8 * b], end = g.bin_count[8 * b + 7];
        const int oi = (int)(b / ((long long)R * R)) * L, oj = (int)((b / R) % R) * L, ok = (int)(b % R) * L;
        for (int q = threadIdx.x; q < NB; q += 256) {
            s_acc[0][q] = s_acc[1][q] = s_acc[2][q] = s_acc[3][q] = 0.f;
            s_hit[q] = 0;
        }
        for (int c0 = beg; c0 < end; c0 += CAP) {
            const int cnt = min(CAP, end - c0);
            for (int q = threadIdx.x; q <= NC; q += 256) s_cnt[q] = 0;
            __syncthreads();
            // pass 1: each particle's cell and its rank among the cell's particles
            int rcell[PPT], rrank[PPT], rp[PPT];
            float rx[PPT][3];
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
                const int q = threadIdx.x + u * 256;
                rcell[u] = -1;
                if (q >= cnt) continue;
                const int p = g.perm[c0 + q];
#pragma unroll
                for (int a = 0; a < 3; ++a) rx[u][a] = __ldg(x + 3 * (long long)p + a);
                const int bi = bspline(rx[u][0], N).base;
                const int bj = bspline(rx[u][1], N).base;
                const int bk = bspline(rx[u][2], N).base;
                rcell[u] = ((bi - oi + 2) * C1 + (bj - oj + 2)) * C1 + (bk - ok + 2);
                rrank[u] = atomicAdd(&s_cnt[rcell[u]], 1);
                rp[u] = p;
            }
            __syncthreads();
            if (threadIdx.x < 32) {  // exclusive scan of the cell counts; occupied cells listed
                int carry = 0, occ = 0;
                for (int base = 0; base < NC; base += 32) {
                    const int i = base + threadIdx.x;
                    const int vv = (i < NC) ? s_cnt[i] : 0;
                    const int inc = warp_incl_scan(vv);
                    if (i < NC) s_start[i] = carry + inc - vv;
                    carry += __shfl_sync(kFull, inc, 31);
                    const unsigned m = __ballot_sync(kFull, vv > 0);
                    if (vv > 0) s_occ[occ + __popc(m & lanemask_lt())] = i;
                    occ += __popc(m);
                }
                if (threadIdx.x == 0) {
                    s_start[NC] = carry;
                    s_nocc = occ;
                }
            }
            __syncthreads();
            // pass 2: stage the particles at their sorted positions (x kept in
            // registers from pass 1, v read here)
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
                if (rcell[u] < 0) continue;
                const int pos = s_start[rcell[u]] + rrank[u];
                const long long p = rp[u];
                const float fx = bspline(rx[u][0], N).fx;
                const float fy = bspline(rx[u][1], N).fx;
                const float fz = bspline(rx[u][2], N).fx;
                const float mv0 = pmass * __ldg(v + 3 * p + 0), mv1 = pmass * __ldg(v + 3 * p + 1),
                            mv2 = pmass * __ldg(v + 3 * p + 2);
                s_rec[0][pos] = make_float4(fx, fy, fz, pmass);
                if (!APIC) {
                    s_rec[1][pos] = make_float4(mv0, mv1, mv2, 0.f);
                } else {
                    float m[9];
                    const float md = pmass * dx;
#pragma unroll
                    for (int e = 0; e < 9; ++e) m[e] = md * __ldg(C + 9 * p + e);
                    const float q0 = mv0 - (m[0] * fx + m[1] * fy + m[2] * fz);
                    const float q1 = mv1 - (m[3] * fx + m[4] * fy + m[5] * fz);
                    const float q2 = mv2 - (m[6] * fx + m[7] * fy + m[8] * fz);
                    s_rec[1][pos] = make_float4(q0, q1, q2, m[0]);
                    s_rec[2][pos] = make_float4(m[1], m[2], m[3], m[4]);
                    s_rec[3][pos] = make_float4(m[5], m[6], m[7], m[8]);
                }
                g.perm[c0 + pos] = rp[u];  // the chunk's order becomes cell order (G2P reads it)
            }
            __syncthreads();
            const int nocc = s_nocc;
            for (int oc = warp; oc < nocc; oc += NWARP) {
                const int cell = s_occ[oc];
                const int p0 = s_start[cell], p1 = s_start[cell + 1];
                const int ci = cell / (C1 * C1), cj = (cell / C1) % C1, ck = cell % C1;
                float m = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f;
                for (int pp = p0; pp < p1; ++pp) {
                    const float4 r0 = s_rec[0][pp];
                    const float w = bs_eval(pa, r0.x) * bs_eval(pb, r0.y) * bs_eval(pc, r0.z);
                    const float4 r1 = s_rec[1][pp];
                    m = fmaf(w, r0.w, m);
                    if (!APIC) {
                        m0 = fmaf(w, r1.x, m0);
                        m1 = fmaf(w, r1.y, m1);
                        m2 = fmaf(w, r1.z, m2);
                    } else {
                        const float4 r2 = s_rec[2][pp], r3 = s_rec[3][pp];
                        // rows of m dx C: (r1.w, r2.x, r2.y), (r2.z, r2.w, r3.x), (r3.y, r3.z, r3.w)
                        const float u0 = fmaf(r1.w, ta, fmaf(r2.x, tb, fmaf(r2.y, tc, r1.x)));
                        const float u1 = fmaf(r2.z, ta, fmaf(r2.w, tb, fmaf(r3.x, tc, r1.y)));
                        const float u2 = fmaf(r3.y, ta, fmaf(r3.z, tb, fmaf(r3.w, tc, r1.z)));
                        m0 = fmaf(w, u0, m0);
                        m1 = fmaf(w, u1, m1);
                        m2 = fmaf(w, u2, m2);
                    }
                }
                const int ni = ci - 2 + la, nj = cj - 2 + lc, nk = ck - 2 + ld;
                if (lane < 27 && ni >= 0 && nj >= 0 && nk >= 0) {  // negative: outside the domain
                    const int nd = (ni * B + nj) * B + nk;
                    atomicAdd(&s_acc[0][nd], m);
                    atomicAdd(&s_acc[1][nd], m0);
                    atomicAdd(&s_acc[2][nd], m1);
                    atomicAdd(&s_acc[3][nd], m2);
                    s_hit[nd] = 1;
                }
            }
            __syncthreads();
        }
        for (int nd = threadIdx.x; nd < NB; nd += 256) {
            if (!s_hit[nd]) continue;
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
            atomicAdd(fm + idx, s_acc[0][nd]);
            atomicAdd(f0 + idx, s_acc[1][nd]);
            atomicAdd(f1 + idx, s_acc[2][nd]);
            atomicAdd(f2 + idx, s_acc[3][nd]);
        }
        __syncthreads();  // the accumulators are zeroed for the next bin
    }
    if (changed) mark_dirty(g);
}

// ---------------------------------------------------------------------------
// Particle reordering: the arrays into the order of the last binning, out[q]
// = in[perm[q]] for nc values per particle (a thread per value, so the writes
// are coalesced), then the order itself becomes the identity.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_sort_gather(const int32_t *__restrict__ perm, long long n, int nc, const T *__restrict__ in,
                              T *__restrict__ out)
{
    const long long total = n * nc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long q = e / nc;
        const int c = (int)(e - q * nc);
        out[e] = in[(long long)perm[q] * nc + c];
    }
}

__global__ void k_iota(int32_t *__restrict__ perm, long long n)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        perm[q] = (int32_t)q;
}

int launch_sort_particles(DevGrid &g, cudaStream_t s, float *x, float *v, float *C, int64_t *ids, long long n,
                          void *tmp, const LaunchCfg &lc)
{
    const unsigned blocks = (unsigned)(lc.num_sms * 8);
    int launches = 0;
    struct Arr { void *p; int nc; bool i64; } arrs[4] = {{x, 3, false}, {v, 3, false}, {C, 9, false}, {ids, 1, true}};
    for (const Arr &a : arrs) {
        if (!a.p) continue;
        if (a.i64)
            k_sort_gather<long long><<<blocks, 256, 0, s>>>(g.perm, n, a.nc, (const long long *)a.p, (long long *)tmp);
        else
            k_sort_gather<float><<<blocks, 256, 0, s>>>(g.perm, n, a.nc, (const float *)a.p, (float *)tmp);
        ++launches;
        cudaMemcpyAsync(a.p, tmp, (size_t)n * a.nc * (a.i64 ? 8 : 4), cudaMemcpyDeviceToDevice, s);
    }
    k_iota<<<blocks, 256, 0, s>>>(g.perm, n);
    return launches + 1;
}

int launch_p2g_binned(DevGrid &g, cudaStream_t s, const float *x, const float *v, const float *C, long long n,
                      float pmass, int f_mass, int f_mom0, bool rebin, const LaunchCfg &lc)
{
    const long long nscan = p2g_num_keys(g.R);
    const int ntiles = (int)((nscan + kBinTile - 1) / kBinTile);
    long long pblocks = (n + 255) / 256;
    if (pblocks > 1 << 20) pblocks = 1 << 20;
    int launches = 0;
    cudaMemsetAsync(g.bin_count, 0, sizeof(int32_t) * nscan, s);
    cudaMemsetAsync(&g.ctrl->bins_used, 0, sizeof(int32_t), s);
    if (rebin) k_p2g_rebin<<<(unsigned)pblocks, 256, 0, s>>>(g, x, n);
    else k_p2g_bin<<<(unsigned)pblocks, 256, 0, s>>>(g, x, n);
    k_bin_scan_tiles<<<ntiles, 256, 0, s>>>(g, nscan);
    launch_alloc_needed(g, s);
    k_bin_scan_top<<<1, 1024, 0, s>>>(g, ntiles);
    k_bin_scan_apply<<<ntiles, 256, 0, s>>>(g, nscan);
    launches += 5;
    if (rebin) {
        k_p2g_reperm<<<(unsigned)pblocks, 256, 0, s>>>(g, n);
        int32_t *t = g.perm;  // the new order is now the current one
        g.perm = g.perm_alt;
        g.perm_alt = t;
    } else {
        k_p2g_perm<<<(unsigned)pblocks, 256, 0, s>>>(g, n);
    }
    ++launches;
#define SG_GATHER(LL, AP) k_p2g_gather<LL, AP><<<resident_ctas(k_p2g_gather<LL, AP>, lc.num_sms), 256, 0, s>>>( \
        g, x, v, C, pmass, f_mass, f_mom0)
    if (C) {
        if (g.L == 4) SG_GATHER(4, true);
        else SG_GATHER(8, true);
    } else {
        if (g.L == 4) SG_GATHER(4, false);
        else SG_GATHER(8, false);
    }
#undef SG_GATHER
    ++launches;
    return launches;
}

}  // namespace sg
