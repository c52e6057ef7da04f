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
                                             int f_mom0)
{
    const int L = g.L, lg2 = g.lg2, N = g.N;
    const float *f0 = g.field[f_mom0], *f1 = g.field[f_mom0 + 1], *f2 = g.field[f_mom0 + 2];
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
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

void launch_g2p(const DevGrid &g, cudaStream_t s, float *x, float *v, long long n, float dt, int f_mom0)
{
    if (n <= 0) return;
    long long blocks = (n + 255) / 256;
    if (blocks > 1 << 20) blocks = 1 << 20;
    k_g2p<<<(unsigned)blocks, 256, 0, s>>>(g, x, v, n, dt, f_mom0);
}

}  // namespace sg
