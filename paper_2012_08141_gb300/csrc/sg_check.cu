// sg_check.cu -- invariant checks of one grid (sg_check and checking grids).
// Not part of the paper's method: a debugging aid that counts violations of
// what every other kernel relies on.  The structure is the two-level tree of
// Sec. 3 (a root of pointer cells over bitmasked leaves), and the stored
// value at an inactive voxel is 0 (Sec. 4: an inactive voxel reads as 0,
// which the whole-leaf loads of the stencil kernels assume).
#include "sg_common.cuh"

namespace sg {

// root cells: null or a handed-out slot, no slot owned twice
__global__ void __launch_bounds__(256) k_check_root(DevGrid g, uint32_t *owner, unsigned long long *cnt)
{
    const long long nr = (long long)g.R * g.R * g.R;
    const long long handed = min((long long)g.ctrl->pool_count, (long long)g.cap);
    unsigned long long bad = 0, shared = 0, leaves = 0;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nr; b += (long long)gridDim.x * blockDim.x) {
        const int r = g.root[b];
        if (r == -1) continue;
        if (r < 0 || r >= handed) {
            ++bad;
            continue;
        }
        ++leaves;
        if (atomicCAS(&owner[r], 0xffffffffu, (uint32_t)b) != 0xffffffffu) ++shared;
    }
    if (bad) atomicAdd(&cnt[kChkRoot], bad);
    if (shared) atomicAdd(&cnt[kChkShared], shared);
    if (leaves) atomicAdd(&cnt[kChkLeaves], leaves);
}

// list entries against the root, and the 27-neighbour table against the root
__global__ void __launch_bounds__(256) k_check_list(DevGrid g, unsigned long long *cnt)
{
    const long long nr = (long long)g.R * g.R * g.R;
    const long long n = g.ctrl->list_n;
    const int R = g.R;
    unsigned long long bad = 0, nbad = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int s = g.list_slot[e], b = g.list_b[e];
        if (b < 0 || b >= nr) {
            ++bad;
            continue;
        }
        if (s < 0 || s >= g.cap || g.root[b] != s || (e > 0 && g.list_b[e - 1] >= b)) ++bad;
        const int bi = b / (R * R), bj = (b / R) % R, bk = b % R;
        for (int q = 0; q < 27; ++q) {
            const int ni = bi + q / 9 - 1, nj = bj + (q / 3) % 3 - 1, nk = bk + q % 3 - 1;
            int want = (int)g.cap;
            if ((unsigned)ni < (unsigned)R && (unsigned)nj < (unsigned)R && (unsigned)nk < (unsigned)R) {
                const int v = g.root[((long long)ni * R + nj) * R + nk];
                if (v >= 0) want = v;
            }
            if (g.nbr[e * 27 + q] != want) ++nbad;
        }
    }
    if (bad) atomicAdd(&cnt[kChkList], bad);
    if (nbad) atomicAdd(&cnt[kChkNbr], nbad);
}

// the zero leaf (slot cap) reads as zeros in every mask word and field
__global__ void __launch_bounds__(256) k_check_zero_leaf(DevGrid g, unsigned long long *cnt)
{
    const long long V = (long long)g.L * g.L * g.L;
    unsigned long long bad = 0;
    for (int w = threadIdx.x; w < g.W; w += blockDim.x)
        if (g.mask[g.cap * g.W + w] != 0u) ++bad;
    for (int f = 0; f < g.F; ++f)
        for (long long v = threadIdx.x; v < V; v += blockDim.x)
            if (g.field[f][g.cap * V + v] != 0.f) ++bad;
    if (bad) atomicAdd(&cnt[kChkZero], bad);
}

// stored values at inactive voxels of listed leaves, for the physical fields
// in field_bits
__global__ void __launch_bounds__(256) k_check_inactive(DevGrid g, uint32_t field_bits, unsigned long long *cnt)
{
    const long long n = g.ctrl->list_n;
    const int V = g.L * g.L * g.L;
    unsigned long long bad = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * V; q += (long long)gridDim.x * blockDim.x) {
        const long long e = q / V;
        const int l = (int)(q - e * V);
        const int s = g.list_slot[e];
        if (s < 0 || s >= g.cap) continue;  // counted by the list check
        if ((g.mask[(long long)s * g.W + (l >> 5)] >> (l & 31)) & 1u) continue;
        for (int f = 0; f < g.F; ++f)
            if (((field_bits >> f) & 1u) && g.field[f][(long long)s * V + l] != 0.f) ++bad;
    }
    if (bad) atomicAdd(&cnt[kChkInactive], bad);
}

void launch_checks(const DevGrid &g, cudaStream_t s, uint32_t *owner, unsigned long long *cnt, bool with_list,
                   uint32_t field_bits, const LaunchCfg &lc)
{
    k_check_root<<<lc.num_sms * 4, 256, 0, s>>>(g, owner, cnt);
    k_check_zero_leaf<<<1, 256, 0, s>>>(g, cnt);
    if (with_list) {
        k_check_list<<<lc.num_sms * 4, 256, 0, s>>>(g, cnt);
        k_check_inactive<<<lc.num_sms * 4, 256, 0, s>>>(g, field_bits, cnt);
    }
}

}  // namespace sg
