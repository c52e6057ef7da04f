// sg_sweep_tma.cu -- the fused diffuse7 -> box27 (+ sum) step over 8^3
// leaves with the leaf blocks and their halo staged in shared memory by the
// tensor memory accelerator (AsyncTaichi Sec. 6.4 task fusion with the
// intermediate t never stored, Sec. 6.5).
//
// Work: the same warp tasks as k_sweep_jruns (runs of up to three leaves
// adjacent in j, from k_region_masks), and the same per-lane arithmetic in
// the same order, so fields are bit-identical to the j-run sweep.  What
// changes is where the x rows come from:
//   - a task's 12 x planes are staged in two halves (region planes 0..5 and
//     6..11) by cp.async.bulk.tensor copies of 4-D boxes of the leaf pool
//     (viewed as [slot][i][j][k]); each half completes on an mbarrier;
//   - every warp owns two half buffers and issues its own copies: one box
//     per lane, so one warp instruction issues up to 32 copies;
//   - while a warp computes the second half of task n, the first half of
//     task n+1 is in flight, and the second half of n+1 while it computes
//     the first half of n+1, so the sweep reads shared memory only;
//   - each task's box sources (27-neighbour slots per j segment) and region
//     masks are laid out once per list by k_tma_tasks.
// No copy uses cluster multicast: every source is this GPU's own leaf pool.
// Every mbarrier wait is bounded in time; a wait that gives up latches
// kErrTimeout (site 4), stops issuing, waits (bounded) for the copies it
// issued and leaves the task loop.
#include <cuda.h>
#include <atomic>
#include <mutex>
#include "sg_common.cuh"

namespace sg {

namespace {

constexpr int kTmaWarps = 8;                  // warps per CTA, one CTA per SM
constexpr int kSegF = 3072;                   // bytes of one half of a full segment (8 rows of one leaf)
constexpr int kSegE = 896;                    // bytes of one half of an end segment (2 rows, boxes padded to 128)
constexpr int kHalfBytes = 12800;             // largest task: E F F E | E F E
constexpr int kRmaskBytes = 480;              // region masks of three leaves (40 words each)
constexpr int kHalfABytes = 13312;            // first half + region masks, rounded to 128
constexpr int kWarpBytes = kHalfABytes + kHalfBytes;
constexpr int kTmaSmem = kTmaWarps * kWarpBytes + 128;  // + alignment slack
constexpr unsigned long long kTmaWaitLimitNs = 1000000000ull;  // 1 s

// Segment types of each task kind (bit s set: segment s is a full leaf) and
// which end segments are the low end (rows j = 6, 7 of the j-1 neighbour).
//   kind 0: three leaves            E F F F E
//   kind 1: two leaves + one leaf   E F F E | E F E
//   kind 2: one leaf + one leaf     E F E | E F E
__host__ __device__ constexpr int kind_nseg(int k) { return k == 0 ? 5 : (k == 1 ? 7 : 6); }
__host__ __device__ constexpr uint32_t kind_fmask(int k) { return k == 0 ? 0x0eu : (k == 1 ? 0x26u : 0x12u); }
__host__ __device__ constexpr uint32_t kind_lomask(int k) { return k == 0 ? 0x01u : (k == 1 ? 0x11u : 0x09u); }
// bytes of the boxes of one half of a task (both halves hold the same amount)
__host__ __device__ constexpr uint32_t kind_tx(int k) { return k == 0 ? 10752u : (k == 1 ? 12288u : 9216u); }

__device__ __forceinline__ int seg_off(int kind, int seg)
{
    const int nf = __popc(kind_fmask(kind) & ((1u << seg) - 1u));
    return nf * kSegF + (seg - nf) * kSegE;
}

// Box b = part * 3 + (dk + 1) of a segment half: byte offset inside the
// segment.  Half 0 holds region planes 0..5 (part 0: 2 planes of the i-1
// leaf, part 1: planes 0..3 of the i leaf); half 1 planes 6..11 (part 0:
// planes 4..7 of the i leaf, part 1: 2 planes of the i+1 leaf).  dk = +-1
// boxes are 4 floats wide (k = 4..7 of the k-1 leaf, k = 0..3 of the k+1
// leaf), dk = 0 boxes 8.  Offsets are multiples of 128 bytes.
__host__ __device__ constexpr uint32_t pack_offs(int a, int b, int c, int d, int e, int f)
{
    return (uint32_t)(a / 128) | (uint32_t)(b / 128) << 5 | (uint32_t)(c / 128) << 10 | (uint32_t)(d / 128) << 15 |
           (uint32_t)(e / 128) << 20 | (uint32_t)(f / 128) << 25;
}
__host__ __device__ constexpr int box_off(bool full, int half, int b)
{
    // six offsets / 128 in 5-bit fields (no local-memory table for runtime b)
    constexpr uint32_t f0 = pack_offs(0, 256, 768, 1024, 1536, 2560);
    constexpr uint32_t f1 = pack_offs(0, 512, 1536, 2048, 2304, 2816);
    constexpr uint32_t e0 = pack_offs(0, 128, 256, 384, 512, 768);
    constexpr uint32_t e1 = pack_offs(0, 128, 384, 512, 640, 768);
    return (int)(((full ? (half == 0 ? f0 : f1) : (half == 0 ? e0 : e1)) >> (5 * b)) & 31u) * 128;
}

// ---- PTX wrappers: mbarrier, bulk tensor copies, proxy fence ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_timer_ns() - t0 > kTmaWaitLimitNs) return false;
    return true;
}

__device__ __forceinline__ void tma_box4(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Generic-proxy reads of a buffer are ordered before the async-proxy copies
// that refill it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void stg4(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ float pick(uint32_t bits, int k, float v) { return ((bits >> k) & 1u) ? v : 0.f; }

// Task kind and piece layout of warp task t (the packing of k_sweep_jruns:
// tasks [0, c3) one piece of three; [c3, c3 + c2) a piece of two plus, while
// pieces of one last, a piece of one; then two pieces of one).
struct TaskShape {
    int kind;
    const int32_t *recA, *recB;  // records (list entries, lowest j first); recB null if absent
    int GA;
};

__device__ __forceinline__ TaskShape task_shape(const DevGrid &g, int t, int c3, int c2, int c1)
{
    const long long cap3 = g.cap * 3;
    const int p = c2 < c1 ? c2 : c1;
    TaskShape s;
    if (t < c3) {
        s.kind = 0;
        s.GA = 3;
        s.recA = g.col_grp + 2 * cap3 + 3LL * t;
        s.recB = nullptr;
    } else if (t < c3 + c2) {
        const int r = t - c3;
        s.kind = 1;
        s.GA = 2;
        s.recA = g.col_grp + cap3 + 3LL * r;
        s.recB = r < p ? g.col_grp + 3LL * r : nullptr;
    } else {
        const int q = p + 2 * (t - c3 - c2);
        s.kind = 2;
        s.GA = 1;
        s.recA = g.col_grp + 3LL * q;
        s.recB = q + 1 < c1 ? g.col_grp + 3LL * (q + 1) : nullptr;
    }
    return s;
}

__device__ __forceinline__ int num_tasks(int c3, int c2, int c1)
{
    const int p = c2 < c1 ? c2 : c1;
    return c3 + c2 + (c1 - p + 1) / 2;
}

}  // namespace

// ---------------------------------------------------------------------------
// Task descriptors, once per list: desc[t][seg * 9 + (di+1) * 3 + (dk+1)] is
// the slot whose leaf is read for the (di, dk) box of segment seg (the zero
// leaf for an absent piece or neighbour), and trm[t][f][40] the region masks
// of the task's full segments in order.  One warp per task.
// ---------------------------------------------------------------------------
__global__ void k_tma_tasks(DevGrid g)
{
    const int c3 = g.col_cnt[2], c2 = g.col_cnt[1], c1 = g.col_cnt[0];
    const int tasks = num_tasks(c3, c2, c1);
    const int lane = lane_id();
    const int Z = (int)g.cap;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < tasks; t += warps) {
        const TaskShape sh = task_shape(g, t, c3, c2, c1);
        const int GA = sh.GA, GB = 1;
        const int nseg = kind_nseg(sh.kind);
        for (int r = 0; r < 2; ++r) {
            const int idx = lane + 32 * r;
            int v = Z;
            const int seg = idx / 9, q9 = idx - seg * 9;
            if (seg < nseg) {
                // which piece, which leaf of it, and which j neighbour of that leaf
                const bool inA = seg < GA + 2;
                const int s = inA ? seg : seg - (GA + 2);
                const int G = inA ? GA : GB;
                const int32_t *rec = inA ? sh.recA : sh.recB;
                if (rec) {
                    const int m = s == 0 ? 0 : (s <= G ? s - 1 : G - 1);
                    const int dj1 = s == 0 ? 0 : (s <= G ? 1 : 2);
                    const int e = rec[m];
                    const int di1 = q9 / 3, dk1 = q9 - di1 * 3;
                    v = g.nbr[(long long)e * 27 + di1 * 9 + dj1 * 3 + dk1];
                }
            }
            if (idx < 64) g.tma_desc[(long long)t * 64 + idx] = (idx < 63) ? v : sh.kind;
        }
        for (int w = lane; w < 120; w += 32) {
            const int f = w / 40, q = w - f * 40;
            // full segments in order: kind 0: A0 A1 A2; kind 1: A0 A1 B0; kind 2: A0 B0
            const int32_t *rec = (f < GA) ? sh.recA : sh.recB;
            const int m = (f < GA) ? f : f - GA;
            uint32_t word = 0;
            if (rec && m < ((f < GA) ? GA : GB)) word = g.rmask[(long long)rec[m] * 40 + q];
            g.tma_rmask[(long long)t * 120 + w] = word;
        }
    }
}

// ---------------------------------------------------------------------------
// The fused kernel.
// ---------------------------------------------------------------------------
struct TmaMaps {
    CUtensorMap m[8];  // box (bk, bj, bi, 1): index (bi == 4) * 4 + (bj == 8) * 2 + (bk == 8)
};

namespace {

// Issue the copies of one half of task u into `buf` (a shared address),
// completing on `bar`.  d0 / d1: desc[u][lane], desc[u][lane + 32].  Called
// by the whole warp.
__device__ __forceinline__ void issue_half(int half, int kind, int d0, int d1, uint32_t buf, uint32_t bar,
                                           const CUtensorMap *maps, const uint32_t *rm_src)
{
    const int lane = lane_id();
    const int nbox = kind_nseg(kind) * 6;
    if (lane == 0) mbar_arrive_expect_tx(bar, kind_tx(kind) + (half == 0 ? (uint32_t)kRmaskBytes : 0u));
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int q = lane + 32 * r;
        const int seg = q / 6, b = q - seg * 6, part = b / 3, dk1 = b - part * 3;
        const int di1 = half == 0 ? part : part + 1;
        const int idx = seg * 9 + di1 * 3 + dk1;
        const int v0 = __shfl_sync(kFull, d0, idx & 31), v1 = __shfl_sync(kFull, d1, idx & 31);
        const int slot = idx < 32 ? v0 : v1;
        if (q < nbox) {
            const bool full = (kind_fmask(kind) >> seg) & 1u;
            const bool lo = (kind_lomask(kind) >> seg) & 1u;
            const int bi4 = (half == 0) ? part : 1 - part;  // box spans 4 planes
            const int mi = bi4 * 4 + (full ? 2 : 0) + (dk1 == 1 ? 1 : 0);
            const int i0 = (half == 0) ? (part == 0 ? 6 : 0) : (part == 0 ? 4 : 0);
            const int j0 = lo ? 6 : 0;
            const int k0 = dk1 == 0 ? 4 : 0;
            const uint32_t dst = buf + seg_off(kind, seg) + box_off(full, half, b);
            tma_box4(dst, maps + mi, k0, j0, i0, slot, bar);
        }
    }
    if (half == 0 && lane == 0) bulk_copy(buf + kHalfBytes, rm_src, kRmaskBytes, bar);
}

// Region row (12 floats) of plane RI for a lane whose segment starts at
// `seg` in the buffer of its half; r16 / r32 = row * 16 / row * 32.
template <int RI>
__device__ __forceinline__ void srow(const uint8_t *segA, const uint8_t *segB, bool full, int r16, int r32, float (&v)[12])
{
    constexpr int H = RI < 6 ? 0 : 1;
    constexpr int P = (RI < 2 || (RI >= 6 && RI < 10)) ? 0 : 1;
    constexpr int PIP = RI < 2 ? RI : (RI < 6 ? RI - 2 : (RI < 10 ? RI - 6 : RI - 10));
    const uint8_t *s = H == 0 ? segA : segB;
    const int o0 = full ? box_off(true, H, P * 3 + 0) + PIP * 128 : box_off(false, H, P * 3 + 0) + PIP * 32;
    const int o1 = full ? box_off(true, H, P * 3 + 1) + PIP * 256 : box_off(false, H, P * 3 + 1) + PIP * 64;
    const int o2 = full ? box_off(true, H, P * 3 + 2) + PIP * 128 : box_off(false, H, P * 3 + 2) + PIP * 32;
    const float2 a = *reinterpret_cast<const float2 *>(s + o0 + r16 + 8);
    const float4 c0 = *reinterpret_cast<const float4 *>(s + o1 + r32);
    const float4 c1 = *reinterpret_cast<const float4 *>(s + o1 + r32 + 16);
    const float2 b = *reinterpret_cast<const float2 *>(s + o2 + r16);
    v[0] = a.x; v[1] = a.y;
    v[2] = c0.x; v[3] = c0.y; v[4] = c0.z; v[5] = c0.w;
    v[6] = c1.x; v[7] = c1.y; v[8] = c1.z; v[9] = c1.w;
    v[10] = b.x; v[11] = b.y;
}

}  // namespace

// One warp task as the kernel body sees it: its descriptors, the tensor maps
// of its source field, its output field, its grid's bucket counts (for the
// lane layout) and control block (for errors), and where its sum goes.
struct TmaRef {
    const int32_t *desc;      // the task's 64 descriptor words
    const uint32_t *trm;      // the task's 120 region-mask words
    const CUtensorMap *maps;  // 8 box shapes over the source field
    float *y;
    Ctrl *ctrl;
    int c1, c2, c3;           // bucket counts of the task's grid
    int t;                    // task index within its grid
    int gi;                   // grid index (0 for one grid)
};

// The tasks of one grid.
struct OneGridTasks {
    DevGrid g;
    const CUtensorMap *maps;
    float *y;
    int c1, c2, c3, tasks;
    __device__ __forceinline__ int total() const { return tasks; }
    __device__ __forceinline__ TmaRef at(int T) const
    {
        TmaRef r;
        r.desc = g.tma_desc + (long long)T * 64;
        r.trm = g.tma_rmask + (long long)T * 120;
        r.maps = maps;
        r.y = y;
        r.ctrl = g.ctrl;
        r.c1 = c1; r.c2 = c2; r.c3 = c3;
        r.t = T;
        r.gi = 0;
        return r;
    }
};

// The concatenated tasks of a batch of grids; s_off (shared memory) holds
// each grid's first task index and the total.
struct BatchTasks {
    const BatchGrid *items;
    const int *s_off;
    int n_grids, total_tasks;
    __device__ __forceinline__ int total() const { return total_tasks; }
    __device__ __forceinline__ TmaRef at(int T) const
    {
        int lo = 0, hi = n_grids - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= T) lo = mid;
            else hi = mid - 1;
        }
        const BatchGrid &it = items[lo];
        const int t = T - s_off[lo];
        TmaRef r;
        r.desc = it.g.tma_desc + (long long)t * 64;
        r.trm = it.g.tma_rmask + (long long)t * 120;
        r.maps = reinterpret_cast<const CUtensorMap *>(it.tma_maps);
        r.y = it.y;
        r.ctrl = it.g.ctrl;
        r.c1 = it.c1; r.c2 = it.c2; r.c3 = it.c3;
        r.t = t;
        r.gi = lo;
        return r;
    }
};

// The per-warp task loop of the staged kernels: warp w of CTA c takes tasks
// c * kTmaWarps + w + k * W (W warps in the launch), each staged in two
// halves as described at the top of the file.  Returns this lane's FP64 sum
// of the outputs it wrote (one grid) or adds each task's warp sum to
// acc[grid] (batch, acc != null).
template <bool SUM, class Tasks>
__device__ __forceinline__ double tma_task_loop(const Tasks &src, float coef, double *acc_batch)
{
    extern __shared__ uint8_t s_dyn[];
    __shared__ __align__(8) uint64_t s_bar[kTmaWarps][2];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    uint8_t *base = s_dyn + ((128u - (smem_addr(s_dyn) & 127u)) & 127u);
    uint8_t *bufA = base + warp * kWarpBytes;
    uint8_t *bufB = bufA + kHalfABytes;
    const uint32_t sA = smem_addr(bufA), sB = smem_addr(bufB);
    const uint32_t barA = smem_addr(&s_bar[warp][0]), barB = smem_addr(&s_bar[warp][1]);
    if (lane == 0) {
        mbar_init(barA, 1);
        mbar_init(barB, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    const int tasks = src.total();
    const int W = gridDim.x * kTmaWarps;
    const float c6 = 1.f - 6.f * coef;
    double acc = 0.0;
    bool ok = true;
    uint32_t phase = 0;
    uint32_t issuedA = 0, doneA = 0, issuedB = 0, doneB = 0;  // half copies issued / seen complete

    int T = blockIdx.x * kTmaWarps + warp;
    TmaRef cur{}, nxt{}, nn{};
    int dc0 = 0, dc1 = 0, dn0 = 0, dn1 = 0, dnn0 = 0, dnn1 = 0;
    if (T < tasks) {
        cur = src.at(T);
        dc0 = __ldg(cur.desc + lane);
        dc1 = __ldg(cur.desc + 32 + lane);
        if (T + W < tasks) {
            nxt = src.at(T + W);
            dn0 = __ldg(nxt.desc + lane);
            dn1 = __ldg(nxt.desc + 32 + lane);
        }
        if (T + 2 * W < tasks) {
            nn = src.at(T + 2 * W);
            dnn0 = __ldg(nn.desc + lane);
            dnn1 = __ldg(nn.desc + 32 + lane);
        }
        const int kind = __shfl_sync(kFull, dc1, 31);
        issue_half(0, kind, dc0, dc1, sA, barA, cur.maps, cur.trm);
        issue_half(1, kind, dc0, dc1, sB, barB, cur.maps, nullptr);
        issuedA = issuedB = 1;
    }
    for (; T < tasks; T += W) {
        const int Tn = T + W;
        const int kind = __shfl_sync(kFull, dc1, 31);
        const int c1 = cur.c1, c2 = cur.c2, c3 = cur.c3, t = cur.t;
        // this lane's piece, row and output leaf (the lane layout of k_sweep_jruns)
        int jj, G, sb;
        bool valid, inA;
        if (kind == 0) {
            inA = true;
            valid = lane < 28; G = 3; sb = 0; jj = lane - 2;
        } else if (kind == 1) {
            const int p = c2 < c1 ? c2 : c1;
            inA = lane < 20;
            valid = inA || (t - c3 < p);
            G = inA ? 2 : 1; sb = inA ? 0 : 4; jj = inA ? lane - 2 : lane - 22;
        } else {
            const int p = c2 < c1 ? c2 : c1;
            const int q = p + 2 * (t - c3 - c2);
            inA = lane < 12;
            valid = inA || (lane < 24 && q + 1 < c1);
            G = 1; sb = inA ? 0 : 3; jj = inA ? lane - 2 : lane - 14;
        }
        const int m = jj < 0 ? 0 : min(jj >> 3, G - 1);
        const int tj = jj - 8 * m + 1;
        const bool full = jj >= 0 && jj < 8 * G;
        const int seg = jj < 0 ? sb : (full ? sb + 1 + (jj >> 3) : sb + G + 1);
        const int row = jj < 0 ? jj + 2 : (full ? (jj & 7) : jj - 8 * G);
        const bool tlane = valid && tj >= 0 && tj <= 9;
        const bool outlane = valid && full;
        const int oidx = (sb + 1 + m) * 9 + 4;
        const int o0 = __shfl_sync(kFull, dc0, oidx & 31), o1 = __shfl_sync(kFull, dc1, oidx & 31);
        const int own = oidx < 32 ? o0 : o1;
        // region masks of the lane's leaf: full segment f of the task
        const int f = inA ? m : (kind == 1 ? 2 : 1);
        const int so = seg_off(kind, seg);
        const uint8_t *segA = bufA + so, *segB = bufB + so;
        const int r16 = row * 16, r32 = row * 32;
        float *__restrict__ y = cur.y;
        float part = 0.f;

        if (mbar_wait(barA, phase)) {
            ++doneA;
        } else {
            ok = false;
            atomicOr(&cur.ctrl->err, kErrTimeout);
            cur.ctrl->timeout_site = 4;
        }
        uint4 rm = make_uint4(0u, 0u, 0u, 0u);
        if (tlane) rm = *reinterpret_cast<const uint4 *>(bufA + kHalfBytes + f * 160 + tj * 16);
        const uint32_t rmw[4] = {rm.x, rm.y, rm.z, rm.w};
        float xa[12], xb[12], xc[12];
        srow<0>(segA, segB, full, r16, r32, xa);
        srow<1>(segA, segB, full, r16, r32, xb);
        float p1[10], p2[10];
        uint32_t mprev = 0;
#define SG_TMA_STEP(S)                                                                                            \
    {                                                                                                            \
        srow<(S) + 2>(segA, segB, full, r16, r32, xc);                                                           \
        const uint32_t mt = (rmw[(S) / 3] >> (10 * ((S) % 3))) & 0x3ffu;                                          \
        float up[12], dn[12];                                                                                    \
        _Pragma("unroll") for (int q = 0; q < 12; ++q)                                                           \
        {                                                                                                        \
            up[q] = __shfl_up_sync(kFull, xb[q], 1);                                                             \
            dn[q] = __shfl_down_sync(kFull, xb[q], 1);                                                           \
        }                                                                                                        \
        float tt[10];                                                                                            \
        _Pragma("unroll") for (int q = 0; q < 10; ++q)                                                           \
        {                                                                                                        \
            const float nb = ((xb[q] + xb[q + 2]) + (xa[q + 1] + xc[q + 1])) + (up[q + 1] + dn[q + 1]);         \
            tt[q] = pick(mt, q, fmaf(coef, nb, c6 * xb[q + 1]));                                                  \
        }                                                                                                        \
        float tu[10], td[10], p0[10];                                                                            \
        _Pragma("unroll") for (int q = 0; q < 10; ++q)                                                           \
        {                                                                                                        \
            tu[q] = __shfl_up_sync(kFull, tt[q], 1);                                                             \
            td[q] = __shfl_down_sync(kFull, tt[q], 1);                                                           \
        }                                                                                                        \
        _Pragma("unroll") for (int q = 0; q < 10; ++q) p0[q] = (tu[q] + tt[q]) + td[q];                           \
        if ((S) >= 2) {                                                                                          \
            float Sm[10];                                                                                        \
            _Pragma("unroll") for (int q = 0; q < 10; ++q) Sm[q] = (p2[q] + p1[q]) + p0[q];                       \
            const uint32_t bits = (mprev >> 1) & 0xffu;                                                          \
            float o[8];                                                                                          \
            _Pragma("unroll") for (int k = 0; k < 8; ++k) o[k] =                                                 \
                pick(bits, k, ((Sm[k] + Sm[k + 1]) + Sm[k + 2]) * (1.f / 27.f));                                 \
            if (outlane) {                                                                                       \
                float *op = y + (long long)own * 512 + ((S) - 2) * 64 + (tj - 1) * 8;                            \
                stg4(op, o[0], o[1], o[2], o[3]);                                                                \
                stg4(op + 4, o[4], o[5], o[6], o[7]);                                                            \
                if (SUM) part += ((o[0] + o[1]) + (o[2] + o[3])) + ((o[4] + o[5]) + (o[6] + o[7]));               \
            }                                                                                                    \
        }                                                                                                        \
        _Pragma("unroll") for (int q = 0; q < 10; ++q)                                                           \
        {                                                                                                        \
            p2[q] = p1[q];                                                                                       \
            p1[q] = p0[q];                                                                                       \
        }                                                                                                        \
        mprev = mt;                                                                                              \
        _Pragma("unroll") for (int q = 0; q < 12; ++q)                                                           \
        {                                                                                                        \
            xa[q] = xb[q];                                                                                       \
            xb[q] = xc[q];                                                                                       \
        }                                                                                                        \
    }
        SG_TMA_STEP(0)
        SG_TMA_STEP(1)
        SG_TMA_STEP(2)
        SG_TMA_STEP(3)
        // the first half is consumed: refill it with the next task's
        __syncwarp();
        fence_proxy_async();
        const int kn = __shfl_sync(kFull, dn1, 31);
        if (ok && Tn < tasks) {
            issue_half(0, kn, dn0, dn1, sA, barA, nxt.maps, nxt.trm);
            ++issuedA;
        }
        if (mbar_wait(barB, phase)) {
            ++doneB;
        } else {
            ok = false;
            atomicOr(&cur.ctrl->err, kErrTimeout);
            cur.ctrl->timeout_site = 4;
        }
        SG_TMA_STEP(4)
        SG_TMA_STEP(5)
        SG_TMA_STEP(6)
        SG_TMA_STEP(7)
        SG_TMA_STEP(8)
        SG_TMA_STEP(9)
#undef SG_TMA_STEP
        __syncwarp();
        fence_proxy_async();
        if (ok && Tn < tasks) {
            issue_half(1, kn, dn0, dn1, sB, barB, nxt.maps, nullptr);
            ++issuedB;
        }
        if (acc_batch) {
            const double w = warp_sum((double)part);
            if (lane == 0) atomicAdd(&acc_batch[cur.gi], w);
        } else {
            acc += (double)part;
        }
        phase ^= 1u;
        cur = nxt;
        dc0 = dn0; dc1 = dn1;
        nxt = nn;
        dn0 = dnn0; dn1 = dnn1;
        if (Tn + 2 * W < tasks) {
            nn = src.at(Tn + 2 * W);
            dnn0 = __ldg(nn.desc + lane);
            dnn1 = __ldg(nn.desc + 32 + lane);
        }
        if (!ok) break;
    }
    // after a wait gave up: wait (bounded) for the copies still in flight
    if (!ok) {
        if (issuedA > doneA) (void)mbar_wait(barA, doneA & 1u);
        if (issuedB > doneB) (void)mbar_wait(barB, doneB & 1u);
    }
    return acc;
}

template <bool SUM>
__global__ void __launch_bounds__(kTmaWarps * 32, 1) k_sweep_tma(DevGrid g, const __grid_constant__ TmaMaps maps,
                                                                  int src, int dst, float coef, int sum_slot)
{
    __shared__ double s_red[kTmaWarps];
    OneGridTasks tk;
    tk.g = g;
    tk.maps = maps.m;
    tk.y = g.field[dst];
    tk.c3 = g.col_cnt[2];
    tk.c2 = g.col_cnt[1];
    tk.c1 = g.col_cnt[0];
    tk.tasks = num_tasks(tk.c3, tk.c2, tk.c1);
    (void)src;
    double acc = tma_task_loop<SUM>(tk, coef, nullptr);
    if (SUM) {
        acc = warp_sum(acc);
        if (lane_id() == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        double tot = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < kTmaWarps; ++w) tot += s_red[w];
        finish_reduction(g, tot, sum_slot);
    }
}

// Batched form: every grid's fused step in one launch over the concatenated
// task lists, each task's warp sum added to acc[grid] (zeroed by the caller).
__global__ void __launch_bounds__(kTmaWarps * 32, 1) k_batch_tma(const BatchGrid *__restrict__ items, int n_grids,
                                                                  int total_tasks, float coef, double *acc)
{
    __shared__ int s_off[kMaxBatch + 1];
    for (int i = threadIdx.x; i <= n_grids; i += blockDim.x) s_off[i] = (i < n_grids) ? items[i].tri0 : total_tasks;
    __syncthreads();
    BatchTasks tk;
    tk.items = items;
    tk.s_off = s_off;
    tk.n_grids = n_grids;
    tk.total_tasks = total_tasks;
    (void)tma_task_loop<true>(tk, coef, acc);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

int sweep_tma_ctas(int num_sms) { return num_sms; }

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// The eight box shapes over field f viewed as [cap + 1][8][8][8] floats.
bool make_maps(const float *base, long long cap, TmaMaps &out)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[4] = {8, 8, 8, (cuuint64_t)(cap + 1)};
    const cuuint64_t strides[3] = {32, 256, 2048};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    for (int mi = 0; mi < 8; ++mi) {
        const cuuint32_t box[4] = {(mi & 1) ? 8u : 4u, (mi & 2) ? 8u : 2u, (mi & 4) ? 4u : 2u, 1u};
        const CUresult r = enc(&out.m[mi], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides,
                               box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

}  // namespace

bool tma_encode_maps(const float *field, long long cap, void *out)
{
    static_assert(sizeof(TmaMaps) == kTmaMapsBytes, "tensor map block size");
    return make_maps(field, cap, *reinterpret_cast<TmaMaps *>(out));
}

int launch_batch_tma(const BatchGrid *items, int n_grids, int total_tri, float coef, double *acc, int num_sms,
                     cudaStream_t s)
{
    static std::atomic<int> attr_set{0};
    if (!attr_set.load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(k_batch_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmem) != cudaSuccess)
            return 1;
        attr_set.store(1, std::memory_order_release);
    }
    k_batch_tma<<<sweep_tma_ctas(num_sms), kTmaWarps * 32, kTmaSmem, s>>>(items, n_grids, total_tri, coef, acc);
    return 0;
}

void launch_tma_tasks(const DevGrid &g, cudaStream_t s, const LaunchCfg &lc)
{
    k_tma_tasks<<<lc.num_sms * 4, 256, 0, s>>>(g);
}


int launch_sweep_tma(const DevGrid &g, cudaStream_t s, int src, int dst, float coef, int sum_slot, const LaunchCfg &lc)
{
    static std::atomic<int> attr_set{0};
    if (!attr_set.load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(k_sweep_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmem) != cudaSuccess ||
            cudaFuncSetAttribute(k_sweep_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmem) != cudaSuccess)
            return 1;
        attr_set.store(1, std::memory_order_release);
    }
    TmaMaps maps;
    if (!make_maps(g.field[src], g.cap, maps)) return 2;
    if (sum_slot >= 0)
        k_sweep_tma<true><<<sweep_tma_ctas(lc.num_sms), kTmaWarps * 32, kTmaSmem, s>>>(g, maps, src, dst, coef, sum_slot);
    else
        k_sweep_tma<false><<<sweep_tma_ctas(lc.num_sms), kTmaWarps * 32, kTmaSmem, s>>>(g, maps, src, dst, coef, sum_slot);
    return 0;
}

}  // namespace sg
