// sg_noalloc.cu -- active-list compaction that allocates no device memory.
//
// The same list generation as k_listgen (non-null pointer cells compacted in
// ascending order with a decoupled look-back prefix sum), for callers that
// cannot allocate: its scratch -- the per-tile look-back words and four
// counters -- lives in a file-scope static device array that every GPU loading
// the library holds until the process exits.  The caller passes the pointer
// array in and the list and count out.
#include <mutex>

#include "../../include/sgrid.h"
#include "sg_common.cuh"

namespace sg {

constexpr long long kNoAllocMaxCells = SG_NOALLOC_MAX_CELLS;  // 4,194,304 pointer cells
constexpr int kNoAllocTiles = (int)(kNoAllocMaxCells / kListTile);     // 4096 look-back words
constexpr int kNaTicket = kNoAllocTiles, kNaTimeout = kNoAllocTiles + 1, kNaDone = kNoAllocTiles + 2,
              kNaTotal = kNoAllocTiles + 3;

// [0, kNoAllocTiles): look-back words; then ticket, timeout flag, finished
// tiles and list length.  32,800 bytes.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocTiles + 4];

constexpr unsigned long long kNaAgg = 1ull << 32, kNaIncl = 2ull << 32;
constexpr unsigned long long kNaWaitLimitNs = 1000000000ull;  // 1 s

__global__ void __launch_bounds__(kListThreads) k_compact_noalloc(const int32_t *__restrict__ root, long long nr,
                                                                   int32_t *list_slot, int32_t *list_b, long long cap,
                                                                   int32_t *count, int num_tiles,
                                                                   unsigned long long *scratch)
{
    __shared__ int s_tile, s_prefix;
    __shared__ int s_wsum[kListThreads / 32];
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    if (tid == 0) s_tile = (int)atomicAdd(&scratch[kNaTicket], 1ull);
    __syncthreads();
    const int tile = s_tile;
    const long long c0 = (long long)tile * kListTile + tid * 4;
    int sl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) sl[q] = (c0 + q < nr) ? root[c0 + q] : -1;
    const int cnt = (sl[0] >= 0) + (sl[1] >= 0) + (sl[2] >= 0) + (sl[3] >= 0);
    const int incl = warp_incl_scan(cnt);
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kListThreads / 32; ++w) {
        wbase += (w < warp) ? s_wsum[w] : 0;
        total += s_wsum[w];
    }
    if (tid == 0) atomicExch(&scratch[tile], (tile == 0 ? kNaIncl : kNaAgg) | (unsigned)total);
    if (warp == 0) {
        int prefix = 0;
        if (tile > 0) {
            int pred = tile - 1;
            const unsigned long long t0 = global_timer_ns();
            for (;;) {
                const int idx = pred - lane;
                unsigned long long w = kNaIncl;
                if (idx >= 0) {
                    for (;;) {
                        w = *(volatile unsigned long long *)&scratch[idx];
                        if (w != 0ull) break;
                        if (global_timer_ns() - t0 > kNaWaitLimitNs) {
                            scratch[kNaTimeout] = 1ull;
                            w = kNaIncl;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                const bool is_incl = (w >> 32) == 2ull;
                const int val = (int)(w & 0xffffffffull);
                const unsigned im = __ballot_sync(kFull, is_incl);
                const int upto = im ? (__ffs(im) - 1) : 31;
                prefix += warp_sum(lane <= upto ? val : 0);
                if (im) break;
                pred -= 32;
            }
            if (lane == 0) atomicExch(&scratch[tile], kNaIncl | (unsigned)(prefix + total));
        }
        if (lane == 0) s_prefix = prefix;
    }
    __syncthreads();
    int pos = s_prefix + wbase + incl - cnt;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (sl[q] >= 0) {
            if (pos < cap) {
                list_slot[pos] = sl[q];
                list_b[pos] = (int32_t)(c0 + q);
            }
            ++pos;
        }
    }
    if (tid == 0) {
        if (tile == num_tiles - 1) scratch[kNaTotal] = (unsigned long long)(s_prefix + total);
        __threadfence();
        const unsigned long long d = atomicAdd(&scratch[kNaDone], 1ull);
        if (d == (unsigned long long)num_tiles - 1ull) {
            __threadfence();
            const bool gave_up = *(volatile unsigned long long *)&scratch[kNaTimeout] != 0ull;
            *count = gave_up ? -1 : (int32_t) * (volatile unsigned long long *)&scratch[kNaTotal];
        }
    }
}

// Address of the scratch array on each device, looked up once per device
// (with that device current) by the first call made on it.
static std::mutex g_noalloc_mutex;
static unsigned long long *g_noalloc_ptr[256];

}  // namespace sg

using namespace sg;

extern "C" int sg_list_gen_noalloc(const int32_t *dev_root, int64_t n_cells, int32_t *dev_list_slot,
                                   int32_t *dev_list_b, int64_t cap, int32_t *dev_count, void *cuda_stream)
{
    if (n_cells < 0 || n_cells > kNoAllocMaxCells || cap < 0 || !dev_count || (n_cells > 0 && !dev_root) ||
        (cap > 0 && (!dev_list_slot || !dev_list_b)))
        return SG_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return SG_ERR_CUDA;
    unsigned long long *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return SG_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = (unsigned long long *)p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    if (n_cells == 0) return cudaMemsetAsync(dev_count, 0, sizeof(int32_t), s) == cudaSuccess ? SG_OK : SG_ERR_CUDA;
    const int num_tiles = (int)((n_cells + kListTile - 1) / kListTile);
    // the array keeps the previous call's contents: zero the look-back words
    // this call uses and the four counters
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * num_tiles, s) != cudaSuccess ||
        cudaMemsetAsync(scratch + kNaTicket, 0, sizeof(unsigned long long) * 4, s) != cudaSuccess)
        return SG_ERR_CUDA;
    k_compact_noalloc<<<num_tiles, kListThreads, 0, s>>>(dev_root, n_cells, dev_list_slot, dev_list_b, cap, dev_count,
                                                         num_tiles, scratch);
    return cudaPeekAtLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}
