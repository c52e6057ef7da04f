// sg_api.cu -- the C ABI of libsgrid: grid lifetime, the deferred op queue,
// and the inter-kernel optimizer that runs on flush.
//
// The queue follows AsyncTaichi's asynchronous engine (Sec. 5, Sec. 7.1):
// calls only enqueue; sg_flush (explicit, non-blocking) or any host read
// (implicit) optimizes the queued ops and launches them.  The optimizer works
// on a fixed op vocabulary instead of a general state-flow graph; what it
// needs of the SFG (Sec. 4) is the version of each grid's mask and list
// states, kept on the host across flushes (the partial garbage collection of
// Sec. 7.1 keeps the latest owners alive for the same purpose):
//   - list-generation removal (Sec. 6.2): a list generated from the current
//     mask version is reused; a device flag lets a launched list generation
//     skip itself when no activation changed anything;
//   - activation demotion (Sec. 6.3): a shell activation identical to one
//     applied since the last deactivation is a no-op and is dropped, and
//     struct-for stores skip the activation check (their targets are the loop
//     indices over the same, unchanged list);
//   - task fusion (Sec. 6.4, Supplement Sec. 2): adjacent struct-fors over the
//     same list are merged when a fused kernel exists for the sequence;
//   - dead-store elimination (Sec. 6.5): a clear fully overwritten before it
//     is read is dropped, and a scratch intermediate consumed inside a fused
//     kernel is never stored.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sgrid.h"
#include "sg_device.h"

using namespace sg;

namespace {

thread_local std::string t_last_error;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return code;
}

enum OpKind { OP_ACT_SHELL, OP_ACT_COORDS, OP_DEACT, OP_LISTGEN, OP_STENCIL, OP_SUM, OP_P2G, OP_GRID_UPDATE, OP_G2P, OP_TEST_WAIT,
              OP_FILL, OP_G2P2G, OP_EW, OP_ADVECT, OP_MAC, OP_WRITE_STAGED, OP_SORT_P };

struct Op {
    OpKind kind;
    int op = 0;          // stencil op code
    int src = 0, dst = 0;  // physical field indices
    bool dst_scratch = false;
    float coef = 0.f;
    long long lo2 = 0, hi2 = 0;
    int strict = 0;
    const void *p0 = nullptr;
    void *p1 = nullptr, *p2 = nullptr, *p3 = nullptr;
    const sg_grid *peer = nullptr, *bins = nullptr;  // G2P2G: source grid, holder of the particle bins
    long long n = 0;
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    int i0 = 0, i1 = 0, i2 = 0;
    long long slot = 0;
};

}  // namespace

// Single stencils switch to the j-run sweep on a list of at least this many
// leaves, after this many sweeps without its run records.
constexpr long long kSingleRunsLeaves = 8192;
constexpr int kSingleRunsAfter = 2;

struct sg_grid {
    sg_desc desc{};
    cudaStream_t stream = nullptr;
    bool dry = false;
    DevGrid dev{};
    LaunchCfg lc{};
    int num_tiles = 1;
    int phys[SG_MAX_FIELDS];
    uint32_t opts = SG_OPT_ALL;
    std::vector<Op> queue;
    // host-side state versions (Sec. 4): mask and list of the grid's structure
    unsigned long long mask_ver = 1, list_ver = 0;
    std::set<std::tuple<long long, long long, int, int>> applied_shells;
    // restrictions applied since the last deactivation: (fine grid, its mask version)
    std::set<std::pair<const sg_grid *, unsigned long long>> applied_restrict;
    unsigned long long lg_calls = 0;
    unsigned long long rmask_ver = 0;  // list version the region masks were built from (0 = never)
    unsigned long long colgrp_ver = 0; // list version the run records were built from (0 = never)
    unsigned long long single_ver = 0; // list version single stencils have swept without run records
    int single_uses = 0;               // how many times
    int colgrp_axis = kGroupNone;      // axis they group leaves along
    unsigned long long tma_ver = 0;    // list version the TMA task descriptors were built from (0 = never)
    unsigned long long rr_calls = 0;   // region-mask launches (tags their look-back words)
    long long tma_entries = 0;         // warp tasks the TMA descriptor arrays hold
    int max_fuse = kMaxEwOps;          // element-wise ops per fused launch
    int flush_period = 0;              // flush once the queue holds this many ops (0: on sync / sg_flush only)
    long long known_leaves = 0;
    sg_stats stats{};
    int latched = SG_OK;
    std::vector<void *> blocks;
    Ctrl *host_ctrl = nullptr;  // pinned
    size_t staging_bytes = 0;
    long long perm_cap = 0;  // particles the binned-P2G order array holds
    void *sort_tmp = nullptr;  // particle reordering scratch, 36 bytes per particle
    long long sort_cap = 0;
    const void *p2g_x = nullptr;  // positions and count the order array was built for
    long long p2g_n = 0;
    unsigned long long *chk_cnt = nullptr;  // invariant-check counters (allocated at the first check)
    long long *act_off = nullptr;           // active-voxel transfer offsets, [cap] and [cap / kOffTile + 2]
    long long *act_tsum = nullptr;
    unsigned long long act_ver = 0;         // list version the offsets were computed for (0 = never)
    long long act_total = 0;
    float *adv_lo[3] = {}, *adv_hi[3] = {}; // advection clamp bounds, (cap + 1) * L^3 each (allocated at first use)
    float4 *adv_vel4 = nullptr;             // packed advection velocity, (cap + 1) * L^3 (allocated at first use)
    // staged uploads (sg_stage_active): two slots filled on a copy stream of
    // the grid's own, each consumed by a queued scatter
    cudaStream_t copy_stream = nullptr;
    float *upload[2] = {};
    cudaEvent_t copied[2] = {}, consumed[2] = {};
    bool slot_used[2] = {};
    long long upload_n[2] = {};
    unsigned upload_seq[2] = {};
    unsigned next_seq = 1;
};

namespace {

void *dev_alloc(sg_grid *g, size_t bytes)
{
    bytes = (bytes + 255) & ~size_t(255);
    void *p = nullptr;
    if (g->desc.alloc) {
        p = g->desc.alloc(bytes, g->desc.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) g->blocks.push_back(p);
    return p;
}

// Free one of g's blocks and forget it; the caller has made sure that no
// queued or running work still uses it.
void dev_release(sg_grid *g, void *p)
{
    if (!p) return;
    const auto it = std::find(g->blocks.begin(), g->blocks.end(), p);
    if (it == g->blocks.end()) return;
    g->blocks.erase(it);
    if (g->desc.free) g->desc.free(p, g->desc.alloc_ctx);
    else cudaFree(p);
}

void dev_free_all(sg_grid *g)
{
    for (void *p : g->blocks) {
        if (g->desc.free) g->desc.free(p, g->desc.alloc_ctx);
        else cudaFree(p);
    }
    g->blocks.clear();
}

int cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SG_OK;
    return fail(SG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int after_launch(sg_grid *g, const char *what)
{
    g->stats.launches++;
    if (g->dry) return SG_OK;
    return cuda_check(cudaPeekAtLastError(), what);
}

bool valid_field(const sg_grid *g, int f) { return f >= 0 && f < g->desc.n_fields; }

// Room in the TMA task-descriptor arrays for `entries` warp tasks (a grid's
// tasks never exceed its list length, nor its pool capacity).  A larger
// request replaces the arrays, grown geometrically up to the pool capacity;
// the old ones are released with the grid, so they total less than the last.
int ensure_tma_desc(sg_grid *g, long long entries)
{
    entries = std::max(1LL, entries);
    if (g->tma_entries >= entries) return SG_OK;
    entries = std::max(entries, std::min(2 * g->tma_entries, (long long)g->dev.cap));
    g->dev.tma_desc = (int32_t *)dev_alloc(g, sizeof(int32_t) * 64 * entries);
    g->dev.tma_rmask = (uint32_t *)dev_alloc(g, sizeof(uint32_t) * 120 * entries);
    if (!g->dev.tma_desc || !g->dev.tma_rmask) {
        g->tma_entries = 0;
        g->dev.tma_desc = nullptr;
        g->dev.tma_rmask = nullptr;
        return fail(SG_ERR_OOM, "TMA task descriptors");
    }
    g->tma_entries = entries;
    g->tma_ver = 0;  // fresh arrays hold no descriptors yet
    return SG_OK;
}

// True while the grid's stream is being recorded into a graph (sg_graph_begin).
bool capturing(const sg_grid *g)
{
    if (g->dry) return false;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(g->stream, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st == cudaStreamCaptureStatusActive;
}

// A change of the grid's structure (new mask version).  Not allowed inside a
// graph recording: the host-side list and demotion state would not follow a
// replay, and list generation numbers its tiles per call.
int bump_structure(sg_grid *g)
{
    g->mask_ver++;
    if (capturing(g)) return fail(SG_ERR_INVALID, "a change of the structure cannot be recorded in a graph");
    return SG_OK;
}

int do_flush(sg_grid *g);

int push(sg_grid *g, Op op)
{
    g->queue.push_back(op);
    g->stats.ops_enqueued++;
    if (g->flush_period > 0 && (int)g->queue.size() >= g->flush_period) return do_flush(g);
    return SG_OK;
}

double leaf_bytes(const sg_grid *g) { return 4.0 * double(g->dev.L) * g->dev.L * g->dev.L; }

// ---- list state ------------------------------------------------------------
int launch_list(sg_grid *g, bool force, int test_wait)
{
    if (capturing(g)) return fail(SG_ERR_INVALID, "list generation cannot be recorded in a graph");
    if (!g->dry) launch_listgen(g->dev, g->stream, force ? 1 : 0, g->lg_calls, g->num_tiles, test_wait);
    g->lg_calls++;
    g->stats.listgen_run++;
    return after_launch(g, "list generation");
}

// Make the list current for a struct-for.  LGR off: the eager form's clear-list
// and list-generation tasks (Sec. 6.1, Fig. 8).  LGR on: nothing if the list was
// generated from the current mask version (Sec. 6.2).
int ensure_list(sg_grid *g)
{
    int rc;
    if (!(g->opts & SG_OPT_LGR)) {
        if (!g->dry) launch_clear_list(g->dev, g->stream);
        if ((rc = after_launch(g, "clear list"))) return rc;
        if ((rc = launch_list(g, true, 0))) return rc;
        g->list_ver = g->mask_ver;
        return SG_OK;
    }
    if (g->list_ver == g->mask_ver) {
        g->stats.listgen_removed++;
        return SG_OK;
    }
    if ((rc = launch_list(g, false, 0))) return rc;
    g->list_ver = g->mask_ver;
    return SG_OK;
}

// Is physical field f read (before being fully overwritten) by queue[from..)?
bool read_later(const sg_grid *g, size_t from, int f)
{
    for (size_t i = from; i < g->queue.size(); ++i) {
        const Op &o = g->queue[i];
        if ((o.kind == OP_STENCIL && o.op != SG_CLEAR && o.src == f) || (o.kind == OP_SUM && o.src == f)) return true;
        if (o.kind == OP_EW && (o.src == f || o.i0 == f)) return true;
        if ((o.kind == OP_ADVECT || o.kind == OP_MAC) &&
            (o.src == f || (f >= o.i0 && f < o.i0 + 3) || (o.kind == OP_MAC && (o.i1 == f || o.i2 == f))))
            return true;
        if (o.kind == OP_EW && o.dst == f) return false;  // fully overwritten
        if (o.kind == OP_P2G || o.kind == OP_GRID_UPDATE || o.kind == OP_G2P) return true;  // conservative
        if (o.kind == OP_STENCIL && o.dst == f) return false;  // fully overwritten
    }
    return false;
}

// The physical fields a leaf allocated by the activation at queue[i] is
// zero-filled in.  With SG_OPT_DSE the fill is a store like any other
// (Sec. 6.5): it is dead in a field whose next access in the queue is a full
// overwrite by a struct-for over the (then current) list, and in a field the
// rest of the flush does not touch that holds a scratch field, whose
// contents no later flush may read.  A read, a partial write (a staged
// upload, the particle ops), a fill or a structure change keeps it.
uint32_t activation_fill_mask(const sg_grid *g, size_t i)
{
    const int F = g->dev.F;
    const uint32_t all = F >= 32 ? 0xffffffffu : ((1u << F) - 1u);
    if (!(g->opts & SG_OPT_DSE)) return all;
    uint32_t scratch_phys = 0;
    for (int f = 0; f < F; ++f)
        if ((g->desc.scratch_mask >> f) & 1u) scratch_phys |= 1u << g->phys[f];
    uint32_t mask = 0;
    for (int pf = 0; pf < F; ++pf) {
        int first = 0;  // 0: untouched, 1: read or kept, 2: fully overwritten
        for (size_t k = i + 1; k < g->queue.size() && first == 0; ++k) {
            const Op &o = g->queue[k];
            switch (o.kind) {
                case OP_LISTGEN:
                case OP_SORT_P:
                    break;
                case OP_FILL:  // sets every voxel of the listed leaves (0 where inactive)
                    if (o.i0 == pf) first = 2;
                    break;
                case OP_STENCIL:
                    if (o.op != SG_CLEAR && o.src == pf) first = 1;
                    else if (o.dst == pf) first = 2;
                    break;
                case OP_SUM:
                    if (o.src == pf) first = 1;
                    break;
                case OP_EW:
                    if (o.src == pf || o.i0 == pf) first = 1;
                    else if (o.dst == pf) first = 2;
                    break;
                case OP_ADVECT:
                case OP_MAC:
                    if (o.src == pf || (pf >= o.i0 && pf < o.i0 + 3) || (o.kind == OP_MAC && (o.i1 == pf || o.i2 == pf)))
                        first = 1;
                    else if (o.dst == pf) first = 2;
                    break;
                default:
                    first = 1;  // conservative
            }
        }
        const bool dead = first == 2 || (first == 0 && ((scratch_phys >> pf) & 1u));
        if (!dead) mask |= 1u << pf;
    }
    return mask;
}

// Dead-store test for a clear at queue[i]: the next access to its field in
// the queue is a full overwrite by a struct-for over the same list.
bool clear_is_dead(const sg_grid *g, size_t i)
{
    const int f = g->queue[i].dst;
    for (size_t k = i + 1; k < g->queue.size(); ++k) {
        const Op &o = g->queue[k];
        if (o.kind == OP_EW) {
            if (o.src == f || o.i0 == f) return false;
            if (o.dst == f) return true;
            continue;
        }
        if (o.kind != OP_STENCIL && o.kind != OP_SUM) return false;  // structure may change
        if (o.kind == OP_SUM && o.src == f) return false;
        if (o.kind == OP_STENCIL && o.op != SG_CLEAR && o.src == f) return false;
        if (o.kind == OP_STENCIL && o.dst == f) return true;
    }
    return false;
}

int run_struct_for_group(sg_grid *g, size_t &i)
{
    int rc;
    const bool ad = (g->opts & SG_OPT_AD) != 0;
    const bool fuse = (g->opts & SG_OPT_FUSE) && (g->opts & SG_OPT_LGR);
    const bool dse = (g->opts & SG_OPT_DSE) != 0;
    const int check = ad ? 0 : 1;
    const Op &a = g->queue[i];
    const double lb = leaf_bytes(g) * double(g->known_leaves);

    if (a.kind == OP_STENCIL && a.op == SG_CLEAR && dse && clear_is_dead(g, i)) {
        g->stats.stores_removed++;
        i += 1;
        return SG_OK;
    }
    if ((rc = ensure_list(g))) return rc;
    auto next = [&](size_t k) -> const Op * { return (i + k < g->queue.size()) ? &g->queue[i + k] : nullptr; };

    if (a.kind == OP_SUM) {
        if (!g->dry) launch_sum(g->dev, g->stream, a.src, (int)a.slot, g->lc);
        g->stats.bytes_model += lb;
        i += 1;
        return after_launch(g, "sum");
    }
    if (a.op == SG_CLEAR) {
        if (!g->dry) launch_clear(g->dev, g->stream, a.dst, check, g->lc);
        g->stats.bytes_model += lb;
        i += 1;
        return after_launch(g, "clear");
    }
    const Op *b = next(1);
    if (fuse && g->dev.L == 8 && a.op == SG_DIFFUSE7 && b && b->kind == OP_STENCIL && b->op == SG_BOX27 &&
        b->src == a.dst && a.src != a.dst && b->dst != a.dst && b->dst != a.src) {
        // fused diffuse7 -> box27 (+ sum of its output)
        const Op *c = next(2);
        const bool with_sum = c && c->kind == OP_SUM && c->src == b->dst;
        const size_t after = i + (with_sum ? 3 : 2);
        const bool store_t = !(dse && a.dst_scratch && !read_later(g, after, a.dst));
        if (!store_t) g->stats.stores_removed++;
        // region masks (and, for the grouped sweeps, the run records) are
        // derived from the structure, cached with the list
        const int v = g->lc.variant;
        const bool sweep = v != kVariantSmem;
        const bool tma = v == kVariantSweepTma && !store_t && !check;
        const int axis = v == kVariantSweepColumns ? kGroupI
                         : ((v == kVariantSweepJRuns || v == kVariantSweepTma) ? kGroupJ : kGroupNone);
        const bool need_runs = axis != kGroupNone && (g->colgrp_ver != g->list_ver || g->colgrp_axis != axis);
        if ((sweep && g->rmask_ver != g->list_ver) || need_runs) {
            if (!g->dry) launch_region_masks(g->dev, g->stream, g->lc, need_runs ? axis : kGroupNone, ++g->rr_calls);
            if ((rc = after_launch(g, "region masks"))) return rc;
            g->rmask_ver = g->list_ver;
            if (need_runs) {
                g->colgrp_ver = g->list_ver;
                g->colgrp_axis = axis;
            }
        }
        if (tma && g->tma_ver != g->list_ver) {
            // the staged kernel's per-task box sources and region masks
            if (!g->dry && (rc = ensure_tma_desc(g, g->dev.cap))) return rc;
            if (!g->dry) launch_tma_tasks(g->dev, g->stream, g->lc);
            if ((rc = after_launch(g, "TMA task descriptors"))) return rc;
            g->tma_ver = g->list_ver;
        }
        if (!g->dry) {
            if (tma) {
                if (launch_sweep_tma(g->dev, g->stream, a.src, b->dst, a.coef, with_sum ? (int)c->slot : -1, g->lc))
                    return fail(SG_ERR_CUDA, "TMA-staged step: tensor maps or launch attributes unavailable");
            } else {
                launch_diffuse_box(g->dev, g->stream, a.src, a.dst, b->dst, a.coef, store_t ? 1 : 0, check,
                                   with_sum ? (int)c->slot : -1, g->lc);
            }
        }
        g->stats.ops_fused += with_sum ? 2 : 1;
        g->stats.bytes_model += lb * (store_t ? 3.0 : 2.0);
        i = after;
        return after_launch(g, "fused diffuse7+box27");
    }
    const Op *c = b;
    const bool with_sum = fuse && c && c->kind == OP_SUM && c->src == a.dst;
    const int sum_slot = with_sum ? (int)c->slot : -1;
    // A single stencil sweeps j-runs (no edge rows) when the run records are
    // current.  Building them is one launch that saves a few microseconds per
    // stencil on a large list, so it is done for a reused list (SG_OPT_LGR) of
    // at least kSingleRunsLeaves leaves (the count at the last sync) that
    // single stencils have already swept kSingleRunsAfter times -- and never
    // while the stream is being captured into a graph, which would replay the
    // one-off build with every launch.
    LaunchCfg lcs = g->lc;
    if (g->dev.L == 8 && g->lc.variant == kVariantSweepJRuns) {
        if (g->colgrp_ver != g->list_ver || g->colgrp_axis != kGroupJ) {
            if (g->single_ver != g->list_ver) {
                g->single_ver = g->list_ver;
                g->single_uses = 0;
            }
            cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
            if (!g->dry) cudaStreamIsCapturing(g->stream, &cap);
            if ((g->opts & SG_OPT_LGR) && ++g->single_uses > kSingleRunsAfter && g->known_leaves >= kSingleRunsLeaves &&
                cap == cudaStreamCaptureStatusNone) {
                if (!g->dry) launch_region_masks(g->dev, g->stream, g->lc, kGroupJ, ++g->rr_calls);
                if ((rc = after_launch(g, "region masks"))) return rc;
                g->rmask_ver = g->list_ver;
                g->colgrp_ver = g->list_ver;
                g->colgrp_axis = kGroupJ;
            }
        }
        lcs.single_runs = (g->colgrp_ver == g->list_ver && g->colgrp_axis == kGroupJ) ? 1 : 0;
    }
    if (a.op == SG_DIFFUSE7) {
        if (!g->dry) launch_diffuse7(g->dev, g->stream, a.src, a.dst, a.coef, check, sum_slot, lcs);
    } else {
        if (!g->dry) launch_box27(g->dev, g->stream, a.src, a.dst, check, sum_slot, lcs);
    }
    g->stats.bytes_model += 2.0 * lb;
    if (with_sum) g->stats.ops_fused += 1;
    i += with_sum ? 2 : 1;
    return after_launch(g, "stencil");
}

// A run of element-wise ops from queue[i] (and at most one reduction inside
// it) as one launch (Sec. 6.4): consecutive ops over the same list whose
// accesses are all at the iteration's voxel, at most max_fuse ops and
// kMaxEwSlots distinct fields.  Fields read before written are loaded once;
// a written field is stored once, and not at all when it is scratch and no
// later queued op reads it (Sec. 6.5).  Without fusion each op is a launch.
//
// Dead ops of a fused run: an op whose result is overwritten before anything
// reads it, and that is not the slot's final stored value, is removed (the
// register-level counterpart of the dead stores above); the loads are then
// the slots the remaining ops read before writing.
void drop_dead_ew_ops(EwProgram &p)
{
    bool live[kMaxEwSlots];
    for (int k = 0; k < p.n_slots; ++k) live[k] = p.store[k] != 0;
    bool keep[kMaxEwOps + 1];
    for (int i = p.n_ops - 1; i >= 0; --i) {
        const EwOp &o = p.op[i];
        keep[i] = o.kind == kEwSum || live[o.dst];
        if (!keep[i]) continue;
        if (o.kind != kEwSum) live[o.dst] = false;
        if (o.kind != kEwFill) live[o.a] = true;
        if (o.kind == kEwAxby || o.kind == kEwGeneral) live[o.b] = true;
    }
    int n = 0;
    for (int i = 0; i < p.n_ops; ++i)
        if (keep[i]) p.op[n++] = p.op[i];
    p.n_ops = n;
    bool written[kMaxEwSlots] = {};
    for (int k = 0; k < p.n_slots; ++k) p.load[k] = 0;
    for (int i = 0; i < p.n_ops; ++i) {
        const EwOp &o = p.op[i];
        if (o.kind != kEwFill && !written[o.a]) p.load[o.a] = 1;
        if ((o.kind == kEwAxby || o.kind == kEwGeneral) && !written[o.b]) p.load[o.b] = 1;
        if (o.kind != kEwSum) written[o.dst] = true;
    }
}

int run_ew_group(sg_grid *g, size_t &i)
{
    int rc;
    if ((rc = ensure_list(g))) return rc;
    const bool fuse = (g->opts & SG_OPT_FUSE) && (g->opts & SG_OPT_LGR);
    const bool dse = (g->opts & SG_OPT_DSE) != 0;
    const int limit = fuse ? std::max(1, std::min(g->max_fuse, kMaxEwOps)) : 1;
    EwProgram p{};
    p.sum_out = -1;
    int slot_of[kMaxFields];
    for (int f = 0; f < kMaxFields; ++f) slot_of[f] = -1;
    bool written[kMaxEwSlots] = {}, scratch[kMaxEwSlots] = {};
    int writes[kMaxEwSlots] = {};
    auto needed = [&](int f) { return (f >= 0 && slot_of[f] < 0) ? 1 : 0; };
    auto use = [&](int f, bool write) -> int8_t {
        if (f < 0) return -1;
        if (slot_of[f] < 0) {
            slot_of[f] = p.n_slots;
            p.field[p.n_slots++] = f;
        }
        const int k = slot_of[f];
        if (!write && !written[k]) p.load[k] = 1;
        return (int8_t)k;
    };
    size_t j = i;
    int nops = 0;
    while (j < g->queue.size()) {
        const Op &o = g->queue[j];
        if (o.kind == OP_EW && nops < limit) {
            int add = needed(o.src) + needed(o.i0);
            add += (o.dst != o.src && o.dst != o.i0) ? needed(o.dst) : 0;
            if (p.n_slots + add > kMaxEwSlots) break;
            EwOp e;
            e.a = use(o.src, false);
            e.b = use(o.i0, false);
            e.dst = use(o.dst, true);
            e.alpha = o.f0;
            e.beta = o.f1;
            e.gamma = o.coef;
            e.delta = o.f2;
            ew_kind(e);
            p.op[p.n_ops++] = e;
            written[e.dst] = true;
            scratch[e.dst] = o.dst_scratch;
            writes[e.dst]++;
            ++nops;
            ++j;
        } else if (fuse && o.kind == OP_SUM && p.sum_out < 0 && nops > 0 && p.n_slots + needed(o.src) <= kMaxEwSlots) {
            EwOp e{};
            e.dst = -1;
            e.a = use(o.src, false);
            e.b = -1;
            ew_kind(e);
            p.op[p.n_ops++] = e;
            p.sum_out = (int)o.slot;
            ++j;
        } else {
            break;
        }
    }
    int stores = 0, loads = 0;
    for (int k = 0; k < p.n_slots; ++k) {
        if (!written[k]) continue;
        p.store[k] = !(dse && scratch[k] && !read_later(g, j, p.field[k]));
        stores += p.store[k];
        g->stats.stores_removed += writes[k] - (p.store[k] ? 1 : 0);
    }
    if (dse) drop_dead_ew_ops(p);
    for (int k = 0; k < p.n_slots; ++k) loads += p.load[k];
    if (!g->dry) launch_ew(g->dev, g->stream, p, g->lc);
    g->stats.ops_fused += (int64_t)(j - i) - 1;
    g->stats.bytes_model += leaf_bytes(g) * double(g->known_leaves) * double(loads + stores);
    i = j;
    return after_launch(g, "element-wise");
}

// ---- MacCormack advection: a run of OP_ADVECT / OP_MAC ops ----------------
// Read and write sets of an advection op (physical fields).
static void advect_sets(const Op &o, std::vector<int> &r, std::vector<int> &w)
{
    r = {o.src, o.i0, o.i0 + 1, o.i0 + 2};
    if (o.kind == OP_MAC) {
        r.push_back(o.i1);
        r.push_back(o.i2);
    }
    w = {o.dst};
}

static bool intersects(const std::vector<int> &a, const std::vector<int> &b)
{
    for (int x : a)
        for (int y : b)
            if (x == y) return true;
    return false;
}

// The run queue[i .. end) of advection ops as fused launches (Sec. 6.4,
// Supp. Sec. 2).  The ops' dependencies come from their read / write sets
// (the state-flow edges between them); ops whose dependencies are all issued
// are ready and mutually independent.  Ready backward advections whose output
// q~ a correction reads at the voxel (an element-wise connection) are fused
// with that correction, q~ then stored only if a later op reads it (Sec. 6.5);
// other ready ops with the same velocity and step are grouped, up to three
// channels per launch.  Without fusion each op is a launch, in queue order.
int run_advect_run(sg_grid *g, size_t &i)
{
    int rc;
    size_t end = i;
    while (end < g->queue.size() && (g->queue[end].kind == OP_ADVECT || g->queue[end].kind == OP_MAC)) ++end;
    const int n = (int)(end - i);
    const bool fuse = (g->opts & SG_OPT_FUSE) && (g->opts & SG_OPT_LGR);
    const bool dse = (g->opts & SG_OPT_DSE) != 0;
    std::vector<std::vector<int>> R(n), W(n), deps(n);
    for (int a = 0; a < n; ++a) advect_sets(g->queue[i + a], R[a], W[a]);
    for (int b = 0; b < n; ++b)
        for (int a = 0; a < b; ++a)
            if (intersects(W[a], R[b]) || intersects(W[a], W[b]) || intersects(R[a], W[b])) deps[b].push_back(a);
    std::vector<char> done(n, 0);
    auto issued = [&](int b, int except) {
        for (int a : deps[b])
            if (!done[a] && a != except) return false;
        return true;
    };
    // Clamp-bound reuse (with fusion): a forward advection whose q, velocity
    // and step a later correction of the run shares stores the min and max of
    // the values its samples read, and the correction reads them instead of
    // tracing the same path again -- provided no op of the run writes q or the
    // velocity.  slot_q[s] etc. describe what bound slot s holds.
    std::vector<int> run_writes;
    for (int a = 0; a < n; ++a) run_writes.insert(run_writes.end(), W[a].begin(), W[a].end());
    auto untouched = [&](int q, int v0) {
        for (int f : run_writes)
            if (f == q || (f >= v0 && f <= v0 + 2)) return false;
        return true;
    };
    int slot_q[3] = {-1, -1, -1}, slot_v0[3] = {-1, -1, -1};
    float slot_dt[3] = {0.f, 0.f, 0.f};
    // the bound arrays (6 x (cap + 1) x L^3 floats); without the memory for
    // them the corrections trace the forward path themselves
    auto ensure_bounds = [&]() -> bool {
        if (g->dry || g->adv_hi[2]) return true;
        const size_t bytes = sizeof(float) * size_t(g->dev.cap + 1) * g->dev.L * g->dev.L * g->dev.L;
        for (int c = 0; c < 3; ++c) {
            if (!g->adv_lo[c]) g->adv_lo[c] = (float *)dev_alloc(g, bytes);
            if (!g->adv_hi[c]) g->adv_hi[c] = (float *)dev_alloc(g, bytes);
            if (!g->adv_lo[c] || !g->adv_hi[c]) return false;
        }
        return true;
    };
    // Velocity packing (with fusion): when two or more advections of the run
    // trace through the velocity of its first advection and no op of the run
    // writes it, the three fields are packed once (before the first launch
    // that traces) and every launch with that velocity reads the packed copy.
    int pack_v0 = -1;
    bool packed = false;
    if (fuse) {
        int tracers = 0;
        for (int a = 0; a < n; ++a) {
            const Op &o = g->queue[i + a];
            if (o.kind != OP_ADVECT) continue;
            if (pack_v0 < 0) pack_v0 = o.i0;
            if (o.i0 == pack_v0) ++tracers;
        }
        if (tracers < 2) pack_v0 = -1;
        for (int f : run_writes)
            if (pack_v0 >= 0 && f >= pack_v0 && f <= pack_v0 + 2) pack_v0 = -1;
    }
    auto ensure_vel4 = [&]() -> bool {
        if (g->dry || g->adv_vel4) return true;
        const size_t per_leaf = size_t(g->dev.L) * g->dev.L * g->dev.L;
        g->adv_vel4 = (float4 *)dev_alloc(g, sizeof(float4) * size_t(g->dev.cap + 1) * per_leaf);
        if (!g->adv_vel4) return false;
        // the zero leaf's block: never written by the packing, read as zeros
        return cudaMemsetAsync(g->adv_vel4 + size_t(g->dev.cap) * per_leaf, 0, sizeof(float4) * per_leaf,
                               g->stream) == cudaSuccess;
    };
    auto launch = [&](int mode, const std::vector<int> &ops, const std::vector<int> &macs) -> int {
        int r2;
        if ((r2 = ensure_list(g))) return r2;
        const Op &f = g->queue[i + ops[0]];
        const float4 *vel4 = nullptr;
        if (pack_v0 >= 0 && f.i0 == pack_v0) {
            if (!packed) {
                if (!ensure_vel4()) {
                    pack_v0 = -1;  // without the memory: read the three fields
                } else {
                    if (!g->dry) launch_pack_velocity(g->dev, g->stream, pack_v0, g->adv_vel4, g->lc);
                    g->stats.velocity_packs++;
                    packed = true;
                    if ((r2 = after_launch(g, "velocity packing"))) return r2;
                }
            }
            if (packed) vel4 = g->adv_vel4;
        }
        int dst[3], src[3], qh[3], qt[3];
        const int C = (int)ops.size();
        for (int c = 0; c < C; ++c) {
            const Op &o = g->queue[i + ops[c]];
            if (mode == 0) {
                dst[c] = o.dst;
                src[c] = o.src;
                qh[c] = qt[c] = -1;
            } else if (mode == 2) {
                dst[c] = o.dst;
                src[c] = o.src;
                qh[c] = o.i1;
                qt[c] = o.i2;
            } else {  // ops[c]: the backward advection, macs[c]: its correction
                const Op &m = g->queue[i + macs[c]];
                dst[c] = m.dst;
                src[c] = m.src;
                qh[c] = m.i1;
                const bool live = !(dse && o.dst_scratch && !read_later(g, end, o.dst));
                bool read_in_run = false;
                for (int b = 0; b < n; ++b)
                    if (!done[b] && b != ops[c] && b != macs[c] && std::count(R[b].begin(), R[b].end(), o.dst))
                        read_in_run = true;
                qt[c] = (live || read_in_run) ? o.dst : -1;
                if (qt[c] < 0) g->stats.stores_removed++;
            }
        }
        const float h = (mode == 1 ? g->queue[i + macs[0]].f0 : f.f0) * (float)g->dev.N;
        const float dt = mode == 1 ? g->queue[i + macs[0]].f0 : f.f0;
        float *lo[3] = {nullptr, nullptr, nullptr}, *hi[3] = {nullptr, nullptr, nullptr};
        bool bnd = false;
        if (fuse && mode == 0) {  // store bounds if a later correction can use them
            for (int c = 0; c < C && !bnd; ++c)
                for (int m = 0; m < n; ++m) {
                    const Op &mc = g->queue[i + m];
                    if (!done[m] && mc.kind == OP_MAC && mc.src == src[c] && mc.i0 == f.i0 && mc.f0 == dt &&
                        untouched(src[c], f.i0)) {
                        bnd = true;
                        break;
                    }
                }
            if (bnd && !ensure_bounds()) bnd = false;
            if (bnd) {
                for (int c = 0; c < 3; ++c) slot_q[c] = -1;
                for (int c = 0; c < C; ++c) {
                    lo[c] = g->adv_lo[c];
                    hi[c] = g->adv_hi[c];
                    slot_q[c] = src[c];
                    slot_v0[c] = f.i0;
                    slot_dt[c] = dt;
                }
            }
        } else if (fuse) {  // a correction: use stored bounds if every channel has them
            bnd = true;
            for (int c = 0; c < C && bnd; ++c) {
                int sl = -1;
                for (int k = 0; k < 3; ++k)
                    if (slot_q[k] == src[c] && slot_v0[k] == f.i0 && slot_dt[k] == dt) sl = k;
                if (sl < 0) bnd = false;
                else {
                    lo[c] = g->adv_lo[sl];
                    hi[c] = g->adv_hi[sl];
                }
            }
            if (!bnd)
                for (int c = 0; c < 3; ++c) lo[c] = hi[c] = nullptr;
        }
        if (bnd) g->stats.bounds_reused += (mode == 0) ? 0 : C;
        if (!g->dry)
            launch_advect_group(g->dev, g->stream, mode, C, dst, src, qh, qt, f.i0, h, bnd ? lo : nullptr,
                                bnd ? hi : nullptr, vel4, g->lc);
        g->stats.ops_fused += (int64_t)(mode == 1 ? 2 * C : C) - 1;
        for (int c : ops) done[c] = 1;
        for (int c : macs) done[c] = 1;
        return after_launch(g, "advection");
    };
    if (!fuse) {
        for (int a = 0; a < n; ++a) {
            const int mode = g->queue[i + a].kind == OP_ADVECT ? 0 : 2;
            rc = launch(mode, std::vector<int>{a}, std::vector<int>{});
            if (rc) return rc;
        }
        i = end;
        return SG_OK;
    }
    int left = n;
    while (left > 0) {
        std::vector<int> ops, macs;
        // (1) ready backward advections fused with the corrections that read their output
        for (int a = 0; a < n && ops.size() < 3; ++a) {
            const Op &o = g->queue[i + a];
            if (done[a] || o.kind != OP_ADVECT || o.f0 >= 0.f || !issued(a, -1)) continue;
            for (int m = a + 1; m < n; ++m) {
                const Op &c = g->queue[i + m];
                if (done[m] || c.kind != OP_MAC || c.i2 != o.dst || c.i0 != o.i0 || c.f0 != -o.f0 || !issued(m, a))
                    continue;
                if (!ops.empty()) {
                    const Op &o0 = g->queue[i + ops[0]];
                    if (o0.i0 != o.i0 || o0.f0 != o.f0) continue;
                }
                ops.push_back(a);
                macs.push_back(m);
                break;
            }
        }
        int mode = 1;
        if (ops.empty()) {  // (2) ready advections with the same velocity and step
            mode = 0;
            for (int a = 0; a < n && ops.size() < 3; ++a) {
                const Op &o = g->queue[i + a];
                if (done[a] || o.kind != OP_ADVECT || !issued(a, -1)) continue;
                if (!ops.empty()) {
                    const Op &o0 = g->queue[i + ops[0]];
                    if (o0.i0 != o.i0 || o0.f0 != o.f0) continue;
                }
                ops.push_back(a);
            }
        }
        if (ops.empty()) {  // (3) ready corrections
            mode = 2;
            for (int a = 0; a < n && ops.size() < 3; ++a) {
                const Op &o = g->queue[i + a];
                if (done[a] || o.kind != OP_MAC || !issued(a, -1)) continue;
                if (!ops.empty()) {
                    const Op &o0 = g->queue[i + ops[0]];
                    if (o0.i0 != o.i0 || o0.f0 != o.f0) continue;
                }
                ops.push_back(a);
            }
        }
        if (ops.empty()) return fail(SG_ERR_INVALID, "advection run has no ready op");  // cannot happen: deps are acyclic
        rc = launch(mode, ops, macs);
        if (rc) return rc;
        left -= (int)(ops.size() + macs.size());
    }
    i = end;
    return SG_OK;
}

// Dead-store elimination of reductions: within one flush nothing on the
// device reads a result slot, so a reduction whose slot a later reduction in
// the queue overwrites is dead (the autodiff microbenchmark's pattern).
void drop_dead_sums(sg_grid *g)
{
    if (!(g->opts & SG_OPT_DSE)) return;
    std::vector<Op> kept;
    kept.reserve(g->queue.size());
    for (size_t k = 0; k < g->queue.size(); ++k) {
        const Op &o = g->queue[k];
        bool dead = false;
        if (o.kind == OP_SUM)
            for (size_t m = k + 1; m < g->queue.size() && !dead; ++m)
                dead = g->queue[m].kind == OP_SUM && g->queue[m].slot == o.slot;
        if (dead) g->stats.stores_removed++;
        else kept.push_back(o);
    }
    g->queue.swap(kept);
}

// Binned-P2G scratch: bin counts and offsets over the root cells, the count
// scan's tile sums, and a particle order array of at least n entries.
int ensure_p2g_scratch(sg_grid *g, long long n)
{
    if (g->dry) return SG_OK;
    const long long nbins = (long long)g->dev.R * g->dev.R * g->dev.R;
    const long long nkeys = p2g_num_keys(g->dev.R);
    if (!g->dev.bin_count) {
        g->dev.bin_count = (int32_t *)dev_alloc(g, sizeof(int32_t) * nkeys);
        g->dev.bin_off = (int32_t *)dev_alloc(g, sizeof(int32_t) * nkeys);
        g->dev.tile_sum = (int32_t *)dev_alloc(g, sizeof(int32_t) * (nkeys / 1024 + 2));
        g->dev.bin_list = (int32_t *)dev_alloc(g, sizeof(int32_t) * (nbins + 1));
        if (!g->dev.bin_count || !g->dev.bin_off || !g->dev.tile_sum || !g->dev.bin_list)
            return fail(SG_ERR_OOM, "p2g bins");
    }
    if (n > g->perm_cap) {
        // grown geometrically: replaced arrays stay allocated until the grid is destroyed
        const long long cap = std::max(n, g->perm_cap * 2);
        g->dev.perm = (int32_t *)dev_alloc(g, sizeof(int32_t) * cap);
        g->dev.perm_alt = (int32_t *)dev_alloc(g, sizeof(int32_t) * cap);
        g->dev.perm_key = (long long *)dev_alloc(g, sizeof(long long) * cap);
        if (!g->dev.perm || !g->dev.perm_alt || !g->dev.perm_key)
            return fail(SG_ERR_OOM, "p2g order of %lld particles", cap);
        g->perm_cap = cap;
        g->p2g_x = nullptr;  // no valid last order in the new arrays
        g->p2g_n = 0;
    }
    return SG_OK;
}

int run_write_staged(sg_grid *g, const Op &o);

int do_flush(sg_grid *g)
{
    int rc = SG_OK;
    g->stats.flushes++;
    drop_dead_sums(g);
    size_t i = 0;
    while (i < g->queue.size() && rc == SG_OK) {
        const Op &o = g->queue[i];
        switch (o.kind) {
            case OP_ACT_SHELL: {
                const auto sig = std::make_tuple(o.lo2, o.hi2, o.strict, o.op);
                if ((g->opts & SG_OPT_AD) && g->applied_shells.count(sig)) {
                    g->stats.act_demoted++;
                } else {
                    const uint32_t fill = activation_fill_mask(g, i);
                    const int F = g->dev.F;
                    for (int f = 0; f < F; ++f)
                        if (!((fill >> f) & 1u)) g->stats.stores_removed++;
                    if (!g->dry) {
                        if (o.op) launch_activate_tube(g->dev, g->stream, o.lo2, o.hi2, fill);
                        else launch_activate_shell(g->dev, g->stream, o.lo2, o.hi2, o.strict, fill);
                    }
                    g->applied_shells.insert(sig);
                    g->stats.act_launched++;
                    rc = after_launch(g, "activate shell");
                    if (!rc) rc = bump_structure(g);
                }
                ++i;
                break;
            }
            case OP_ACT_COORDS: {
                const uint32_t fill = activation_fill_mask(g, i);
                for (int f = 0; f < g->dev.F; ++f)
                    if (!((fill >> f) & 1u)) g->stats.stores_removed++;
                if (!g->dry) launch_mark_coords(g->dev, g->stream, (const int32_t *)o.p0, o.n);
                if (!(rc = after_launch(g, "mark coords"))) {
                    if (!g->dry) launch_alloc_needed(g->dev, g->stream, fill);
                    if (!(rc = after_launch(g, "allocate"))) {
                        if (!g->dry) launch_setbits_coords(g->dev, g->stream, (const int32_t *)o.p0, o.n);
                        rc = after_launch(g, "set bits");
                    }
                }
                if (!rc) rc = bump_structure(g);
                g->stats.act_launched++;
                ++i;
                break;
            }
            case OP_DEACT:
                if (!g->dry) launch_deactivate_all(g->dev, g->stream);
                g->applied_shells.clear();
                g->applied_restrict.clear();
                rc = after_launch(g, "deactivate");
                if (!rc) rc = bump_structure(g);
                ++i;
                break;
            case OP_LISTGEN:
                rc = ensure_list(g);
                ++i;
                break;
            case OP_FILL:
                if (!(rc = ensure_list(g))) {
                    if (!g->dry) launch_fill_hash(g->dev, g->stream, o.i0, (unsigned long long)o.slot, g->lc);
                    rc = after_launch(g, "fill");
                }
                ++i;
                break;
            case OP_TEST_WAIT:
                rc = launch_list(g, false, 1);
                ++i;
                break;
            case OP_STENCIL:
            case OP_SUM:
                rc = run_struct_for_group(g, i);
                break;
            case OP_EW:
                rc = run_ew_group(g, i);
                break;
            case OP_ADVECT:
            case OP_MAC:
                rc = run_advect_run(g, i);
                break;
            case OP_P2G:
                if (!(rc = ensure_p2g_scratch(g, o.n))) {
                    // the same particles binned before: rebin from their last order
                    const bool rebin = g->p2g_x == o.p0 && g->p2g_n == o.n;
                    const int k = g->dry ? 7
                                         : launch_p2g_binned(g->dev, g->stream, (const float *)o.p0,
                                                             (const float *)o.p1, (const float *)o.p3, o.n, o.f0,
                                                             o.i0, o.i1, rebin, g->lc);
                    g->stats.launches += k - 1;
                    rc = after_launch(g, "binned p2g");
                    g->p2g_x = o.p0;
                    g->p2g_n = o.n;
                }
                if (!rc) rc = bump_structure(g);
                g->stats.act_launched++;
                ++i;
                break;
            case OP_GRID_UPDATE:
                if (!(rc = ensure_list(g))) {
                    if (!g->dry) launch_grid_update(g->dev, g->stream, o.i0, o.i1, o.f0, o.f1, o.i2, g->lc);
                    rc = after_launch(g, "grid update");
                }
                ++i;
                break;
            case OP_G2P2G:
                if (!g->dry)
                    launch_g2p2g(o.peer->dev, g->dev, o.bins->dev, g->stream, (float *)o.p1, (float *)o.p2, o.n, o.f0,
                                 o.i0, o.f1, o.i1, o.i2, g->lc);
                rc = after_launch(g, "g2p2g");
                if (!rc) rc = bump_structure(g);
                g->stats.act_launched++;
                ++i;
                break;
            case OP_WRITE_STAGED:
                rc = run_write_staged(g, o);
                ++i;
                break;
            case OP_G2P:
                if (!g->dry)
                    launch_g2p(g->dev, g->stream, (float *)o.p1, (float *)o.p2, (float *)o.p3, o.n, o.f0, o.i0,
                               o.p1 == g->p2g_x && o.n == g->p2g_n, g->lc);
                rc = after_launch(g, "g2p");
                ++i;
                break;
            case OP_SORT_P: {
                if (o.p0 != g->p2g_x || o.n != g->p2g_n) {
                    rc = fail(SG_ERR_INVALID, "sort_particles: no binned P2G of these particles is current");
                    ++i;
                    break;
                }
                if (!g->dry && o.n > g->sort_cap) {
                    // grown geometrically: replaced blocks stay allocated until
                    // the grid is destroyed, so their total stays below 2x the last
                    const long long cap = std::max<long long>(o.n, 2 * g->sort_cap);
                    g->sort_tmp = dev_alloc(g, (size_t)cap * 36);
                    if (!g->sort_tmp) {
                        rc = fail(SG_ERR_OOM, "particle reordering scratch");
                        ++i;
                        break;
                    }
                    g->sort_cap = cap;
                }
                const int k = g->dry ? 1 + (o.p0 ? 1 : 0) + (o.p1 ? 1 : 0) + (o.p2 ? 1 : 0) + (o.p3 ? 1 : 0)
                                     : launch_sort_particles(g->dev, g->stream, (float *)o.p0, (float *)o.p1,
                                                             (float *)o.p2, (int64_t *)o.p3, o.n, g->sort_tmp, g->lc);
                g->stats.launches += k - 1;
                rc = after_launch(g, "sort particles");
                ++i;
                break;
            }
        }
    }
    g->queue.clear();
    return rc;
}

int map_device_error(int bits)
{
    if (bits & kErrPool) return fail(SG_ERR_POOL_EXHAUSTED, "leaf pool exhausted (max_leaves too small)");
    if (bits & kErrTimeout) return fail(SG_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (bits & kErrCheck) return fail(SG_ERR_CUDA, "a kernel's address self-check failed (the access was skipped)");
    return SG_OK;
}

int ensure_staging(sg_grid *g);

// The invariant checks of sg_check; the list-dependent ones only with a
// current list.  Check kernels are not counted in sg_stats.
int run_checks(sg_grid *g, sg_check_report *r, bool with_list)
{
    *r = sg_check_report{};
    int rc;
    if (!g->chk_cnt && !(g->chk_cnt = (unsigned long long *)dev_alloc(g, sizeof(unsigned long long) * kNumChk)))
        return fail(SG_ERR_OOM, "check counters");
    if ((rc = ensure_staging(g))) return rc;  // slot -> root cell map
    uint32_t field_bits = 0;
    for (int f = 0; f < g->dev.F; ++f)
        if (!((g->desc.scratch_mask >> f) & 1u)) field_bits |= 1u << g->phys[f];
    cudaStream_t s = g->stream;
    if ((rc = cuda_check(cudaMemsetAsync(g->chk_cnt, 0, sizeof(unsigned long long) * kNumChk, s), "check counters")) ||
        (rc = cuda_check(cudaMemsetAsync(g->dev.staging_u, 0xff, sizeof(uint32_t) * g->dev.cap, s), "owner map")))
        return rc;
    launch_checks(g->dev, s, g->dev.staging_u, g->chk_cnt, with_list, field_bits, g->lc);
    if ((rc = cuda_check(cudaPeekAtLastError(), "invariant checks"))) return rc;
    unsigned long long c[kNumChk];
    if ((rc = cuda_check(cudaMemcpyAsync(c, g->chk_cnt, sizeof c, cudaMemcpyDeviceToHost, s), "read check counters")) ||
        (rc = cuda_check(cudaStreamSynchronize(s), "stream synchronize")))
        return rc;
    // the counters that each launch's last CTA resets must be zero between launches
    // (host_ctrl was read by the sync before the checks)
    r->ctrl_bad = (int64_t)(g->host_ctrl->red_ticket != 0u);
    r->root_bad = (int64_t)c[kChkRoot];
    r->slot_shared = (int64_t)c[kChkShared];
    r->leaves = (int64_t)c[kChkLeaves];
    r->zero_leaf_bad = (int64_t)c[kChkZero];
    if (with_list) {
        const long long d = (long long)g->host_ctrl->list_n - (long long)c[kChkLeaves];
        r->list_bad = (int64_t)c[kChkList] + (d < 0 ? -d : d);
        r->nbr_bad = (int64_t)c[kChkNbr];
        r->inactive_nonzero = (int64_t)c[kChkInactive];
    }
    return SG_OK;
}

// Flush, wait, read the control block; latch and clear device errors.
int do_sync(sg_grid *g)
{
    int rc = do_flush(g);
    if (g->dry) return rc;
    if (rc) return rc;
    if ((rc = cuda_check(cudaMemcpyAsync(g->host_ctrl, g->dev.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, g->stream),
                         "read control block")))
        return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize"))) return rc;
    const int bits = g->host_ctrl->err;
    if (bits) {
        cudaMemsetAsync(&g->dev.ctrl->err, 0, sizeof(int32_t), g->stream);
        cudaStreamSynchronize(g->stream);
        const int code = map_device_error(bits);
        if (g->latched == SG_OK) g->latched = code;
    }
    if ((g->desc.flags & SG_CREATE_CHECK) && g->latched == SG_OK) {
        sg_check_report r;
        const bool with_list = g->list_ver == g->mask_ver;
        if ((rc = run_checks(g, &r, with_list))) return rc;
        if (r.root_bad | r.slot_shared | r.list_bad | r.nbr_bad | r.zero_leaf_bad | r.inactive_nonzero | r.ctrl_bad)
            g->latched = fail(SG_ERR_CHECK,
                              "invariant check: root %lld, shared slots %lld, list %lld, neighbours %lld, zero leaf %lld, "
                              "inactive values %lld, control counters %lld",
                              (long long)r.root_bad, (long long)r.slot_shared, (long long)r.list_bad,
                              (long long)r.nbr_bad, (long long)r.zero_leaf_bad, (long long)r.inactive_nonzero,
                              (long long)r.ctrl_bad);
    }
    if (g->list_ver == g->mask_ver) g->known_leaves = g->host_ctrl->list_n;
    const int out = g->latched;
    g->latched = SG_OK;
    return out;
}

// Implicit sync with a current list (reads need list order).
int sync_with_list(sg_grid *g)
{
    if (g->dry) return fail(SG_ERR_INVALID, "a dry-run grid holds no data");
    int rc = do_flush(g);
    if (rc) return rc;
    if (g->list_ver != g->mask_ver) {
        // a read needs the list even when LGR is off; generate it without a clear
        if ((rc = launch_list(g, false, 0))) return rc;
        g->list_ver = g->mask_ver;
    }
    return do_sync(g);
}

int ensure_staging(sg_grid *g)
{
    const size_t need = size_t(g->desc.max_leaves) * size_t(g->dev.L) * g->dev.L * g->dev.L * 4;
    if (g->staging_bytes >= need) return SG_OK;
    void *p = dev_alloc(g, need);
    if (!p) return fail(SG_ERR_OOM, "staging buffer of %zu bytes", need);
    g->dev.staging = (float *)p;
    g->dev.staging_u = (uint32_t *)p;
    g->staging_bytes = need;
    return SG_OK;
}

// Packed positions of every list entry's active voxels (a current list of n
// entries); returns their total through *total (implicit wait).  Kept while
// the structure is unchanged: the list version keys them.
int active_offsets(sg_grid *g, long long n, long long *total)
{
    // reused while no activation has touched the structure since (the list
    // is current and the device dirty flag, read at the last sync, is clear)
    if (g->act_ver == g->list_ver && g->act_ver != 0 && g->host_ctrl->dirty == 0) {
        *total = g->act_total;
        return SG_OK;
    }
    if (!g->act_off) {
        g->act_off = (long long *)dev_alloc(g, sizeof(long long) * size_t(g->dev.cap));
        g->act_tsum = (long long *)dev_alloc(g, sizeof(long long) * size_t(g->dev.cap / kOffTile + 2));
        if (!g->act_off || !g->act_tsum) return fail(SG_ERR_OOM, "transfer offsets");
    }
    launch_active_offsets(g->dev, g->stream, n, g->act_off, g->act_tsum);
    int rc = after_launch(g, "active offsets");
    if (rc) return rc;
    const int ntiles = (int)((n + kOffTile - 1) / kOffTile);
    if ((rc = cuda_check(cudaMemcpyAsync(total, g->act_tsum + ntiles, sizeof(long long), cudaMemcpyDeviceToHost,
                                         g->stream),
                         "read active total")) ||
        (rc = cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize")))
        return rc;
    g->act_ver = g->list_ver;
    g->act_total = *total;
    return SG_OK;
}

// The queued half of a staged upload: wait for the slot's copy, check the
// count and scatter the slot into the field.  The active count comes from the
// kept offsets when the structure is unchanged since they were computed;
// otherwise they are computed here, which waits for the device once.
int run_write_staged(sg_grid *g, const Op &o)
{
    const int k = (int)o.slot;
    if (g->upload_seq[k] != (unsigned)o.i1)
        return fail(SG_ERR_INVALID, "staged upload %u was replaced by a later one", (unsigned)o.i1);
    if (g->dry) return after_launch(g, "scatter staged");
    if (capturing(g)) return fail(SG_ERR_INVALID, "a staged upload cannot be recorded in a graph");
    int rc = ensure_list(g);
    if (rc) return rc;
    long long total = 0;
    if (!(g->act_ver == g->list_ver && g->act_ver != 0 && g->host_ctrl->dirty == 0)) {
        // the list length, on the host: wait for the work launched so far and
        // read the control block (no flush -- this runs inside one; device
        // errors stay latched for the next sync)
        if ((rc = cuda_check(cudaMemcpyAsync(g->host_ctrl, g->dev.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                                             g->stream),
                             "read control block")) ||
            (rc = cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize")))
            return rc;
    }
    const long long n = g->host_ctrl->list_n;
    if (n > 0 && (rc = active_offsets(g, n, &total))) return rc;
    if (total != o.n)
        return fail(SG_ERR_INVALID, "the grid has %lld active voxels, the upload holds %lld", total, o.n);
    if (n == 0) return SG_OK;
    if ((rc = cuda_check(cudaStreamWaitEvent(g->stream, g->copied[k], 0), "wait for the upload"))) return rc;
    launch_scatter_active(g->dev, g->stream, o.i0, g->upload[k], total, g->act_off, g->act_tsum, g->lc);
    if ((rc = after_launch(g, "scatter staged"))) return rc;
    return cuda_check(cudaEventRecord(g->consumed[k], g->stream), "record upload consumed");
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
namespace sg {

int grid_create(const sg_desc *desc, void *cuda_stream, sg_grid **out, bool init_sync)
{
    if (!desc || !out) return fail(SG_ERR_INVALID, "null argument");
    *out = nullptr;
    const int lg2 = desc->leaf_log2;
    if (lg2 != 2 && lg2 != 3) return fail(SG_ERR_INVALID, "leaf_log2 must be 2 or 3");
    const int L = 1 << lg2;
    if (desc->res <= 0 || desc->res > 4096 || desc->res % L) return fail(SG_ERR_INVALID, "res must be a positive multiple of the leaf edge <= 4096");
    if (desc->n_fields < 1 || desc->n_fields > SG_MAX_FIELDS) return fail(SG_ERR_INVALID, "n_fields out of range");
    if (desc->max_leaves < 1 || desc->max_leaves > (1LL << 30)) return fail(SG_ERR_INVALID, "max_leaves out of range");
    if (desc->max_sums < 0) return fail(SG_ERR_INVALID, "max_sums < 0");
    if ((desc->alloc == nullptr) != (desc->free == nullptr)) return fail(SG_ERR_INVALID, "alloc and free come together");

    sg_grid *g = new (std::nothrow) sg_grid();
    if (!g) return fail(SG_ERR_OOM, "host allocation");
    g->desc = *desc;
    g->stream = (cudaStream_t)cuda_stream;
    g->dry = (desc->flags & SG_CREATE_DRY_RUN) != 0;
    for (int f = 0; f < SG_MAX_FIELDS; ++f) g->phys[f] = f;
    DevGrid &d = g->dev;
    d.N = desc->res;
    d.L = L;
    d.lg2 = lg2;
    d.R = desc->res / L;
    d.W = (L * L * L) / 32;
    d.F = desc->n_fields;
    d.cap = desc->max_leaves;
    const long long nr = (long long)d.R * d.R * d.R;
    g->num_tiles = (int)((nr + kListTile - 1) / kListTile);
    g->lc.variant = kVariantSweepJRuns;
    if (g->dry) {
        g->lc.num_sms = 152;
        g->lc.persistent_ctas = 152;
        *out = g;
        return SG_OK;
    }
    int dev = 0;
    int rc;
    if ((rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice")) ||
        (rc = cuda_check(cudaDeviceGetAttribute(&g->lc.num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count"))) {
        delete g;
        return rc;
    }
    g->lc.persistent_ctas = g->lc.num_sms;
    const size_t V = size_t(L) * L * L;
    const int max_ctas = 8192;
    struct Need { void **dst; size_t bytes; } needs[] = {
        {(void **)&d.root, sizeof(int32_t) * nr},
        {(void **)&d.mask, sizeof(uint32_t) * d.W * (d.cap + 1)},
        {(void **)&d.list_slot, sizeof(int32_t) * d.cap},
        {(void **)&d.list_b, sizeof(int32_t) * d.cap},
        {(void **)&d.nbr, sizeof(int32_t) * 27 * d.cap},
        {(void **)&d.ent_of_slot, sizeof(int32_t) * d.cap},
        {(void **)&d.col_grp, sizeof(int32_t) * 9 * d.cap},
        {(void **)&d.col_cnt, sizeof(int32_t) * 4},
        {(void **)&d.rr_status, sizeof(unsigned long long) * 3 * (d.cap / 256 + 1)},
        {(void **)&d.rmask, (L == 8 ? sizeof(uint32_t) * 40 : size_t(4)) * d.cap},
        {(void **)&d.need, (size_t)nr},
        {(void **)&d.tile_status, sizeof(unsigned long long) * g->num_tiles},
        {(void **)&d.partials, sizeof(double) * max_ctas},
        {(void **)&d.sums, sizeof(double) * std::max(1, desc->max_sums)},
        {(void **)&d.ctrl, sizeof(Ctrl)},
    };
    for (auto &nd : needs) {
        *nd.dst = dev_alloc(g, nd.bytes);
        if (!*nd.dst) {
            dev_free_all(g);
            delete g;
            return fail(SG_ERR_OOM, "device allocation of %zu bytes", nd.bytes);
        }
    }
    for (int f = 0; f < d.F; ++f) {
        d.field[f] = (float *)dev_alloc(g, sizeof(float) * V * (d.cap + 1));
        if (!d.field[f]) {
            dev_free_all(g);
            delete g;
            return fail(SG_ERR_OOM, "field allocation");
        }
    }
    if (cudaMallocHost((void **)&g->host_ctrl, sizeof(Ctrl)) != cudaSuccess) {
        cudaGetLastError();
        dev_free_all(g);
        delete g;
        return fail(SG_ERR_OOM, "pinned host control block");
    }
    // initial state: all pointers null, empty pool and list, structure dirty
    cudaStream_t s = g->stream;
    rc = cuda_check(cudaMemsetAsync(d.root, 0xff, sizeof(int32_t) * nr, s), "init root");
    if (!rc) rc = cuda_check(cudaMemsetAsync(d.need, 0, (size_t)nr, s), "init need");
    if (!rc) rc = cuda_check(cudaMemsetAsync(d.tile_status, 0, sizeof(unsigned long long) * g->num_tiles, s), "init status");
    if (!rc)
        rc = cuda_check(cudaMemsetAsync(d.rr_status, 0, sizeof(unsigned long long) * 3 * (d.cap / 256 + 1), s),
                        "init run-record status");
    if (!rc) rc = cuda_check(cudaMemsetAsync(d.sums, 0, sizeof(double) * std::max(1, desc->max_sums), s), "init sums");
    // the zero leaf (slot cap): never allocated, read in place of null neighbours
    if (!rc) rc = cuda_check(cudaMemsetAsync(d.mask + d.W * d.cap, 0, sizeof(uint32_t) * d.W, s), "init zero leaf");
    for (int f = 0; f < d.F && !rc; ++f)
        rc = cuda_check(cudaMemsetAsync(d.field[f] + V * d.cap, 0, sizeof(float) * V, s), "init zero leaf");
    if (!rc) {
        Ctrl c{};
        c.dirty = 1;
        std::memcpy(g->host_ctrl, &c, sizeof c);
        rc = cuda_check(cudaMemcpyAsync(d.ctrl, g->host_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, s), "init ctrl");
    }
    if (!rc && init_sync) rc = cuda_check(cudaStreamSynchronize(s), "init sync");
    if (rc) {
        cudaStreamSynchronize(s);  // the queued initialisation still reads host_ctrl
        cudaFreeHost(g->host_ctrl);
        dev_free_all(g);
        delete g;
        return rc;
    }
    *out = g;
    return SG_OK;
}

}  // namespace sg

extern "C" {

int sg_create(const sg_desc *desc, void *cuda_stream, sg_grid **out)
{
    return grid_create(desc, cuda_stream, out, true);
}

int sg_destroy(sg_grid *g)
{
    if (!g) return SG_OK;
    int rc = SG_OK;
    if (!g->dry) {
        rc = cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize");
        if (g->copy_stream) {
            cudaStreamSynchronize(g->copy_stream);
            cudaStreamDestroy(g->copy_stream);
        }
        for (int k = 0; k < 2; ++k) {
            if (g->copied[k]) cudaEventDestroy(g->copied[k]);
            if (g->consumed[k]) cudaEventDestroy(g->consumed[k]);
        }
        dev_free_all(g);
        if (g->host_ctrl) cudaFreeHost(g->host_ctrl);
    }
    delete g;
    return rc;
}

int sg_set_opts(sg_grid *g, uint32_t opts)
{
    if (!g || (opts & ~SG_OPT_ALL)) return fail(SG_ERR_INVALID, "bad grid or options");
    g->opts = opts;
    return SG_OK;
}

int sg_activate_shell(sg_grid *g, int64_t lo2, int64_t hi2, int32_t lo_strict)
{
    if (!g) return fail(SG_ERR_INVALID, "null grid");
    Op o{OP_ACT_SHELL};
    o.lo2 = lo2;
    o.hi2 = hi2;
    o.strict = lo_strict ? 1 : 0;
    return push(g, o);
}

int sg_activate_coords(sg_grid *g, const int32_t *dev_xyz, int64_t n)
{
    if (!g || n < 0 || (n > 0 && !dev_xyz)) return fail(SG_ERR_INVALID, "bad coordinates");
    if (n == 0) return SG_OK;
    Op o{OP_ACT_COORDS};
    o.p0 = dev_xyz;
    o.n = n;
    return push(g, o);
}

int sg_deactivate_all(sg_grid *g)
{
    if (!g) return fail(SG_ERR_INVALID, "null grid");
    return push(g, Op{OP_DEACT});
}

int sg_list_gen(sg_grid *g)
{
    if (!g) return fail(SG_ERR_INVALID, "null grid");
    return push(g, Op{OP_LISTGEN});
}

int sg_launch_stencil(sg_grid *g, int32_t op, int32_t src, int32_t dst, float coef)
{
    if (!g) return fail(SG_ERR_INVALID, "null grid");
    if (op != SG_CLEAR && op != SG_DIFFUSE7 && op != SG_BOX27) return fail(SG_ERR_INVALID, "unknown stencil op %d", op);
    if (!valid_field(g, dst) || (op != SG_CLEAR && (!valid_field(g, src) || src == dst)))
        return fail(SG_ERR_INVALID, "bad field indices src=%d dst=%d", src, dst);
    Op o{OP_STENCIL};
    o.op = op;
    o.src = (op == SG_CLEAR) ? g->phys[dst] : g->phys[src];
    o.dst = g->phys[dst];
    o.dst_scratch = (g->desc.scratch_mask >> dst) & 1u;
    o.coef = coef;
    return push(g, o);
}

int sg_launch_ew(sg_grid *g, int32_t dst, int32_t a, int32_t b, float alpha, float beta, float gamma, float delta)
{
    if (!g || !valid_field(g, dst) || (a != -1 && !valid_field(g, a)) || (b != -1 && !valid_field(g, b)))
        return fail(SG_ERR_INVALID, "bad element-wise fields dst=%d a=%d b=%d", dst, a, b);
    Op o{OP_EW};
    o.dst = g->phys[dst];
    o.src = a >= 0 ? g->phys[a] : -1;
    o.i0 = b >= 0 ? g->phys[b] : -1;
    o.dst_scratch = (g->desc.scratch_mask >> dst) & 1u;
    o.f0 = alpha;
    o.f1 = beta;
    o.coef = gamma;
    o.f2 = delta;
    return push(g, o);
}

int sg_activate_tube(sg_grid *g, int64_t lo2, int64_t hi2)
{
    if (!g || lo2 < 0 || hi2 < lo2) return fail(SG_ERR_INVALID, "bad tube bounds");
    Op o{OP_ACT_SHELL};
    o.lo2 = lo2;
    o.hi2 = hi2;
    o.op = 1;  // tube
    return push(g, o);
}

// Velocity fields v0, v0+1, v0+2 valid and stored consecutively.
static bool valid_velocity(const sg_grid *g, int v0)
{
    return valid_field(g, v0) && valid_field(g, v0 + 2) && g->phys[v0 + 1] == g->phys[v0] + 1 &&
           g->phys[v0 + 2] == g->phys[v0] + 2;
}

int sg_advect(sg_grid *g, int32_t dst, int32_t src, int32_t v0, float dt)
{
    if (!g || !valid_field(g, dst) || !valid_field(g, src) || !valid_velocity(g, v0) || dst == src ||
        (dst >= v0 && dst <= v0 + 2))
        return fail(SG_ERR_INVALID, "bad advection fields dst=%d src=%d vel=%d", dst, src, v0);
    Op o{OP_ADVECT};
    o.dst = g->phys[dst];
    o.src = g->phys[src];
    o.i0 = g->phys[v0];
    o.f0 = dt;
    o.dst_scratch = (g->desc.scratch_mask >> dst) & 1u;
    return push(g, o);
}

int sg_maccormack(sg_grid *g, int32_t dst, int32_t q, int32_t qhat, int32_t qtilde, int32_t v0, float dt)
{
    if (!g || !valid_field(g, dst) || !valid_field(g, q) || !valid_field(g, qhat) || !valid_field(g, qtilde) ||
        !valid_velocity(g, v0) || dst == q || dst == qhat || dst == qtilde || (dst >= v0 && dst <= v0 + 2))
        return fail(SG_ERR_INVALID, "bad MacCormack fields");
    Op o{OP_MAC};
    o.dst = g->phys[dst];
    o.src = g->phys[q];
    o.i0 = g->phys[v0];
    o.i1 = g->phys[qhat];
    o.i2 = g->phys[qtilde];
    o.f0 = dt;
    o.dst_scratch = (g->desc.scratch_mask >> dst) & 1u;
    return push(g, o);
}

int sg_set_flush_period(sg_grid *g, int32_t ops)
{
    if (!g || ops < 0) return fail(SG_ERR_INVALID, "flush period must be >= 0");
    g->flush_period = ops;
    return SG_OK;
}

int sg_set_max_fuse(sg_grid *g, int32_t max_ops)
{
    if (!g || max_ops < 1) return fail(SG_ERR_INVALID, "max_fuse must be >= 1");
    g->max_fuse = max_ops;
    return SG_OK;
}

int sg_reduce_sum(sg_grid *g, int32_t src, int64_t out_slot)
{
    if (!g || !valid_field(g, src) || out_slot < 0 || out_slot >= g->desc.max_sums)
        return fail(SG_ERR_INVALID, "bad reduction arguments");
    Op o{OP_SUM};
    o.src = g->phys[src];
    o.slot = out_slot;
    return push(g, o);
}

int sg_p2g(sg_grid *g, const float *dev_x, const float *dev_v, int64_t n, float pmass, int32_t f_mass, int32_t f_mom0)
{
    return sg_p2g_apic(g, dev_x, dev_v, nullptr, n, pmass, f_mass, f_mom0);
}

int sg_p2g_apic(sg_grid *g, const float *dev_x, const float *dev_v, const float *dev_C, int64_t n, float pmass,
                int32_t f_mass, int32_t f_mom0)
{
    if (!g || n < 0 || (n > 0 && (!dev_x || !dev_v)) || !valid_field(g, f_mass) || !valid_field(g, f_mom0) ||
        !valid_field(g, f_mom0 + 2) || (f_mass >= f_mom0 && f_mass <= f_mom0 + 2))
        return fail(SG_ERR_INVALID, "bad p2g arguments");
    if (n == 0) return SG_OK;
    Op o{OP_P2G};
    o.p0 = dev_x;
    o.p1 = (void *)dev_v;
    o.p3 = (void *)dev_C;
    o.n = n;
    o.f0 = pmass;
    o.i0 = g->phys[f_mass];
    o.i1 = g->phys[f_mom0];
    if (g->phys[f_mom0 + 1] != o.i1 + 1 || g->phys[f_mom0 + 2] != o.i1 + 2)
        return fail(SG_ERR_INVALID, "momentum fields must be three consecutive unswapped fields");
    return push(g, o);
}

int sg_grid_update(sg_grid *g, int32_t f_mass, int32_t f_mom0, float dt, float gz, int32_t bound)
{
    if (!g || !valid_field(g, f_mass) || !valid_field(g, f_mom0) || !valid_field(g, f_mom0 + 2))
        return fail(SG_ERR_INVALID, "bad grid update arguments");
    Op o{OP_GRID_UPDATE};
    o.i0 = g->phys[f_mass];
    o.i1 = g->phys[f_mom0];
    o.i2 = bound;
    o.f0 = dt;
    o.f1 = gz;
    if (g->phys[f_mom0 + 1] != o.i1 + 1 || g->phys[f_mom0 + 2] != o.i1 + 2)
        return fail(SG_ERR_INVALID, "momentum fields must be three consecutive unswapped fields");
    return push(g, o);
}

int sg_g2p(sg_grid *g, float *dev_x, float *dev_v, int64_t n, float dt, int32_t f_mom0)
{
    return sg_g2p_apic(g, dev_x, dev_v, nullptr, n, dt, f_mom0);
}

int sg_sort_particles(sg_grid *g, float *dev_x, float *dev_v, float *dev_C, int64_t *dev_ids, int64_t n)
{
    if (!g || n < 0 || (n > 0 && (!dev_x || !dev_v))) return fail(SG_ERR_INVALID, "bad sort_particles arguments");
    if (n == 0) return SG_OK;
    if (n > INT32_MAX) return fail(SG_ERR_INVALID, "at most 2^31 - 1 particles");
    Op o{OP_SORT_P};
    o.p0 = dev_x;
    o.p1 = dev_v;
    o.p2 = dev_C;
    o.p3 = dev_ids;
    o.n = n;
    return push(g, o);
}

int sg_g2p_apic(sg_grid *g, float *dev_x, float *dev_v, float *dev_C, int64_t n, float dt, int32_t f_mom0)
{
    if (!g || n < 0 || (n > 0 && (!dev_x || !dev_v)) || !valid_field(g, f_mom0) || !valid_field(g, f_mom0 + 2))
        return fail(SG_ERR_INVALID, "bad g2p arguments");
    if (n == 0) return SG_OK;
    Op o{OP_G2P};
    o.p1 = dev_x;
    o.p2 = dev_v;
    o.p3 = dev_C;
    o.n = n;
    o.f0 = dt;
    o.i0 = g->phys[f_mom0];
    if (g->phys[f_mom0 + 1] != o.i0 + 1 || g->phys[f_mom0 + 2] != o.i0 + 2)
        return fail(SG_ERR_INVALID, "momentum fields must be three consecutive unswapped fields");
    return push(g, o);
}

int sg_g2p2g(sg_grid *src, sg_grid *dst, float *dev_x, float *dev_v, int64_t n, float dt, int32_t f_vel0, float pmass,
             int32_t f_mass, int32_t f_mom0)
{
    if (!src || !dst || src == dst || n < 0 || (n > 0 && (!dev_x || !dev_v)))
        return fail(SG_ERR_INVALID, "bad g2p2g arguments");
    if (src->dev.N != dst->dev.N || src->dev.L != dst->dev.L || src->stream != dst->stream || src->dry != dst->dry)
        return fail(SG_ERR_INVALID, "g2p2g grids must share resolution, leaf size and stream");
    if (!valid_field(src, f_vel0) || !valid_field(src, f_vel0 + 2) || !valid_field(dst, f_mass) ||
        !valid_field(dst, f_mom0) || !valid_field(dst, f_mom0 + 2) || (f_mass >= f_mom0 && f_mass <= f_mom0 + 2))
        return fail(SG_ERR_INVALID, "bad g2p2g field indices");
    Op o{OP_G2P2G};
    o.i0 = src->phys[f_vel0];
    o.i1 = dst->phys[f_mass];
    o.i2 = dst->phys[f_mom0];
    if (src->phys[f_vel0 + 1] != o.i0 + 1 || src->phys[f_vel0 + 2] != o.i0 + 2 || dst->phys[f_mom0 + 1] != o.i2 + 1 ||
        dst->phys[f_mom0 + 2] != o.i2 + 2)
        return fail(SG_ERR_INVALID, "velocity and momentum fields must be three consecutive unswapped fields");
    if (n == 0) return SG_OK;
    // queued work of both grids (src's P2G and grid update, dst's deactivation)
    // runs first on the shared stream
    int rc = do_flush(src);
    if (rc || (rc = do_flush(dst))) return rc;
    const sg_grid *bins = (src->p2g_x == dev_x && src->p2g_n == n)   ? src
                          : (dst->p2g_x == dev_x && dst->p2g_n == n) ? dst
                                                                     : nullptr;
    if (!bins) return fail(SG_ERR_INVALID, "g2p2g needs a binned P2G over the same particles on src or dst first");
    o.p1 = dev_x;
    o.p2 = dev_v;
    o.n = n;
    o.f0 = dt;
    o.f1 = pmass;
    o.peer = src;
    o.bins = bins;
    if ((rc = push(dst, o))) return rc;
    return do_flush(dst);  // launched now: later src ops cannot run before it
}

// Both grids: distinct, same leaf size and stream, fine edge twice the coarse.
static int check_pair(const sg_grid *fine, const sg_grid *coarse, const char *what)
{
    if (!fine || !coarse || fine == coarse) return fail(SG_ERR_INVALID, "%s: two distinct grids are needed", what);
    if (fine->dev.N != 2 * coarse->dev.N || fine->dev.L != coarse->dev.L || fine->stream != coarse->stream ||
        fine->dry != coarse->dry)
        return fail(SG_ERR_INVALID, "%s: the fine grid's res must be twice the coarse one's, same leaf size and stream",
                    what);
    return SG_OK;
}

int sg_restrict(sg_grid *fine, sg_grid *coarse, int32_t f_src, int32_t f_dst, float w)
{
    int rc = check_pair(fine, coarse, "restrict");
    if (rc) return rc;
    if (!valid_field(fine, f_src) || !valid_field(coarse, f_dst)) return fail(SG_ERR_INVALID, "bad restrict fields");
    // queued work of both grids runs first; the loop runs over the fine list
    if ((rc = do_flush(fine)) || (rc = do_flush(coarse)) || (rc = ensure_list(fine))) return rc;
    const auto key = std::make_pair((const sg_grid *)fine, fine->mask_ver);
    const bool demote = (coarse->opts & SG_OPT_AD) && coarse->applied_restrict.count(key);
    if (demote) {
        coarse->stats.act_demoted++;
    } else {
        if (!coarse->dry) launch_restrict_mark(fine->dev, coarse->dev, coarse->stream, coarse->lc);
        if ((rc = after_launch(coarse, "restrict: mark"))) return rc;
        if (!coarse->dry) launch_alloc_needed(coarse->dev, coarse->stream);
        if ((rc = after_launch(coarse, "restrict: allocate"))) return rc;
        coarse->applied_restrict.insert(key);
        coarse->stats.act_launched++;
        if ((rc = bump_structure(coarse))) return rc;
    }
    if (!coarse->dry)
        launch_restrict(fine->dev, coarse->dev, coarse->stream, fine->phys[f_src], coarse->phys[f_dst], w, !demote,
                        coarse->lc);
    return after_launch(coarse, "restrict");
}

int sg_prolong(sg_grid *coarse, sg_grid *fine, int32_t f_src, int32_t f_dst, float w)
{
    int rc = check_pair(fine, coarse, "prolong");
    if (rc) return rc;
    if (!valid_field(coarse, f_src) || !valid_field(fine, f_dst)) return fail(SG_ERR_INVALID, "bad prolong fields");
    if ((rc = do_flush(coarse)) || (rc = do_flush(fine)) || (rc = ensure_list(fine))) return rc;
    if (!fine->dry)
        launch_prolong(coarse->dev, fine->dev, fine->stream, coarse->phys[f_src], fine->phys[f_dst], w, fine->lc);
    return after_launch(fine, "prolong");
}

int sg_swap(sg_grid *g, int32_t a, int32_t b)
{
    if (!g || !valid_field(g, a) || !valid_field(g, b)) return fail(SG_ERR_INVALID, "bad field indices");
    std::swap(g->phys[a], g->phys[b]);
    return SG_OK;
}

int sg_flush(sg_grid *g)
{
    if (!g) return fail(SG_ERR_INVALID, "null grid");
    return do_flush(g);
}

int sg_sync(sg_grid *g)
{
    if (!g) return fail(SG_ERR_INVALID, "null grid");
    return do_sync(g);
}

int sg_num_leaves(sg_grid *g, int64_t *n_leaves)
{
    if (!g || !n_leaves) return fail(SG_ERR_INVALID, "null argument");
    if (g->dry) {
        *n_leaves = 0;
        return do_flush(g);
    }
    int rc = sync_with_list(g);
    *n_leaves = g->host_ctrl->list_n;
    return rc;
}

int sg_read_structure(sg_grid *g, int64_t cap, int64_t *n_leaves, int32_t *leaf_b, uint32_t *masks)
{
    if (!g || !n_leaves || cap < 0) return fail(SG_ERR_INVALID, "null argument");
    int rc = sync_with_list(g);
    if (rc) return rc;
    const long long n = g->host_ctrl->list_n;
    *n_leaves = n;
    if (n > cap) return fail(SG_ERR_INVALID, "buffer holds %lld leaves, list has %lld", (long long)cap, n);
    if (n == 0) return SG_OK;
    if (leaf_b && (rc = cuda_check(cudaMemcpyAsync(leaf_b, g->dev.list_b, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, g->stream),
                                   "copy list")))
        return rc;
    if (masks) {
        if ((rc = ensure_staging(g))) return rc;
        launch_gather_masks(g->dev, g->stream, g->lc);
        if ((rc = after_launch(g, "gather masks"))) return rc;
        if ((rc = cuda_check(cudaMemcpyAsync(masks, g->dev.staging_u, sizeof(uint32_t) * g->dev.W * n,
                                             cudaMemcpyDeviceToHost, g->stream),
                             "copy masks")))
            return rc;
    }
    return cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize");
}

// The device address of a host buffer of `bytes` bytes that the device can
// read and write in place -- page-locked, mapped into the device's address
// space over its whole range, 16-byte aligned -- or null (then transfers go
// through the staging buffer with cudaMemcpyAsync).
void *mapped_host(void *host, size_t bytes)
{
    if (!host || bytes == 0 || ((uintptr_t)host & 15)) return nullptr;
    cudaPointerAttributes a{}, z{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess ||
        cudaPointerGetAttributes(&z, (char *)host + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || z.type != cudaMemoryTypeHost || !a.devicePointer || !z.devicePointer ||
        (char *)z.devicePointer != (char *)a.devicePointer + bytes - 1)
        return nullptr;
    return a.devicePointer;
}

int sg_read_field(sg_grid *g, int32_t f, int64_t cap, float *host_vals)
{
    if (!g || !valid_field(g, f) || !host_vals || cap < 0) return fail(SG_ERR_INVALID, "bad arguments");
    int rc = sync_with_list(g);
    if (rc) return rc;
    const long long n = g->host_ctrl->list_n;
    if (n > cap) return fail(SG_ERR_INVALID, "buffer holds %lld leaves, list has %lld", (long long)cap, n);
    if (n == 0) return SG_OK;
    const size_t bytes = sizeof(float) * size_t(n) * g->dev.L * g->dev.L * g->dev.L;
    float *direct = (float *)mapped_host(host_vals, bytes);
    if (!direct && (rc = ensure_staging(g))) return rc;
    launch_gather_field(g->dev, g->stream, g->phys[f], direct, g->lc);
    if ((rc = after_launch(g, "gather field"))) return rc;
    if (!direct && (rc = cuda_check(cudaMemcpyAsync(host_vals, g->dev.staging, bytes, cudaMemcpyDeviceToHost, g->stream),
                                    "copy field")))
        return rc;
    return cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize");
}

int sg_write_field(sg_grid *g, int32_t f, const float *host_vals, int64_t n_leaves)
{
    if (!g || !valid_field(g, f) || !host_vals || n_leaves < 0) return fail(SG_ERR_INVALID, "bad arguments");
    int rc = sync_with_list(g);
    if (rc) return rc;
    const long long n = g->host_ctrl->list_n;
    if (n != n_leaves) return fail(SG_ERR_INVALID, "list has %lld leaves, got %lld", n, (long long)n_leaves);
    if (n == 0) return SG_OK;
    const size_t bytes = sizeof(float) * size_t(n) * g->dev.L * g->dev.L * g->dev.L;
    // a mapped pinned buffer is read by the scatter kernel in place (one pass
    // over the host link, no staging copy)
    const float *direct = (const float *)mapped_host(const_cast<float *>(host_vals), bytes);
    if (!direct) {
        if ((rc = ensure_staging(g))) return rc;
        if ((rc = cuda_check(cudaMemcpyAsync(g->dev.staging, host_vals, bytes, cudaMemcpyHostToDevice, g->stream),
                             "copy field")))
            return rc;
    }
    launch_scatter_field(g->dev, g->stream, g->phys[f], direct, g->lc);
    if ((rc = after_launch(g, "scatter field"))) return rc;
    return cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize");
}

int sg_check(sg_grid *g, sg_check_report *out)
{
    if (!g || !out) return fail(SG_ERR_INVALID, "null argument");
    if (g->dry) return fail(SG_ERR_INVALID, "a dry-run grid holds no data");
    int rc = sync_with_list(g);
    if (rc && rc != SG_ERR_CHECK) return rc;  // a checking grid's own sync counts the same violations
    return run_checks(g, out, true);
}

int sg_debug_poke(sg_grid *g, int32_t array, int64_t index, uint32_t bits)
{
    if (!g || g->dry || array < 0 || array >= 2 + g->desc.n_fields || index < 0)
        return fail(SG_ERR_INVALID, "bad poke target");
    const long long nr = (long long)g->dev.R * g->dev.R * g->dev.R;
    const long long V = (long long)g->dev.L * g->dev.L * g->dev.L;
    void *dst = nullptr;
    if (array == 0) {
        const int32_t v = (int32_t)bits;
        if (index >= nr || v < -1 || v >= g->dev.cap) return fail(SG_ERR_INVALID, "root poke out of range");
        dst = g->dev.root + index;
    } else if (array == 1) {
        if (index >= (g->dev.cap + 1) * g->dev.W) return fail(SG_ERR_INVALID, "mask poke out of range");
        dst = g->dev.mask + index;
    } else {
        if (index >= (g->dev.cap + 1) * V) return fail(SG_ERR_INVALID, "field poke out of range");
        dst = g->dev.field[g->phys[array - 2]] + index;
    }
    int rc = do_sync(g);
    if (rc) return rc;
    if ((rc = cuda_check(cudaMemcpyAsync(dst, &bits, sizeof bits, cudaMemcpyHostToDevice, g->stream), "poke")))
        return rc;
    return cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize");
}

int sg_stage_active(sg_grid *g, const float *host_vals, int64_t n_active, int32_t *ticket)
{
    if (!g || !ticket || n_active < 0 || (n_active > 0 && !host_vals)) return fail(SG_ERR_INVALID, "bad arguments");
    const long long V = (long long)g->dev.L * g->dev.L * g->dev.L;
    if (n_active > g->dev.cap * V) return fail(SG_ERR_INVALID, "more values than the pool holds voxels");
    const int k = (int)(g->next_seq & 1u);
    const unsigned seq = g->next_seq++;
    if (!g->dry) {
        if (!g->copy_stream) {
            int rc;
            if ((rc = cuda_check(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking), "copy stream")))
                return rc;
            for (int j = 0; j < 2; ++j)
                if ((rc = cuda_check(cudaEventCreateWithFlags(&g->copied[j], cudaEventDisableTiming), "event")) ||
                    (rc = cuda_check(cudaEventCreateWithFlags(&g->consumed[j], cudaEventDisableTiming), "event")))
                    return rc;
        }
        if (!g->upload[k]) {
            g->upload[k] = (float *)dev_alloc(g, sizeof(float) * size_t(g->dev.cap * V));
            if (!g->upload[k]) return fail(SG_ERR_OOM, "upload slot");
        }
        int rc;
        // the slot's previous copy has finished reading its host buffer once
        // this returns (it ran two uploads ago; the wait is normally free)
        if (g->slot_used[k] &&
            ((rc = cuda_check(cudaEventSynchronize(g->copied[k]), "previous upload")) ||
             (rc = cuda_check(cudaStreamWaitEvent(g->copy_stream, g->consumed[k], 0), "wait for the slot"))))
            return rc;
        if (n_active > 0 &&
            (rc = cuda_check(cudaMemcpyAsync(g->upload[k], host_vals, sizeof(float) * size_t(n_active),
                                             cudaMemcpyHostToDevice, g->copy_stream),
                             "stage upload")))
            return rc;
        if ((rc = cuda_check(cudaEventRecord(g->copied[k], g->copy_stream), "record upload"))) return rc;
        // until a scatter consumes it, reusing the slot waits for this copy
        if ((rc = cuda_check(cudaEventRecord(g->consumed[k], g->copy_stream), "record slot"))) return rc;
        g->slot_used[k] = true;
    }
    g->upload_n[k] = n_active;
    g->upload_seq[k] = seq;
    *ticket = (int32_t)seq;
    return SG_OK;
}

int sg_write_field_staged(sg_grid *g, int32_t f, int32_t ticket)
{
    if (!g || !valid_field(g, f) || ticket <= 0) return fail(SG_ERR_INVALID, "bad arguments");
    const int k = (int)((unsigned)ticket & 1u);
    if (g->upload_seq[k] != (unsigned)ticket) return fail(SG_ERR_INVALID, "unknown or replaced upload ticket");
    Op o{OP_WRITE_STAGED};
    o.i0 = g->phys[f];
    o.i1 = ticket;
    o.slot = k;
    o.n = g->upload_n[k];
    return push(g, o);
}

int sg_write_field_active(sg_grid *g, int32_t f, const float *host_vals, int64_t n_active)
{
    if (!g || !valid_field(g, f) || n_active < 0 || (n_active > 0 && !host_vals))
        return fail(SG_ERR_INVALID, "bad arguments");
    int rc = sync_with_list(g);
    if (rc) return rc;
    const long long n = g->host_ctrl->list_n;
    long long total = 0;
    if (n > 0 && (rc = active_offsets(g, n, &total))) return rc;
    if (total != n_active)
        return fail(SG_ERR_INVALID, "the grid has %lld active voxels, got %lld", total, (long long)n_active);
    if (n == 0) return SG_OK;
    const size_t bytes = sizeof(float) * size_t(total);
    const float *direct = total > 0 ? (const float *)mapped_host(const_cast<float *>(host_vals), bytes) : nullptr;
    if (!direct) {
        if ((rc = ensure_staging(g))) return rc;
        if (bytes && (rc = cuda_check(cudaMemcpyAsync(g->dev.staging, host_vals, bytes, cudaMemcpyHostToDevice,
                                                      g->stream),
                                      "copy active values")))
            return rc;
    }
    launch_scatter_active(g->dev, g->stream, g->phys[f], direct ? direct : g->dev.staging, total, g->act_off,
                          g->act_tsum, g->lc);
    if ((rc = after_launch(g, "scatter active"))) return rc;
    return cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize");
}

int sg_read_field_active(sg_grid *g, int32_t f, int64_t cap, int64_t *n_active, float *host_vals)
{
    if (!g || !valid_field(g, f) || cap < 0 || !n_active) return fail(SG_ERR_INVALID, "bad arguments");
    int rc = sync_with_list(g);
    if (rc) return rc;
    const long long n = g->host_ctrl->list_n;
    long long total = 0;
    if (n > 0 && (rc = active_offsets(g, n, &total))) return rc;
    *n_active = total;
    if (total > cap) return fail(SG_ERR_INVALID, "buffer holds %lld values, the grid has %lld active voxels",
                                 (long long)cap, total);
    if (total == 0) return SG_OK;
    if (!host_vals) return fail(SG_ERR_INVALID, "null buffer");
    const size_t bytes = sizeof(float) * size_t(total);
    float *direct = (float *)mapped_host(host_vals, bytes);
    if (!direct && (rc = ensure_staging(g))) return rc;
    launch_gather_active(g->dev, g->stream, g->phys[f], direct ? direct : g->dev.staging, total, g->act_off,
                         g->act_tsum, g->lc);
    if ((rc = after_launch(g, "gather active"))) return rc;
    if (!direct && (rc = cuda_check(cudaMemcpyAsync(host_vals, g->dev.staging, bytes, cudaMemcpyDeviceToHost,
                                                    g->stream),
                                    "copy active values")))
        return rc;
    return cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize");
}

struct sg_graph {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

int sg_graph_begin(void *cuda_stream)
{
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s) return fail(SG_ERR_INVALID, "the legacy default stream cannot be recorded");
    return cuda_check(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "begin recording");
}

int sg_graph_end(void *cuda_stream, sg_graph **out)
{
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s || !out) return fail(SG_ERR_INVALID, "null argument");
    *out = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return fail(SG_ERR_INVALID, "recording failed (%s): a call made while recording needed the host",
                    cudaGetErrorString(e));
    }
    sg_graph *gr = new (std::nothrow) sg_graph();
    if (!gr) {
        cudaGraphDestroy(graph);
        return fail(SG_ERR_OOM, "host allocation");
    }
    gr->stream = s;
    gr->graph = graph;
    int rc = cuda_check(cudaGraphInstantiate(&gr->exec, graph, 0), "instantiate graph");
    if (rc) {
        cudaGraphDestroy(graph);
        delete gr;
        return rc;
    }
    *out = gr;
    return SG_OK;
}

int sg_graph_launch(sg_graph *gr)
{
    if (!gr) return fail(SG_ERR_INVALID, "null graph");
    return cuda_check(cudaGraphLaunch(gr->exec, gr->stream), "launch graph");
}

int sg_graph_destroy(sg_graph *gr)
{
    if (!gr) return SG_OK;
    cudaStreamSynchronize(gr->stream);
    if (gr->exec) cudaGraphExecDestroy(gr->exec);
    if (gr->graph) cudaGraphDestroy(gr->graph);
    delete gr;
    return SG_OK;
}

int sg_write_structure(sg_grid *g, int64_t n_leaves, const int32_t *leaf_b, const uint32_t *masks)
{
    if (!g || n_leaves < 0 || (n_leaves > 0 && (!leaf_b || !masks))) return fail(SG_ERR_INVALID, "bad arguments");
    const long long nr = (long long)g->dev.R * g->dev.R * g->dev.R;
    for (long long e = 0; e < n_leaves; ++e)
        if (leaf_b[e] < 0 || leaf_b[e] >= nr || (e > 0 && leaf_b[e] <= leaf_b[e - 1]))
            return fail(SG_ERR_INVALID, "leaf_b[%lld] = %d out of range or order", e, leaf_b[e]);
    if (n_leaves > g->dev.cap)
        return fail(SG_ERR_POOL_EXHAUSTED, "%lld saved leaves, max_leaves %lld", (long long)n_leaves,
                    (long long)g->dev.cap);
    if (g->dry) return fail(SG_ERR_INVALID, "a dry-run grid holds no data");
    int rc = do_sync(g);
    if (rc) return rc;
    const long long n = n_leaves;
    // both arrays go through the staging buffer: n * (1 + W) words <= cap * L^3
    if (n > 0 && (rc = ensure_staging(g))) return rc;
    const size_t b_words = (size_t(n) + 3) & ~size_t(3);  // masks start 16-byte aligned
    int32_t *dev_b = (int32_t *)g->dev.staging_u;
    uint32_t *dev_m = g->dev.staging_u + b_words;
    launch_deactivate_all(g->dev, g->stream);
    if ((rc = after_launch(g, "deactivate"))) return rc;
    if (n > 0) {
        if ((rc = cuda_check(cudaMemcpyAsync(dev_b, leaf_b, sizeof(int32_t) * n, cudaMemcpyHostToDevice, g->stream),
                             "copy leaf_b")) ||
            (rc = cuda_check(cudaMemcpyAsync(dev_m, masks, sizeof(uint32_t) * g->dev.W * n, cudaMemcpyHostToDevice,
                                             g->stream),
                             "copy masks")))
            return rc;
        launch_restore_structure(g->dev, g->stream, dev_b, dev_m, n, g->lc);
        if ((rc = after_launch(g, "restore structure"))) return rc;
    }
    g->mask_ver++;
    g->applied_shells.clear();
    g->applied_restrict.clear();
    return sync_with_list(g);
}

int sg_read_sums(sg_grid *g, double *host, int64_t n)
{
    if (!g || n < 0 || n > g->desc.max_sums || (n > 0 && !host)) return fail(SG_ERR_INVALID, "bad arguments");
    if (g->dry) return fail(SG_ERR_INVALID, "a dry-run grid holds no data");
    int rc = do_sync(g);
    if (rc) return rc;
    if (n == 0) return SG_OK;
    if ((rc = cuda_check(cudaMemcpyAsync(host, g->dev.sums, sizeof(double) * n, cudaMemcpyDeviceToHost, g->stream), "copy sums")))
        return rc;
    return cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize");
}

int sg_set_stencil_variant(sg_grid *g, int32_t variant)
{
    if (!g || variant < SG_VARIANT_SWEEP || variant > SG_VARIANT_SWEEP_TMA)
        return fail(SG_ERR_INVALID, "bad grid or variant");
    g->lc.variant = variant;
    return SG_OK;
}

int sg_get_stats(sg_grid *g, sg_stats *out)
{
    if (!g || !out) return fail(SG_ERR_INVALID, "null argument");
    *out = g->stats;
    return SG_OK;
}

int sg_debug_wait_test(sg_grid *g)
{
    if (!g) return fail(SG_ERR_INVALID, "null grid");
    return push(g, Op{OP_TEST_WAIT});
}

int sg_num_active(sg_grid *g, int64_t *n_active)
{
    if (!g || !n_active) return fail(SG_ERR_INVALID, "null argument");
    int rc = sync_with_list(g);
    if (rc) return rc;
    launch_count_active(g->dev, g->stream, g->lc);
    if ((rc = after_launch(g, "count active"))) return rc;
    if ((rc = do_sync(g))) return rc;
    *n_active = (int64_t)g->host_ctrl->n_active;
    return SG_OK;
}

int sg_fill_hash(sg_grid *g, int32_t f, int64_t seed)
{
    if (!g || !valid_field(g, f) || seed < 0 || seed >= (1LL << 24)) return fail(SG_ERR_INVALID, "bad fill arguments");
    Op o{OP_FILL};
    o.i0 = g->phys[f];
    o.slot = seed;
    return push(g, o);
}

}  // extern "C"

// ============================================================================
// Batched stepping: many grids, one persistent launch per step
// ============================================================================
struct sg_batch {
    std::vector<sg_grid *> grids;
    cudaStream_t stream = nullptr;
    int32_t src = 0, tmp = 1, dst = 2;
    float coef = 0.f;
    int total_tri = 0;
    long long total_leaves = 0;
    BatchGrid *dev_items[2] = {nullptr, nullptr};  // parity 0: src -> dst; parity 1: dst -> src
    double *dev_acc = nullptr;
    void *blocks[2] = {nullptr, nullptr};  // descriptors (and sums), from grid 0's allocator
    void *maps = nullptr;                  // the staged body's tensor maps, from grid 0's allocator
    int parity = 0;
    int warps = 4;
    int use_graph = 1;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t own = nullptr;            // capture / replay stream (the caller's may be the legacy stream)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int num_sms = 0;
    long long launches = 0;
    int staged = 0;                        // body: 0 register sweep, 1 staged by bulk tensor copies
    bool staged_ready = false;             // descriptors and tensor maps of the staged body are set up
    std::vector<BatchGrid> host_items[2];
};

namespace {

void batch_drop_graphs(sg_batch *b)
{
    for (auto &e : b->exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
}

int batch_enqueue(sg_batch *b, int parity)
{
    const size_t nacc = sizeof(double) * b->grids.size();
    int rc = cuda_check(cudaMemsetAsync(b->dev_acc, 0, nacc, b->stream), "batch accumulator reset");
    if (rc) return rc;
    if (b->staged) {
        if (launch_batch_tma(b->dev_items[parity], (int)b->grids.size(), b->total_tri, b->coef, b->dev_acc, b->num_sms,
                             b->stream))
            return fail(SG_ERR_CUDA, "staged batched step: launch attributes unavailable");
    } else {
        launch_batch_diffuse_box(b->dev_items[parity], (int)b->grids.size(), b->total_tri, b->coef, b->dev_acc,
                                 b->warps, b->num_sms, b->stream);
    }
    return cuda_check(cudaPeekAtLastError(), "batched step launch");
}

int batch_capture(sg_batch *b, int parity)
{
    cudaGraph_t graph = nullptr;
    int rc = cuda_check(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (rc) return rc;
    cudaStream_t user = b->stream;
    b->stream = b->own;  // enqueue into the capturing stream
    const int rc_enq = batch_enqueue(b, parity);
    b->stream = user;
    rc = cuda_check(cudaStreamEndCapture(b->own, &graph), "end capture");
    if (rc_enq) {
        if (graph) cudaGraphDestroy(graph);
        return rc_enq;
    }
    if (rc) return rc;
    rc = cuda_check(cudaGraphInstantiate(&b->exec[parity], graph, 0), "graph instantiate");
    cudaGraphDestroy(graph);
    return rc;
}

}  // namespace

namespace sg {

int grid_num_sms(const sg_grid *g) { return g->lc.num_sms; }

// The queued part of preparing a grid for the batched step: the queued ops,
// a current list, the region masks and j-run records, and the active count.
static int prepare_batch_queue(sg_grid *g, int src, int tmp, int dst)
{
    if (!g || g->dry || g->dev.L != 8) return fail(SG_ERR_INVALID, "batched grids must be live 8^3-leaf grids");
    if (!valid_field(g, src) || !valid_field(g, tmp) || !valid_field(g, dst) || src == tmp || src == dst || tmp == dst)
        return fail(SG_ERR_INVALID, "bad field indices");
    int rc = do_flush(g);
    if (!rc && g->list_ver != g->mask_ver) {
        rc = launch_list(g, false, 0);
        g->list_ver = g->mask_ver;
    }
    // region masks and the j-run records of the batched kernel
    const bool need_runs = g->colgrp_ver != g->list_ver || g->colgrp_axis != kGroupJ;
    if (!rc && (g->rmask_ver != g->list_ver || need_runs)) {
        launch_region_masks(g->dev, g->stream, g->lc, need_runs ? kGroupJ : kGroupNone, ++g->rr_calls);
        rc = after_launch(g, "region masks");
        g->rmask_ver = g->list_ver;
        if (need_runs) {
            g->colgrp_ver = g->list_ver;
            g->colgrp_axis = kGroupJ;
        }
    }
    if (!rc) {
        launch_count_active(g->dev, g->stream, g->lc);
        rc = after_launch(g, "count active");
    }
    return rc;
}

// The two parities' descriptors from the host copies of the control block and
// the run-record counts.
static void batch_items(sg_grid *g, int src, int tmp, int dst, const int32_t *cnt, BatchGrid out[2],
                        long long *n_active)
{
    if (n_active) *n_active = (long long)g->host_ctrl->n_active;
    const int nl = g->host_ctrl->list_n;
    const int pairs = std::min(cnt[1], cnt[0]);
    for (int p = 0; p < 2; ++p) {
        BatchGrid it{};
        it.g = g->dev;
        it.x = g->dev.field[g->phys[p == 0 ? src : dst]];
        it.y = g->dev.field[g->phys[p == 0 ? dst : src]];
        it.t = g->dev.field[g->phys[tmp]];
        it.n = nl;
        it.c1 = cnt[0];
        it.c2 = cnt[1];
        it.c3 = cnt[2];
        it.tasks = cnt[2] + cnt[1] + (cnt[0] - pairs + 1) / 2;
        it.tri0 = 0;
        out[p] = it;
    }
}

int grid_prepare_batch(sg_grid *g, int src, int tmp, int dst, BatchGrid out[2], long long *n_active)
{
    int rc = prepare_batch_queue(g, src, tmp, dst);
    if (!rc) rc = do_sync(g);
    int32_t cnt[3] = {0, 0, 0};
    if (!rc)
        rc = cuda_check(cudaMemcpy(cnt, g->dev.col_cnt, sizeof cnt, cudaMemcpyDeviceToHost), "run record counts");
    if (rc) return rc;
    batch_items(g, src, tmp, dst, cnt, out, n_active);
    return SG_OK;
}

int grid_prepare_batch_async(sg_grid *g, int src, int tmp, int dst, int32_t *cnt)
{
    if (g && (g->desc.flags & SG_CREATE_CHECK)) return fail(SG_ERR_INVALID, "checking grids prepare synchronously");
    int rc = prepare_batch_queue(g, src, tmp, dst);
    if (!rc)
        rc = cuda_check(cudaMemcpyAsync(g->host_ctrl, g->dev.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, g->stream),
                        "read control block");
    if (!rc)
        rc = cuda_check(cudaMemcpyAsync(cnt, g->dev.col_cnt, sizeof(int32_t) * 3, cudaMemcpyDeviceToHost, g->stream),
                        "run record counts");
    return rc;
}

int grid_prepare_batch_finish(sg_grid *g, int src, int tmp, int dst, const int32_t *cnt, BatchGrid out[2],
                              long long *n_active)
{
    const int bits = g->host_ctrl->err;
    if (bits) {
        cudaMemsetAsync(&g->dev.ctrl->err, 0, sizeof(int32_t), g->stream);
        cudaStreamSynchronize(g->stream);
        return map_device_error(bits);
    }
    if (g->latched != SG_OK) {
        const int out_rc = g->latched;
        g->latched = SG_OK;
        return out_rc;
    }
    if (g->list_ver == g->mask_ver) g->known_leaves = g->host_ctrl->list_n;
    batch_items(g, src, tmp, dst, cnt, out, n_active);
    return SG_OK;
}

}  // namespace sg

extern "C" {

int sg_batch_create(sg_grid *const *grids, int32_t n, int32_t src, int32_t tmp, int32_t dst, float coef,
                    void *cuda_stream, sg_batch **out)
{
    if (!grids || !out || n < 1 || n > kMaxBatch) return fail(SG_ERR_INVALID, "batch needs 1..%d grids", kMaxBatch);
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        sg_grid *g = grids[i];
        if (!g || g->dry || g->dev.L != 8) return fail(SG_ERR_INVALID, "batched grids must be live 8^3-leaf grids");
        if (!valid_field(g, src) || !valid_field(g, tmp) || !valid_field(g, dst) || src == tmp || src == dst || tmp == dst)
            return fail(SG_ERR_INVALID, "bad field indices for grid %d", i);
    }
    sg_batch *b = new (std::nothrow) sg_batch();
    if (!b) return fail(SG_ERR_OOM, "host allocation");
    b->grids.assign(grids, grids + n);
    b->stream = (cudaStream_t)cuda_stream;
    b->src = src;
    b->tmp = tmp;
    b->dst = dst;
    b->coef = coef;
    b->num_sms = grids[0]->lc.num_sms;
    std::vector<BatchGrid> items[2];
    int rc = SG_OK;
    for (int i = 0; i < n && !rc; ++i) {
        BatchGrid two[2];
        long long na = 0;
        rc = grid_prepare_batch(grids[i], src, tmp, dst, two, &na);
        if (rc) break;
        for (int p = 0; p < 2; ++p) {
            two[p].tri0 = b->total_tri;
            items[p].push_back(two[p]);
        }
        b->total_tri += two[0].tasks;
        b->total_leaves += two[0].n;
    }
    if (rc) {
        delete b;
        return rc;
    }
    sg_grid *g0 = grids[0];
    b->host_items[0] = items[0];
    b->host_items[1] = items[1];
    for (int p = 0; p < 2 && !rc; ++p) {
        b->blocks[p] = dev_alloc(g0, sizeof(BatchGrid) * n + (p == 0 ? sizeof(double) * n : 0));
        if (!b->blocks[p]) rc = fail(SG_ERR_OOM, "batch descriptors");
    }
    if (!rc) {
        b->dev_items[0] = (BatchGrid *)b->blocks[0];
        b->dev_acc = (double *)((char *)b->blocks[0] + sizeof(BatchGrid) * n);
        b->dev_items[1] = (BatchGrid *)b->blocks[1];
        for (int p = 0; p < 2 && !rc; ++p)
            rc = cuda_check(cudaMemcpyAsync(b->dev_items[p], items[p].data(), sizeof(BatchGrid) * n,
                                            cudaMemcpyHostToDevice, b->stream),
                            "batch descriptors");
        if (!rc) rc = cuda_check(cudaMemsetAsync(b->dev_acc, 0, sizeof(double) * n, b->stream), "batch sums");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(b->stream), "batch sync");
    }
    if (!rc) rc = cuda_check(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking), "batch stream");
    if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming), "batch event");
    if (!rc) rc = cuda_check(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming), "batch event");
    if (rc) {
        // blocks belong to grid 0's allocation list and are released with it
        if (b->ev_in) cudaEventDestroy(b->ev_in);
        if (b->own) cudaStreamDestroy(b->own);
        delete b;
        return rc;
    }
    *out = b;
    return SG_OK;
}

// The staged body's inputs, once per batch: every grid's TMA task
// descriptors (its j-run records are current since sg_batch_create) and the
// tensor maps over x for both src/dst parities, uploaded with the
// descriptors of the batch.
int batch_prepare_staged(sg_batch *b)
{
    if (b->staged_ready) return SG_OK;
    const int n = (int)b->grids.size();
    int rc;
    for (sg_grid *g : b->grids) {
        if ((rc = ensure_tma_desc(g, std::max<long long>(g->host_ctrl->list_n, 1)))) return rc;
        if (g->tma_ver != g->list_ver) {
            launch_tma_tasks(g->dev, g->stream, g->lc);
            if ((rc = after_launch(g, "TMA task descriptors"))) return rc;
            g->tma_ver = g->list_ver;
        }
        if ((rc = cuda_check(cudaStreamSynchronize(g->stream), "stream synchronize"))) return rc;
    }
    std::vector<unsigned char> host(size_t(2) * n * kTmaMapsBytes + 64);
    unsigned char *h = host.data() + ((64 - (reinterpret_cast<uintptr_t>(host.data()) & 63)) & 63);
    for (int i = 0; i < n; ++i)
        for (int p = 0; p < 2; ++p)
            if (!tma_encode_maps(b->host_items[p][i].x, b->grids[i]->dev.cap, h + size_t(2 * i + p) * kTmaMapsBytes))
                return fail(SG_ERR_CUDA, "tensor maps of batched grid %d could not be encoded", i);
    unsigned char *dmaps = (unsigned char *)dev_alloc(b->grids[0], size_t(2) * n * kTmaMapsBytes);
    if (!dmaps) return fail(SG_ERR_OOM, "batch tensor maps");
    b->maps = dmaps;
    for (int i = 0; i < n; ++i) {
        const DevGrid &d = b->grids[i]->dev;
        if (!d.tma_desc || !d.tma_rmask) return fail(SG_ERR_INVALID, "batched grid %d has no TMA task descriptors", i);
        for (int p = 0; p < 2; ++p) {
            // the items hold copies of the grids' device descriptors, taken at
            // sg_batch_create: refresh them so they carry the arrays above
            b->host_items[p][i].g.tma_desc = d.tma_desc;
            b->host_items[p][i].g.tma_rmask = d.tma_rmask;
            b->host_items[p][i].tma_maps = dmaps + size_t(2 * i + p) * kTmaMapsBytes;
        }
    }
    if ((rc = cuda_check(cudaMemcpyAsync(dmaps, h, size_t(2) * n * kTmaMapsBytes, cudaMemcpyHostToDevice, b->stream),
                         "batch tensor maps")))
        return rc;
    for (int p = 0; p < 2; ++p)
        if ((rc = cuda_check(cudaMemcpyAsync(b->dev_items[p], b->host_items[p].data(), sizeof(BatchGrid) * n,
                                             cudaMemcpyHostToDevice, b->stream),
                             "batch descriptors")))
            return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(b->stream), "batch sync"))) return rc;
    b->staged_ready = true;
    return SG_OK;
}

int sg_batch_set(sg_batch *b, int32_t warps_per_cta, int32_t use_graph)
{
    if (!b || (warps_per_cta != 2 && warps_per_cta != 4 && warps_per_cta != 8))
        return fail(SG_ERR_INVALID, "warps_per_cta must be 2, 4 or 8");
    if (warps_per_cta != b->warps) batch_drop_graphs(b);
    b->warps = warps_per_cta;
    b->use_graph = use_graph ? 1 : 0;
    return SG_OK;
}

int sg_batch_step(sg_batch *b)
{
    if (!b) return fail(SG_ERR_INVALID, "null batch");
    int rc;
    const int p = b->parity;
    if (b->use_graph) {
        if (!b->exec[p] && (rc = batch_capture(b, p))) return rc;
        // replay on the batch's own stream, ordered after and before the caller's stream
        if ((rc = cuda_check(cudaEventRecord(b->ev_in, b->stream), "event record")) ||
            (rc = cuda_check(cudaStreamWaitEvent(b->own, b->ev_in, 0), "stream wait")) ||
            (rc = cuda_check(cudaGraphLaunch(b->exec[p], b->own), "graph launch")) ||
            (rc = cuda_check(cudaEventRecord(b->ev_out, b->own), "event record")) ||
            (rc = cuda_check(cudaStreamWaitEvent(b->stream, b->ev_out, 0), "stream wait")))
            return rc;
    } else if ((rc = batch_enqueue(b, p))) {
        return rc;
    }
    b->launches++;
    for (sg_grid *g : b->grids) {
        std::swap(g->phys[b->src], g->phys[b->dst]);
        g->stats.launches++;
        g->stats.ops_fused += 2;
        g->stats.stores_removed += 1;
    }
    b->parity ^= 1;
    return SG_OK;
}

int sg_batch_read_sums(sg_batch *b, double *host, int32_t n)
{
    if (!b || n < 0 || n > (int32_t)b->grids.size() || (n > 0 && !host)) return fail(SG_ERR_INVALID, "bad arguments");
    int rc = cuda_check(cudaMemcpyAsync(host, b->dev_acc, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream),
                        "copy batch sums");
    if (rc) return rc;
    return cuda_check(cudaStreamSynchronize(b->stream), "batch sync");
}

int sg_batch_set_staging(sg_batch *b, int32_t staged)
{
    if (!b || (staged != 0 && staged != 1)) return fail(SG_ERR_INVALID, "staged must be 0 or 1");
    int rc;
    if (staged && (rc = batch_prepare_staged(b))) return rc;
    if (staged != b->staged) batch_drop_graphs(b);
    b->staged = staged;
    return SG_OK;
}

int sg_batch_config(sg_batch *b, int32_t *warps_per_cta, int32_t *staged)
{
    if (!b) return fail(SG_ERR_INVALID, "null batch");
    if (warps_per_cta) *warps_per_cta = b->staged ? 8 : b->warps;
    if (staged) *staged = b->staged;
    return SG_OK;
}

int sg_batch_info(sg_batch *b, int64_t *total_leaves, int64_t *launches, int32_t *warps_per_cta)
{
    if (!b) return fail(SG_ERR_INVALID, "null batch");
    if (total_leaves) *total_leaves = b->total_leaves;
    if (launches) *launches = b->launches;
    if (warps_per_cta) *warps_per_cta = b->warps;
    return SG_OK;
}

int sg_batch_autotune(sg_batch *b, int32_t trial_steps, int32_t *chosen)
{
    if (!b || trial_steps < 1) return fail(SG_ERR_INVALID, "bad autotune arguments");
    // (halo staging, warps per CTA): the register sweep at 2, 4 and 8 warps
    // per CTA, and the body staged by bulk tensor copies (eight warps per CTA,
    // one CTA per SM, fixed by its shared-memory buffers)
    const int cands[4][2] = {{0, 2}, {0, 4}, {0, 8}, {1, 8}};
    float best = 1e30f;
    int best_w = b->warps, best_s = b->staged, rc = SG_OK;
    cudaEvent_t e0, e1;
    if ((rc = cuda_check(cudaEventCreate(&e0), "event"))) return rc;
    if ((rc = cuda_check(cudaEventCreate(&e1), "event"))) {
        cudaEventDestroy(e0);
        return rc;
    }
    for (const auto &c : cands) {
        if ((rc = sg_batch_set_staging(b, c[0]))) break;
        if ((rc = sg_batch_set(b, c[1], b->use_graph))) break;
        if ((rc = sg_batch_step(b))) break;  // warm-up (and graph capture)
        if ((rc = cuda_check(cudaEventRecord(e0, b->stream), "event"))) break;
        for (int st = 0; st < trial_steps && !rc; ++st) rc = sg_batch_step(b);
        if (rc) break;
        if ((rc = cuda_check(cudaEventRecord(e1, b->stream), "event"))) break;
        if ((rc = cuda_check(cudaEventSynchronize(e1), "event sync"))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_w = c[1];
            best_s = c[0];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = sg_batch_set_staging(b, best_s)) || (rc = sg_batch_set(b, best_w, b->use_graph))) return rc;
    if (chosen) *chosen = best_w;
    return SG_OK;
}

int sg_batch_destroy(sg_batch *b)
{
    if (!b) return SG_OK;
    int rc = cuda_check(cudaStreamSynchronize(b->stream), "batch sync");
    if (b->own) cudaStreamSynchronize(b->own);
    batch_drop_graphs(b);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->own) cudaStreamDestroy(b->own);
    // the batch's work has finished: its blocks go back to grid 0's allocator
    if (!b->grids.empty()) {
        dev_release(b->grids[0], b->blocks[0]);
        dev_release(b->grids[0], b->blocks[1]);
        dev_release(b->grids[0], b->maps);
    }
    delete b;
    return rc;
}

const char *sg_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"
