// sg_device.h -- device-side layout of one sparse grid and the launch
// wrappers the host queue calls.  Internal to libsgrid.
//
// HBM layout of a grid (all arrays allocated once at creation):
//   root[R^3]            int32   leaf slot of each pointer cell, -1 = null
//   mask[cap][W]         uint32  W = L^3/32 bit words per leaf slot
//   field[f][cap][L^3]   float   one array per field (structure of arrays),
//                                each leaf a contiguous 2 KB (L=8) block
//   list_slot[cap], list_b[cap]  the active-leaf list, ascending b
//   nbr[cap][27]         int32   slots of the 3x3x3 leaf neighbourhood of each
//                                list entry (index (di+1)*9+(dj+1)*3+(dk+1));
//                                a null or out-of-domain neighbour is slot
//                                `cap`, the zero leaf: field and mask arrays
//                                hold cap + 1 leaves and leaf `cap` is never
//                                allocated, so it reads as zeros everywhere
//   need[R^3]            uint8   activation requests (coords / particles)
//   tile_status[tiles]   uint64  list-compaction look-back words
//   partials[max_ctas]   double  per-CTA reduction partials
//   sums[max_sums]       double  reduction results
//   ctrl                 Ctrl    counters and flags below
// Invariant kept by every kernel: a stored value at an inactive voxel of an
// allocated leaf is 0, so whole-leaf loads need no mask to read 0 there.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sgrid.h"

namespace sg {

constexpr int kMaxFields = 16;

enum ErrBits : int32_t {
    kErrPool = 1,     // leaf pool exhausted
    kErrTimeout = 2,  // a bounded wait gave up
    kErrCheck = 4,    // a kernel's own address check failed; the access was skipped
};

struct Ctrl {
    int32_t pool_count;   // slots handed out (may exceed cap after exhaustion)
    int32_t dirty;        // structure changed since the list was generated
    int32_t list_n;       // entries in the active-leaf list
    int32_t err;          // ErrBits
    unsigned long long lg_ticket;  // list-compaction tile tickets (monotone)
    unsigned long long lg_done;    // list-compaction finished tiles (monotone)
    unsigned long long n_active;   // active voxels of the listed leaves (count kernel)
    unsigned int red_ticket;       // reduction finished CTAs (reset by the last)
    int32_t never_set;    // a flag nothing writes (bounded-wait test)
    int32_t timeout_site; // which wait gave up (0 none, 1 look-back, 2 test, 3 leaf allocation)
                          // or, with kErrCheck, 100 + the failed check
    int32_t bins_used;    // leaves holding particles in the last binned P2G
    uint32_t rr_ticket;   // run-record tiles handed out (zeroed before each region-mask launch)
    int32_t pad[1];
};

struct DevGrid {
    int32_t N, L, R, lg2, W, F;
    int64_t cap;
    int32_t *root;
    uint32_t *mask;
    float *field[kMaxFields];
    int32_t *list_slot;
    int32_t *list_b;
    int32_t *nbr;
    uint32_t *rmask;     // [cap][10][4]: region masks of the fused kernel, see launch_region_masks
    uint8_t *need;
    unsigned long long *tile_status;
    double *partials;
    double *sums;
    Ctrl *ctrl;
    float *staging;      // n * L^3 floats for host reads/writes
    uint32_t *staging_u; // aliases staging for mask gathers
    // binned P2G scratch (allocated at the first P2G): per-key counts/cursors
    // and offsets, tile sums of the count scan, particle order
    int32_t *bin_count;
    int32_t *bin_off;
    int32_t *tile_sum;
    int32_t *perm;
    int32_t *perm_alt;  // the next binning's order, built from the last one (then swapped)
    long long *perm_key;  // each particle's key, stored by the count pass for the order pass
    int32_t *bin_list;  // the leaves holding particles, in no particular order
    // grouped sweeps of the fused step: list entry of each slot (written by
    // the list generation), the records of runs of adjacent leaves (along i
    // for the column sweep, along j for the j-run sweep) bucketed by length,
    // and their counts (built with the region masks); allocated with the grid
    int32_t *ent_of_slot;
    int32_t *col_grp;   // [3][cap][3]
    int32_t *col_cnt;   // [4]
    unsigned long long *rr_status; // [cap / 256 + 1][3]: run-record look-back words, per 256-entry tile and length
    // TMA-staged fused step (allocated at its first use): per j-run warp task,
    // the source slot of each staged box and the kind (64 words), and the
    // region masks of its leaves (120 words); see k_tma_tasks
    int32_t *tma_desc;  // [cap][64]
    uint32_t *tma_rmask; // [cap][120]
};

// Stencil kernel families for 8^3 leaves (sg_set_stencil_variant picks one).
enum StencilVariant : int {
    kVariantSweep = 0,  // register sweep, rows loaded through the read-only path
    kVariantSmem = 1,   // leaf + halo staged in shared memory by plain loads
    kVariantSweepColumns = 2,  // register sweep; the fused step sweeps columns of
                               // leaves adjacent in i (see k_sweep_columns)
    kVariantSweepJRuns = 3,    // register sweep; a warp's leaves are runs of leaves
                               // adjacent in j (see k_sweep_jruns)
    kVariantSweepTma = 4,      // the j-run tasks with every x row staged in shared
                               // memory by bulk tensor copies (see k_sweep_tma)
};

// Axis along which launch_region_masks groups adjacent leaves into records.
enum GroupAxis : int { kGroupNone = 0, kGroupI = 1, kGroupJ = 2 };

// Launch shapes chosen by the host.
struct LaunchCfg {
    int num_sms;
    int persistent_ctas;  // CTAs of the persistent leaf loops
    int variant;          // StencilVariant
    int single_runs = 0;  // the j-run records are current: single stencils sweep j-runs
};

constexpr int kListTile = 1024;  // root cells per compaction CTA
constexpr int kListThreads = 256;
constexpr int kSpinLimit = 1 << 22;  // bounded waits: polls before giving up

// ---- structure kernels (sg_structure.cu) ----
// fill_mask: the physical fields a newly allocated leaf is zero-filled in
// (bit f for field f; all of them unless the caller knows a field's zeros are
// never read).
void launch_activate_shell(const DevGrid &g, cudaStream_t s, long long lo2, long long hi2, int strict,
                           uint32_t fill_mask);
void launch_mark_coords(const DevGrid &g, cudaStream_t s, const int32_t *xyz, long long n);
// fill_mask as for launch_activate_shell (default: every field)
void launch_alloc_needed(const DevGrid &g, cudaStream_t s, uint32_t fill_mask = 0xffffffffu);
void launch_setbits_coords(const DevGrid &g, cudaStream_t s, const int32_t *xyz, long long n);
void launch_deactivate_all(const DevGrid &g, cudaStream_t s);
// Invariant checks (sg_check): violation counters, indexed by CheckKind.
enum CheckKind { kChkRoot, kChkShared, kChkList, kChkNbr, kChkZero, kChkInactive, kChkLeaves, kNumChk };
// owner: cap words set to 0xffffffff before the launch (slot -> root cell);
// cnt: kNumChk zeroed counters.  The list checks need a current list.
void launch_checks(const DevGrid &g, cudaStream_t s, uint32_t *owner, unsigned long long *cnt, bool with_list,
                   uint32_t field_bits, const LaunchCfg &lc);
// Slot e <- saved leaf e: root[leaf_b[e]] = e, mask words copied, fields
// zeroed; pool_count = n.  Runs after launch_deactivate_all.
void launch_restore_structure(const DevGrid &g, cudaStream_t s, const int32_t *leaf_b, const uint32_t *masks,
                              long long n, const LaunchCfg &lc);
void launch_clear_list(const DevGrid &g, cudaStream_t s);
// For each list entry (8^3 leaves) and each of the 10 columns tj of the
// 10^3 region around the leaf, the activity bits of the 10 rows ti = 0..9 of
// that column: row (ti, tj) covers region voxels (ti+1, tj+1, r+1), r = 0..9,
// as 10 bits; rows 3w..3w+2 are packed into word w of rmask[e][tj][0..3].
// The fused sweep's region masks of the current list; with columns also the
// column records of the column sweep (ent_of_slot is written by the list
// generation).
// call: a per-grid counter of these launches (tags the look-back words, so
// stale words of earlier launches are ignored without a reset).
void launch_region_masks(const DevGrid &g, cudaStream_t s, const LaunchCfg &lc, int group_axis,
                         unsigned long long call);
void launch_listgen(const DevGrid &g, cudaStream_t s, int force, unsigned long long call_idx,
                    int num_tiles, int test_wait);
// Field f of the listed leaves to / from a dense list-order buffer: the
// staging buffer when the pointer is null, else a device-addressable one
// (16-byte aligned; e.g. mapped pinned host memory, read or written in place).
void launch_gather_field(const DevGrid &g, cudaStream_t s, int f, float *dst, const LaunchCfg &lc);
void launch_gather_masks(const DevGrid &g, cudaStream_t s, const LaunchCfg &lc);
void launch_scatter_field(const DevGrid &g, cudaStream_t s, int f, const float *src, const LaunchCfg &lc);
// Active-voxel transfers: off[n] and tsum[n / kOffTile + 2] are scratch;
// launch_active_offsets leaves the packed position of each list entry's first
// active voxel in off[e] + tsum[e / kOffTile] and the total in
// tsum[ceil(n / kOffTile)].  src / out hold exactly that many values.
constexpr int kOffTile = 1024;
void launch_active_offsets(const DevGrid &g, cudaStream_t s, long long n, long long *off, long long *tsum);
void launch_scatter_active(const DevGrid &g, cudaStream_t s, int f, const float *src, long long total,
                           const long long *off, const long long *tsum, const LaunchCfg &lc);
void launch_gather_active(const DevGrid &g, cudaStream_t s, int f, float *out, long long total, const long long *off,
                          const long long *tsum, const LaunchCfg &lc);

// ---- stencil kernels (sg_stencil.cu) ----
// check_act: eager activation-on-write check on every store (Sec. 6.3 off).
void launch_clear(const DevGrid &g, cudaStream_t s, int dst, int check_act, const LaunchCfg &lc);
void launch_diffuse7(const DevGrid &g, cudaStream_t s, int src, int dst, float coef,
                     int check_act, int sum_slot, const LaunchCfg &lc);
void launch_box27(const DevGrid &g, cudaStream_t s, int src, int dst, int check_act,
                  int sum_slot, const LaunchCfg &lc);
void launch_sweep_columns(const DevGrid &g, cudaStream_t s, int src, int tmp, int dst, float coef, int store_tmp,
                          int check_act, int sum_slot, const LaunchCfg &lc);
void launch_sweep_jruns(const DevGrid &g, cudaStream_t s, int src, int tmp, int dst, float coef, int store_tmp,
                        int check_act, int sum_slot, const LaunchCfg &lc);
void launch_diffuse_box(const DevGrid &g, cudaStream_t s, int src, int tmp, int dst, float coef,
                        int store_tmp, int check_act, int sum_slot, const LaunchCfg &lc);
void launch_sum(const DevGrid &g, cudaStream_t s, int src, int sum_slot, const LaunchCfg &lc);
int stencil_persistent_ctas(int num_sms, int which);

// ---- TMA-staged fused step (sg_sweep_tma.cu), 8^3 leaves ----
// Task descriptors of the j-run tasks (after launch_region_masks with the
// j-run records); then the fused diffuse7 -> box27 (+ sum) step, t never
// stored and no activation checks.  Returns 0, or nonzero if the tensor maps
// or the launch attributes could not be set up (nothing launched).
void launch_tma_tasks(const DevGrid &g, cudaStream_t s, const LaunchCfg &lc);
int launch_sweep_tma(const DevGrid &g, cudaStream_t s, int src, int dst, float coef, int sum_slot, const LaunchCfg &lc);

// ---- batched fused step over many grids (sg_sweep.cu) ----
constexpr int kMaxBatch = 1024;
struct BatchGrid {
    DevGrid g;
    const float *x;  // diffuse7 input
    float *y;        // box27 output
    float *t;        // intermediate (not stored by the batched kernel)
    int n;           // list length
    int c3, c2, c1;  // j-run pieces of three, two and one leaves (records in g.col_grp)
    int tasks;       // warp tasks of this grid (see k_sweep_jruns)
    int tri0;        // first global task index of this grid
    const void *tma_maps;  // staged body: 8 tensor maps (1 KB, device memory) over x, else null
};
// One launch: every grid's fused diffuse7 -> box27 step, per-grid sums
// added to acc[grid] (acc zeroed by the caller).  warps = warps per CTA.
void launch_batch_diffuse_box(const BatchGrid *items, int n_grids, int total_tri, float coef, double *acc, int warps,
                              int num_sms, cudaStream_t s);
int batch_ctas(int num_sms, int warps);
// The same step with the staged (TMA) body of sg_sweep_tma.cu: needs every
// grid's TMA task descriptors (launch_tma_tasks) and tma_maps.  Returns
// nonzero if the launch attributes could not be set (nothing launched).
int launch_batch_tma(const BatchGrid *items, int n_grids, int total_tri, float coef, double *acc, int num_sms,
                     cudaStream_t s);
constexpr int kTmaMapsBytes = 1024;  // 8 tensor maps of 128 bytes
// Encode the staged kernel's 8 tensor maps over a field of (cap + 1) 8^3
// leaves into host memory (kTmaMapsBytes, 64-byte aligned).  False if the
// driver's encoder is unavailable or refuses.
bool tma_encode_maps(const float *field, long long cap, void *out);

// ---- active-voxel count of the listed leaves into ctrl->n_active ----
void launch_count_active(const DevGrid &g, cudaStream_t s, const LaunchCfg &lc);

// ---- host helpers shared by the batch and the server (sg_api.cu) ----
// Flush the grid, make its list, neighbour table and region masks current,
// count its active voxels, synchronize, and fill the descriptors of both
// src/dst parities (tri0 left 0).  Returns an SG_* code.
int grid_prepare_batch(sg_grid *g, int src, int tmp, int dst, BatchGrid out[2], long long *n_active);
// The same in two halves, for a caller that overlaps them with other work:
// _async queues everything on the grid's stream, ending with copies of the
// control block and the three run-record counts to the host (cnt: pinned);
// _finish, once the stream has passed them, checks the device error word and
// fills out[2] and *n_active.  Not for grids created with SG_CREATE_CHECK.
int grid_prepare_batch_async(sg_grid *g, int src, int tmp, int dst, int32_t *cnt);
int grid_prepare_batch_finish(sg_grid *g, int src, int tmp, int dst, const int32_t *cnt, BatchGrid out[2],
                              long long *n_active);
// sg_create, with the final wait for the grid's initialisation optional
// (init_sync false: it stays queued on the grid's stream, ahead of any later
// work there).
int grid_create(const sg_desc *desc, void *cuda_stream, sg_grid **out, bool init_sync);
int grid_num_sms(const sg_grid *g);

// ---- device-side fill with the counter-based generator (sg_structure.cu) ----
void launch_fill_hash(const DevGrid &g, cudaStream_t s, int f, unsigned long long seed, const LaunchCfg &lc);

// ---- register-sweep stencil kernels (sg_sweep.cu), 8^3 leaves ----
void launch_sweep_diffuse_box(const DevGrid &g, cudaStream_t s, int src, int tmp, int dst, float coef,
                              int store_tmp, int check_act, int sum_slot, const LaunchCfg &lc);
// op: 1 = diffuse7, 2 = box27
// (with lc.single_runs: the j-run form, k_sweep_single_jruns)
void launch_sweep_single(const DevGrid &g, cudaStream_t s, int op, int src, int dst, float coef, int check_act,
                         int sum_slot, const LaunchCfg &lc);

// ---- particle kernels (sg_particle.cu) ----
// Binned P2G (count, allocate, scan, order, accumulate per bin); returns the
// number of kernels launched.  Needs bin_count/bin_off (p2g_num_keys each),
// tile_sum, perm and bin_list (R^3).  Keys: 8 reach classes per leaf plus one
// for particles whose stencil misses the domain.
constexpr long long p2g_num_keys(int R) { return 8LL * R * R * R + 1; }
// C: NULL for PIC, else the APIC matrices (n x 9 FP32, row-major).
// rebin: the particle order of the last binning of the same particles is
// valid in g.perm; the new order is built from it in g.perm_alt (fewer
// conflicting count atomics) and the two are swapped in g.
int launch_p2g_binned(DevGrid &g, cudaStream_t s, const float *x, const float *v, const float *C, long long n,
                      float pmass, int f_mass, int f_mom0, bool rebin, const LaunchCfg &lc);
void launch_grid_update(const DevGrid &g, cudaStream_t s, int f_mass, int f_mom0, float dt,
                        float gz, int bound, const LaunchCfg &lc);
// binned: use the bins of the last binned P2G over the same particles (the
// particle order, leaf list and key ranges) to stage each leaf's
// neighbourhood of node velocities in shared memory; otherwise input order.
// C: NULL for PIC, else APIC, the matrices written there (n x 9 FP32).
// The particle arrays (x, v: n x 3 FP32; C: n x 9 FP32; ids: n int64; any of
// the last two may be null) permuted into the order g.perm of the last
// binning, in place through tmp (n x 9 x 4 bytes), and g.perm reset to the
// identity.  Returns the number of kernels launched.
int launch_sort_particles(DevGrid &g, cudaStream_t s, float *x, float *v, float *C, int64_t *ids, long long n,
                          void *tmp, const LaunchCfg &lc);
void launch_g2p(const DevGrid &g, cudaStream_t s, float *x, float *v, float *C, long long n, float dt, int f_mom0,
                int binned, const LaunchCfg &lc);

// ---- MacCormack / RK3 advection (sg_advect.cu) ----
// mode 0: dst[c] = src[c] at the RK3 backtrace over h = dt * N;
// mode 1: backward advection of qhat[c] over -h fused with the correction
//         dst[c] = clamp(qhat + (src - q~) / 2), q~ stored to qtil[c] if >= 0;
// mode 2: the correction with q~ read from qtil[c].  C <= 3 channels.
// lo / hi (or null): per channel, arrays of (cap + 1) * L^3 floats.  Mode 0
// stores there the clamp bounds of each sample (min and max of the 8 values
// it reads); modes 1 and 2 read the bounds there instead of tracing the
// forward path (they must come from a mode-0 launch with the same q,
// velocity and h, nothing written to q or the velocity since).
// vel4: fields v0..v0+2 packed by launch_pack_velocity since they last
// changed, or null.
void launch_advect_group(const DevGrid &g, cudaStream_t s, int mode, int C, const int *dst, const int *src,
                         const int *qhat, const int *qtil, int v0, float h, float *const *lo, float *const *hi,
                         const float4 *vel4, const LaunchCfg &lc);
// vel4 ((cap + 1) * L^3 float4): the listed leaves' velocity (fields v0..v0+2)
void launch_pack_velocity(const DevGrid &g, cudaStream_t s, int v0, float4 *vel4, const LaunchCfg &lc);
void launch_activate_tube(const DevGrid &g, cudaStream_t s, long long lo2, long long hi2, uint32_t fill_mask);

// ---- fused element-wise struct-fors (sg_elementwise.cu) ----
constexpr int kMaxEwOps = 16;   // ops (and at most one reduction) per fused launch
constexpr int kMaxEwSlots = 8;  // distinct fields per fused launch
// r[dst] = alpha r[a] + beta r[b] + gamma r[a] r[b] + delta on the active
// voxels (0 elsewhere); a, b = -1: absent (0).  dst = -1: add the active
// values of r[a] to the launch's reduction.  `kind` names the terms present
// (set by the host with ew_kind), so the kernel evaluates only those.
enum EwKind : int8_t {
    kEwGeneral = 0,  // gamma a b + alpha a + beta b + delta
    kEwFill = 1,     // delta                      (a, b absent)
    kEwAx = 2,       // alpha a + delta            (b absent)
    kEwAxby = 3,     // alpha a + beta b + delta   (gamma = 0)
    kEwSum = 4,      // reduction of r[a]
};
struct EwOp {
    int8_t dst, a, b, kind;
    float alpha, beta, gamma, delta;
};
// Normalise an op and set its kind: an op reading only b is rewritten to read
// a; kinds follow from the absent operands and gamma == 0.
inline void ew_kind(EwOp &o)
{
    if (o.dst < 0) {
        o.kind = kEwSum;
        return;
    }
    if (o.a < 0 && o.b >= 0) {
        o.a = o.b;
        o.alpha = o.beta;
        o.b = -1;
        o.beta = 0.f;
    }
    if (o.a < 0) o.kind = kEwFill;
    else if (o.b < 0) o.kind = kEwAx;
    else if (o.gamma == 0.f) o.kind = kEwAxby;
    else o.kind = kEwGeneral;
}
struct EwProgram {
    int n_ops, n_slots;
    int field[kMaxEwSlots];      // physical field of each slot
    uint8_t load[kMaxEwSlots];   // read before written: load it
    uint8_t store[kMaxEwSlots];  // final value live: store it
    EwOp op[kMaxEwOps + 1];
    int sum_out;                 // result index of the reduction, -1 none
    float *fp[kMaxEwSlots];      // field[field[k]], filled in by launch_ew
};
void launch_ew(const DevGrid &g, cudaStream_t s, const EwProgram &prog, const LaunchCfg &lc);

// ---- restriction / prolongation to a half-edge grid (sg_multigrid.cu) ----
void launch_restrict_mark(const DevGrid &fine, const DevGrid &coarse, cudaStream_t s, const LaunchCfg &lc);
// activate: set the coarse bits (the coarse leaves are allocated); else the
// activation is demoted (bits known to be set).
void launch_restrict(const DevGrid &fine, const DevGrid &coarse, cudaStream_t s, int f_src, int f_dst, float w,
                     bool activate, const LaunchCfg &lc);
void launch_prolong(const DevGrid &coarse, const DevGrid &fine, cudaStream_t s, int f_src, int f_dst, float w,
                    const LaunchCfg &lc);

// ---- fused G2P2G (sg_g2p2g.cu) ----
// APIC G2P from src (velocities f_vel0..+2) then APIC P2G with activation
// into dst (f_mass, f_mom0..+2), C kept on chip; the particles visited in the
// order and bins of the last binned P2G held by `bins` (src or dst).
void launch_g2p2g(const DevGrid &src, const DevGrid &dst, const DevGrid &bins, cudaStream_t s, float *x, float *v,
                  long long n, float dt, int f_vel0, float pmass, int f_mass, int f_mom0, const LaunchCfg &lc);

}  // namespace sg
