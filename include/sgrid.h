/*
 * sgrid.h -- C ABI of libsgrid, a GB300 (sm_103a) library for time steps on a
 * two-level spatially sparse grid: a pointer root over bitmasked leaf blocks.
 *
 * The operations follow the problem statement of AsyncTaichi (Hu et al.,
 * "AsyncTaichi: On-the-fly Inter-kernel Optimizations for Imperative and
 * Spatially Sparse Programming", 2021):
 *   - the data structure is Sec. 3.1 / Fig. 3 (pointer cells are active iff
 *     non-null, bitmasked cells iff their bit is set; Sec. 4 "States");
 *   - an inactive voxel reads as 0 (Sec. 4 "States", Fig. 5 caption);
 *   - writing activates and zero-fills (Sec. 3.2 item 3, Fig. 4);
 *   - struct-for loops run over a generated list of active leaves
 *     (Sec. 3.2 item 2);
 *   - calls are queued and launched lazily: flush is explicit and
 *     non-blocking, and every device-to-host transfer flushes implicitly
 *     (Sec. 5, Sec. 7.1);
 *   - on flush the queue goes through list-generation removal (Sec. 6.2),
 *     activation demotion (Sec. 6.3), task fusion (Sec. 6.4, Supplement
 *     Sec. 2) and dead-store elimination (Sec. 6.5), each of which can be
 *     switched off with sg_set_opts; all four off is the eager form that
 *     regenerates the list and checks activation in every kernel.
 *
 * Conventions shared by every call:
 *   - Return value: SG_OK (0) or one of the SG_ERR_* codes below; no C++
 *     exception crosses this boundary.  sg_last_error() gives a message for
 *     the last failing call on the calling thread.
 *   - Domain: N^3 voxels, N = res, leaves of edge L = 2^leaf_log2, root edge
 *     R = N / L.  Root index b = (bi*R + bj)*R + bk; local voxel index
 *     l = (li*L + lj)*L + lk (k fastest); mask bit l is bit (l % 32) of 32-bit
 *     word l / 32 of the leaf's mask.
 *   - Fields are FP32 scalar channels identified by an index 0..n_fields-1;
 *     sg_swap exchanges the storage behind two indices.
 *   - List order (used by every read and write of per-leaf data) is
 *     ascending root index b.
 *   - Device pointers passed to queued calls are BORROWED: they must stay
 *     valid, and their contents unchanged by the caller, until the next
 *     sg_sync (or any call documented as an implicit sync) returns.
 *   - All device work of a grid runs in order on the CUDA stream given to
 *     sg_create.  A grid must not be used from two threads at once.
 *   - Device-side errors (pool exhausted, a bounded wait that gave up) are
 *     latched in the grid and returned by the next sg_sync or implicit sync.
 */
#ifndef SGRID_H
#define SGRID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SG_OK 0
#define SG_ERR_INVALID 1         /* bad argument or call order */
#define SG_ERR_OOM 2             /* device memory could not be allocated */
#define SG_ERR_POOL_EXHAUSTED 3  /* an activation needed more than max_leaves leaves */
#define SG_ERR_TIMEOUT 4         /* a bounded device-side wait gave up */
#define SG_ERR_CUDA 5            /* a CUDA runtime call failed */
#define SG_ERR_CHECK 6           /* an invariant check of a checking grid failed (sg_check) */

/* ---- optimizer passes (sg_set_opts); all four on is the default ---- */
#define SG_OPT_LGR 1u  /* list-generation removal, Sec. 6.2 */
#define SG_OPT_AD 2u   /* activation demotion, Sec. 6.3 */
#define SG_OPT_FUSE 4u /* task fusion, Sec. 6.4 (needs SG_OPT_LGR) */
#define SG_OPT_DSE 8u  /* dead-store elimination, Sec. 6.5 */
#define SG_OPT_ALL 15u
#define SG_OPT_EAGER 0u

/* ---- stencil operations (sg_launch_stencil) ---- */
#define SG_CLEAR 0    /* dst = 0 on active voxels */
#define SG_DIFFUSE7 1 /* dst = src + coef*(sum of 6 face neighbours - 6 src) */
#define SG_BOX27 2    /* dst = (1/27) * sum over the 3x3x3 neighbourhood of src */

/* ---- sg_desc.flags ---- */
#define SG_CREATE_DRY_RUN 1u /* no device memory and no launches: the queue and
                                optimizer run and sg_stats counts what would
                                have been launched (host-logic testing) */
#define SG_CREATE_CHECK 2u   /* checking grid: every sync also runs sg_check's
                                invariant checks (the list-dependent ones when
                                the list is current) and a violation is
                                returned as SG_ERR_CHECK.  A debugging mode:
                                each sync costs a few extra kernels */

#define SG_MAX_FIELDS 16

/* Device memory provider.  alloc returns a device pointer of at least `bytes`
 * bytes aligned to 256 bytes, or NULL; free releases it.  When both are NULL
 * the library uses cudaMalloc / cudaFree. */
typedef void *(*sg_alloc_fn)(size_t bytes, void *ctx);
typedef void (*sg_free_fn)(void *ptr, void *ctx);

typedef struct sg_desc {
    int32_t res;           /* N: virtual domain edge, a multiple of L, <= 4096 */
    int32_t leaf_log2;     /* 2 (4^3 leaves) or 3 (8^3 leaves) */
    int32_t n_fields;      /* FP32 scalar fields, 1..SG_MAX_FIELDS */
    int32_t max_sums;      /* FP64 reduction result slots (>= 0) */
    int64_t max_leaves;    /* leaf pool capacity, >= 1 */
    uint32_t scratch_mask; /* bit f set: field f is scratch -- its contents are
                              undefined once the flush that wrote it ends, which
                              licenses dead-store elimination of its stores */
    uint32_t flags;        /* SG_CREATE_* */
    sg_alloc_fn alloc;     /* optional device memory provider */
    sg_free_fn free;
    void *alloc_ctx;
} sg_desc;

typedef struct sg_stats {
    int64_t launches;        /* device kernels launched (copies not counted) */
    int64_t listgen_run;     /* list-generation kernels launched */
    int64_t listgen_removed; /* list generations removed on the host (Sec. 6.2) */
    int64_t act_launched;    /* activation kernels launched */
    int64_t act_demoted;     /* activations demoted away (Sec. 6.3) */
    int64_t ops_enqueued;    /* calls queued */
    int64_t ops_fused;       /* queued ops that ran inside another op's kernel */
    int64_t stores_removed;  /* dead stores removed (Sec. 6.5) */
    int64_t flushes;
    double bytes_model;      /* algorithmic HBM bytes of the launched stencil,
                                clear and reduction kernels (whole leaves) */
    int64_t bounds_reused;   /* MacCormack corrections (per channel) that read the
                                clamp bounds their forward advection stored */
    int64_t velocity_packs;  /* advection runs whose velocity was packed once
                                for all their launches (one launch each) */
} sg_stats;

typedef struct sg_grid sg_grid; /* opaque; owned by the library */

/* Create a grid whose device work runs on `cuda_stream` (a cudaStream_t; NULL
 * is the legacy default stream).  All leaves are inactive.  On success *out
 * receives the grid.  Errors: SG_ERR_INVALID (bad desc), SG_ERR_OOM.
 * Passage: Sec. 3.2 and Fig. 3 (a pointer array over dense blocks, every
 * pointer null while inactive; here the blocks carry a bitmask, the
 * pointer-over-bitmasked-leaf layout of the benchmarks) and Sec. 4 "States"
 * (the value, mask, list and allocator states the grid holds; the allocator
 * state is the leaf pool of max_leaves). */
int sg_create(const sg_desc *desc, void *cuda_stream, sg_grid **out);

/* Synchronize the grid's stream, then release the grid and its memory.
 * Passage: Sec. 4 "States" (it ends the grid's states, the allocator state
 * included; the paper releases them with the program and prints no call). */
int sg_destroy(sg_grid *g);

/* Select optimizer passes (SG_OPT_* bits) for ops flushed from now on.
 * Passage: Sec. 6.2-6.5 (the four passes) and Sec. 8 Table 3 (the per-pass
 * ablation, which turns each pass off in turn). */
int sg_set_opts(sg_grid *g, uint32_t opts);

/* Queue: activate every voxel with lo2 <= D < hi2 (lo2 < D when lo_strict),
 * D = sum_a (2 i_a + 1 - N)^2 = 4 * (distance from the voxel centre to the
 * domain centre)^2.  Newly allocated leaves are zero-filled (Sec. 3.2).
 * With SG_OPT_AD, a call identical to one already applied since the last
 * sg_deactivate_all activates nothing new and is demoted (Sec. 6.3). */
int sg_activate_shell(sg_grid *g, int64_t lo2, int64_t hi2, int32_t lo_strict);

/* Queue: activate n voxels given as int32 (i,j,k) triples in device memory
 * (borrowed).  Triples outside the domain are ignored.  Passage: Sec. 3.2
 * item 3 and Fig. 4 (activation on write: a missing leaf is allocated and
 * zero-filled, the voxel's bit set), modifying the mask and allocator states
 * of Sec. 4. */
int sg_activate_coords(sg_grid *g, const int32_t *dev_xyz, int64_t n);

/* Queue: deactivate every voxel and return every leaf to the pool.
 * Passage: Sec. 4 "States" (a task that clears the mask and allocator
 * states); the MLS-MPM case of Sec. 8.3 starts each substep's grid empty. */
int sg_deactivate_all(sg_grid *g);

/* Queue: (re)generate the active-leaf list and its 27-neighbour table.  With
 * SG_OPT_LGR it is removed when the structure is known unchanged (Sec. 6.2),
 * and skipped on the device when no activation since the last list changed
 * anything. */
int sg_list_gen(sg_grid *g);

/* Queue a struct-for over the active voxels: op is SG_CLEAR (src ignored),
 * SG_DIFFUSE7 (coef used) or SG_BOX27.  src != dst.  Reads of inactive or
 * out-of-domain voxels give 0; dst at inactive voxels stays 0.  Passage:
 * Sec. 3.2 item 1 (sparse struct-for loops over the active voxels, fed by the
 * list of item 2) and Sec. 4 "States" with Fig. 5 (an inactive voxel reads as
 * its ambient value 0); the stencils are the microbenchmark kind of Supp.
 * Sec. 1 (stencil_reduction). */
int sg_launch_stencil(sg_grid *g, int32_t op, int32_t src, int32_t dst, float coef);

/* Queue activation of a tube along the k axis: every voxel with
 * lo2 <= (2i+1-N)^2 + (2j+1-N)^2 < hi2 (4 N^2 times the squared distance of
 * its cell centre from the axis through the domain centre), at every k (the
 * advection domain of Sec. 8.2 / Supp. Sec. 4.2).  Activation demotion as for
 * sg_activate_shell. */
int sg_activate_tube(sg_grid *g, int64_t lo2, int64_t hi2);

/* Queue semi-Lagrangian advection (Sec. 8.2): on every active voxel, dst =
 * src sampled at the cell centre's backtrace over dt (negative: backward)
 * through the velocity fields v0, v0+1, v0+2 (domain units per time; three
 * consecutive unswapped fields).  Collocated cells, Ralston's RK3 for the
 * backtrace, trilinear samples read through the mask (inactive or
 * out-of-domain cells read 0); dst keeps 0 at inactive voxels.  dst must
 * differ from src and the velocity fields. */
int sg_advect(sg_grid *g, int32_t dst, int32_t src, int32_t v0, float dt);

/* Queue the MacCormack correction (Selle et al., as used in Sec. 8.2): on
 * every active voxel dst = qhat + (q - qtilde) / 2, clamped to the min / max
 * of the 8 values of q that the forward sample (the backtrace over dt)
 * interpolates; dst keeps 0 at inactive voxels and differs from every input.
 * With SG_OPT_FUSE (and SG_OPT_LGR) the queue schedules a run of advection
 * ops by their field dependencies: independent advections with the same
 * velocity and step are one launch of up to three channels sharing the
 * backtrace, and a backward advection whose output a correction reads is
 * fused with it (that output, if scratch and read later by nothing, is not
 * stored) -- the channel fusion of Sec. 8.2.  A forward advection of q with
 * the same velocity and step in the same run, when no op of the run writes q
 * or the velocity, also stores the clamp bounds, and the correction reads them
 * instead of tracing the forward path again (identical results;
 * sg_stats.bounds_reused counts it).  When two or more advections of such a
 * run share a velocity that no op of the run writes, its three fields are
 * first packed into one 16-byte value per voxel (one extra launch, counted in
 * sg_stats.velocity_packs; identical results), so each velocity corner of a
 * backtrace is one load. */
int sg_maccormack(sg_grid *g, int32_t dst, int32_t q, int32_t qhat, int32_t qtilde, int32_t v0, float dt);

/* Queue an element-wise struct-for: on every active voxel
 *   dst = alpha * a + beta * b + gamma * a * b + delta,
 * a and b read at the same voxel (field index -1: absent, reads 0); dst
 * keeps 0 at inactive voxels; dst may equal a or b.  It covers the general
 * kernels of the paper's microbenchmarks (copies, increments, fills, saxpy,
 * products; Supp. Sec. 1).  With SG_OPT_FUSE (and SG_OPT_LGR) a run of
 * consecutive element-wise ops, with at most one reduction among them, is one
 * launch (Sec. 6.4; at most sg_set_max_fuse ops, default 16, and 8 distinct
 * fields); with SG_OPT_DSE a scratch field written in the run and read by no
 * later queued op is not stored (Sec. 6.5). */
int sg_launch_ew(sg_grid *g, int32_t dst, int32_t a, int32_t b, float alpha, float beta, float gamma,
                 float delta);

/* Flush the queue automatically once it holds `ops` queued ops (the flush
 * period of the paper's asynchronous engine, Sec. 7.1; 1 issues every op as
 * it is queued, as a synchronous engine would; 0, the default, flushes only on
 * sg_flush and on implicit syncs).  Optimizations apply within a flush. */
int sg_set_flush_period(sg_grid *g, int32_t ops);

/* Largest number of element-wise ops fused into one launch (>= 1; the
 * role of the paper's async_max_fuse_per_task, Supp. Sec. 2 item 4). */
int sg_set_max_fuse(sg_grid *g, int32_t max_ops);

/* Queue: sum of field src over the active voxels into result slot out_slot
 * (FP64; per-leaf partials are FP32).  Read with sg_read_sums.  The reduction
 * of the paper's stencil-and-reduce microbenchmark (Supp. Sec. 1); with task
 * fusion (Sec. 6.4) it runs inside the stencil kernel that writes src. */
int sg_reduce_sum(sg_grid *g, int32_t src, int64_t out_slot);
/* (With SG_OPT_DSE, a reduction whose result slot a later queued reduction
 * overwrites within the same flush is not run: nothing reads it.) */

/* Queue P2G with activation: for each of n particles (positions dev_x and
 * velocities dev_v, n*3 FP32 in (x,y,z) order, device memory, borrowed) and
 * each of its 27 quadratic B-spline stencil nodes inside the domain (unit
 * cube, dx = 1/N): activate the node, add w*pmass to field f_mass and
 * w*pmass*v to fields f_mom0, f_mom0+1, f_mom0+2 (Sec. 8.3 workload).
 * Accumulation order is unspecified (FP32 atomics). */
int sg_p2g(sg_grid *g, const float *dev_x, const float *dev_v, int64_t n,
           float pmass, int32_t f_mass, int32_t f_mom0);

/* Queue the grid update on active nodes: where mass > 0, v = momentum/mass,
 * v_z -= dt*gz, and along each axis a node with index < bound loses a negative
 * component and one with index > N - bound a positive one; massless nodes get
 * v = 0.  v replaces the momentum in f_mom0..f_mom0+2.  Passage: Sec. 8.3
 * and Supp. Sec. 4.3 (the MLS-MPM grid operation between P2G and G2P:
 * gravity 9.8, the ground along z). */
int sg_grid_update(sg_grid *g, int32_t f_mass, int32_t f_mom0, float dt,
                   float gz, int32_t bound);

/* Queue G2P: v_p = sum of w * v over the 27 stencil nodes (fields
 * f_mom0..f_mom0+2), then x_p += dt * v_p; dev_x and dev_v (n*3 FP32, device,
 * borrowed) are overwritten.  Passage: Sec. 8.3 (the G2P task of MLS-MPM,
 * Fig. 12), with the quadratic B-spline weights of the MLS-MPM method it
 * cites. */
int sg_g2p(sg_grid *g, float *dev_x, float *dev_v, int64_t n, float dt, int32_t f_mom0);

/* Queue APIC P2G with activation (the affine transfer of MLS-MPM, Sec. 8.3):
 * as sg_p2g, with the momentum contribution of particle p to stencil node n
 *   w * pmass * (v_p + C_p (x_n - x_p)),
 * where dev_C holds one 3x3 matrix per particle, n*9 FP32 row-major
 * ((C d)_a = sum_b C[9p + 3a + b] d_b), device memory, borrowed until the
 * next sync.  dev_C == NULL is the PIC transfer of sg_p2g. */
int sg_p2g_apic(sg_grid *g, const float *dev_x, const float *dev_v, const float *dev_C, int64_t n,
                float pmass, int32_t f_mass, int32_t f_mom0);

/* Queue APIC G2P: as sg_g2p, and C_p = (4/dx^2) sum_n w v_n (x_n - x_p)^T
 * (quadratic B-splines: sum_n w d d^T = dx^2/4 I) is written to dev_C (n*9
 * FP32 row-major, device, borrowed).  dev_C == NULL is sg_g2p. */
int sg_g2p_apic(sg_grid *g, float *dev_x, float *dev_v, float *dev_C, int64_t n, float dt, int32_t f_mom0);

/* Fused G2P2G (Sec. 8.3): the APIC G2P of one step and the APIC P2G of the
 * next in one pass over the particles, the affine matrix C held on chip and
 * never stored (Sec. 6.5, dead-store elimination).  The result is that of
 *   sg_g2p_apic(src, dev_x, dev_v, C, n, dt, f_vel0);
 *   sg_p2g_apic(dst, dev_x, dev_v, C, n, pmass, f_mass, f_mom0);
 * for some C that is then discarded: velocities are read from src fields
 * f_vel0..f_vel0+2 (after its grid update), x and v are overwritten, and
 * dst's stencil nodes of the new positions are activated (its leaves are
 * allocated inside the kernel) and receive mass and affine momentum.  src and
 * dst are distinct grids with the same res and leaf size created on the same
 * stream; a binned P2G over the same dev_x and n must have run on src or dst
 * (its particle order and bins are reused; particles that have since left
 * their bin's neighbourhood take slower exact paths).  Flushes src, then
 * queues and flushes the op on dst; dev_x, dev_v borrowed until the next sync
 * of dst.  Errors: SG_ERR_INVALID (arguments, no bins), pool exhaustion and
 * timeouts latched on dst. */
int sg_g2p2g(sg_grid *src, sg_grid *dst, float *dev_x, float *dev_v, int64_t n, float dt, int32_t f_vel0,
             float pmass, int32_t f_mass, int32_t f_mom0);

/* Queue a reordering of the particle arrays into the order of the last binned
 * P2G of the same particles on g (dev_x and n as given to that sg_p2g or
 * sg_p2g_apic, which must still be current: no other binning of other arrays
 * since).  dev_x and dev_v (n*3 FP32), dev_C (n*9 FP32, APIC) and dev_ids (n
 * int64, e.g. the caller's particle numbers) are each permuted in place by
 * the same permutation -- dev_C and dev_ids may be NULL -- and the binning's
 * order becomes the identity, so the bins stay valid for sg_g2p, sg_g2p_apic
 * and sg_g2p2g.  Afterwards the particles of a leaf, and within it of a cell,
 * are adjacent in memory: the next binnings, the P2G gather and G2P read and
 * write them in order instead of one scattered 12-byte access each.  The
 * particle order a caller sees changes; dev_ids says which particle is where.
 * An addition of this library (the paper keeps particles in their own order);
 * particles move little per step, so calling it every few steps keeps them
 * ordered.  One gather kernel per array plus one reset, and a device copy per
 * array (scratch: 36 bytes per particle, allocated at first use).  Arrays
 * borrowed until the next sync.  Errors: SG_ERR_INVALID (bad arguments; at
 * the flush, no current binning of these particles), SG_ERR_OOM. */
int sg_sort_particles(sg_grid *g, float *dev_x, float *dev_v, float *dev_C, int64_t *dev_ids, int64_t n);

/* Restriction onto a grid of half the edge (the multigrid pattern of Sec. 6.3,
 * Fig. 13): for every active voxel i of `fine`, activate voxel i // 2
 * (componentwise) of `coarse` and add w * fine[f_src][i] to coarse[f_dst]
 * there.  fine and coarse are distinct grids with fine res = 2 * coarse res,
 * the same leaf size, created on the same stream.  Both grids' queued work is
 * flushed first (a scratch field's contents are undefined after a flush), the
 * fine list is made current, and the restriction is launched at once on the
 * stream.  With SG_OPT_AD on `coarse`, a restriction from the same fine grid
 * whose mask has not changed since one already applied (and no deactivation
 * of coarse since) is demoted: it adds values without activating, and
 * coarse's structure stays unchanged, so its list generation can be removed
 * (Sec. 6.3).  Errors: SG_ERR_INVALID; pool exhaustion latched on coarse. */
int sg_restrict(sg_grid *fine, sg_grid *coarse, int32_t f_src, int32_t f_dst, float w);

/* Prolongation: for every active voxel i of `fine`, fine[f_dst][i] +=
 * w * coarse[f_src][i // 2], reading coarse through its mask (an inactive or
 * absent coarse voxel reads 0).  No activation.  Same grid requirements and
 * flushing as sg_restrict; launched at once on the stream. */
int sg_prolong(sg_grid *coarse, sg_grid *fine, int32_t f_src, int32_t f_dst, float w);

/* Exchange the storage behind field indices a and b (no device work).
 * Passage: Sec. 8.3 (two grids swapped before each substep); the same
 * ping-pong of value states serves the stencil steps. */
int sg_swap(sg_grid *g, int32_t a, int32_t b);

/* Optimize and launch every queued op; does not wait.  Passage: Sec. 7.1
 * "Flushing" (an explicit, non-blocking flush of the task queue through the
 * optimizer to the device) and Sec. 5 (lazy kernel launches). */
int sg_flush(sg_grid *g);

/* Flush, wait for the stream, and return the first latched device error.
 * Passage: Sec. 7.1 (an implicit synchronization event flushes the queue;
 * the evaluation synchronizes after each run, Sec. 8). */
int sg_sync(sg_grid *g);

/* Implicit sync, then the number of leaves in the (current) list. */
int sg_num_leaves(sg_grid *g, int64_t *n_leaves);

/* Implicit sync, then copy the list state to host memory: leaf_b gets the
 * root index of each leaf in ascending order, masks gets L^3/32 uint32 words
 * per leaf (either may be NULL).  cap is the number of leaves the buffers
 * hold; if the list is longer, nothing is copied, *n_leaves is set and
 * SG_ERR_INVALID is returned.  Passage: Sec. 4 "States" (the list and mask
 * states) and Sec. 7.1 (a device-to-host transfer is an implicit
 * synchronization event). */
int sg_read_structure(sg_grid *g, int64_t cap, int64_t *n_leaves, int32_t *leaf_b,
                      uint32_t *masks);

/* Implicit sync, then copy field f to host memory in list order, L^3 values
 * per leaf, 0 at inactive voxels.  cap = leaves the buffer holds.  A
 * page-locked buffer mapped into the device's address space (16-byte
 * aligned) is written in place by the gather kernel; any other buffer gets a
 * staged copy.  Passage: Sec. 4 "States" and Fig. 5 (the value state, an
 * inactive voxel reading 0) and Sec. 7.1 (the read is an implicit
 * synchronization event). */
int sg_read_field(sg_grid *g, int32_t f, int64_t cap, float *host_vals);

/* Set field f from host memory in list order (n_leaves * L^3 FP32 values;
 * n_leaves must equal the current list length).  Values at inactive voxels
 * are ignored (stored as 0).  The copy is made before the call returns, so
 * the host buffer may be reused at once.  A page-locked buffer mapped into
 * the device's address space (16-byte aligned) is read in place by the
 * scatter kernel, one pass over the host link; any other buffer is first
 * copied to a device staging buffer. */
int sg_write_field(sg_grid *g, int32_t f, const float *host_vals, int64_t n_leaves);

/* Active-voxel ("packed") transfers of field f: only the values at active
 * voxels, in list order and, within a leaf, ascending local index l -- the
 * order of the set mask bits.  Implicit syncs.  A page-locked buffer mapped
 * into the device's address space (16-byte aligned) is read or written in
 * place by the transfer kernel; any other buffer is staged.
 *
 * write: n_active must equal the grid's active voxel count (else
 * SG_ERR_INVALID, nothing written); every inactive voxel of the listed
 * leaves is set to 0.  The host buffer may be reused when the call returns.
 * read: *n_active receives the count; if it exceeds cap nothing is copied
 * and SG_ERR_INVALID is returned. */
int sg_write_field_active(sg_grid *g, int32_t f, const float *host_vals, int64_t n_active);
int sg_read_field_active(sg_grid *g, int32_t f, int64_t cap, int64_t *n_active, float *host_vals);

/* Staged (overlapped) active-voxel uploads.  sg_stage_active starts copying
 * n_active packed values from host memory into one of the grid's two upload
 * slots, on a copy stream of the grid's own, and returns a ticket; the copy
 * runs while device work already queued runs.  host_vals (page-locked, or the
 * call waits for the copy) is borrowed until the next upload into the same
 * slot has been staged (that call waits for the earlier copy) or the grid has
 * been synced after the ticket's write.  A slot is refilled only after the
 * write that read it has run, so two uploads can be in flight.  sg_write_field_staged queues: field f = the staged
 * values (as sg_write_field_active); at flush the grid's stream waits for the
 * copy.  The count must equal the grid's active voxels when the write runs
 * (else SG_ERR_INVALID at flush, the field unchanged).  When the structure
 * changed since the packed offsets were last computed, the flush waits for
 * the device once to compute them.  A staged write cannot be recorded in a
 * graph (sg_graph_begin).  Errors: SG_ERR_INVALID (arguments, a
 * ticket replaced by a later upload into its slot), SG_ERR_OOM. */
int sg_stage_active(sg_grid *g, const float *host_vals, int64_t n_active, int32_t *ticket);
int sg_write_field_staged(sg_grid *g, int32_t f, int32_t ticket);

/* ---- CUDA graphs of steady-state steps ----
 * Record the device work that flushes of grids on `cuda_stream` issue
 * between sg_graph_begin and sg_graph_end into a graph, and replay it with
 * sg_graph_launch (on the same stream, in stream order).  Only queued calls
 * and sg_flush may be made while recording: a call that waits for the device
 * (sg_sync, reads, implicit syncs) ends the recording with an error, and so
 * does a change of a grid's structure or a list generation (activation,
 * deactivation, particle transfers, an activating restriction), since the
 * host-side list and demotion state would not follow a replay.  Record after
 * a warm-up step, so the structure and lists are current and every scratch
 * buffer exists.  Host state (sg_stats, versions) counts the recorded step
 * once; replays run the same kernels on the same fields: sg_swap is resolved
 * when a call is queued, so a step that swaps fields needs one graph per
 * parity.  After a failed recording the grids' contents are undefined.
 * Errors: SG_ERR_INVALID (null stream, failed recording), SG_ERR_CUDA. */
typedef struct sg_graph sg_graph;
int sg_graph_begin(void *cuda_stream);
int sg_graph_end(void *cuda_stream, sg_graph **out);
int sg_graph_launch(sg_graph *graph);
int sg_graph_destroy(sg_graph *graph);

/* Replace the whole structure with a saved one (the restore half of a
 * checkpoint whose save half is sg_read_structure + sg_read_field): leaf_b
 * holds n_leaves root indices in strictly ascending order, each in [0, R^3),
 * and masks holds L^3/32 uint32 words per leaf, in the layout
 * sg_read_structure writes (the voxel bit of local index (li*L + lj)*L + lk,
 * Sec. 3).  Implicit sync: queued work runs first and its latched error, if
 * any, is returned without changing the structure.  Every field of the
 * restored leaves is zero afterwards (write them with sg_write_field); the
 * list is current and in leaf_b's order; reduction slots are untouched.
 * Both host buffers are copied before the call returns.  Errors:
 * SG_ERR_INVALID (null buffers with n_leaves > 0, order or range of leaf_b,
 * a dry-run grid), SG_ERR_POOL_EXHAUSTED (n_leaves > max_leaves; nothing is
 * changed). */
int sg_write_structure(sg_grid *g, int64_t n_leaves, const int32_t *leaf_b, const uint32_t *masks);

/* Implicit sync, then copy result slots [0, n) to host memory.  Passage:
 * Sec. 7.1 (a device-to-host transfer flushes the queue and synchronizes);
 * the slots hold reductions such as those of the stencil_reduction
 * microbenchmark (Supp. Sec. 1). */
int sg_read_sums(sg_grid *g, double *host, int64_t n);

/* Counters since creation.  Passage: Sec. 8 "Metrics" (tasks launched is
 * the paper's third metric; list generations and demoted activations are the
 * counts behind Sec. 8.4's 420,912 -> 8,004 list generations). */
int sg_get_stats(sg_grid *g, sg_stats *out);

/* ---- stencil kernel family for 8^3 leaves (tuning; results are identical
 * up to FP32 rounding order; the four sweeps give bit-identical fields) ---- */
#define SG_VARIANT_SWEEP 0 /* register sweep along i, rows via the read-only path; a warp
                              takes three consecutive list entries */
#define SG_VARIANT_SMEM 1  /* leaf + halo staged in shared memory */
#define SG_VARIANT_SWEEP_COLUMNS 2 /* register sweep; the fused step sweeps columns of up
                                      to three leaves adjacent in i (same results; slower
                                      on the band: fewer, longer tasks) */
#define SG_VARIANT_SWEEP_JRUNS 3   /* the default: register sweep; the fused step gives each
                                      warp up to three leaves from runs adjacent in j, so rows
                                      at the leaves' shared faces are loaded once */
#define SG_VARIANT_SWEEP_TMA 4     /* the j-run tasks of SG_VARIANT_SWEEP_JRUNS with every x row
                                      of the fused step staged in shared memory by bulk tensor
                                      copies (two half-regions per warp in flight, completed
                                      on mbarriers); bit-identical fields to SG_VARIANT_SWEEP_JRUNS.
                                      Slower than it on the bands: a task needs 60 to 84 small
                                      copies and each costs about 70 SM cycles of copy-engine
                                      time.  Other stencil ops use the j-run kernels. */

/* Select the stencil kernel family used by ops flushed from now on (a new grid
 * uses SG_VARIANT_SWEEP_JRUNS). */
int sg_set_stencil_variant(sg_grid *g, int32_t variant);

/* Implicit sync, then the number of active voxels of the listed leaves. */
int sg_num_active(sg_grid *g, int64_t *n_active);

/* Queue: set field f at every active voxel (i,j,k) to the uniform [0,1)
 * value top24(splitmix64(seed * 2^40 + (i*N + j)*N + k)) * 2^-24 (the
 * splitmix64 output function of Steele, Lea & Flood 2014), and to 0 at
 * inactive voxels.  0 <= seed < 2^24.  Gives device-side initial values
 * identical to the ones a host generator with the same definition uploads. */
int sg_fill_hash(sg_grid *g, int32_t f, int64_t seed);

/* ---- batched stepping: many grids, one persistent launch per step ----
 *
 * (Small sparse problems are dominated by per-task launch overhead, Sec. 8.4;
 * the batch removes it across grids as task fusion does within one.)
 *
 * A batch binds n (1..1024) live grids with 8^3 leaves.  Each sg_batch_step
 * runs, for every grid, the fused step dst = box27(diffuse7(src, coef)) with
 * the per-grid sum of dst accumulated, as ONE kernel launch over the
 * concatenated work of all grids (a persistent kernel whose warps stride
 * over the grids' j-run pieces, as SG_VARIANT_SWEEP_JRUNS does for one
 * grid), then exchanges src and dst in every grid (as
 * sg_swap).  The intermediate field tmp is not stored (every grid's tmp is
 * treated as scratch).  Steps are captured as CUDA graphs (one per src/dst
 * parity) unless disabled.  Results equal stepping each grid alone up to
 * FP32 rounding order (the fused kernel body is the same).
 *
 * sg_batch_create flushes every grid, makes its list, neighbour table,
 * region masks and j-run records current, and synchronizes; the structure of the grids must
 * not change while the batch exists, and between batch steps the grids
 * must not be used except for reads (which synchronize).  All work runs on
 * cuda_stream.  Descriptor memory comes from grid 0's allocator and goes
 * back to it at sg_batch_destroy, so the grids must outlive the batch:
 * destroy the batch first. */
typedef struct sg_batch sg_batch;
int sg_batch_create(sg_grid *const *grids, int32_t n, int32_t src, int32_t tmp, int32_t dst, float coef,
                    void *cuda_stream, sg_batch **out);
/* Enqueue one batched step (no host wait). */
int sg_batch_step(sg_batch *b);
/* Wait, then copy the n first grids' sums of the last step to host memory. */
int sg_batch_read_sums(sg_batch *b, double *host, int32_t n);
/* Warps per CTA of the persistent kernel (2, 4 or 8: up to 6, 12 or 24 leaves
 * per CTA) and whether steps run as captured CUDA graphs. */
int sg_batch_set(sg_batch *b, int32_t warps_per_cta, int32_t use_graph);
/* Halo staging of the batched kernel: 0 (the default) the register sweep,
 * whose lanes read their x rows, halo included, from L2/HBM; 1 every task's
 * x region (leaves plus halo) staged in shared memory by bulk tensor copies
 * completed on mbarriers, eight warps per CTA, one CTA per SM (the body of
 * SG_VARIANT_SWEEP_TMA; warps_per_cta does not apply).  The first switch to 1
 * builds every grid's task descriptors and tensor maps and synchronizes.
 * Fields are bit-identical either way. */
int sg_batch_set_staging(sg_batch *b, int32_t staged);
/* The launch shape a step uses now (warps per CTA, halo staging). */
int sg_batch_config(sg_batch *b, int32_t *warps_per_cta, int32_t *staged);
/* Autotuner: time trial_steps steps with each (halo staging, warps per CTA)
 * choice -- the register sweep at 2, 4 and 8 warps per CTA and the staged
 * body -- (these are real steps: they advance every grid) and keep the
 * fastest; *chosen_warps gets its warps per CTA (sg_batch_config gives
 * both). */
int sg_batch_autotune(sg_batch *b, int32_t trial_steps, int32_t *chosen_warps);
int sg_batch_info(sg_batch *b, int64_t *total_leaves, int64_t *launches, int32_t *warps_per_cta);
int sg_batch_destroy(sg_batch *b);

/* ---- serving: a continuous-batching request loop ----
 *
 * Jobs are independent sparse diffusion runs: a shell/band activation
 * (res, lo2, hi2, lo_strict as in sg_activate_shell, 8^3 leaves), initial
 * field values from sg_fill_hash(seed), and `steps` fused steps
 * x <- box27(diffuse7(x, coef)) with the sum of x kept after each step.
 * sg_server_submit only queues a job.  Each sg_server_tick waits once, for
 * the device work the previous tick queued, then
 *   1. advances the jobs of the previous tick's step and retires those that
 *      reached their step count, keeping their last sum and their submit /
 *      admit / done times (seconds, host steady clock), and copying their
 *      final field to out_values when one is given;
 *   2. adds the jobs admitted by the previous tick to the resident set;
 *   3. launches one batched step (one persistent launch, see
 *      sg_batch_create) over every resident job, so jobs admitted while
 *      others run share it, and does not wait for it;
 *   4. while that step runs, admits pending jobs in submission order while a
 *      slot is free and cudaMemGetInfo's free memory covers the job's
 *      footprint plus hbm_reserve (a job that cannot fit even on an idle
 *      server fails): the job's grid is allocated and its creation,
 *      activation, list, fill and counts are queued behind the step on the
 *      server's stream; the job stays resident until it completes.
 * So an admitted job joins the next tick's step, and a job's last step
 * completes in one tick and is retired by the next.  sg_server_stats.resident
 * counts admitted jobs.  A job's result equals the same job run alone up to
 * FP32 rounding order. */
#define SG_JOB_PENDING 0
#define SG_JOB_RUNNING 1
#define SG_JOB_DONE 2
#define SG_JOB_FAILED 3

typedef struct sg_server sg_server;
typedef struct sg_server_desc {
    int32_t max_jobs;      /* resident job slots, 1..1024 */
    int32_t warps_per_cta; /* batched kernel: 2, 4 or 8 */
    int64_t hbm_reserve;   /* bytes of device memory to leave free when admitting */
    float coef;            /* diffusion coefficient of every job */
    sg_alloc_fn alloc;     /* device memory provider for job grids (NULL: cudaMalloc) */
    sg_free_fn free;
    void *alloc_ctx;
} sg_server_desc;
typedef struct sg_job_desc {
    int32_t res;      /* N, a multiple of 8 */
    int32_t lo_strict;
    int64_t lo2, hi2; /* band, as sg_activate_shell */
    int32_t steps;    /* >= 1 */
    int32_t pad;
    int64_t seed;     /* sg_fill_hash seed, 0 <= seed < 2^24 */
    float *out_values; /* optional (NULL: none): host buffer that receives the
                          job's final x at its active voxels when it completes,
                          packed as sg_read_field_active writes them; owned by
                          the caller and borrowed until the job is done */
    int64_t out_cap;   /* values out_values holds; a job with more active
                          voxels fails at completion instead of writing */
} sg_job_desc;
typedef struct sg_job_status {
    int32_t state;      /* SG_JOB_* */
    int32_t steps_done;
    int64_t n_active;   /* active voxels (known once admitted) */
    double sum;         /* sum of x after the last completed step */
    double t_submit, t_admit, t_done;
} sg_job_status;
typedef struct sg_server_stats {
    int64_t submitted, completed, failed, ticks, launches, admission_waits;
    int32_t resident, pending;
    double voxel_steps; /* sum over ticks of the resident jobs' active voxels */
} sg_server_stats;

int sg_server_create(const sg_server_desc *desc, void *cuda_stream, sg_server **out);
int sg_server_submit(sg_server *s, const sg_job_desc *job, int64_t *job_id);
int sg_server_tick(sg_server *s);
int sg_server_job(sg_server *s, int64_t job_id, sg_job_status *out);
/* Forget a finished job (SG_JOB_DONE or SG_JOB_FAILED): its record is freed
 * and sg_server_job no longer knows its id.  A server keeps every job's
 * record until this call or sg_server_destroy, so a long-running server
 * releases the jobs whose results it has read.  SG_ERR_INVALID for an
 * unknown id or a job that is still pending or running. */
int sg_server_release(sg_server *s, int64_t job_id);
int sg_server_get_stats(sg_server *s, sg_server_stats *out);
int sg_server_destroy(sg_server *s);

/* ---- list generation for callers that cannot allocate device memory ----
 *
 * Some callers cannot call cudaMalloc: a process whose device memory is owned
 * by another allocator (a framework's caching allocator, or a pool sized at
 * start-up that a stray cudaMalloc would fail against or fragment), or code
 * in a time-critical loop, where cudaMalloc and cudaFree would synchronize
 * the device.  sg_list_gen_noalloc gives them the active-list compaction that
 * sg_list_gen runs, without any allocation: it calls no cudaMalloc, cudaFree
 * or allocating library routine.  The paper has no counterpart; it is an
 * addition of this library.
 *
 * Input: dev_root, n_cells int32 pointer cells in device memory (a cell is
 * active iff its value is >= 0).  Output, in device memory: the active cells
 * in ascending index order -- dev_list_b gets the cell index, dev_list_slot
 * its value -- at most `cap` entries (NULL allowed when cap == 0), and
 * *dev_count the number of active cells (even when more than cap), or -1 if
 * a bounded device wait gave up (after about 1 s).  The work is queued on
 * `cuda_stream`; read the outputs after it completes.
 *
 * Scratch: a 32,800-byte static device array, which every GPU that loads
 * this library holds until the process exits; n_cells is limited to
 * 4,194,304 (SG_ERR_INVALID beyond).  All calls on a device share that
 * array, and each call clears the parts it uses on the stream before its
 * kernel runs, so two calls whose work overlaps on the GPU (different
 * streams, no ordering between them) race and give wrong results.  The first
 * call on a device, with that device current, looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it for the process; make that
 * first call before any stream capture begins.  A reset of the device
 * (cudaDeviceReset) unloads the library's device code there and makes the
 * kept address stale, which the library does not detect: do not call this
 * entry point on a device after resetting it.
 *
 * Returns SG_OK, SG_ERR_INVALID (bad arguments or too many cells) or
 * SG_ERR_CUDA (the address lookup, a memset or the launch failed). */
#define SG_NOALLOC_MAX_CELLS 4194304
int sg_list_gen_noalloc(const int32_t *dev_root, int64_t n_cells, int32_t *dev_list_slot,
                        int32_t *dev_list_b, int64_t cap, int32_t *dev_count, void *cuda_stream);

/* Fault injection for testing bounded waits: queue a list generation whose
 * first CTA also waits on a device flag that nothing ever sets.  The wait
 * gives up after about 0.2 s and latches SG_ERR_TIMEOUT, which the next sync
 * returns; the grid stays usable.  No counterpart in the paper. */
int sg_debug_wait_test(sg_grid *g);

/* Invariant checks of the structure and the stored values, counted per kind
 * (0 everywhere for a sound grid).  The structure is the two-level tree of
 * Sec. 3: a root of R^3 pointer cells over a pool of bitmasked leaves. */
typedef struct sg_check_report {
    int64_t root_bad;         /* root cells neither null (-1) nor a handed-out slot < max_leaves */
    int64_t slot_shared;      /* slots referenced by more than one root cell */
    int64_t list_bad;         /* list entries whose slot is not root[b] or whose b are not
                                 strictly ascending, plus |list length - allocated leaves| */
    int64_t nbr_bad;          /* neighbour-table entries differing from the root's */
    int64_t zero_leaf_bad;    /* nonzero mask words or values in the zero leaf */
    int64_t inactive_nonzero; /* nonzero values stored at inactive voxels of listed leaves
                                 (fields not marked scratch) */
    int64_t leaves;           /* allocated leaves found in the root */
    int64_t ctrl_bad;         /* control-block counters that the last CTA of a kernel resets
                                 (the reduction ticket) found nonzero between launches: a
                                 launch that stopped early would leave them so, and the next
                                 launch would pick the wrong last CTA */
} sg_check_report;

/* Implicit sync (with a current list), then run every check and fill *out.
 * Returns SG_OK whatever the counts are; errors are those of the sync, or
 * SG_ERR_INVALID (null arguments, a dry-run grid), SG_ERR_OOM (scratch for
 * the checks).  Not part of the paper's method: a debugging aid. */
int sg_check(sg_grid *g, sg_check_report *out);

/* Test hook for the checks above: after an implicit sync, overwrite one
 * 32-bit word of the grid's device arrays behind the queue's back (no host
 * state changes).  array 0 = root (index < R^3; bits, read as int32, must lie
 * in [-1, max_leaves), so every later access stays in bounds), 1 = mask words
 * (index < (max_leaves + 1) * L^3/32), 2 + f = field f (index <
 * (max_leaves + 1) * L^3; bits are the FP32 pattern).  The last leaf of the
 * mask and field arrays is the zero leaf.  Errors: SG_ERR_INVALID (an index or
 * value outside those ranges, a dry-run grid). */
int sg_debug_poke(sg_grid *g, int32_t array, int64_t index, uint32_t bits);

/* Message of the last failing call on this thread ("" if none). */
const char *sg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SGRID_H */
