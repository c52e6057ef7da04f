/*
 * oracle.c -- plain FP64 CPU oracle of the sparse-grid time-stepping path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * What it models (AsyncTaichi, Hu et al. 2021):
 *   - a two-level sparse grid: a pointer root over bitmasked leaf blocks of
 *     edge L (Sec. 3.1, Fig. 3; Sec. 4 "States": a pointer cell is active iff
 *     non-null, a bitmasked cell is active iff its bit is set);
 *   - value state: every voxel has a value; an inactive voxel reads as the
 *     ambient value 0 (Sec. 4 "States", Fig. 5 caption);
 *   - activation on write, which allocates the parent pointer cell and
 *     zero-fills (Sec. 3.2 item 3, Fig. 4);
 *   - list state: the active leaves (Sec. 3.2 item 2).  The paper does not fix
 *     the list order; this oracle lists leaves in ascending root index b.
 *   - the stencil, reduction and particle kernels of the workloads, written as
 *     their plain definitions, every read going through the mask as the
 *     Fig. 5 caption describes.
 *
 * The method's optimizations (list-generation removal, activation demotion,
 * task fusion, dead-store elimination; Sec. 6) are exact transformations, so
 * this file contains none of them: the oracle computes the unoptimized
 * definition, one plain loop per operation.
 *
 * Precision: all arithmetic on field values is FP64.  Inputs that arrive as
 * FP32 (initial field values, particle state) are widened.  Particle state is
 * stored back as FP32 because it is FP32 by definition of the workload; where
 * an FP32 number decides an integer (the particle's base node), the decision
 * is taken in FP32, the same precision the GPU path takes it in.
 *
 * Parity status of each function is recorded in its comment; every function
 * below is pinned by the CPU tests (brute force on dense arrays, closed-form
 * eigenmode decay, conservation identities, library special cases).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct og_grid {
    int32_t N;       /* virtual domain edge, a multiple of L */
    int32_t L;       /* leaf edge */
    int32_t R;       /* root edge = N / L */
    int32_t F;       /* number of scalar fields */
    int64_t cap;     /* allocated leaf capacity (grows) */
    int64_t n;       /* leaves allocated */
    int32_t *root;   /* R^3 cells: leaf index or -1 (null pointer) */
    int32_t *leaf_b; /* per leaf: its root cell index */
    uint8_t *act;    /* per leaf: L^3 booleans, the bitmask as bytes */
    double **val;    /* F arrays of cap * L^3 values */
} og_grid;

static int64_t cube(int64_t a) { return a * a * a; }

og_grid *og_create(int32_t N, int32_t L, int32_t F)
{
    if (N <= 0 || L <= 0 || N % L != 0 || F <= 0) return NULL;
    og_grid *g = (og_grid *)calloc(1, sizeof(og_grid));
    g->N = N; g->L = L; g->R = N / L; g->F = F;
    int64_t nr = cube(g->R);
    g->root = (int32_t *)malloc(sizeof(int32_t) * nr);
    for (int64_t b = 0; b < nr; b++) g->root[b] = -1;
    g->cap = 0; g->n = 0;
    g->val = (double **)calloc(F, sizeof(double *));
    return g;
}

void og_destroy(og_grid *g)
{
    if (!g) return;
    for (int f = 0; f < g->F; f++) free(g->val[f]);
    free(g->val); free(g->act); free(g->leaf_b); free(g->root); free(g);
}

static void og_grow(og_grid *g)
{
    int64_t nc = g->cap ? 2 * g->cap : 64;
    int64_t v = cube(g->L);
    g->leaf_b = (int32_t *)realloc(g->leaf_b, sizeof(int32_t) * nc);
    g->act = (uint8_t *)realloc(g->act, (size_t)(nc * v));
    for (int f = 0; f < g->F; f++)
        g->val[f] = (double *)realloc(g->val[f], sizeof(double) * nc * v);
    g->cap = nc;
}

/* Is (i,j,k) inside the virtual domain [0,N)^3? */
static int in_domain(const og_grid *g, int64_t i, int64_t j, int64_t k)
{
    return i >= 0 && j >= 0 && k >= 0 && i < g->N && j < g->N && k < g->N;
}

/* Root cell and local voxel index of a voxel (k is the fastest axis). */
static int64_t root_of(const og_grid *g, int64_t i, int64_t j, int64_t k)
{
    int64_t L = g->L, R = g->R;
    return ((i / L) * R + (j / L)) * R + (k / L);
}
static int64_t local_of(const og_grid *g, int64_t i, int64_t j, int64_t k)
{
    int64_t L = g->L;
    return ((i % L) * L + (j % L)) * L + (k % L);
}

/* Activation on write (Sec. 3.2 item 3, Fig. 4): allocate the pointer cell's
 * leaf if it is null (the new leaf is zero-filled and fully inactive), then
 * set the voxel's bit.  Returns 1 when the voxel was newly activated. */
static int og_activate_voxel(og_grid *g, int64_t i, int64_t j, int64_t k)
{
    int64_t b = root_of(g, i, j, k), l = local_of(g, i, j, k);
    int64_t v = cube(g->L);
    if (g->root[b] < 0) {
        if (g->n == g->cap) og_grow(g);
        int64_t s = g->n++;
        g->leaf_b[s] = (int32_t)b;
        memset(g->act + s * v, 0, (size_t)v);
        for (int f = 0; f < g->F; f++)
            for (int64_t q = 0; q < v; q++) g->val[f][s * v + q] = 0.0;
        g->root[b] = (int32_t)s;
    }
    uint8_t *a = g->act + (int64_t)g->root[b] * v + l;
    if (*a) return 0;
    *a = 1;
    return 1;
}

/* Read a voxel's value through the mask (Fig. 5 caption): out of the domain,
 * a null pointer or a clear bit all read as 0. */
static double og_get(const og_grid *g, int f, int64_t i, int64_t j, int64_t k)
{
    if (!in_domain(g, i, j, k)) return 0.0;
    int32_t s = g->root[root_of(g, i, j, k)];
    if (s < 0) return 0.0;
    int64_t idx = (int64_t)s * cube(g->L) + local_of(g, i, j, k);
    if (!g->act[idx]) return 0.0;
    return g->val[f][idx];
}

static int og_is_active(const og_grid *g, int64_t i, int64_t j, int64_t k)
{
    if (!in_domain(g, i, j, k)) return 0;
    int32_t s = g->root[root_of(g, i, j, k)];
    if (s < 0) return 0;
    return g->act[(int64_t)s * cube(g->L) + local_of(g, i, j, k)];
}

/* Global coordinates of local voxel l of leaf s. */
static void coords_of(const og_grid *g, int64_t s, int64_t l,
                      int64_t *i, int64_t *j, int64_t *k)
{
    int64_t L = g->L, R = g->R, b = g->leaf_b[s];
    int64_t bi = b / (R * R), bj = (b / R) % R, bk = b % R;
    *i = bi * L + l / (L * L);
    *j = bj * L + (l / L) % L;
    *k = bk * L + l % L;
}

/* Activate every voxel of the domain whose squared doubled distance from the
 * domain centre, D = sum_a (2 i_a + 1 - N)^2, lies in the band
 *   lo2 <= D < hi2  (lo_strict = 0)   or   lo2 < D < hi2  (lo_strict = 1).
 * D is 4x the squared distance from the voxel centre to the domain centre, so
 * a spherical shell of radii (r0, r1) is lo2 = ceil(4 r0^2), hi2 = ceil(4 r1^2).
 * Brute force over all N^3 voxels.  Returns the number of voxels newly
 * activated. */
int64_t og_activate_shell(og_grid *g, int64_t lo2, int64_t hi2, int32_t lo_strict)
{
    int64_t N = g->N, cnt = 0;
    for (int64_t i = 0; i < N; i++)
        for (int64_t j = 0; j < N; j++)
            for (int64_t k = 0; k < N; k++) {
                int64_t a = 2 * i + 1 - N, b = 2 * j + 1 - N, c = 2 * k + 1 - N;
                int64_t D = a * a + b * b + c * c;
                int lo_ok = lo_strict ? (lo2 < D) : (lo2 <= D);
                if (lo_ok && D < hi2) cnt += og_activate_voxel(g, i, j, k);
            }
    return cnt;
}

/* Activate explicit voxels given as n (i,j,k) int32 triples.  Coordinates
 * outside the domain are ignored.  Returns the number newly activated. */
/* Activate every voxel whose cell centre lies in the tube lo2 <= D < hi2
 * around the k axis through the domain centre, D = (2i+1-N)^2 + (2j+1-N)^2
 * (4 N^2 times the squared distance from the axis), at every k.  Returns the
 * number of newly activated voxels. */
int64_t og_activate_tube(og_grid *g, int64_t lo2, int64_t hi2)
{
    int64_t N = g->N, cnt = 0;
    for (int64_t i = 0; i < N; i++)
        for (int64_t j = 0; j < N; j++) {
            int64_t a = 2 * i + 1 - N, b = 2 * j + 1 - N, D = a * a + b * b;
            if (D < lo2 || D >= hi2) continue;
            for (int64_t k = 0; k < N; k++) cnt += og_activate_voxel(g, i, j, k);
        }
    return cnt;
}

int64_t og_activate_coords(og_grid *g, const int32_t *xyz, int64_t n)
{
    int64_t cnt = 0;
    for (int64_t p = 0; p < n; p++) {
        int64_t i = xyz[3 * p], j = xyz[3 * p + 1], k = xyz[3 * p + 2];
        if (in_domain(g, i, j, k)) cnt += og_activate_voxel(g, i, j, k);
    }
    return cnt;
}

/* Deactivate everything: all pointer cells null, no leaves. */
void og_deactivate_all(og_grid *g)
{
    int64_t nr = cube(g->R);
    for (int64_t b = 0; b < nr; b++) g->root[b] = -1;
    g->n = 0;
}

int64_t og_num_leaves(const og_grid *g) { return g->n; }

int64_t og_num_active(const og_grid *g)
{
    int64_t v = cube(g->L), c = 0;
    for (int64_t q = 0; q < g->n * v; q++) c += g->act[q];
    return c;
}

/* The list state: leaves in ascending root index b, each with its mask packed
 * as bit l of 32-bit word l/32 (l = local index, k fastest).  leaf_b gets
 * og_num_leaves entries, masks gets og_num_leaves * ceil(L^3/32) words. */
void og_read_structure(const og_grid *g, int32_t *leaf_b, uint32_t *masks)
{
    int64_t nr = cube(g->R), v = cube(g->L), W = (v + 31) / 32, e = 0;
    for (int64_t b = 0; b < nr; b++) {
        int32_t s = g->root[b];
        if (s < 0) continue;
        leaf_b[e] = (int32_t)b;
        for (int64_t w = 0; w < W; w++) masks[e * W + w] = 0;
        for (int64_t l = 0; l < v; l++)
            if (g->act[(int64_t)s * v + l]) masks[e * W + l / 32] |= 1u << (l % 32);
        e++;
    }
}

/* Field values in list order (ascending b), L^3 per leaf, 0 at inactive
 * voxels (the ambient value). */
void og_read_field(const og_grid *g, int32_t f, double *out)
{
    int64_t nr = cube(g->R), v = cube(g->L), e = 0;
    for (int64_t b = 0; b < nr; b++) {
        int32_t s = g->root[b];
        if (s < 0) continue;
        for (int64_t l = 0; l < v; l++) {
            int64_t idx = (int64_t)s * v + l;
            out[e * v + l] = g->act[idx] ? g->val[f][idx] : 0.0;
        }
        e++;
    }
}

/* Set field values from an FP32 array in list order; entries at inactive
 * voxels are ignored (an inactive voxel holds the ambient value). */
void og_write_field(og_grid *g, int32_t f, const float *in)
{
    int64_t nr = cube(g->R), v = cube(g->L), e = 0;
    for (int64_t b = 0; b < nr; b++) {
        int32_t s = g->root[b];
        if (s < 0) continue;
        for (int64_t l = 0; l < v; l++) {
            int64_t idx = (int64_t)s * v + l;
            g->val[f][idx] = g->act[idx] ? (double)in[e * v + l] : 0.0;
        }
        e++;
    }
}

/* As og_write_field, from FP64 data (used to set exact test fields). */
void og_write_field64(og_grid *g, int32_t f, const double *in)
{
    int64_t nr = cube(g->R), v = cube(g->L), e = 0;
    for (int64_t b = 0; b < nr; b++) {
        int32_t s = g->root[b];
        if (s < 0) continue;
        for (int64_t l = 0; l < v; l++) {
            int64_t idx = (int64_t)s * v + l;
            g->val[f][idx] = g->act[idx] ? in[e * v + l] : 0.0;
        }
        e++;
    }
}

/* clear: x = 0 on every active voxel (struct-for over active voxels). */
void og_clear(og_grid *g, int32_t f)
{
    int64_t v = cube(g->L);
    for (int64_t q = 0; q < g->n * v; q++) g->val[f][q] = 0.0;
}

/* 7-point explicit diffusion step on the active voxels:
 *   dst_i = src_i + coef * (sum over the 6 face neighbours n of src_n - 6 src_i)
 * with src read through the mask (inactive or out-of-domain neighbours are 0).
 * dst at inactive voxels is left at the ambient value 0.  src != dst. */
void og_diffuse7(og_grid *g, int32_t src, int32_t dst, double coef)
{
    int64_t v = cube(g->L);
    int64_t total = g->n * v;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < total; q++) {
        int64_t s = q / v, l = q % v, i, j, k;
        if (!g->act[q]) { g->val[dst][q] = 0.0; continue; }
        coords_of(g, s, l, &i, &j, &k);
        double c = og_get(g, src, i, j, k);
        double nb = og_get(g, src, i - 1, j, k) + og_get(g, src, i + 1, j, k)
                  + og_get(g, src, i, j - 1, k) + og_get(g, src, i, j + 1, k)
                  + og_get(g, src, i, j, k - 1) + og_get(g, src, i, j, k + 1);
        g->val[dst][q] = c + coef * (nb - 6.0 * c);
    }
}

/* 27-point box smoothing on the active voxels:
 *   dst_i = (1/27) * sum over the 3x3x3 neighbourhood n of src_n
 * with src read through the mask.  src != dst. */
void og_box27(og_grid *g, int32_t src, int32_t dst)
{
    int64_t v = cube(g->L);
    int64_t total = g->n * v;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < total; q++) {
        int64_t s = q / v, l = q % v, i, j, k;
        if (!g->act[q]) { g->val[dst][q] = 0.0; continue; }
        coords_of(g, s, l, &i, &j, &k);
        double acc = 0.0;
        for (int di = -1; di <= 1; di++)
            for (int dj = -1; dj <= 1; dj++)
                for (int dk = -1; dk <= 1; dk++)
                    acc += og_get(g, src, i + di, j + dj, k + dk);
        g->val[dst][q] = acc / 27.0;
    }
}

/* Sum of a field over the active voxels. */
double og_sum(const og_grid *g, int32_t f)
{
    int64_t v = cube(g->L), total = g->n * v;
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t q = 0; q < total; q++)
        if (g->act[q]) s += g->val[f][q];
    return s;
}

/* ---------------------------------------------------------------------------
 * Particle-grid transfer (hybrid Lagrangian-Eulerian workload, Sec. 8.3).
 * The paper names MLS-MPM but does not print the transfer formulas; these are
 * the standard quadratic B-spline PIC transfers of that method family.
 * The domain is the unit cube, dx = 1/N, node (i,j,k) sits at (i,j,k)*dx.
 * Particle arrays are AoS float triples (x, y, z) mapping to (i, j, k).
 * ------------------------------------------------------------------------- */

/* Base node and FP64 weights of one particle along one axis.  X = x * N and
 * base = floor(X - 0.5) are taken in FP32; fx = X - base is exact. */
static void og_bspline(float x, int32_t N, int64_t *base, double w[3])
{
    float X = x * (float)N;
    float bf = floorf(X - 0.5f);
    double fx = (double)X - (double)bf;
    *base = (int64_t)bf;
    w[0] = 0.5 * (1.5 - fx) * (1.5 - fx);
    w[1] = 0.75 - (fx - 1.0) * (fx - 1.0);
    w[2] = 0.5 * (fx - 0.5) * (fx - 0.5);
}

/* P2G with activation: for each particle p and each of its 27 stencil nodes n
 * inside the domain, activate n (activation on write) and accumulate
 *   mass_n += w_pn * pmass,   mom_n[a] += w_pn * pmass * v_p[a].
 * Fields f_mom0, f_mom0+1, f_mom0+2 hold the three momentum components.
 * Serial, in particle order. */
void og_p2g(og_grid *g, const float *x, const float *vel, int64_t n,
            double pmass, int32_t f_mass, int32_t f_mom0)
{
    int64_t v = cube(g->L);
    for (int64_t p = 0; p < n; p++) {
        int64_t base[3];
        double w[3][3];
        for (int a = 0; a < 3; a++) og_bspline(x[3 * p + a], g->N, &base[a], w[a]);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                for (int c = 0; c < 3; c++) {
                    int64_t i = base[0] + a, j = base[1] + b, k = base[2] + c;
                    if (!in_domain(g, i, j, k)) continue;
                    og_activate_voxel(g, i, j, k);
                    int64_t idx = (int64_t)g->root[root_of(g, i, j, k)] * v + local_of(g, i, j, k);
                    double wm = w[0][a] * w[1][b] * w[2][c] * pmass;
                    g->val[f_mass][idx] += wm;
                    for (int d = 0; d < 3; d++)
                        g->val[f_mom0 + d][idx] += wm * (double)vel[3 * p + d];
                }
    }
}

/* Grid update on the active nodes: where mass > 0, velocity = momentum/mass,
 * then gravity  v_z -= dt * gz  and the boundary condition: along each axis a,
 * a node with index < bound has a negative v_a set to 0, and a node with index
 * > N - bound has a positive v_a set to 0.  Nodes with mass <= 0 get velocity
 * 0.  The velocity replaces the momentum in fields f_mom0..f_mom0+2. */
void og_grid_update(og_grid *g, int32_t f_mass, int32_t f_mom0, double dt,
                    double gz, int32_t bound)
{
    int64_t v = cube(g->L);
    for (int64_t q = 0; q < g->n * v; q++) {
        if (!g->act[q]) continue;
        int64_t s = q / v, l = q % v, idx[3];
        coords_of(g, s, l, &idx[0], &idx[1], &idx[2]);
        double m = g->val[f_mass][q], u[3] = {0.0, 0.0, 0.0};
        if (m > 0.0) {
            for (int d = 0; d < 3; d++) u[d] = g->val[f_mom0 + d][q] / m;
            u[2] -= dt * gz;
            for (int d = 0; d < 3; d++) {
                if (idx[d] < bound && u[d] < 0.0) u[d] = 0.0;
                if (idx[d] > g->N - bound && u[d] > 0.0) u[d] = 0.0;
            }
        }
        for (int d = 0; d < 3; d++) g->val[f_mom0 + d][q] = u[d];
    }
}

/* G2P: v_p = sum over the 27 stencil nodes of w_pn * v_n (velocity read
 * through the mask), then x_p += dt * v_p.  Particle state is stored back as
 * FP32. */
void og_g2p(og_grid *g, float *x, float *vel, int64_t n, double dt, int32_t f_mom0)
{
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++) {
        int64_t base[3];
        double w[3][3], u[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; a++) og_bspline(x[3 * p + a], g->N, &base[a], w[a]);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                for (int c = 0; c < 3; c++) {
                    double wt = w[0][a] * w[1][b] * w[2][c];
                    for (int d = 0; d < 3; d++)
                        u[d] += wt * og_get(g, f_mom0 + d, base[0] + a, base[1] + b, base[2] + c);
                }
        for (int d = 0; d < 3; d++) {
            vel[3 * p + d] = (float)u[d];
            x[3 * p + d] = (float)((double)x[3 * p + d] + dt * u[d]);
        }
    }
}

/* ---------------------------------------------------------------------------
 * Affine (APIC) transfers, the particle-grid transfers of MLS-MPM (Sec. 8.3).
 * The paper does not print them; these are the affine particle-in-cell
 * transfers with quadratic B-splines, for which the inertia-like tensor
 * D_p = sum_n w_pn d_pn d_pn^T equals dx^2/4 times the identity.  Each
 * particle carries a 3x3 matrix C_p, stored row-major as 9 FP32 values
 * (C[9p + 3a + b] = C_ab), acting as (C d)_a = sum_b C_ab d_b.  The offset of
 * stencil node base + (a,b,c) from the particle is d = ((a,b,c) - fx) * dx
 * with fx the per-axis spline offsets X - base (X = x * N in FP32).
 * ------------------------------------------------------------------------- */

/* APIC P2G with activation: as og_p2g, with the momentum contribution
 *   mom_n += w_pn * pmass * (v_p + C_p d_pn). */
void og_p2g_apic(og_grid *g, const float *x, const float *vel, const float *C, int64_t n,
                 double pmass, int32_t f_mass, int32_t f_mom0)
{
    int64_t v = cube(g->L);
    double dx = 1.0 / (double)g->N;
    for (int64_t p = 0; p < n; p++) {
        int64_t base[3];
        double w[3][3], fx[3];
        for (int a = 0; a < 3; a++) {
            og_bspline(x[3 * p + a], g->N, &base[a], w[a]);
            fx[a] = (double)(x[3 * p + a] * (float)g->N) - (double)base[a];
        }
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                for (int c = 0; c < 3; c++) {
                    int64_t i = base[0] + a, j = base[1] + b, k = base[2] + c;
                    if (!in_domain(g, i, j, k)) continue;
                    og_activate_voxel(g, i, j, k);
                    int64_t idx = (int64_t)g->root[root_of(g, i, j, k)] * v + local_of(g, i, j, k);
                    double d[3] = {((double)a - fx[0]) * dx, ((double)b - fx[1]) * dx, ((double)c - fx[2]) * dx};
                    double wm = w[0][a] * w[1][b] * w[2][c] * pmass;
                    g->val[f_mass][idx] += wm;
                    for (int e = 0; e < 3; e++) {
                        double u = (double)vel[3 * p + e];
                        for (int f = 0; f < 3; f++) u += (double)C[9 * p + 3 * e + f] * d[f];
                        g->val[f_mom0 + e][idx] += wm * u;
                    }
                }
    }
}

/* APIC G2P: v_p = sum_n w_pn v_n, C_p = (4 / dx^2) sum_n w_pn v_n d_pn^T,
 * x_p += dt * v_p.  x, vel and C are stored back as FP32. */
void og_g2p_apic(og_grid *g, float *x, float *vel, float *C, int64_t n, double dt, int32_t f_mom0)
{
    double dx = 1.0 / (double)g->N, inv_d = 4.0 / (dx * dx);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; p++) {
        int64_t base[3];
        double w[3][3], fx[3], u[3] = {0.0, 0.0, 0.0}, B[3][3] = {{0.0}};
        for (int a = 0; a < 3; a++) {
            og_bspline(x[3 * p + a], g->N, &base[a], w[a]);
            fx[a] = (double)(x[3 * p + a] * (float)g->N) - (double)base[a];
        }
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
                for (int c = 0; c < 3; c++) {
                    double wt = w[0][a] * w[1][b] * w[2][c];
                    double d[3] = {((double)a - fx[0]) * dx, ((double)b - fx[1]) * dx, ((double)c - fx[2]) * dx};
                    for (int e = 0; e < 3; e++) {
                        double vn = og_get(g, f_mom0 + e, base[0] + a, base[1] + b, base[2] + c);
                        u[e] += wt * vn;
                        for (int f = 0; f < 3; f++) B[e][f] += wt * vn * d[f];
                    }
                }
        for (int e = 0; e < 3; e++) {
            vel[3 * p + e] = (float)u[e];
            x[3 * p + e] = (float)((double)x[3 * p + e] + dt * u[e]);
            for (int f = 0; f < 3; f++) C[9 * p + 3 * e + f] = (float)(inv_d * B[e][f]);
        }
    }
}

/* ---------------------------------------------------------------------------
 * Grid transfers between a fine grid and a coarse grid of half its edge, the
 * restriction / prolongation pattern of multigrid solvers that Sec. 6.3 uses
 * to motivate activation demotion (Fig. 13, the loop y[i // 2] += x[i] * w).
 * ------------------------------------------------------------------------- */

/* Restriction with activation on write: for every active fine voxel i,
 * activate coarse voxel i // 2 (componentwise floor division) and add
 * w * x_i to coarse field f_dst there.  coarse->N == fine->N / 2.  Serial, in
 * list order. */
void og_restrict(const og_grid *fine, og_grid *coarse, int32_t f_src, int32_t f_dst, double w)
{
    int64_t v = cube(fine->L), vc = cube(coarse->L);
    for (int64_t q = 0; q < fine->n * v; q++) {
        if (!fine->act[q]) continue;
        int64_t i, j, k;
        coords_of(fine, q / v, q % v, &i, &j, &k);
        og_activate_voxel(coarse, i / 2, j / 2, k / 2);
        int64_t idx = (int64_t)coarse->root[root_of(coarse, i / 2, j / 2, k / 2)] * vc
                    + local_of(coarse, i / 2, j / 2, k / 2);
        coarse->val[f_dst][idx] += w * fine->val[f_src][q];
    }
}

/* Prolongation: for every active fine voxel i, x_i += w * y_{i // 2}, with y
 * (coarse field f_src) read through the coarse mask (an inactive or absent
 * coarse voxel reads 0).  No activation. */
void og_prolong(const og_grid *coarse, og_grid *fine, int32_t f_src, int32_t f_dst, double w)
{
    int64_t v = cube(fine->L);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < fine->n * v; q++) {
        if (!fine->act[q]) continue;
        int64_t i, j, k;
        coords_of(fine, q / v, q % v, &i, &j, &k);
        fine->val[f_dst][q] += w * og_get(coarse, f_src, i / 2, j / 2, k / 2);
    }
}

/* Element-wise struct-for (the general kernels of the paper's
 * microbenchmarks, Supp. Sec. 1: chain_copy, increments, fill_array,
 * sparse_saxpy, autodiff): on every active voxel
 *   dst = alpha * a + beta * b + gamma * a * b + delta,
 * with a, b read at the same voxel (field index -1: absent, reads 0); dst
 * stays 0 at inactive voxels.  dst may equal a or b. */
void og_ew(og_grid *g, int32_t dst, int32_t a, int32_t b, double alpha, double beta, double gamma, double delta)
{
    int64_t total = g->n * cube(g->L);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < total; q++) {
        if (!g->act[q]) { g->val[dst][q] = 0.0; continue; }
        double va = a >= 0 ? g->val[a][q] : 0.0, vb = b >= 0 ? g->val[b][q] : 0.0;
        g->val[dst][q] = alpha * va + beta * vb + gamma * va * vb + delta;
    }
}

/* ---------------------------------------------------------------------------
 * MacCormack advection with RK3 path integration (Sec. 8.2; Supp. Sec. 4.2).
 * Collocated grid: every field lives at cell centres, voxel (i,j,k) at grid
 * position (i+0.5, j+0.5, k+0.5) in cell units.  Velocities are in domain
 * units (the unit cube) per time, so a time step dt moves h = dt * N cells
 * per unit velocity.  Samples between cells are trilinear over the 8
 * surrounding cell centres, each read through the mask (inactive or
 * out-of-domain cells read 0).  The paper does not print the scheme; the
 * readings are: Ralston's third-order Runge-Kutta for the backtrace, and the
 * MacCormack correction of Selle et al. clamped to the 8 values the forward
 * sample interpolates.
 * ------------------------------------------------------------------------- */

/* Trilinear sample of field f at position p (cell units); optionally the
 * min / max of the 8 cell values it interpolates. */
static double og_trilinear(const og_grid *g, int f, const double p[3], double *mn, double *mx)
{
    double X[3], fr[3];
    int64_t b[3];
    for (int a = 0; a < 3; a++) {
        X[a] = p[a] - 0.5;
        b[a] = (int64_t)floor(X[a]);
        fr[a] = X[a] - (double)b[a];
    }
    double s = 0.0, lo = INFINITY, hi = -INFINITY;
    for (int a = 0; a < 2; a++)
        for (int c = 0; c < 2; c++)
            for (int d = 0; d < 2; d++) {
                double v = og_get(g, f, b[0] + a, b[1] + c, b[2] + d);
                double w = (a ? fr[0] : 1.0 - fr[0]) * (c ? fr[1] : 1.0 - fr[1]) * (d ? fr[2] : 1.0 - fr[2]);
                s += w * v;
                if (v < lo) lo = v;
                if (v > hi) hi = v;
            }
    if (mn) *mn = lo;
    if (mx) *mx = hi;
    return s;
}

/* Velocity (fields v0, v0+1, v0+2) interpolated at p. */
static void og_velocity(const og_grid *g, int v0, const double p[3], double u[3])
{
    for (int a = 0; a < 3; a++) u[a] = og_trilinear(g, v0 + a, p, NULL, NULL);
}

/* Backtrace of the centre of voxel (i,j,k) over h cells per unit velocity
 * with Ralston's RK3: k1 = u(x), k2 = u(x - h/2 k1), k3 = u(x - 3h/4 k2),
 * x_back = x - h (2 k1 + 3 k2 + 4 k3) / 9. */
static void og_backtrace(const og_grid *g, int v0, double h, int64_t i, int64_t j, int64_t k, double out[3])
{
    double x[3] = {(double)i + 0.5, (double)j + 0.5, (double)k + 0.5}, k1[3], k2[3], k3[3], p[3];
    og_velocity(g, v0, x, k1);
    for (int a = 0; a < 3; a++) p[a] = x[a] - 0.5 * h * k1[a];
    og_velocity(g, v0, p, k2);
    for (int a = 0; a < 3; a++) p[a] = x[a] - 0.75 * h * k2[a];
    og_velocity(g, v0, p, k3);
    for (int a = 0; a < 3; a++) out[a] = x[a] - h * (2.0 * k1[a] + 3.0 * k2[a] + 4.0 * k3[a]) / 9.0;
}

/* Semi-Lagrangian advection: dst = src sampled at the backtrace of every
 * active voxel over time step dt (negative: backward); 0 at inactive voxels.
 * dst must differ from src and the velocity fields. */
void og_advect(og_grid *g, int32_t dst, int32_t src, int32_t v0, double dt)
{
    int64_t v = cube(g->L), total = g->n * v;
    double h = dt * (double)g->N;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < total; q++) {
        if (!g->act[q]) { g->val[dst][q] = 0.0; continue; }
        int64_t i, j, k;
        double p[3];
        coords_of(g, q / v, q % v, &i, &j, &k);
        og_backtrace(g, v0, h, i, j, k, p);
        g->val[dst][q] = og_trilinear(g, src, p, NULL, NULL);
    }
}

/* MacCormack correction: dst = qhat + (q - qtilde) / 2 at every active voxel,
 * clamped to the min / max of the 8 values of q that the forward sample (the
 * backtrace over dt) interpolates; 0 at inactive voxels.  dst must differ
 * from q and the velocity fields. */
void og_maccormack(og_grid *g, int32_t dst, int32_t qf, int32_t qhat, int32_t qtilde, int32_t v0, double dt)
{
    int64_t v = cube(g->L), total = g->n * v;
    double h = dt * (double)g->N;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < total; q++) {
        if (!g->act[q]) { g->val[dst][q] = 0.0; continue; }
        int64_t i, j, k;
        double p[3], lo, hi;
        coords_of(g, q / v, q % v, &i, &j, &k);
        og_backtrace(g, v0, h, i, j, k, p);
        og_trilinear(g, qf, p, &lo, &hi);
        double r = g->val[qhat][q] + 0.5 * (g->val[qf][q] - g->val[qtilde][q]);
        g->val[dst][q] = r < lo ? lo : (r > hi ? hi : r);
    }
}

/* Value of one voxel of a field read through the mask (for sampled checks). */
double og_get_voxel(const og_grid *g, int32_t f, int64_t i, int64_t j, int64_t k)
{
    return og_get(g, f, i, j, k);
}

int32_t og_voxel_active(const og_grid *g, int64_t i, int64_t j, int64_t k)
{
    return og_is_active(g, i, j, k);
}
