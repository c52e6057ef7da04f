"""Pins of the FP64 oracle against things other than itself.

Each test fixes a part of the oracle to brute force on dense arrays (library
filters), to a closed form, to an exact identity, or to a worked example the
paper prints, chosen so that a dropped term, a wrong sign or index, or a
transposed operand in oracle.c fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import dense_twin as dt
from sgtest import mask_bits
import oracle
from advect_cases import clamp_case
from workload import band_bounds, band512, leaf_values, spheres_particles, tiny_shell

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        k, v = (s.strip() for s in line.split("=", 1))
        out[k] = [int(t) for t in v.split()]
    return out


def _coords(b, N, L):
    return oracle.leaf_coords(b, N, L)


# ---------------------------------------------------------------------------
# Structure: activation, list state, bit layout
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,L,r0,r1,strict", [
    (16, 8, 3.0, 7.5, False),
    (24, 8, 5.2, 9.9, True),
    (32, 8, 10.0, 14.0, False),
    (32, 4, 6.5, 12.25, True),
    (40, 8, 0.0, 9.0, False),      # ball
    (64, 8, 22.0, 26.0, False),    # the 64^3 shell of radius 24
])
def test_shell_structure_matches_bruteforce(N, L, r0, r1, strict):
    lo2, hi2 = band_bounds(r0, r1)
    g = oracle.Grid(N, L, 1)
    n_new = g.activate_shell(lo2, hi2, strict)
    act = dt.shell_active(N, lo2, hi2, strict)
    assert n_new == int(act.sum()) == g.num_active()
    b, m = g.structure()
    b2, m2 = dt.structure(act, L)
    np.testing.assert_array_equal(b, b2)
    np.testing.assert_array_equal(m, m2)
    assert np.all(np.diff(b) > 0)            # list in ascending root index


def test_shell_counts_64_and_512():
    """The 64^3 radius-24 shell and the 512^3 |dist-200|<8 band, counted by
    brute force over every voxel with numpy (independent of the oracle)."""
    lo2, hi2 = band_bounds(22.0, 26.0)
    g = oracle.Grid(64, 8, 1)
    g.activate_shell(lo2, hi2, False)
    act = dt.shell_active(64, lo2, hi2, False)
    assert g.num_active() == int(act.sum())
    assert g.num_leaves() == len(dt.structure(act, 8)[0])
    s = band512()
    g2 = oracle.Grid(s.N, s.L, 1)
    g2.activate_shell(s.lo2, s.hi2, s.lo_strict)
    c = (2 * np.arange(s.N, dtype=np.int64) + 1 - s.N) ** 2
    total, leaves = 0, set()
    for i in range(s.N):
        D = c[i] + c[:, None] + c[None, :]
        a = (D > s.lo2) & (D < s.hi2)
        total += int(a.sum())
        jj, kk = np.nonzero(a)
        leaves.update(((i // 8) * 64 + jj // 8) * 64 + kk // 8)
    assert g2.num_active() == total
    assert g2.num_leaves() == len(leaves)


def test_shell_activation_idempotent():
    lo2, hi2 = band_bounds(5.0, 9.0)
    g = oracle.Grid(24, 8, 1)
    first = g.activate_shell(lo2, hi2, False)
    assert first > 0
    assert g.activate_shell(lo2, hi2, False) == 0


def test_activate_coords_zero_fill_and_domain():
    """Activation on write zero-fills (Sec. 3.2 item 3): a voxel activated
    after values were written reads 0, a new leaf reads 0 everywhere, and
    coordinates outside the domain are ignored."""
    N, L = 16, 8
    g = oracle.Grid(N, L, 2)
    g.activate_coords([[1, 2, 3], [4, 4, 4]])
    b, _ = g.structure()
    g.write_field64(0, np.full((len(b), L ** 3), 5.0))
    assert g.get(0, 1, 2, 3) == 5.0 and g.get(0, 4, 4, 4) == 5.0
    assert g.get(0, 1, 2, 4) == 0.0                     # inactive reads ambient 0
    n = g.activate_coords([[1, 2, 4], [9, 9, 9], [-1, 0, 0], [16, 0, 0], [0, 0, 16]])
    assert n == 2
    assert g.get(0, 1, 2, 4) == 0.0 and g.get(0, 9, 9, 9) == 0.0
    assert g.get(0, 1, 2, 3) == 5.0
    assert g.num_leaves() == 2 and g.num_active() == 4
    assert g.activate_coords([[1, 2, 3]]) == 0


def test_fig4_activation_on_write_bitmasked():
    """Fig. 4: for i in x: y[i // 2] += 1 activates y[1], y[3].  Bitmasked
    leaves activate only the written cells, not their siblings."""
    gold = golden()
    x = oracle.Grid(8, 8, 1)
    x.activate_coords([[0, 0, k] for k in (2, 3, 6, 7)])
    b, m = x.structure()
    ks = [l % 8 for l in range(512) if (m[0, l // 32] >> (l % 32)) & 1]
    y = oracle.Grid(8, 8, 1)
    y.activate_coords([[0, 0, k // 2] for k in ks])
    yk = sorted(k for k in range(8) if y.is_active(0, 0, k))
    assert yk == gold["fig4_written_cells"]
    for k in gold["fig4_dense_leaf_extra_cells"]:
        assert not y.is_active(0, 0, k)
    assert y.num_leaves() == 1


def test_deactivate_all():
    g = oracle.Grid(16, 8, 1)
    g.activate_coords([[0, 0, 0], [15, 15, 15]])
    assert g.num_leaves() == 2
    g.deactivate_all()
    assert g.num_leaves() == 0 and g.num_active() == 0
    assert g.get(0, 0, 0, 0) == 0.0
    g.activate_coords([[15, 15, 15]])
    assert g.num_leaves() == 1 and g.get(0, 15, 15, 15) == 0.0


# ---------------------------------------------------------------------------
# 7-point diffusion
# ---------------------------------------------------------------------------

def _box_grid(n, N=32, L=8, F=2):
    g = oracle.Grid(N, L, F)
    ii, jj, kk = np.meshgrid(*(np.arange(s) for s in n), indexing="ij")
    g.activate_coords(np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1))
    return g


@pytest.mark.parametrize("n,m", [((20, 24, 28), (1, 1, 1)), ((20, 24, 28), (1, 2, 3)),
                                 ((8, 8, 8), (2, 1, 4)), ((13, 5, 30), (3, 2, 7))])
def test_diffusion_eigenmode_closed_form(n, m):
    """On a fully active box [0,n)^3 with zero outside, the discrete Dirichlet
    mode u = prod_a sin(pi m_a (i_a+1)/(n_a+1)) is an eigenvector of the 7-point
    step: u_s = lambda^s u_0 with lambda = 1 - 0.1 sum_a (2 - 2 cos(pi m_a/(n_a+1)))."""
    N, L = 32, 8
    g = _box_grid(n, N, L)
    b, _ = g.structure()
    c = oracle.leaf_coords(b, N, L)
    u0 = np.ones(c.shape[:2])
    for a in range(3):
        u0 *= np.sin(math.pi * m[a] * (c[:, :, a] + 1) / (n[a] + 1))
    inside = np.all(c < np.array(n), axis=2)
    u0 = np.where(inside, u0, 0.0)
    g.write_field64(0, u0)
    lam = 1.0 - 0.1 * sum(2.0 - 2.0 * math.cos(math.pi * m[a] / (n[a] + 1)) for a in range(3))
    src, dst = 0, 1
    amp = np.max(np.abs(u0))
    for s in range(1, 101):
        g.diffuse7(src, dst, 0.1)
        src, dst = dst, src
        if s in (1, 5, 100):
            # every mode has |lambda| <= 1, so rounding errors stay below ~s*eps*amp
            err = np.max(np.abs(g.read_field(src) - lam ** s * u0))
            assert err <= 1e-13 * s * amp, (s, err)


def test_diffusion_mass_identity():
    """sum(t) - sum(x) = -coef * sum_i x_i b_i, b_i = number of inactive or
    out-of-domain face neighbours of i (the flux leaving the active set)."""
    N, L = 32, 8
    lo2, hi2 = band_bounds(6.0, 13.0)
    g = oracle.Grid(N, L, 2)
    g.activate_shell(lo2, hi2, False)
    b, _ = g.structure()
    x = leaf_values(7, N, L, b).astype(np.float64)
    g.write_field64(0, x)
    g.diffuse7(0, 1, 0.1)
    act = dt.shell_active(N, lo2, hi2, False)
    pad = np.pad(act, 1)
    nb_inactive = np.zeros_like(act, dtype=np.int64)
    for ax in range(3):
        for s in (-1, 1):
            nb_inactive += ~np.roll(pad, s, axis=ax)[1:-1, 1:-1, 1:-1]
    xd = dt.from_leaves(g.read_field(0), b, N, L)
    lhs = g.sum(1) - g.sum(0)
    rhs = -0.1 * float(np.sum(xd * nb_inactive * act))
    assert abs(lhs - rhs) <= 1e-11 * abs(rhs)


@pytest.mark.parametrize("N,L,r0,r1", [(24, 8, 4.0, 10.0), (32, 4, 7.0, 13.0), (16, 8, 0.0, 20.0)])
def test_diffusion_matches_dense_convolution(N, L, r0, r1):
    lo2, hi2 = band_bounds(r0, r1)
    g = oracle.Grid(N, L, 2)
    g.activate_shell(lo2, hi2, False)
    b, _ = g.structure()
    x = leaf_values(3, N, L, b)
    g.write_field(0, x)
    g.diffuse7(0, 1, 0.1)
    act = dt.shell_active(N, lo2, hi2, False)
    xd = dt.from_leaves(x.astype(np.float64), b, N, L)
    want = dt.to_leaves(dt.diffuse7(xd, act, 0.1), b, L)
    np.testing.assert_allclose(g.read_field(1), want, rtol=0, atol=1e-13)


# ---------------------------------------------------------------------------
# 27-point box smoothing and the sum reduction
# ---------------------------------------------------------------------------

def test_box27_full_domain_is_uniform_filter():
    """Fully active domain, zero outside: box27 is scipy's uniform_filter of
    size 3 with constant-zero boundary (a library special case)."""
    from scipy import ndimage
    N, L = 16, 8
    g = oracle.Grid(N, L, 2)
    g.activate_shell(0, 10 ** 9, False)
    b, _ = g.structure()
    t = leaf_values(11, N, L, b).astype(np.float64)
    g.write_field64(0, t)
    g.box27(0, 1)
    td = dt.from_leaves(t, b, N, L)
    want = dt.to_leaves(ndimage.uniform_filter(td, size=3, mode="constant", cval=0.0), b, L)
    np.testing.assert_allclose(g.read_field(1), want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("N,L,r0,r1", [(24, 8, 4.0, 10.0), (32, 4, 7.0, 13.0)])
def test_box27_matches_dense_and_sum_identity(N, L, r0, r1):
    lo2, hi2 = band_bounds(r0, r1)
    g = oracle.Grid(N, L, 2)
    g.activate_shell(lo2, hi2, False)
    b, _ = g.structure()
    t = leaf_values(5, N, L, b).astype(np.float64)
    g.write_field64(0, t)
    g.box27(0, 1)
    act = dt.shell_active(N, lo2, hi2, False)
    td = dt.from_leaves(t, b, N, L) * act
    want = dt.to_leaves(dt.box27(td, act), b, L)
    np.testing.assert_allclose(g.read_field(1), want, rtol=0, atol=1e-14)
    # sum x' = (1/27) sum_n t_n c_n, c_n = active voxels in n's 3^3 neighbourhood
    from scipy import ndimage
    cnt = ndimage.convolve(act.astype(np.float64), np.ones((3, 3, 3)), mode="constant")
    rhs = float(np.sum(td * cnt)) / 27.0
    assert abs(g.sum(1) - rhs) <= 1e-12 * abs(rhs)


def test_box27_constant_fixed_point():
    N, L = 32, 8
    g = _box_grid((20, 20, 20), N, L)
    b, _ = g.structure()
    c = oracle.leaf_coords(b, N, L)
    inside = np.all(c < 20, axis=2)
    g.write_field64(0, np.where(inside, 0.75, 0.0))
    g.box27(0, 1)
    out = g.read_field(1)
    interior = np.all((c >= 1) & (c < 19), axis=2)
    np.testing.assert_allclose(out[interior], 0.75, rtol=0, atol=1e-15)
    corner = np.all(c == 0, axis=2)
    np.testing.assert_allclose(out[corner], 0.75 * 8 / 27, rtol=0, atol=1e-15)


def test_sum_matches_numpy():
    N, L = 24, 8
    lo2, hi2 = band_bounds(3.0, 11.0)
    g = oracle.Grid(N, L, 1)
    g.activate_shell(lo2, hi2, False)
    b, m = g.structure()
    x = leaf_values(9, N, L, b).astype(np.float64)
    g.write_field64(0, x)
    act = dt.to_leaves(dt.shell_active(N, lo2, hi2, False), b, L)
    assert g.sum(0) == pytest.approx(float(np.sum(x * act)), rel=1e-14)


def test_read_write_roundtrip_inactive_zero():
    N, L = 16, 8
    g = oracle.Grid(N, L, 1)
    g.activate_coords([[0, 0, 0], [3, 5, 7]])
    b, _ = g.structure()
    g.write_field(0, np.full((1, 512), 2.5, dtype=np.float32))
    out = g.read_field(0)
    assert out.sum() == 5.0 and out[0, 0] == 2.5 and out[0, (3 * 8 + 5) * 8 + 7] == 2.5


# ---------------------------------------------------------------------------
# Particle transfers
# ---------------------------------------------------------------------------

def _small_particles(n=3000, N=32, seed=1):
    spec = spheres_particles(seed=seed, n=n, N=N, L=4, r_min=0.1, r_max=0.2)
    return spec


def test_p2g_matches_dense_add_at_and_activation_union():
    spec = _small_particles()
    N, L = spec.N, spec.L
    g = oracle.Grid(N, L, 4)
    g.p2g(spec.x, spec.v, spec.pmass, 0, 1)
    act, mass, mom = dt.p2g(spec.x, spec.v, N, spec.pmass)
    b, m = g.structure()
    b2, m2 = dt.structure(act, L)
    np.testing.assert_array_equal(b, b2)
    np.testing.assert_array_equal(m, m2)
    np.testing.assert_allclose(g.read_field(0), dt.to_leaves(mass, b, L), rtol=0, atol=1e-12)
    for d in range(3):
        np.testing.assert_allclose(g.read_field(1 + d), dt.to_leaves(mom[d], b, L), rtol=0, atol=1e-12)


def test_p2g_conservation():
    """Partition of unity: total mass = n * pmass, total momentum =
    pmass * sum v (all stencils inside the domain)."""
    spec = _small_particles(n=5000, N=32, seed=4)
    g = oracle.Grid(spec.N, spec.L, 4)
    g.p2g(spec.x, spec.v, 2.0, 0, 1)
    assert g.sum(0) == pytest.approx(2.0 * spec.n, rel=1e-12)
    for d in range(3):
        want = 2.0 * float(np.sum(spec.v[:, d].astype(np.float64)))
        assert abs(g.sum(1 + d) - want) <= 1e-11 * float(np.sum(np.abs(spec.v[:, d])))


def test_g2p_reproduces_linear_field():
    """Quadratic B-splines reproduce linear functions: with grid velocity
    v(node) = A node*dx + c, G2P returns A x_p + c (up to FP32 storage)."""
    spec = _small_particles(n=2000, N=32, seed=2)
    N, L = spec.N, spec.L
    g = oracle.Grid(N, L, 4)
    g.p2g(spec.x, spec.v, 1.0, 0, 1)
    b, _ = g.structure()
    c = oracle.leaf_coords(b, N, L).astype(np.float64) / N
    A = np.array([[0.3, -1.2, 0.5], [2.0, 0.1, -0.7], [-0.4, 0.9, 1.1]])
    off = np.array([0.05, -0.2, 0.3])
    for d in range(3):
        g.write_field64(1 + d, c @ A[d] + off[d])
    x = spec.x.copy()
    v = np.zeros_like(spec.v)
    dtime = 1e-3
    g.g2p(x, v, dtime, 1)
    xp = (spec.x.astype(np.float32) * np.float32(N)).astype(np.float64) / N
    want = xp @ A.T + off
    np.testing.assert_allclose(v, want, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(x, (spec.x.astype(np.float64) + dtime * v.astype(np.float64)),
                               rtol=0, atol=1e-7)


def test_g2p_uniform_velocity_exact():
    spec = _small_particles(n=500, N=32, seed=3)
    g = oracle.Grid(spec.N, spec.L, 4)
    g.p2g(spec.x, spec.v, 1.0, 0, 1)
    n = g.num_leaves()
    for d, val in enumerate((0.25, -0.5, 0.125)):
        g.write_field64(1 + d, np.full((n, 64), val))
    x = spec.x.copy()
    v = np.zeros_like(spec.v)
    g.g2p(x, v, 0.0, 1)
    np.testing.assert_allclose(v, np.broadcast_to([0.25, -0.5, 0.125], v.shape), rtol=1e-15, atol=0)
    np.testing.assert_array_equal(x, spec.x)


def test_g2p_apic_reproduces_affine_field():
    """APIC G2P on an affine grid velocity v(node) = A node*dx + c returns
    v_p = A x_p + c and C_p = A: quadratic B-splines reproduce linear
    functions and sum_n w d d^T = dx^2/4 I, so (4/dx^2) sum_n w v_n d^T = A.
    A is not symmetric, so a transposed C fails, as do a wrong sign of d or a
    wrong 4/dx^2 factor."""
    spec = _small_particles(n=2000, N=32, seed=5)
    N, L = spec.N, spec.L
    g = oracle.Grid(N, L, 4)
    g.p2g(spec.x, spec.v, 1.0, 0, 1)
    b, _ = g.structure()
    c = oracle.leaf_coords(b, N, L).astype(np.float64) / N
    A = np.array([[0.3, -1.2, 0.5], [2.0, 0.1, -0.7], [-0.4, 0.9, 1.1]])
    off = np.array([0.05, -0.2, 0.3])
    for d in range(3):
        g.write_field64(1 + d, c @ A[d] + off[d])
    x = spec.x.copy()
    v = np.zeros_like(spec.v)
    C = np.zeros((spec.n, 9), dtype=np.float32)
    dtime = 1e-3
    g.g2p_apic(x, v, C, dtime, 1)
    xp = (spec.x.astype(np.float32) * np.float32(N)).astype(np.float64) / N
    np.testing.assert_allclose(v, xp @ A.T + off, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(C.reshape(-1, 3, 3), np.broadcast_to(A, (spec.n, 3, 3)), rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(x, (spec.x.astype(np.float64) + dtime * v.astype(np.float64)), rtol=0, atol=1e-7)


def test_p2g_apic_zero_affine_is_pic():
    """With C = 0 the APIC P2G reduces to the PIC P2G: identical fields and
    structure (v + 0 is exact)."""
    spec = _small_particles(n=3000, N=32, seed=6)
    g1, g2 = oracle.Grid(spec.N, spec.L, 4), oracle.Grid(spec.N, spec.L, 4)
    g1.p2g(spec.x, spec.v, 1.25, 0, 1)
    g2.p2g_apic(spec.x, spec.v, np.zeros((spec.n, 9), np.float32), 1.25, 0, 1)
    b1, m1 = g1.structure()
    b2, m2 = g2.structure()
    np.testing.assert_array_equal(b1, b2)
    np.testing.assert_array_equal(m1, m2)
    for f in range(4):
        np.testing.assert_array_equal(g1.read_field(f), g2.read_field(f))


def test_p2g_apic_momentum_and_angular_momentum():
    """APIC P2G conserves linear momentum (sum_n w d = 0) and transfers the
    affine part as angular momentum: with every stencil inside the domain,
    sum_n x_n x p_n = pmass * sum_p [x_p x v_p + dx^2/4 (C21 - C12, C02 - C20,
    C10 - C01)], from sum_n w d d^T = dx^2/4 I."""
    spec = _small_particles(n=4000, N=32, seed=7)
    N, L, pm = spec.N, spec.L, 1.5
    rng = np.random.default_rng(8)
    C = rng.normal(0.0, 5.0, size=(spec.n, 9)).astype(np.float32)
    g = oracle.Grid(N, L, 4)
    g.p2g_apic(spec.x, spec.v, C, pm, 0, 1)
    assert g.sum(0) == pytest.approx(pm * spec.n, rel=1e-12)
    v64 = spec.v.astype(np.float64)
    for d in range(3):
        assert abs(g.sum(1 + d) - pm * v64[:, d].sum()) <= 1e-10 * pm * np.abs(v64[:, d]).sum()
    b, _ = g.structure()
    xn = (oracle.leaf_coords(b, N, L).astype(np.float64) / N).reshape(-1, 3)
    pn = np.stack([g.read_field(1 + d).reshape(-1) for d in range(3)], axis=1)
    got = np.cross(xn, pn).sum(axis=0)
    xp = (spec.x.astype(np.float32) * np.float32(N)).astype(np.float64) / N
    Cm = C.astype(np.float64).reshape(-1, 3, 3)
    spin = np.stack([Cm[:, 2, 1] - Cm[:, 1, 2], Cm[:, 0, 2] - Cm[:, 2, 0], Cm[:, 1, 0] - Cm[:, 0, 1]], axis=1)
    want = pm * (np.cross(xp, v64).sum(axis=0) + (1.0 / N) ** 2 / 4.0 * spin.sum(axis=0))
    scale = pm * (np.abs(np.cross(xp, v64)).sum() + np.abs(spin).sum() / (4.0 * N * N))
    assert np.max(np.abs(got - want)) <= 1e-11 * scale


# ---------------------------------------------------------------------------
# Restriction / prolongation between a grid and its half-edge coarse grid
# ---------------------------------------------------------------------------

def _fine_grid(N, L, seed, frac=0.05):
    rng = np.random.default_rng(seed)
    pts = rng.integers(0, N, size=(int(frac * N ** 3), 3)).astype(np.int32)
    g = oracle.Grid(N, L, 2)
    g.activate_coords(pts)
    b, _ = g.structure()
    g.write_field64(0, rng.uniform(-1.0, 1.0, size=(len(b), L ** 3)))
    return g


@pytest.mark.parametrize("N,L", [(32, 8), (32, 4), (16, 2)])
def test_restrict_matches_dense_block_sums(N, L):
    """Coarse structure = the set of i // 2 over active fine voxels (bit-exact)
    and coarse values = w * the sum of the active children, against a dense
    block-sum twin."""
    f = _fine_grid(N, L, seed=N + L)
    c = oracle.Grid(N // 2, L, 2)
    f.restrict_to(c, 0, 1, 0.125)
    fb, fm = f.structure()
    x = dt.from_leaves(f.read_field(0), fb, N, L)
    act = dt.from_leaves(mask_bits(fm, L ** 3).astype(float), fb, N, L) > 0
    want, want_act = dt.restrict(x, act, 0.125)
    cb, cm = c.structure()
    b2, m2 = dt.structure(want_act, L)
    np.testing.assert_array_equal(cb, b2)
    np.testing.assert_array_equal(cm, m2)
    np.testing.assert_allclose(c.read_field(1), dt.to_leaves(want, cb, L), rtol=0, atol=1e-13)


def test_restrict_conservation_and_accumulation():
    """sum(coarse) = w * sum(fine); a second restriction adds the same amount
    again and activates nothing new."""
    f = _fine_grid(32, 8, seed=3, frac=0.2)
    c = oracle.Grid(16, 8, 2)
    f.restrict_to(c, 0, 1, 0.25)
    b1, m1 = c.structure()
    s1 = c.sum(1)
    assert s1 == pytest.approx(0.25 * f.sum(0), rel=1e-12, abs=1e-12)
    f.restrict_to(c, 0, 1, 0.25)
    b2, m2 = c.structure()
    np.testing.assert_array_equal(b1, b2)
    np.testing.assert_array_equal(m1, m2)
    assert c.sum(1) == pytest.approx(2 * s1, rel=1e-12, abs=1e-12)


def test_prolong_then_restrict_closed_form():
    """With every fine voxel of a box active, restricting the prolongation of
    y gives 8 * w_r * w_p * y on every coarse voxel of the box's image."""
    N, L = 16, 4
    f = oracle.Grid(N, L, 2)
    box = np.stack(np.meshgrid(*[np.arange(4, 12)] * 3, indexing="ij"), -1).reshape(-1, 3)
    f.activate_coords(box)
    c = oracle.Grid(N // 2, L, 2)
    c.activate_coords(box // 2)
    cb, _ = c.structure()
    rng = np.random.default_rng(9)
    y = rng.uniform(-2.0, 2.0, size=(len(cb), L ** 3))
    c.write_field64(0, y)
    f.prolong_from(c, 0, 0, 0.5)
    f.restrict_to(c, 0, 1, 0.125)
    cc = oracle.leaf_coords(cb, N // 2, L)
    inside = np.all((cc >= 2) & (cc < 6), axis=2)
    got, y0 = c.read_field(1), c.read_field(0)
    np.testing.assert_allclose(got[inside], 8 * 0.125 * 0.5 * y0[inside], rtol=1e-14, atol=1e-15)
    assert np.all(got[~inside] == 0.0)


# ---------------------------------------------------------------------------
# Element-wise struct-fors (the microbenchmark kernels)
# ---------------------------------------------------------------------------

def _shell_grid(F=4, seed=1):
    spec = tiny_shell(seed)
    g = oracle.Grid(spec.N, spec.L, F)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    b, m = g.structure()
    g.write_field(0, leaf_values(seed, spec.N, spec.L, b))
    return g, b, m


def test_ew_algebra_identities():
    """2a - a = a exactly; a * a - a^2 via gamma = 0; fill gives delta on the
    active voxels and 0 elsewhere; ten increments add 10."""
    g, b, m = _shell_grid()
    x = g.read_field(0)
    act = mask_bits(m, 512)
    g.ew(1, 0, 0, 2.0, -1.0)                       # 2x - x
    np.testing.assert_array_equal(g.read_field(1), x)
    g.ew(2, 0, 0, gamma=1.0)                       # x * x
    np.testing.assert_array_equal(g.read_field(2), np.where(act, x * x, 0.0))
    g.ew(3, delta=0.75)                            # fill
    np.testing.assert_array_equal(g.read_field(3), np.where(act, 0.75, 0.0))
    assert g.sum(3) == pytest.approx(0.75 * act.sum(), rel=1e-15)
    for _ in range(10):
        g.ew(1, 1, alpha=1.0, delta=1.0)           # increments
    np.testing.assert_allclose(g.read_field(1), np.where(act, x + 10.0, 0.0), rtol=0, atol=1e-12)


def test_ew_saxpy_chain_in_place():
    """z = 3x + y; y = y - z (in place, reads its own old value); against the
    same arithmetic on the dense values."""
    g, b, m = _shell_grid(seed=2)
    act = mask_bits(m, 512)
    g.ew(1, 0, alpha=0.5, delta=-0.25)             # y = 0.5 x - 0.25
    x, y = g.read_field(0), g.read_field(1)
    g.ew(2, 0, 1, 3.0, 1.0)
    g.ew(1, 1, 2, 1.0, -1.0)
    z = np.where(act, 3.0 * x + y, 0.0)
    np.testing.assert_allclose(g.read_field(2), z, rtol=1e-15, atol=0)
    np.testing.assert_allclose(g.read_field(1), np.where(act, y - z, 0.0), rtol=1e-15, atol=1e-15)


# ---------------------------------------------------------------------------
# Tube activation and MacCormack / RK3 advection
# ---------------------------------------------------------------------------

def test_tube_structure_matches_bruteforce():
    N, L = 32, 8
    lo2, hi2 = 4 * N * N * 0.32 ** 2, 4 * N * N * 0.45 ** 2
    lo2, hi2 = int(np.ceil(lo2)), int(np.ceil(hi2))
    g = oracle.Grid(N, L, 1)
    n = g.activate_tube(lo2, hi2)
    c = (2 * np.arange(N) + 1 - N) ** 2
    D = c[:, None] + c[None, :]
    act2 = (D >= lo2) & (D < hi2)
    act = np.broadcast_to(act2[:, :, None], (N, N, N))
    assert n == int(act.sum())
    b, m = g.structure()
    b2, m2 = dt.structure(act, L)
    np.testing.assert_array_equal(b, b2)
    np.testing.assert_array_equal(m, m2)


def _box_advect_grid(N=32, L=8, lo=4, hi=28, F=6):
    g = oracle.Grid(N, L, F)
    r = np.arange(lo, hi)
    box = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.int32)
    g.activate_coords(box)
    b, _ = g.structure()
    cells = oracle.leaf_coords(b, N, L).astype(np.float64) + 0.5      # cell centres, cell units
    return g, b, cells


def test_advect_uniform_integer_shift_is_exact():
    """Uniform velocity moving exactly (2, -1, 0) cells per step: every voxel
    whose source stays inside the box gets the source value exactly."""
    N, dtime = 32, 0.01
    g, b, cells = _box_advect_grid(N)
    shift = np.array([2.0, -1.0, 0.0])
    u = shift / (dtime * N)
    for a in range(3):
        g.write_field64(1 + a, np.full(cells.shape[:2], u[a]))
    q = np.sin(cells[..., 0]) + 0.1 * cells[..., 1] * cells[..., 2]
    g.write_field64(0, q)
    g.advect(4, 0, 1, dtime)
    src = cells - shift
    inside = np.all((src > 4) & (src < 28), axis=2) & np.all((cells > 7) & (cells < 25), axis=2)
    want = np.sin(src[..., 0]) + 0.1 * src[..., 1] * src[..., 2]
    got = g.read_field(4)
    np.testing.assert_allclose(got[inside], want[inside], rtol=0, atol=1e-12)


def test_advect_linear_fields_rk3_taylor():
    """Linear velocity u(c) = B (c - c0) and linear scalar q(c) = w . (c - c0)
    + q0, both reproduced exactly by trilinear interpolation: the RK3
    backtrace of a linear ODE is the third-order Taylor polynomial of
    exp(-hB), so q_hat(c) = w . T (c - c0) + q0 with T = I - hB + (hB)^2/2 -
    (hB)^3/6 on voxels whose stages stay inside the box.  A wrong RK3
    coefficient or a sign of h changes T."""
    N, dtime = 32, 0.004          # displacements below 2 cells: every sample stays in the box
    g, b, cells = _box_advect_grid(N)
    c0 = np.array([16.0, 16.0, 16.0])
    B = np.array([[0.3, -1.1, 0.2], [0.9, 0.1, -0.4], [-0.2, 0.5, -0.3]])
    d = cells - c0
    for a in range(3):
        g.write_field64(1 + a, d @ B[a])
    w, q0 = np.array([0.7, -0.3, 1.2]), 2.5
    g.write_field64(0, d @ w + q0)
    g.advect(4, 0, 1, dtime)
    hB = dtime * N * B
    T = np.eye(3) - hB + hB @ hB / 2 - hB @ hB @ hB / 6
    want = (d @ T.T) @ w + q0
    inside = np.all(np.abs(d) < 8.5, axis=2)
    np.testing.assert_allclose(g.read_field(4)[inside], want[inside], rtol=0, atol=1e-11)


def test_maccormack_linear_field_and_clamp():
    """Uniform fractional velocity on a linear field: q_hat = q(x - d),
    q_tilde = q, so the correction returns q_hat exactly; the corrected value
    always lies within the forward sample's 8 values."""
    N, dtime = 32, 0.01
    g, b, cells = _box_advect_grid(N, F=7)   # q 0, velocity 1..3, q^ 4, q~ 5, result 6
    u = np.array([0.7, -0.35, 1.3]) / (dtime * N)
    for a in range(3):
        g.write_field64(1 + a, np.full(cells.shape[:2], u[a]))
    w = np.array([0.5, 1.5, -0.25])
    g.write_field64(0, (cells - 16.0) @ w)
    g.advect(4, 0, 1, dtime)
    g.advect(5, 4, 1, -dtime)
    g.maccormack(6, 0, 4, 5, 1, dtime)
    inside = np.all(np.abs(cells - 16.0) < 8, axis=2)
    np.testing.assert_allclose(g.read_field(6)[inside], g.read_field(4)[inside], rtol=0, atol=1e-12)
    # bounds on a rough field
    rng = np.random.default_rng(4)
    g.write_field64(0, rng.uniform(-1, 1, size=cells.shape[:2]))
    g.advect(4, 0, 1, dtime)
    g.advect(5, 4, 1, -dtime)
    g.maccormack(6, 0, 4, 5, 1, dtime)
    q, r = g.read_field(0), g.read_field(6)
    assert np.all(r <= max(q.max(), 0.0) + 1e-15) and np.all(r >= min(q.min(), 0.0) - 1e-15)


def test_maccormack_clamp_acts_on_the_forward_sample_values():
    """Near a spike the correction qhat + (q - q~)/2 leaves the range of the
    forward sample's 8 values of q, and the oracle must clamp it to exactly
    those 8 (Sec. 8.2, the clamped MacCormack of Selle et al.).  The expected
    field comes from the definitions on a dense array; the case is chosen so
    that a clamp to the voxel's own 8 cells or to the 8 cells around the
    backward sample gives a different field, so either mistake fails."""
    N = 32
    dtime, d, dense, m, rr, fw, own, bw = clamp_case(N)
    want = np.clip(rr, fw[0], fw[1])
    acts = (rr < fw[0]) | (rr > fw[1])
    assert acts.sum() >= 8                                     # the clamp acts here
    assert np.abs(np.clip(rr, own[0], own[1]) - want).max() > 1e-3
    assert np.abs(np.clip(rr, bw[0], bw[1]) - want).max() > 1e-3
    g, b, cells = _box_advect_grid(N, F=7)   # q 0, velocity 1..3, q^ 4, q~ 5, result 6
    idx = cells.astype(np.int64)
    u = d / (dtime * N)
    for a in range(3):
        g.write_field64(1 + a, np.full(cells.shape[:2], u[a]))
    g.write_field64(0, dense[idx[..., 0], idx[..., 1], idx[..., 2]])
    g.advect(4, 0, 1, dtime)
    g.advect(5, 4, 1, -dtime)
    g.maccormack(6, 0, 4, 5, 1, dtime)
    got = np.array([[[g.get(6, i, j, k) for k in range(m, N - m)] for j in range(m, N - m)] for i in range(m, N - m)])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_grid_update_hand_case():
    """v = p/m, v_z -= dt g, then the boundary clamp (index < bound with
    negative component, index > N - bound with positive component)."""
    N, L = 16, 4
    g = oracle.Grid(N, L, 4)
    nodes = np.array([[8, 8, 8], [1, 8, 8], [15, 8, 8], [8, 14, 2], [5, 5, 5]])
    g.activate_coords(nodes)
    b, _ = g.structure()
    coords = oracle.leaf_coords(b, N, L)
    mass = np.zeros((len(b), 64))
    mom = np.zeros((3, len(b), 64))
    vals = {(8, 8, 8): (2.0, (2.0, -4.0, 6.0)), (1, 8, 8): (1.0, (-1.0, 1.0, 1.0)),
            (15, 8, 8): (4.0, (4.0, 4.0, 4.0)), (8, 14, 2): (1.0, (0.5, 0.5, -0.5)),
            (5, 5, 5): (0.0, (0.0, 0.0, 0.0))}
    for key, (mm, p) in vals.items():
        sel = np.all(coords == np.array(key), axis=2)
        mass[sel] = mm
        for d in range(3):
            mom[d][sel] = p[d]
    g.write_field64(0, mass)
    for d in range(3):
        g.write_field64(1 + d, mom[d])
    g.grid_update(0, 1, 0.01, 9.8, 3)
    got = {key: tuple(g.get(1 + d, *key) for d in range(3)) for key in vals}
    assert got[(8, 8, 8)] == pytest.approx((1.0, -2.0, 3.0 - 0.098))
    assert got[(1, 8, 8)] == pytest.approx((0.0, 1.0, 1.0 - 0.098))      # i=1 < 3, v_x<0 -> 0
    assert got[(15, 8, 8)] == pytest.approx((0.0, 1.0, 1.0 - 0.098))     # i=15 > 13, v_x>0 -> 0
    assert got[(8, 14, 2)] == pytest.approx((0.5, 0.0, 0.0))             # j>13 v_y>0, k<3 v_z<0
    assert got[(5, 5, 5)] == (0.0, 0.0, 0.0)                            # massless node


def test_inputs_deterministic():
    a, b = tiny_shell(3), tiny_shell(3)
    assert (a.lo2, a.hi2) == (b.lo2, b.hi2)
    v1 = leaf_values(5, 64, 8, np.array([0, 17, 300]))
    v2 = leaf_values(5, 64, 8, np.array([0, 17, 300]))
    np.testing.assert_array_equal(v1, v2)
    assert v1.dtype == np.float32 and v1.min() >= 0.0 and v1.max() < 1.0
    p1, p2 = spheres_particles(2, n=100, N=32), spheres_particles(2, n=100, N=32)
    np.testing.assert_array_equal(p1.x, p2.x)
    lo, hi = 3 / 32, 1 - 3 / 32
    assert p1.x.min() >= lo and p1.x.max() <= hi
