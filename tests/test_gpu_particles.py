"""GPU parity of the particle-grid transfers (P2G with activation, grid
update, G2P) against the FP64 oracle.

The active node set must match bit-exactly (both sides take the base-node
decision in FP32 from the same FP32 positions).  Grid fields agree within a
normwise relative L-inf of 1e-4 (the FP32 atomic accumulation order is
unspecified); particle velocities within 1e-4 of their scale; positions within
a few FP32 ulps."""
import numpy as np
import pytest

import oracle
from sgtest import rel_linf
from workload import cube_particles, spheres_particles

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def make(spec, max_leaves):
    import paper_2012_08141_gb300 as sg
    g = sg.Grid(spec.N, int(np.log2(spec.L)), 4, max_leaves=max_leaves)
    og = oracle.Grid(spec.N, spec.L, 4)
    return g, og


def stencil_union_leaves(x, N, L):
    """Leaves touched by the 27-node stencils of FP32 positions x (numpy)."""
    X = (x.astype(np.float32) * np.float32(N)).astype(np.float32)
    base = np.floor(X - np.float32(0.5)).astype(np.int64)
    R = N // L
    out = set()
    for a in range(3):
        for b in range(3):
            for c in range(3):
                i, j, k = base[:, 0] + a, base[:, 1] + b, base[:, 2] + c
                ok = (i >= 0) & (j >= 0) & (k >= 0) & (i < N) & (j < N) & (k < N)
                out.update((((i[ok] // L) * R + j[ok] // L) * R + k[ok] // L).tolist())
    return np.array(sorted(out), dtype=np.int32)


def one_step_compare(spec, max_leaves, interior=True):
    import torch
    g, og = make(spec, max_leaves)
    x = torch.from_numpy(spec.x).cuda()
    v = torch.from_numpy(spec.v).cuda()
    ox, ov = spec.x.copy(), spec.v.copy()
    g.deactivate_all()
    g.p2g(x, v, spec.pmass, 0, 1)
    og.deactivate_all()
    og.p2g(ox, ov, spec.pmass, 0, 1)
    gb, gm = g.read_structure()
    ob, om = og.structure()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gm, om)
    for f in range(4):
        assert rel_linf(g.read_field(f), og.read_field(f)) <= TOL, f
    if interior:  # totals: partition of unity
        assert abs(g.read_field(0).astype(np.float64).sum() - spec.n * spec.pmass) <= 1e-4 * spec.n * spec.pmass
    g.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
    og.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
    for f in range(1, 4):
        assert rel_linf(g.read_field(f), og.read_field(f)) <= TOL, f
    g.g2p(x, v, spec.dt, 1)
    og.g2p(ox, ov, spec.dt, 1)
    g.sync()
    gv, gx = v.cpu().numpy(), x.cpu().numpy()
    assert rel_linf(gv, ov) <= TOL
    assert np.max(np.abs(gx.astype(np.float64) - ox)) <= 4e-7
    g.close()


def test_p2g_g2p_small():
    spec = spheres_particles(seed=3, n=20000, N=64, L=4, r_min=0.1, r_max=0.2)
    one_step_compare(spec, 8192)


@pytest.mark.parametrize("L", [4, 8])
def test_p2g_g2p_domain_faces(L):
    """Particles across every face of the domain and beyond it: stencils cut by
    the faces, bases at -2 and -1 (binned to leaf 0), and particles with no
    stencil node inside the domain (no activation, zero velocity)."""
    spec = cube_particles(seed=11 + L, n=3000, N=64, L=L, pad_cells=3.0)
    one_step_compare(spec, (64 // L) ** 3, interior=False)


def test_g2p_positions_moved_after_p2g():
    """G2P over the bins of the last P2G when the positions have changed since
    (shifted by up to 6 cells, some out of the domain): particles that left
    their bin's staged neighbourhood read the grid node by node."""
    import torch
    spec = spheres_particles(seed=4, n=20000, N=64, L=4, r_min=0.1, r_max=0.2)
    g, og = make(spec, 4096)
    x = torch.from_numpy(spec.x).cuda()
    v = torch.from_numpy(spec.v).cuda()
    ox, ov = spec.x.copy(), spec.v.copy()
    g.p2g(x, v, spec.pmass, 0, 1)
    g.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
    og.p2g(ox, ov, spec.pmass, 0, 1)
    og.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
    g.sync()
    rng = np.random.default_rng(5)
    shift = rng.uniform(-6.0, 6.0, size=ox.shape) / spec.N
    shift[rng.random(spec.n) < 0.5] = 0.0                   # half keep their bin
    xm = (ox + shift).astype(np.float32)
    x.copy_(torch.from_numpy(xm))
    torch.cuda.synchronize()
    ox = xm.copy()
    g.g2p(x, v, spec.dt, 1)
    og.g2p(ox, ov, spec.dt, 1)
    g.sync()
    assert rel_linf(v.cpu().numpy(), ov) <= TOL
    assert np.max(np.abs(x.cpu().numpy().astype(np.float64) - ox)) <= 4e-7
    g.close()


def test_p2g_g2p_unaligned_views():
    """Positions and velocities in views that start 4 bytes past an 8-byte
    boundary (the G2P stores fall back to single floats)."""
    import torch
    spec = spheres_particles(seed=6, n=9999, N=64, L=4, r_min=0.1, r_max=0.2)
    g, og = make(spec, 4096)
    xb = torch.zeros(3 * spec.n + 1, dtype=torch.float32, device="cuda")
    vb = torch.zeros(3 * spec.n + 1, dtype=torch.float32, device="cuda")
    x, v = xb[1:], vb[1:]
    assert x.data_ptr() % 8 == 4
    x.copy_(torch.from_numpy(spec.x.reshape(-1)))
    v.copy_(torch.from_numpy(spec.v.reshape(-1)))
    torch.cuda.synchronize()
    ox, ov = spec.x.copy(), spec.v.copy()
    for G, X, V in ((g, x, v), (og, ox, ov)):
        G.p2g(X, V, spec.pmass, 0, 1)
        G.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        G.g2p(X, V, spec.dt, 1)
    g.sync()
    assert rel_linf(v.cpu().numpy().reshape(-1, 3), ov) <= TOL
    assert np.max(np.abs(x.cpu().numpy().reshape(-1, 3).astype(np.float64) - ox)) <= 4e-7
    assert xb[0].item() == 0.0 and vb[0].item() == 0.0
    g.close()


def apic_step_compare(spec, max_leaves, C0, interior=True, shift=None):
    """APIC P2G, grid update, APIC G2P against the oracle: structure exact,
    fields, v and C within TOL normwise, x within a few ulps.  shift, if
    given, moves the positions between the grid update and G2P (same shift on
    both sides)."""
    import torch
    g, og = make(spec, max_leaves)
    x = torch.from_numpy(spec.x).cuda()
    v = torch.from_numpy(spec.v).cuda()
    C = torch.from_numpy(C0).cuda()
    ox, ov, oC = spec.x.copy(), spec.v.copy(), C0.copy()
    g.p2g_apic(x, v, C, spec.pmass, 0, 1)
    og.p2g_apic(ox, ov, oC, spec.pmass, 0, 1)
    gb, gm = g.read_structure()
    ob, om = og.structure()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gm, om)
    for f in range(4):
        assert rel_linf(g.read_field(f), og.read_field(f)) <= TOL, f
    g.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
    og.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
    if shift is not None:
        g.sync()
        xm = (ox + shift).astype(np.float32)
        x.copy_(torch.from_numpy(xm))
        torch.cuda.synchronize()
        ox = xm.copy()
    g.g2p_apic(x, v, C, spec.dt, 1)
    og.g2p_apic(ox, ov, oC, spec.dt, 1)
    g.sync()
    assert rel_linf(v.cpu().numpy(), ov) <= TOL
    assert rel_linf(C.cpu().numpy(), oC) <= TOL
    assert np.max(np.abs(x.cpu().numpy().astype(np.float64) - ox)) <= 4e-7
    g.close()


def _affine(n, seed, scale=5.0):
    return np.random.default_rng(seed).normal(0.0, scale, size=(n, 9)).astype(np.float32)


@pytest.mark.parametrize("L", [4, 8])
def test_apic_p2g_g2p_small(L):
    spec = spheres_particles(seed=21, n=20000, N=64, L=L, r_min=0.1, r_max=0.2)
    apic_step_compare(spec, (64 // L) ** 3, _affine(spec.n, 22))


@pytest.mark.parametrize("L", [4, 8])
def test_apic_domain_faces(L):
    spec = cube_particles(seed=23 + L, n=3000, N=64, L=L, pad_cells=3.0)
    apic_step_compare(spec, (64 // L) ** 3, _affine(spec.n, 24), interior=False)


def test_apic_g2p_positions_moved():
    spec = spheres_particles(seed=25, n=20000, N=64, L=4, r_min=0.1, r_max=0.2)
    rng = np.random.default_rng(26)
    shift = rng.uniform(-6.0, 6.0, size=spec.x.shape) / spec.N
    shift[rng.random(spec.n) < 0.5] = 0.0
    apic_step_compare(spec, 4096, _affine(spec.n, 27), shift=shift)


def test_apic_full_size_one_step():
    spec = spheres_particles(seed=0)            # 2M particles, 256^3, 4^3 leaves
    apic_step_compare(spec, 262144, _affine(spec.n, 28))


def test_p2g_g2p_full_size_one_step():
    spec = spheres_particles(seed=0)            # 2M particles, 256^3, 4^3 leaves
    one_step_compare(spec, 262144)


def test_particle_steps_full_size():
    """Five full steps (deactivate, P2G, grid update, G2P) on 2M particles run
    independently on both sides.  The node set is compared with the union of
    the 27-node stencils of the GPU's own positions (valid at any size), the
    particle state with the oracle's."""
    import torch
    import paper_2012_08141_gb300 as sg
    spec = spheres_particles(seed=1)
    g = sg.Grid(spec.N, 2, 4, max_leaves=262144)
    og = oracle.Grid(spec.N, spec.L, 4)
    x = torch.from_numpy(spec.x).cuda()
    v = torch.from_numpy(spec.v).cuda()
    ox, ov = spec.x.copy(), spec.v.copy()
    for _ in range(5):
        xs = x.cpu().numpy().copy()
        g.deactivate_all()
        g.p2g(x, v, spec.pmass, 0, 1)
        g.list_gen()
        g.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        gb, _ = g.read_structure()
        np.testing.assert_array_equal(gb, stencil_union_leaves(xs, spec.N, spec.L))
        g.g2p(x, v, spec.dt, 1)
        og.deactivate_all()
        og.p2g(ox, ov, spec.pmass, 0, 1)
        og.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        og.g2p(ox, ov, spec.dt, 1)
    g.sync()
    assert rel_linf(v.cpu().numpy(), ov) <= TOL
    assert np.max(np.abs(x.cpu().numpy().astype(np.float64) - ox)) <= 2e-6
    g.close()


def test_p2g_pool_exhaustion():
    import torch
    import paper_2012_08141_gb300 as sg
    spec = spheres_particles(seed=2, n=5000, N=64, L=4, r_min=0.1, r_max=0.2)
    g = sg.Grid(spec.N, 2, 4, max_leaves=16)
    g.p2g(torch.from_numpy(spec.x).cuda(), torch.from_numpy(spec.v).cuda(), 1.0, 0, 1)
    with pytest.raises(sg.SgError) as e:
        g.sync()
    assert e.value.code == sg.SG_ERR_POOL_EXHAUSTED
    g.close()


def _spec_from(x, v, N, L):
    from workload import ParticleSpec
    x = np.ascontiguousarray(x, dtype=np.float32)
    v = np.ascontiguousarray(v, dtype=np.float32)
    return ParticleSpec(N, L, len(x), np.zeros((3, 3)), np.zeros(3), x, v)


@pytest.mark.parametrize("L", [4, 8])
def test_crowded_cells_and_boundaries(L):
    """Degenerate particle layouts: 6,000 particles inside one cell (a bin
    several staging chunks long), particles exactly on cell faces and leaf
    faces (fractional offsets 0 and 0.5), and particles whose stencil lies
    wholly outside the domain (they touch nothing)."""
    rng = np.random.default_rng(50 + L)
    N = 64
    dx = 1.0 / N
    crowd = (np.array([20.5, 9.5, 33.5]) + rng.uniform(-0.49, 0.49, size=(6000, 3))) * dx
    faces = np.array([[i, j, k] for i in (8, 16, 31.5) for j in (0.5, 8.0, 24.0) for k in (1.0, 40.5, 63.5)]) * dx
    faces = np.repeat(faces, 5, axis=0)
    outside = np.array([[-0.2, 0.5, 0.5], [0.5, 1.3, 0.5], [0.5, 0.5, -0.5], [1.5, 1.5, 1.5]])
    x = np.concatenate([crowd, faces, outside])
    v = rng.normal(0.0, 0.1, size=x.shape)
    one_step_compare(_spec_from(x, v, N, L), (N // L) ** 3, interior=False)


def test_empty_particle_set_is_a_no_op():
    import torch
    import paper_2012_08141_gb300 as sg
    g = sg.Grid(64, 2, 4, max_leaves=64)
    x = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    v = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    l0 = g.stats()["launches"]
    g.p2g(x, v, 1.0, 0, 1)
    g.g2p(x, v, 1e-3, 1)
    g.sync()
    assert g.stats()["launches"] == l0                  # nothing queued, nothing launched
    assert g.num_leaves() == 0
    g.close()


def test_particles_all_outside_activate_nothing():
    import torch
    import paper_2012_08141_gb300 as sg
    x = np.array([[-0.3, 0.5, 0.5], [0.5, 1.2, 0.5], [2.0, 2.0, 2.0], [0.5, 0.5, -0.04]], dtype=np.float32)
    v = np.zeros_like(x)
    g = sg.Grid(64, 2, 4, max_leaves=64)
    og = oracle.Grid(64, 4, 4)
    g.p2g(torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda(), 1.0, 0, 1)
    og.p2g(x.copy(), v.copy(), 1.0, 0, 1)
    gb, gm = g.read_structure()
    ob, om = og.structure()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gm, om)
    assert gb.size == 0
    g.close()


def test_particle_50_steps_full_size():
    """The particle workload at its stated length: 50 steps (deactivate, P2G,
    grid update, G2P, dt = 1e-4) on 2M particles, run independently on both
    sides.  The node set is compared with the union of the 27-node stencils of
    the GPU's own positions at the first, a middle and the last step; the
    particle state with the oracle's at the end: velocities within 1e-4 of
    their scale (the P2G tolerance; each step's G2P interpolates grid
    velocities that agree to that bound, and the B-spline weights are
    continuous, so a base node decided differently near a cell face moves
    the result continuously, not by a jump), positions within 1e-5 (50
    steps of dt * v with v ~ 0.1-1)."""
    import torch
    import paper_2012_08141_gb300 as sg
    spec = spheres_particles(seed=1)
    g = sg.Grid(spec.N, 2, 4, max_leaves=262144)
    og = oracle.Grid(spec.N, spec.L, 4)
    x = torch.from_numpy(spec.x).cuda()
    v = torch.from_numpy(spec.v).cuda()
    ox, ov = spec.x.copy(), spec.v.copy()
    for step in range(50):
        check = step in (0, 24, 49)
        if check:
            g.sync()  # the queued steps run before the positions are read on the host
            xs = x.cpu().numpy().copy()
        g.deactivate_all()
        g.p2g(x, v, spec.pmass, 0, 1)
        g.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        if check:
            g.list_gen()
            gb, _ = g.read_structure()
            np.testing.assert_array_equal(gb, stencil_union_leaves(xs, spec.N, spec.L))
        g.g2p(x, v, spec.dt, 1)
        og.deactivate_all()
        og.p2g(ox, ov, spec.pmass, 0, 1)
        og.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        og.g2p(ox, ov, spec.dt, 1)
    g.sync()
    assert rel_linf(v.cpu().numpy(), ov) <= TOL
    assert np.max(np.abs(x.cpu().numpy().astype(np.float64) - ox)) <= 1e-5
    g.close()


def _bin_keys(x, N, L):
    """The binning key order of FP32 positions: leaf of the clamped base node
    (row-major over the root), the ordering sg_sort_particles leaves bins in."""
    X = (x.astype(np.float32) * np.float32(N)).astype(np.float32)
    base = np.floor(X - np.float32(0.5)).astype(np.int64)
    n0 = np.maximum(base, 0)
    R = N // L
    return ((n0[:, 0] // L) * R + n0[:, 1] // L) * R + n0[:, 2] // L


def test_sort_particles_reorders_and_keeps_the_physics():
    """Steps with the particle arrays reordered into bin order every other
    step (sg_sort_particles, the ids carried along) against the oracle's
    steps on the particles in their own order: after each sort the arrays
    hold the same particles (bit-exact, by id) grouped by bin, and after five
    steps every particle's state matches the oracle's by id."""
    import torch
    import paper_2012_08141_gb300 as sg
    spec = spheres_particles(seed=5, n=200000, N=128, L=4, r_min=0.1, r_max=0.25)
    g = sg.Grid(spec.N, 2, 4, max_leaves=(spec.N // 4) ** 3)
    og = oracle.Grid(spec.N, spec.L, 4)
    x = torch.from_numpy(spec.x).cuda()
    v = torch.from_numpy(spec.v).cuda()
    ids = torch.arange(spec.n, dtype=torch.int64, device="cuda")
    ox, ov = spec.x.copy(), spec.v.copy()
    for s in range(5):
        g.sync()                                  # the queued steps have run
        xb = x.cpu().numpy().copy()               # the positions this step bins
        g.deactivate_all()
        g.p2g(x, v, spec.pmass, 0, 1)
        g.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        g.g2p(x, v, spec.dt, 1)
        og.deactivate_all()
        og.p2g(ox, ov, spec.pmass, 0, 1)
        og.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        og.g2p(ox, ov, spec.dt, 1)
        if s % 2 == 0:
            g.sync()
            x_before, v_before, id_before = x.clone(), v.clone(), ids.clone()
            g.sort_particles(x, v, ids=ids)
            g.sync()
            perm_ids = ids.cpu().numpy()
            assert np.array_equal(np.sort(perm_ids), np.arange(spec.n))
            # the same particles: position q now holds what sat where its id was
            where = np.empty(spec.n, np.int64)
            where[id_before.cpu().numpy()] = np.arange(spec.n)
            src = where[perm_ids]
            np.testing.assert_array_equal(x.cpu().numpy(), x_before.cpu().numpy()[src])
            np.testing.assert_array_equal(v.cpu().numpy(), v_before.cpu().numpy()[src])
            keys = _bin_keys(xb[src], spec.N, spec.L)   # grouped by the step's bins
            inside = np.all((xb[src] * spec.N >= 0.5) & (xb[src] * spec.N < spec.N - 1.5), axis=1)
            assert np.all(np.diff(keys[inside]) >= 0)
    g.sync()
    order = ids.cpu().numpy()
    assert rel_linf(v.cpu().numpy(), ov[order]) <= TOL
    assert np.max(np.abs(x.cpu().numpy().astype(np.float64) - ox[order])) <= 2e-6
    g.close()
