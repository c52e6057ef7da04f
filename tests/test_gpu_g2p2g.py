"""GPU parity of the fused G2P2G (APIC G2P from one grid and APIC P2G into
another in one pass, the affine matrix C never stored) against the oracle's
separate APIC G2P and APIC P2G.

The oracle's P2G is fed the GPU's new positions: activation is decided by the
FP32 positions, which the GPU and the FP64 oracle round differently in the
last place, so this makes the structure comparable bit-exactly.  Velocities,
C and grid fields agree within a normwise relative L-inf of 1e-4 (FP32
atomic order), positions within a few FP32 ulps."""
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


def _affine(n, seed, scale=5.0):
    return np.random.default_rng(seed).normal(0.0, scale, size=(n, 9)).astype(np.float32)


def _setup(spec, C0, max_leaves, dst_leaves=None):
    """GPU grids A (binned APIC P2G + grid update done) and B, and the oracle's A."""
    import torch
    import paper_2012_08141_gb300 as sg
    lg = int(np.log2(spec.L))
    A = sg.Grid(spec.N, lg, 4, max_leaves=max_leaves)
    B = sg.Grid(spec.N, lg, 4, max_leaves=dst_leaves or max_leaves)
    x = torch.from_numpy(spec.x).cuda()
    v = torch.from_numpy(spec.v).cuda()
    C = torch.from_numpy(C0).cuda()
    A.p2g_apic(x, v, C, spec.pmass, 0, 1)
    A.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
    oA = oracle.Grid(spec.N, spec.L, 4)
    ox, ov = spec.x.copy(), spec.v.copy()
    oA.p2g_apic(ox, ov, C0, spec.pmass, 0, 1)
    oA.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
    return A, B, oA, x, v, ox, ov


def fused_step_check(spec, C0, max_leaves, shift=None):
    import torch
    A, B, oA, x, v, ox, ov = _setup(spec, C0, max_leaves)
    if shift is not None:          # positions changed since the binning
        A.sync()
        xm = (ox + shift).astype(np.float32)
        x.copy_(torch.from_numpy(xm))
        torch.cuda.synchronize()
        ox = xm.copy()
    B.deactivate_all()
    A.g2p2g(B, x, v, spec.dt, 1, spec.pmass, 0, 1)
    B.sync()
    oC = np.zeros((spec.n, 9), np.float32)
    oA.g2p_apic(ox, ov, oC, spec.dt, 1)
    gx, gv = x.cpu().numpy(), v.cpu().numpy()
    assert rel_linf(gv, ov) <= TOL
    assert np.max(np.abs(gx.astype(np.float64) - ox)) <= 4e-7
    oB = oracle.Grid(spec.N, spec.L, 4)
    oB.p2g_apic(gx, ov, oC, spec.pmass, 0, 1)
    gb, gm = B.read_structure()
    ob, om = oB.structure()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gm, om)
    for f in range(4):
        assert rel_linf(B.read_field(f), oB.read_field(f)) <= TOL, f
    A.close()
    B.close()


@pytest.mark.parametrize("L", [4, 8])
def test_g2p2g_one_step(L):
    spec = spheres_particles(seed=31, n=20000, N=64, L=L, r_min=0.1, r_max=0.2)
    fused_step_check(spec, _affine(spec.n, 32), (64 // L) ** 3)


@pytest.mark.parametrize("L", [4, 8])
def test_g2p2g_domain_faces(L):
    """Particles across and beyond every face: the out-of-domain key and the
    node-by-node paths."""
    spec = cube_particles(seed=33 + L, n=3000, N=64, L=L, pad_cells=3.0)
    fused_step_check(spec, _affine(spec.n, 34), (64 // L) ** 3)


def test_g2p2g_positions_moved():
    """Half the particles moved up to 6 cells since the binning: G2P reads the
    grid node by node and P2G scatters node by node with in-kernel leaf
    allocation."""
    spec = spheres_particles(seed=35, n=20000, N=64, L=4, r_min=0.1, r_max=0.2)
    rng = np.random.default_rng(36)
    shift = rng.uniform(-6.0, 6.0, size=spec.x.shape) / spec.N
    shift[rng.random(spec.n) < 0.5] = 0.0
    fused_step_check(spec, _affine(spec.n, 37), 4096, shift=shift)


def test_g2p2g_full_size_one_step():
    spec = spheres_particles(seed=0)            # 2M particles, 256^3, 4^3 leaves
    fused_step_check(spec, _affine(spec.n, 38, scale=1.0), 262144)


def test_g2p2g_steps_against_separate_oracle_steps():
    """Five fused steps (deactivate dst, G2P2G, grid update, swap the grids)
    against five separate oracle steps (G2P, deactivate, P2G, grid update):
    particle state within tolerance, and the last grid's structure equal to
    the oracle's activation from the GPU's positions."""
    import torch
    spec = spheres_particles(seed=39, n=20000, N=64, L=4, r_min=0.1, r_max=0.2)
    C0 = _affine(spec.n, 40)
    A, B, oA, x, v, ox, ov = _setup(spec, C0, 4096)
    oB = oracle.Grid(spec.N, spec.L, 4)
    oC = np.zeros((spec.n, 9), np.float32)
    for _ in range(5):
        B.deactivate_all()
        A.g2p2g(B, x, v, spec.dt, 1, spec.pmass, 0, 1)
        B.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        A, B = B, A
        oA.g2p_apic(ox, ov, oC, spec.dt, 1)
        oB.deactivate_all()
        oB.p2g_apic(ox, ov, oC, spec.pmass, 0, 1)
        oB.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        oA, oB = oB, oA
    A.sync()
    gx, gv = x.cpu().numpy(), v.cpu().numpy()
    assert rel_linf(gv, ov) <= TOL
    assert np.max(np.abs(gx.astype(np.float64) - ox)) <= 2e-6
    # the last fused step scattered at the final positions into the grid now in A
    gb, gm = A.read_structure()
    chk = oracle.Grid(spec.N, spec.L, 4)
    chk.p2g_apic(gx, np.zeros_like(gv), np.zeros((spec.n, 9), np.float32), 1.0, 0, 1)
    cb, cm = chk.structure()
    np.testing.assert_array_equal(gb, cb)
    np.testing.assert_array_equal(gm, cm)
    A.close()
    B.close()


def test_g2p2g_pool_exhaustion_reports():
    import paper_2012_08141_gb300 as sg
    spec = spheres_particles(seed=41, n=5000, N=64, L=4, r_min=0.1, r_max=0.2)
    A, B, oA, x, v, ox, ov = _setup(spec, _affine(spec.n, 42), 4096, dst_leaves=16)
    B.deactivate_all()
    A.g2p2g(B, x, v, spec.dt, 1, spec.pmass, 0, 1)
    with pytest.raises(sg.SgError) as e:
        B.sync()
    assert e.value.code == sg.SG_ERR_POOL_EXHAUSTED
    A.close()
    B.close()


def test_g2p2g_steps_after_a_sort():
    """The fused steps of the test above with the particle arrays reordered
    into the bin order right after the binned P2G (sg_sort_particles on the
    grid holding the bins, the ids carried along): the bins stay valid, and
    after five steps every particle's state matches the oracle's by id."""
    import torch
    spec = spheres_particles(seed=39, n=20000, N=64, L=4, r_min=0.1, r_max=0.2)
    C0 = _affine(spec.n, 40)
    A, B, oA, x, v, ox, ov = _setup(spec, C0, 4096)
    ids = torch.arange(spec.n, dtype=torch.int64, device="cuda")
    C = torch.from_numpy(C0).cuda()
    A.sort_particles(x, v, C, ids)
    oB = oracle.Grid(spec.N, spec.L, 4)
    oC = np.zeros((spec.n, 9), np.float32)
    for _ in range(5):
        B.deactivate_all()
        A.g2p2g(B, x, v, spec.dt, 1, spec.pmass, 0, 1)
        B.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        A, B = B, A
        oA.g2p_apic(ox, ov, oC, spec.dt, 1)
        oB.deactivate_all()
        oB.p2g_apic(ox, ov, oC, spec.pmass, 0, 1)
        oB.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        oA, oB = oB, oA
    A.sync()
    order = ids.cpu().numpy()
    assert not np.array_equal(order, np.arange(spec.n))      # the arrays were reordered
    np.testing.assert_array_equal(C.cpu().numpy(), C0[order])
    gx, gv = x.cpu().numpy(), v.cpu().numpy()
    assert rel_linf(gv, ov[order]) <= TOL
    assert np.max(np.abs(gx.astype(np.float64) - ox[order])) <= 2e-6
    A.close()
    B.close()
