"""GPU parity of the MacCormack / RK3 advection over a tube against the FP64
oracle: tube structure bit-exact; advected and corrected fields within 2e-5
normwise relative L-inf of the oracle's (smooth channels; FP32 sampling
positions); the fused (channel-grouped, backward advection + correction) and
unfused orders give the same fields."""
import numpy as np
import pytest

import oracle
from sgtest import rel_linf
from workload import tube, tube_fields

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def fields_of(spec, b):
    cells = oracle.leaf_coords(b, spec.N, spec.L).astype(np.float64)
    return tube_fields(spec, cells)


def setup(spec, opts):
    import paper_2012_08141_gb300 as sg
    F = 15          # velocity 0..2; channel c: q 3+4c, q^ 4+4c, q~ 5+4c, q' 6+4c
    scratch = sum(1 << (5 + 4 * c) for c in range(3))
    g = sg.Grid(spec.N, int(np.log2(spec.L)), F, max_leaves=(spec.N // spec.L) ** 3, scratch_mask=scratch)
    g.set_opts(opts)
    og = oracle.Grid(spec.N, spec.L, F)
    g.activate_tube(spec.lo2, spec.hi2)
    og.activate_tube(spec.lo2, spec.hi2)
    b, m = g.read_structure()
    ob, om = og.structure()
    np.testing.assert_array_equal(b, ob)
    np.testing.assert_array_equal(m, om)
    vel, ch = fields_of(spec, b)
    for a in range(3):
        g.write_field(a, vel[a])
        og.write_field(a, vel[a])
    for c in range(3):
        g.write_field(3 + 4 * c, ch[c])
        og.write_field(3 + 4 * c, ch[c])
    return g, og


def step(g, dt):
    for c in range(3):
        q, qh, qt, qn = 3 + 4 * c, 4 + 4 * c, 5 + 4 * c, 6 + 4 * c
        g.advect(qh, q, 0, dt)
        g.advect(qt, qh, 0, -dt)
        g.maccormack(qn, q, qh, qt, 0, dt)


@pytest.mark.parametrize("L", [8, 4])
@pytest.mark.parametrize("mode", ["all", "nofuse"])
def test_one_step(L, mode):
    import paper_2012_08141_gb300 as sg
    spec = tube(N=64, L=L)
    opts = sg.SG_OPT_ALL if mode == "all" else sg.SG_OPT_ALL & ~sg.SG_OPT_FUSE
    g, og = setup(spec, opts)
    step(g, spec.dt)
    step(og, spec.dt)
    for c in range(3):
        for f in (4 + 4 * c, 6 + 4 * c):        # q^ and the corrected q' (q~ is scratch)
            assert rel_linf(g.read_field(f), og.read_field(f)) <= TOL, (mode, c, f)
    g.close()


def test_ten_steps_fused():
    """Ten fused steps (swapping q and q' after each) against ten oracle steps."""
    import paper_2012_08141_gb300 as sg
    spec = tube(N=64, L=8)
    g, og = setup(spec, sg.SG_OPT_ALL)
    for _ in range(10):
        for G in (g, og):
            step(G, spec.dt)
        for c in range(3):
            g.swap(3 + 4 * c, 6 + 4 * c)
            og_q = og.read_field(6 + 4 * c)
            og.write_field64(3 + 4 * c, og_q)
    for c in range(3):
        assert rel_linf(g.read_field(3 + 4 * c), og.read_field(3 + 4 * c)) <= 1e-4, c
    g.close()


@pytest.mark.parametrize("mode", ["all", "nofuse"])
def test_clamp_case_matches_oracle(mode):
    """The case of the oracle's clamp pin (a spike on a ramp, uniform
    fractional velocity): the library's MacCormack correction, fused with the
    backward advection (and reading the forward advection's stored bounds) or
    not, matches the oracle within 2e-5, and where the unclamped correction
    leaves the forward sample's range the library's value is the clamp bound,
    not the unclamped value."""
    import torch
    import paper_2012_08141_gb300 as sg
    from advect_cases import clamp_case
    N = 32
    dtime, d, dense, m, rr, fw, _, _ = clamp_case(N)
    r = np.arange(4, 28)
    box = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.int32)
    g = sg.Grid(N, 3, 7, max_leaves=(N // 8) ** 3, scratch_mask=1 << 5)
    g.set_opts(sg.SG_OPT_ALL if mode == "all" else sg.SG_OPT_ALL & ~sg.SG_OPT_FUSE)
    og = oracle.Grid(N, 8, 7)
    xyz = torch.from_numpy(box).cuda()
    g.activate_coords(xyz)
    og.activate_coords(box)
    b, msk = g.read_structure()
    ob, om = og.structure()
    np.testing.assert_array_equal(b, ob)
    np.testing.assert_array_equal(msk, om)
    cells = oracle.leaf_coords(b, N, 8)
    u = d / (dtime * N)
    vals = dense[cells[..., 0], cells[..., 1], cells[..., 2]]
    for G in (g, og):
        for a in range(3):
            G.write_field(1 + a, np.full(cells.shape[:2], u[a]))
        G.write_field(0, vals)
        G.advect(4, 0, 1, dtime)        # q^ = q at x - d
        G.advect(5, 4, 1, -dtime)       # q~ = q^ at x + d (scratch)
        G.maccormack(6, 0, 4, 5, 1, dtime)
    got, ref = g.read_field(6), og.read_field(6)
    assert rel_linf(got, ref) <= TOL
    # the voxels where the clamp acts, by the definitions
    dense_got = np.zeros((N, N, N))
    dense_got[cells[..., 0], cells[..., 1], cells[..., 2]] = got
    inner = dense_got[m:N - m, m:N - m, m:N - m]
    acts = (rr < fw[0]) | (rr > fw[1])
    want = np.clip(rr, fw[0], fw[1])
    strong = acts & (np.abs(want - rr) > 1e-3)   # clearly clamped
    assert strong.sum() >= 4
    np.testing.assert_allclose(inner[acts], want[acts], rtol=0, atol=2e-6)
    assert np.all(np.abs(inner[strong] - rr[strong]) > 5e-4)
    g.close()
