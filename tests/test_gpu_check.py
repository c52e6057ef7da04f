"""GPU tests of the invariant checks (sg_check, checking grids): a grid driven
through every kind of op reports no violation; each kind of planted
violation (sg_debug_poke, in-bounds words written behind the queue's back) is
counted exactly, and a checking grid returns SG_ERR_CHECK at its next sync."""
import numpy as np
import pytest

from workload import band_bounds, leaf_values, tiny_shell

pytestmark = pytest.mark.gpu

CLEAN = dict(root_bad=0, slot_shared=0, list_bad=0, nbr_bad=0, zero_leaf_bad=0, inactive_nonzero=0, ctrl_bad=0)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _violations(r):
    return {k: r[k] for k in CLEAN}


def _grid(checking=False, L=8):
    import paper_2012_08141_gb300 as sg
    spec = tiny_shell(2, N=64, L=L)
    g = sg.Grid(64, int(np.log2(L)), 3, max_leaves=(64 // L) ** 3, max_sums=1, checking=checking)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    b, _ = g.read_structure()
    g.write_field(0, leaf_values(2, 64, L, b))
    return g


@pytest.mark.parametrize("L", [8, 4])
def test_sound_after_every_kind_of_op(L):
    import torch
    import paper_2012_08141_gb300 as sg
    from workload import cube_particles
    g = _grid(checking=True, L=L)
    g.diffuse7(0, 1, 0.1)
    g.box27(1, 2)
    g.reduce_sum(2, 0)
    g.ew(1, 0, 2, 1.0, -1.0)
    g.swap(0, 2)
    g.sync()
    r = g.check()
    assert _violations(r) == CLEAN and r["leaves"] == g.num_leaves()
    # particles: activation by P2G onto a second grid, grid update, G2P
    p = cube_particles(3, 4000, 64, L)
    x = torch.from_numpy(p.x).cuda()
    v = torch.from_numpy(p.v).cuda()
    h = sg.Grid(64, int(np.log2(L)), 4, max_leaves=(64 // L) ** 3, checking=True)
    h.p2g(x, v, 1.0, 0, 1)
    h.grid_update(0, 1, 1e-3, -9.8, 2)
    h.g2p(x, v, 1e-3, 1)
    h.sync()
    assert _violations(h.check()) == CLEAN
    # restriction onto a coarse grid, then deactivation and re-activation
    c = sg.Grid(32, int(np.log2(L)), 2, max_leaves=(32 // L) ** 3, checking=True)
    g.restrict_to(c, 0, 1, 0.125)
    c.sync()
    assert _violations(c.check()) == CLEAN
    lo2, hi2 = band_bounds(4.0, 12.0)
    g.deactivate_all()
    g.activate_shell(lo2, hi2, False)
    g.fill_hash(0, 9)
    g.sync()
    assert _violations(g.check()) == CLEAN
    for grid in (g, h, c):
        grid.close()


def _first_inactive(g):
    """List entry and local index of the first inactive voxel of a listed
    leaf (on a restored grid the entry is also the leaf's slot)."""
    b, m = g.read_structure()
    bits = np.unpackbits(m.view(np.uint8), bitorder="little").reshape(b.size, g.V)
    e, l = np.argwhere(bits == 0)[0]
    return int(e), int(l), b, m


def _restored(L=8):
    """A grid whose slots equal its list entries (restored from its own
    structure), so a test can name a slot."""
    g = _grid(L=L)
    b, m = g.read_structure()
    vals = g.read_field(0)
    g.write_structure(b, m)
    g.write_field(0, vals)
    return g


def test_inactive_value_is_counted():
    import paper_2012_08141_gb300 as sg
    g = _restored()
    e, l, b, m = _first_inactive(g)
    g.lib.sg_debug_poke(g.h, 2 + 0, e * g.V + l, int(np.float32(0.5).view(np.uint32)))
    assert _violations(g.check()) == dict(CLEAN, inactive_nonzero=1)
    g.lib.sg_debug_poke(g.h, 2 + 1, e * g.V + l, int(np.float32(-2.0).view(np.uint32)))
    assert g.check()["inactive_nonzero"] == 2
    g.close()


def _null_next_to_leaf(g, b):
    """A null root cell that is the +k neighbour of a listed leaf."""
    R = g.res // g.L
    have = set(int(x) for x in b)
    for x in b:
        x = int(x)
        if x % R + 1 < R and x + 1 not in have:
            return x + 1
    raise AssertionError("no null cell next to a leaf")


def test_zero_leaf_and_root_violations_are_counted():
    g = _restored()
    n = g.num_leaves()
    cap = g.max_leaves
    g.lib.sg_debug_poke(g.h, 2 + 2, cap * g.V + 17, int(np.float32(1.0).view(np.uint32)))
    g.lib.sg_debug_poke(g.h, 1, cap * g.W + 3, 0x10)
    assert _violations(g.check()) == dict(CLEAN, zero_leaf_bad=2)
    g.close()
    g = _restored()
    b, _ = g.read_structure()
    null = _null_next_to_leaf(g, b)
    assert n < cap
    g.lib.sg_debug_poke(g.h, 0, null, cap - 1)          # a slot never handed out
    r = g.check()
    assert r["root_bad"] == 1 and r["slot_shared"] == 0
    g.close()


def test_shared_slot_is_counted():
    g = _restored()
    b, _ = g.read_structure()
    null = _null_next_to_leaf(g, b)
    g.lib.sg_debug_poke(g.h, 0, null, 0)                # a second cell pointing at slot 0
    r = g.check()
    assert r["slot_shared"] == 1 and r["root_bad"] == 0
    assert r["leaves"] == b.size + 1
    assert r["list_bad"] == 1                           # the list misses one allocated leaf
    assert r["nbr_bad"] >= 1                            # neighbours of the new cell still see null
    g.close()


def test_checking_grid_raises_at_sync():
    import paper_2012_08141_gb300 as sg
    g = _grid(checking=True)
    b, m = g.read_structure()
    vals = g.read_field(0)
    g.write_structure(b, m)
    g.write_field(0, vals)
    e, l, _, _ = _first_inactive(g)
    assert g.lib.sg_debug_poke(g.h, 2, e * g.V + l, int(np.float32(3.0).view(np.uint32))) == sg.SG_OK
    with pytest.raises(sg.SgError) as exc:
        g.sync()
    assert exc.value.code == sg.SG_ERR_CHECK
    assert "inactive values 1" in str(exc.value)
    g.close()


def test_poke_rejects_out_of_range_targets():
    import paper_2012_08141_gb300 as sg
    g = _grid()
    cap, nr = g.max_leaves, (g.res // g.L) ** 3
    bad = [(0, nr, 0), (0, 0, cap), (0, 0, (-2) & 0xffffffff), (1, (cap + 1) * g.W, 0),
           (2, (cap + 1) * g.V, 0), (5, 0, 0), (-1, 0, 0), (2, -1, 0)]
    for arr, idx, bits in bad:
        assert g.lib.sg_debug_poke(g.h, arr, idx, bits) == sg.SG_ERR_INVALID, (arr, idx, bits)
    assert _violations(g.check()) == CLEAN
    g.close()
