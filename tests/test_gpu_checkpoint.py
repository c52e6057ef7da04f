"""GPU tests of checkpoint and restore (sg_write_structure + sg_write_field
behind paper_2012_08141_gb300.checkpoint): a restored grid has the saved
structure bit-exact, the saved fields bit-exact, and time steps continued from
it give bit-identical fields, and sums equal to FP64 rounding, to the
original grid's."""
import numpy as np
import pytest

import oracle
from workload import leaf_values, tiny_shell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _stepped(L, seed=4):
    import paper_2012_08141_gb300 as sg
    spec = tiny_shell(seed, N=64, L=L)
    g = sg.Grid(spec.N, int(np.log2(L)), 3, max_leaves=(64 // L) ** 3, max_sums=2)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    b, _ = g.read_structure()
    g.write_field(0, leaf_values(seed, spec.N, L, b))
    g.diffuse7(0, 1, 0.1)
    g.box27(1, 2)
    g.diffuse7(2, 0, 0.05)
    return spec, g


def _continue(g):
    g.diffuse7(0, 1, 0.1)
    g.box27(1, 2)
    g.reduce_sum(2, 0)
    g.diffuse7(2, 0, 0.1)
    g.reduce_sum(0, 1)


def _same(a, b, fields):
    ab, am = a.read_structure()
    bb, bm = b.read_structure()
    np.testing.assert_array_equal(ab, bb)
    np.testing.assert_array_equal(am, bm)
    for f in fields:
        np.testing.assert_array_equal(a.read_field(f), b.read_field(f))


@pytest.mark.parametrize("L", [8, 4])
def test_round_trip_then_identical_steps(L, tmp_path):
    from paper_2012_08141_gb300 import checkpoint
    spec, g = _stepped(L)
    path = tmp_path / "ck.npz"
    checkpoint.save(g, path)
    h = checkpoint.load(path, max_sums=2)
    _same(g, h, range(3))
    og = oracle.Grid(spec.N, L, 1)               # the restored structure is the shell's, by definition
    og.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    ob, om = og.structure()
    hb, hm = h.read_structure()
    np.testing.assert_array_equal(hb, ob)
    np.testing.assert_array_equal(hm, om)
    for grid in (g, h):
        _continue(grid)
    _same(g, h, range(3))
    np.testing.assert_allclose(g.read_sums(2), h.read_sums(2), rtol=1e-12)   # FP64 partials
    g.close()
    h.close()


def test_restore_replaces_an_existing_structure(tmp_path):
    """Restoring into a grid that holds another shell drops its leaves and
    values; fields left out of the checkpoint read 0; a later activation of the
    saved shell is launched (not demoted) and changes nothing."""
    import paper_2012_08141_gb300 as sg
    from paper_2012_08141_gb300 import checkpoint
    spec, g = _stepped(8)
    path = tmp_path / "ck.npz"
    checkpoint.save(g, path, fields=[0, 2])
    other = tiny_shell(9, N=64, L=8)
    h = sg.Grid(64, 3, 3, max_leaves=512, max_sums=2)
    h.activate_shell(other.lo2 // 2, other.hi2 * 2, False)
    h.fill_hash(0, 3)
    h.fill_hash(1, 4)
    assert h.num_leaves() != g.num_leaves()
    checkpoint.restore(h, path)
    _same(g, h, [0, 2])
    assert not h.read_field(1).any()
    d0 = h.stats()["act_demoted"]
    h.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    h.flush()
    assert h.stats()["act_demoted"] == d0
    _same(g, h, [0, 2])
    g.close()
    h.close()


def test_empty_and_maskless_leaves(tmp_path):
    """An empty structure restores to an empty grid; leaves whose masks are all
    zero are kept (allocated, no active voxel) and listed in order."""
    import paper_2012_08141_gb300 as sg
    g = sg.Grid(64, 3, 1, max_leaves=512)
    g.fill_hash(0, 1)
    g.write_structure(np.zeros(0, np.int32), np.zeros((0, g.W), np.uint32))
    assert g.num_leaves() == 0 and g.num_active() == 0
    b = np.array([0, 7, 64, 511], np.int32)
    m = np.zeros((4, g.W), np.uint32)
    m[1, 3] = 0x80000001
    m[3, g.W - 1] = 0xffffffff
    g.write_structure(b, m)
    gb, gm = g.read_structure()
    np.testing.assert_array_equal(gb, b)
    np.testing.assert_array_equal(gm, m)
    assert g.num_active() == 34
    g.fill_hash(0, 2)
    v = g.read_field(0)
    bits = np.unpackbits(m.view(np.uint8), bitorder="little").reshape(4, g.V).astype(bool)
    assert (v[~bits] == 0).all() and (v[bits] > 0).sum() >= 30
    g.close()


def test_too_many_leaves_leaves_the_grid_unchanged(tmp_path):
    import paper_2012_08141_gb300 as sg
    from paper_2012_08141_gb300 import checkpoint
    spec, g = _stepped(8)
    path = tmp_path / "ck.npz"
    checkpoint.save(g, path)
    small = sg.Grid(64, 3, 3, max_leaves=8)
    import torch
    small.activate_coords(torch.tensor([[1, 2, 3]], dtype=torch.int32).cuda())
    small.fill_hash(0, 5)
    before_b, before_m = small.read_structure()
    before_v = small.read_field(0)
    with pytest.raises(sg.SgError) as e:
        checkpoint.restore(small, path)
    assert e.value.code == sg.SG_ERR_POOL_EXHAUSTED
    b, m = small.read_structure()
    np.testing.assert_array_equal(b, before_b)
    np.testing.assert_array_equal(m, before_m)
    np.testing.assert_array_equal(small.read_field(0), before_v)
    with pytest.raises(ValueError):
        checkpoint.restore(sg.Grid(32, 3, 3, max_leaves=64), path)   # another resolution
    g.close()
    small.close()


def test_band512_round_trip(tmp_path):
    """The 512^3 band (26,104 leaves of 8^3): structure and a hashed field
    round-trip bit-exact; one fused step from each gives the same sum."""
    import paper_2012_08141_gb300 as sg
    from paper_2012_08141_gb300 import checkpoint
    from workload import band512
    spec = band512()
    g = sg.Grid(512, 3, 3, max_leaves=32768, max_sums=1, scratch_mask=0b010)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    g.fill_hash(0, 17)
    path = tmp_path / "band.npz"
    checkpoint.save(g, path, fields=[0])
    h = checkpoint.load(path, max_sums=1, scratch_mask=0b010)
    _same(g, h, [0])
    for grid in (g, h):
        grid.diffuse7(0, 1, 0.1)
        grid.box27(1, 2)
        grid.reduce_sum(2, 0)
    np.testing.assert_allclose(g.read_sums(1), h.read_sums(1), rtol=1e-12)
    np.testing.assert_array_equal(g.read_field(2), h.read_field(2))
    g.close()
    h.close()


@pytest.mark.parametrize("L", [8, 4])
def test_pinned_transfers_equal_pageable(L):
    """Field writes and reads through mapped pinned host buffers (read and
    written in place by the transfer kernels) give the same values as through
    pageable buffers (staged copies), for aligned and unaligned pinned views."""
    import torch
    import paper_2012_08141_gb300 as sg
    spec = tiny_shell(6, N=64, L=L)
    g = sg.Grid(64, int(np.log2(L)), 2, max_leaves=(64 // L) ** 3)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    b, _ = g.read_structure()
    vals = leaf_values(6, 64, L, b)
    g.write_field(0, vals)                                  # pageable: staged
    pinned = torch.empty(vals.size + 1, dtype=torch.float32).pin_memory()
    pinned[:vals.size] = torch.from_numpy(vals.reshape(-1))
    g.write_field(1, pinned[:vals.size])                    # pinned, aligned: in place
    np.testing.assert_array_equal(g.read_field(0), g.read_field(1))
    out = torch.zeros(vals.size + 1, dtype=torch.float32).pin_memory()
    g.read_field(1, out=out[:vals.size].numpy().reshape(vals.shape))
    np.testing.assert_array_equal(out[:vals.size].numpy().reshape(vals.shape), g.read_field(0))
    shifted = torch.empty(vals.size + 1, dtype=torch.float32).pin_memory()
    shifted[1:] = torch.from_numpy(vals.reshape(-1))
    g.write_field(1, shifted[1:])                           # 4-byte aligned view: staged
    np.testing.assert_array_equal(g.read_field(0), g.read_field(1))
    g.close()


def _bits(m, V):
    n = m.shape[0]
    return np.unpackbits(m.view(np.uint8), bitorder="little").reshape(n, V).astype(bool)


@pytest.mark.parametrize("L", [8, 4])
def test_active_value_transfers(L):
    """Writes and reads of the active voxels only (list order, then mask-bit
    order) agree bit-exactly with the dense transfers, through pageable and
    mapped pinned buffers; a wrong count is refused."""
    import torch
    import paper_2012_08141_gb300 as sg
    spec = tiny_shell(7, N=64, L=L)
    g = sg.Grid(64, int(np.log2(L)), 2, max_leaves=(64 // L) ** 3)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    b, m = g.read_structure()
    vals = leaf_values(7, 64, L, b)
    packed = vals[_bits(m, g.V)]
    assert packed.size == g.num_active()
    g.write_field_active(0, packed)                     # pageable: staged
    g.write_field(1, vals)
    np.testing.assert_array_equal(g.read_field(0), g.read_field(1))
    np.testing.assert_array_equal(g.read_field_active(0), packed)
    pin = torch.from_numpy(packed).pin_memory()
    g.fill_hash(0, 3)
    g.write_field_active(0, pin)                        # pinned: read in place
    np.testing.assert_array_equal(g.read_field(0), g.read_field(1))
    out = torch.zeros(packed.size, dtype=torch.float32).pin_memory()
    np.testing.assert_array_equal(g.read_field_active(1, out=out.numpy()), packed)
    with pytest.raises(sg.SgError) as e:
        g.write_field_active(0, packed[:-1])
    assert e.value.code == sg.SG_ERR_INVALID
    with pytest.raises(sg.SgError):
        g.read_field_active(0, out=np.empty(packed.size - 1, np.float32))
    np.testing.assert_array_equal(g.read_field(0), g.read_field(1))   # the refused write changed nothing
    # the structure changes: the packed order follows it
    g.activate_coords(torch.tensor([[0, 0, 0], [63, 63, 63], [31, 32, 33]], dtype=torch.int32).cuda())
    b2, m2 = g.read_structure()
    assert g.num_active() > packed.size
    with pytest.raises(sg.SgError):
        g.write_field_active(0, packed)
    dense = leaf_values(8, 64, L, b2)
    g.write_field(1, dense)
    np.testing.assert_array_equal(g.read_field_active(1), dense[_bits(m2, g.V)])
    g.write_field_active(0, dense[_bits(m2, g.V)])
    np.testing.assert_array_equal(g.read_field(0), g.read_field(1))
    g.close()


def test_active_value_transfers_band512_and_empty():
    """26,104 leaves (26 scan tiles): the packed read equals the dense read at
    the set bits; an empty grid transfers nothing."""
    import paper_2012_08141_gb300 as sg
    from workload import band512
    spec = band512()
    g = sg.Grid(512, 3, 1, max_leaves=32768)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    g.fill_hash(0, 23)
    b, m = g.read_structure()
    packed = g.read_field_active(0)
    assert packed.size == 8047608
    np.testing.assert_array_equal(packed, g.read_field(0)[_bits(m, g.V)])
    g.write_field_active(0, packed[::-1].copy())
    np.testing.assert_array_equal(g.read_field_active(0), packed[::-1])
    g.close()
    e = sg.Grid(64, 3, 1, max_leaves=8)
    assert e.read_field_active(0).size == 0
    e.write_field_active(0, np.zeros(0, np.float32))
    e.close()


def test_staged_uploads_overlap_and_match():
    """Staged uploads (copy on the grid's copy stream, scatter queued) give the
    same fields as synchronous active-value writes in a pipelined loop where
    the next input is staged while the current step runs; a count that no
    longer matches the structure and a replaced ticket are refused."""
    import torch
    import paper_2012_08141_gb300 as sg
    spec = tiny_shell(12, N=64, L=8)
    mk = lambda: sg.Grid(64, 3, 3, max_leaves=512, max_sums=1, scratch_mask=0b010)
    a, b = mk(), mk()
    for g in (a, b):
        g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    n = a.num_active()
    rng = np.random.default_rng(12)
    inputs = [torch.from_numpy(rng.random(n, dtype=np.float32)).pin_memory() for _ in range(4)]
    t = a.stage_active(inputs[0])
    for s in range(4):
        a.write_field_staged(0, t)
        a.diffuse7(0, 1, 0.1)
        a.box27(1, 2)
        a.reduce_sum(2, 0)
        a.flush()
        if s + 1 < 4:
            t = a.stage_active(inputs[s + 1])          # overlaps the step just queued
        got = a.read_sums(1)
        b.write_field_active(0, inputs[s])
        b.diffuse7(0, 1, 0.1)
        b.box27(1, 2)
        b.reduce_sum(2, 0)
        np.testing.assert_array_equal(got, b.read_sums(1))
        np.testing.assert_array_equal(a.read_field(2), b.read_field(2))
    # a ticket whose slot was refilled is refused
    t1 = a.stage_active(inputs[0])
    a.stage_active(inputs[1])
    a.stage_active(inputs[2])                          # same slot as t1
    with pytest.raises(sg.SgError):
        a.write_field_staged(0, t1)
    # the structure changes between staging and writing: refused at the flush
    before = a.read_field(0)
    t2 = a.stage_active(inputs[3])
    a.activate_coords(torch.tensor([[1, 1, 1]], dtype=torch.int32).cuda())
    a.write_field_staged(0, t2)
    with pytest.raises(sg.SgError) as e:
        a.sync()
    assert e.value.code == sg.SG_ERR_INVALID
    after = a.read_field(0)                            # field 0 unchanged; the new voxel reads 0
    assert after.astype(np.float64).sum() == before.astype(np.float64).sum()
    assert np.count_nonzero(after) == np.count_nonzero(before)
    a.close()
    b.close()
