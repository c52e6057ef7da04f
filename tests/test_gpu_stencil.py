"""GPU parity of the stencil path against the FP64 oracle, through the C ABI.

Structure (lists and masks) must match bit-exactly; FP32 fields within a
normwise relative L-inf of 2e-5 after the stated number of steps; the
per-step sums within 2e-5 relative."""
import numpy as np
import pytest

import oracle
from sgtest import mask_bits, rel_linf, shell_pair
from workload import ShellSpec, band_bounds, band512, leaf_values, tiny_shell

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_08141_gb300 as sg
    sg.load_library()
    yield


def sgmod():
    import paper_2012_08141_gb300 as sg
    return sg


OPTS = {
    "fused": 15,
    "eager": 0,
    "no_lgr": 15 & ~1,
    "no_ad": 15 & ~2,
    "no_fuse": 15 & ~4,
    "no_dse": 15 & ~8,
}


# ---------------------------------------------------------------------------
# 64^3 shell, 20 steps of activate -> list -> diffuse7 -> swap
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("mode", list(OPTS))
@pytest.mark.parametrize("seed", [0, 5])
def test_tiny_shell_20_steps(mode, seed, variant):
    spec = tiny_shell(seed)
    g, og = shell_pair(spec, n_fields=2, opts=OPTS[mode], variant=variant)
    ob, om = og.structure()
    cur, oth = 0, 1
    for _ in range(20):
        g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
        g.list_gen()
        g.diffuse7(0, 1, 0.1)
        g.swap(0, 1)
        og.diffuse7(cur, oth, 0.1)
        cur, oth = oth, cur
    gb, gm = g.read_structure()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gm, om)
    got = g.read_field(0)
    ref = og.read_field(cur)
    assert rel_linf(got, ref) <= TOL
    # inactive voxels hold exactly 0
    assert np.all(got[~mask_bits(gm, 512)] == 0.0)
    g.close()


# ---------------------------------------------------------------------------
# Band workload: clear(t), diffuse7(x->t), box27(t->y), swap(x,y), sum(x)
# ---------------------------------------------------------------------------

def run_band(g, og, steps, slot0=0):
    cur, y = 0, 2
    sums_ref = []
    for s in range(steps):
        g.clear(1)
        g.diffuse7(0, 1, 0.1)
        g.box27(1, 2)
        g.swap(0, 2)
        g.reduce_sum(0, slot0 + s)
        og.clear(1)
        og.diffuse7(cur, 1, 0.1)
        og.box27(1, y)
        cur, y = y, cur
        sums_ref.append(og.sum(cur))
    return cur, np.array(sums_ref)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("mode", list(OPTS))
def test_band_128_100_steps(mode, variant):
    lo2, hi2 = band_bounds(40.0, 56.0)
    spec = ShellSpec(128, 8, lo2, hi2, True, 3)
    g, og = shell_pair(spec, n_fields=3, opts=OPTS[mode], scratch_mask=0b010, variant=variant)
    cur, sums_ref = run_band(g, og, 100)
    sums = g.read_sums(100)
    assert np.max(np.abs(sums - sums_ref) / np.abs(sums_ref)) <= TOL
    assert rel_linf(g.read_field(0), og.read_field(cur)) <= TOL
    if mode in ("fused", "no_dse"):
        assert g.stats()["ops_fused"] >= 100
    g.close()


def test_band512_full_size_fused_and_eager():
    """The full 512^3 band (26,104 leaves): 100 steps fused (register-sweep,
    TMA-staged kernels) and eager, every per-step sum and the final field
    compared with one oracle run."""
    spec = band512()
    og = oracle.Grid(spec.N, spec.L, 3)
    og.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    ob, om = og.structure()
    assert len(ob) == 26104
    og.write_field(0, leaf_values(spec.seed, spec.N, spec.L, ob))
    grids = {}
    for mode in ("fused", "eager", "fused_tma"):
        sg = sgmod()
        g = sg.Grid(spec.N, 3, 3, max_leaves=32768, max_sums=100, scratch_mask=0b010)
        g.set_opts(OPTS[mode.split("_")[0]])
        g.set_stencil_variant(sg.SG_VARIANT_SWEEP_TMA if mode == "fused_tma" else sg.SG_VARIANT_SWEEP_JRUNS)
        g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
        g.list_gen()
        gb, gm = g.read_structure()
        np.testing.assert_array_equal(gb, ob)
        np.testing.assert_array_equal(gm, om)
        g.write_field(0, leaf_values(spec.seed, spec.N, spec.L, gb))
        grids[mode] = g
    cur, y = 0, 2
    sums_ref = []
    for s in range(100):
        for g in grids.values():
            g.clear(1)
            g.diffuse7(0, 1, 0.1)
            g.box27(1, 2)
            g.swap(0, 2)
            g.reduce_sum(0, s)
            g.flush()
        og.diffuse7(cur, 1, 0.1)
        og.box27(1, y)
        cur, y = y, cur
        sums_ref.append(og.sum(cur))
    sums_ref = np.array(sums_ref)
    ref = og.read_field(cur)
    for mode, g in grids.items():
        sums = g.read_sums(100)
        assert np.max(np.abs(sums - sums_ref) / np.abs(sums_ref)) <= TOL, mode
        assert rel_linf(g.read_field(0), ref) <= TOL, mode
        g.close()


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def test_empty_grid():
    sg = sgmod()
    g = sg.Grid(64, 3, 3, max_leaves=16, max_sums=2)
    g.list_gen()
    assert g.num_leaves() == 0
    g.clear(1)
    g.diffuse7(0, 1, 0.1)
    g.box27(1, 2)
    g.reduce_sum(2, 0)
    g.diffuse7(0, 1, 0.1)
    g.reduce_sum(1, 1)
    np.testing.assert_array_equal(g.read_sums(2), [0.0, 0.0])
    b, m = g.read_structure()
    assert b.size == 0 and m.shape == (0, 16)
    g.close()


@pytest.mark.parametrize("N,r0,r1,strict", [(40, 4.0, 17.0, False),   # R=5: 125 root cells, ragged tile
                                             (8, 0.0, 3.0, False),     # a single leaf
                                             (200, 60.0, 99.0, True)]) # 15,625 cells, tail tile, leaves on the border
def test_ragged_domains(N, r0, r1, strict):
    lo2, hi2 = band_bounds(r0, r1)
    spec = ShellSpec(N, 8, lo2, hi2, strict, 11)
    for mode, variant in [("fused", 0), ("eager", 0), ("fused", 1), ("eager", 1), ("fused", 2), ("fused", 3), ("eager", 3),
                          ("fused", 4)]:
        g, og = shell_pair(spec, n_fields=3, opts=OPTS[mode], scratch_mask=0b010, variant=variant)
        cur, sums_ref = run_band(g, og, 7)
        assert rel_linf(g.read_field(0), og.read_field(cur)) <= TOL
        sums = g.read_sums(7)
        assert np.max(np.abs(sums - sums_ref) / np.maximum(np.abs(sums_ref), 1e-30)) <= TOL
        g.close()


def test_full_domain_boundary_reads_zero():
    """Every voxel active: out-of-domain neighbours read 0 at all six faces."""
    spec = ShellSpec(24, 8, 0, 10 ** 9, False, 2)
    for mode, variant in [("fused", 0), ("eager", 0), ("fused", 1), ("eager", 1), ("fused", 2), ("fused", 3), ("eager", 3),
                          ("fused", 4)]:
        g, og = shell_pair(spec, n_fields=3, opts=OPTS[mode], variant=variant)
        cur, _ = run_band(g, og, 5)
        assert rel_linf(g.read_field(0), og.read_field(cur)) <= TOL
        g.close()


def test_activate_coords_parity():
    sg = sgmod()
    import torch
    rng = np.random.default_rng(4)
    xyz = rng.integers(-3, 99, size=(5000, 3)).astype(np.int32)   # some outside the 96^3 domain
    g = sg.Grid(96, 3, 2, max_leaves=2048)
    og = oracle.Grid(96, 8, 2)
    g.activate_coords(torch.from_numpy(xyz).cuda())
    og.activate_coords(xyz)
    gb, gm = g.read_structure()
    ob, om = og.structure()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gm, om)
    # a second batch: new bits in existing leaves and new leaves
    xyz2 = rng.integers(0, 96, size=(3000, 3)).astype(np.int32)
    g.activate_coords(torch.from_numpy(xyz2).cuda())
    og.activate_coords(xyz2)
    g.diffuse7(0, 1, 0.1)
    gb, gm = g.read_structure()
    ob, om = og.structure()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gm, om)
    g.close()


def test_activation_zero_fills_after_values():
    """A voxel activated after its leaf holds values reads 0 (Sec. 3.2)."""
    sg = sgmod()
    import torch
    g = sg.Grid(16, 3, 2, max_leaves=8)
    g.activate_coords(torch.tensor([[1, 2, 3], [4, 4, 4]], dtype=torch.int32, device="cuda"))
    g.list_gen()
    n = g.num_leaves()
    g.write_field(0, np.full((n, 512), 5.0, dtype=np.float32))
    g.activate_coords(torch.tensor([[1, 2, 4], [9, 9, 9]], dtype=torch.int32, device="cuda"))
    b, m = g.read_structure()
    vals = g.read_field(0)
    act = mask_bits(m, 512)
    assert act.sum() == 4
    assert sorted(vals[act].tolist()) == [0.0, 0.0, 5.0, 5.0]
    assert np.all(vals[~act] == 0.0)
    g.close()


def test_activation_fill_elimination_on_reused_slots():
    """After a deactivation the pool's slots still hold the old values.  With
    dead-store elimination a re-activation zero-fills a new leaf only in the
    fields the queue reads (or leaves alone) before overwriting them; every
    non-scratch field then holds exactly what the ops wrote: 0 at inactive
    voxels, the written values at active ones, zeros where it was read
    first.  Without DSE every field is filled; the results are the same."""
    sg = sgmod()
    A = band_bounds(12.0, 20.0)
    B = band_bounds(13.0, 21.0)
    for opts in (15, 15 & ~8):
        g = sg.Grid(64, 3, 4, max_leaves=512, scratch_mask=0b0010)
        g.set_opts(opts)
        g.activate_shell(A[0], A[1], True)
        for f in range(4):
            g.ew(f, delta=7.0)                     # stale values in every field's slots
        g.sync()
        g.deactivate_all()
        g.activate_shell(B[0], B[1], True)        # the same slots, other cells
        g.ew(2, delta=3.0)                         # 2 overwritten first: its fill is dead
        g.diffuse7(0, 3, 0.1)                      # 0 read first (filled); 3 overwritten
        g.sync()
        b, m = g.read_structure()
        act = mask_bits(m, 512)
        assert act.sum() > 0
        v0, v2, v3 = g.read_field(0), g.read_field(2), g.read_field(3)
        assert np.all(v0 == 0.0)
        assert np.all(v2[act] == 3.0) and np.all(v2[~act] == 0.0)
        assert np.all(v3 == 0.0)
        g.close()


def test_deactivate_and_reactivate():
    spec = tiny_shell(1)
    g, og = shell_pair(spec, n_fields=2)
    g.deactivate_all()
    assert g.num_leaves() == 0
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    b, m = g.read_structure()
    ob, om = og.structure()
    np.testing.assert_array_equal(b, ob)
    np.testing.assert_array_equal(m, om)
    assert np.all(g.read_field(0) == 0.0)      # fresh leaves are zero-filled
    g.close()


def test_pool_exhaustion_is_reported_and_grid_recovers():
    sg = sgmod()
    spec = tiny_shell(0)                    # 248 leaves
    g = sg.Grid(64, 3, 2, max_leaves=100)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    with pytest.raises(sg.SgError) as e:
        g.sync()
    assert e.value.code == sg.SG_ERR_POOL_EXHAUSTED
    g.deactivate_all()
    lo2, hi2 = band_bounds(0.0, 10.0)
    g.activate_shell(lo2, hi2, False)
    g.sync()
    assert 0 < g.num_leaves() <= 100
    g.close()


def test_bounded_wait_reports_timeout():
    """A device wait on a flag that nothing sets gives up, the next sync
    returns SG_ERR_TIMEOUT, and the grid keeps working."""
    sg = sgmod()
    spec = tiny_shell(2)
    g, og = shell_pair(spec, n_fields=2)
    g.debug_wait_test()
    with pytest.raises(sg.SgError) as e:
        g.sync()
    assert e.value.code == sg.SG_ERR_TIMEOUT
    g.diffuse7(0, 1, 0.1)
    og.diffuse7(0, 1, 0.1)
    assert rel_linf(g.read_field(1), og.read_field(1)) <= TOL
    g.close()


def test_generic_leaf4_stencils():
    """4^3 leaves run the generic kernels (tree-walk reads)."""
    lo2, hi2 = band_bounds(6.0, 13.0)
    spec = ShellSpec(32, 4, lo2, hi2, False, 8)
    for mode in ("fused", "eager"):
        g, og = shell_pair(spec, n_fields=3, opts=OPTS[mode], scratch_mask=0b010)
        cur, sums_ref = run_band(g, og, 10)
        assert rel_linf(g.read_field(0), og.read_field(cur)) <= TOL
        assert np.max(np.abs(g.read_sums(10) - sums_ref) / np.abs(sums_ref)) <= TOL
        g.close()


def test_scratch_intermediate_kept_when_read_later():
    lo2, hi2 = band_bounds(10.0, 20.0)
    spec = ShellSpec(48, 8, lo2, hi2, False, 9)
    g, og = shell_pair(spec, n_fields=3, scratch_mask=0b010)
    g.diffuse7(0, 1, 0.1)
    g.box27(1, 2)
    g.reduce_sum(1, 0)      # reads the scratch intermediate: it must be stored
    og.diffuse7(0, 1, 0.1)
    og.box27(1, 2)
    s = g.read_sums(1)[0]
    assert abs(s - og.sum(1)) <= TOL * abs(og.sum(1))
    assert rel_linf(g.read_field(2), og.read_field(2)) <= TOL
    g.close()


@pytest.mark.parametrize("L", [8, 4])
def test_maximum_resolution_sparse_clusters(L):
    """The largest domain the library accepts (4096^3: 512^3 or 1024^3 root
    cells): clusters of voxels at the eight corners, on faces and edges and at
    the centre, activated from coordinates; structure bit-exact and five fused
    and eager steps within tolerance of the oracle."""
    sg = sgmod()
    import torch
    N = 4096
    rng = np.random.default_rng(17)
    boxes = [(a, b, c) for a in (0, N - 20) for b in (0, N - 20) for c in (0, N - 20)]
    boxes += [(N // 2 - 10, N // 2 - 10, N // 2 - 10), (0, N // 2 - 10, N // 2 - 10), (N - 20, 7, N // 2 + 3)]
    xyz = np.concatenate([np.array(o) + rng.integers(0, 20, size=(400, 3)) for o in boxes]).astype(np.int32)
    assert xyz.min() >= 0 and xyz.max() < N
    lg = int(np.log2(L))
    for opts in (sg.SG_OPT_ALL, sg.SG_OPT_EAGER):
        g = sg.Grid(N, lg, 3, max_leaves=8192, max_sums=5, scratch_mask=0b010)
        g.set_opts(opts)
        og = oracle.Grid(N, L, 3)
        g.activate_coords(torch.from_numpy(xyz).cuda())
        og.activate_coords(xyz)
        gb, gm = g.read_structure()
        ob, om = og.structure()
        np.testing.assert_array_equal(gb, ob)
        np.testing.assert_array_equal(gm, om)
        vals = leaf_values(9, N, L, gb)
        g.write_field(0, vals)
        og.write_field(0, vals)
        cur, sums_ref = run_band(g, og, 5)
        assert rel_linf(g.read_field(0), og.read_field(cur)) <= TOL
        sums = g.read_sums(5)
        assert np.max(np.abs(sums - sums_ref) / np.maximum(np.abs(sums_ref), 1e-30)) <= TOL
        g.close()
        del og


@pytest.mark.parametrize("grouped", ["columns", "jruns", "tma"])
@pytest.mark.parametrize("store_t", [False, True])
def test_grouped_sweeps_equal_leaf_sweep(store_t, grouped):
    """The column sweep (runs of leaves adjacent in i swept in one pass), the
    j-run sweep (a warp's leaves taken from runs adjacent in j), the same
    j-run tasks with every x row staged in shared memory by bulk tensor copies,
    and the leaf-triple sweep run the same arithmetic per voxel: fields after
    five fused steps on the 512^3 band are bit-identical, sums agree to FP32
    partial-sum rounding; with the intermediate stored (not scratch) that field
    is bit-identical too."""
    sg = sgmod()
    spec = band512()
    grids = []
    first = {"columns": sg.SG_VARIANT_SWEEP_COLUMNS, "jruns": sg.SG_VARIANT_SWEEP_JRUNS,
             "tma": sg.SG_VARIANT_SWEEP_TMA}[grouped]
    for variant in (first, sg.SG_VARIANT_SWEEP):
        g = sg.Grid(spec.N, 3, 3, max_leaves=32768, max_sums=5, scratch_mask=0 if store_t else 0b010)
        g.set_stencil_variant(variant)
        g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
        g.fill_hash(0, 41)
        grids.append(g)
    for s in range(5):
        for g in grids:
            g.clear(1)
            g.diffuse7(0, 1, 0.1)
            g.box27(1, 2)
            g.swap(0, 2)
            g.reduce_sum(0, s)
            if store_t:
                g.reduce_sum(1, s)   # reads t later: the intermediate is stored
            g.flush()
    a, b = grids
    np.testing.assert_array_equal(a.read_field(0), b.read_field(0))
    if store_t:
        np.testing.assert_array_equal(a.read_field(1), b.read_field(1))
    np.testing.assert_allclose(a.read_sums(5), b.read_sums(5), rtol=1e-6)
    for g in grids:
        g.close()


@pytest.mark.parametrize("mode", ["no_fuse", "no_fuse_no_ad"])
def test_single_jruns_equal_leaf_sweep(mode):
    """Without fusion the stencils run one by one; on a large reused list they
    sweep j-runs from the third stencil on (k_sweep_single_jruns: x-only outer
    lanes, no edge rows), under the leaf-triple variant k_sweep_single.  Each
    output takes the same operands in the same order, so six steps on the
    512^3 band give bit-identical fields and sums; without activation demotion
    every written row is also checked against the mask (the kernels' checking
    instances)."""
    sg = sgmod()
    spec = band512()
    opts = 15 & ~4 if mode == "no_fuse" else 15 & ~6
    grids = []
    for variant in (sg.SG_VARIANT_SWEEP_JRUNS, sg.SG_VARIANT_SWEEP):
        g = sg.Grid(spec.N, 3, 3, max_leaves=32768, max_sums=6, scratch_mask=0b010)
        g.set_opts(opts)
        g.set_stencil_variant(variant)
        g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
        g.fill_hash(0, 43)
        g.sync()                                  # the leaf count the switch looks at
        grids.append(g)
    for s in range(6):
        for g in grids:
            g.clear(1)
            g.diffuse7(0, 1, 0.1)
            g.box27(1, 2)
            g.swap(0, 2)
            g.reduce_sum(0, s)
            g.flush()
    a, b = grids
    assert a.stats()["launches"] == b.stats()["launches"] + 1   # the run records, built once
    np.testing.assert_array_equal(a.read_field(0), b.read_field(0))
    np.testing.assert_array_equal(a.read_field(1), b.read_field(1))
    np.testing.assert_array_equal(a.read_sums(6), b.read_sums(6))
    for g in grids:
        g.close()


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_fused_steps_across_structure_changes(variant):
    """Fused steps; a wider band activated (new leaves, new bits in listed
    leaves, zero-filled); fused steps; everything deactivated and a third band
    activated and filled; fused steps.  Structure bit-exact and fields and
    sums within tolerance of the oracle at every stage, so the list, region
    masks and run records cached with the list follow every change."""
    sg = sgmod()
    N = 128
    A, B, C = band_bounds(40.0, 46.0), band_bounds(36.0, 52.0), band_bounds(20.0, 30.0)
    spec = ShellSpec(N, 8, A[0], A[1], False, 13)
    g, og = shell_pair(spec, n_fields=3, scratch_mask=0b010, variant=variant, max_leaves=(N // 8) ** 3)
    state = {"cur": 0, "slot": 0, "ref": []}

    def steps(n):
        for _ in range(n):
            y = 2 if state["cur"] == 0 else 0
            g.clear(1)
            g.diffuse7(0, 1, 0.1)
            g.box27(1, 2)
            g.swap(0, 2)
            g.reduce_sum(0, state["slot"])
            og.clear(1)
            og.diffuse7(state["cur"], 1, 0.1)
            og.box27(1, y)
            state["cur"] = y
            state["ref"].append(og.sum(y))
            state["slot"] += 1

    def check():
        gb, gm = g.read_structure()
        ob, om = og.structure()
        np.testing.assert_array_equal(gb, ob)
        np.testing.assert_array_equal(gm, om)
        got = g.read_field(0)
        assert rel_linf(got, og.read_field(state["cur"])) <= TOL
        assert np.all(got[~mask_bits(gm, 512)] == 0.0)
        sums = g.read_sums(state["slot"])
        ref = np.array(state["ref"])
        assert np.max(np.abs(sums - ref) / np.maximum(np.abs(ref), 1e-30)) <= TOL

    steps(3)
    check()
    n0 = g.num_leaves()
    g.activate_shell(B[0], B[1], False)
    og.activate_shell(B[0], B[1], False)
    assert g.num_leaves() > n0
    steps(3)
    check()
    g.deactivate_all()
    og.deactivate_all()
    g.activate_shell(C[0], C[1], False)
    og.activate_shell(C[0], C[1], False)
    gb, _ = g.read_structure()
    ob, _ = og.structure()
    g.write_field(0, leaf_values(17, N, 8, gb))
    og.write_field(state["cur"], leaf_values(17, N, 8, ob))
    steps(3)
    check()
    g.close()
