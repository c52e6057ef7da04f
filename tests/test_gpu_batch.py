"""GPU tests of the batched fused step (many grids, one persistent launch per
step, CUDA graph) and of the device-side counter-based fill: each grid's
result in the batch equals the same grid stepped alone (within the stencil
tolerance) and, for small grids, the FP64 oracle."""
import numpy as np
import pytest

import oracle
from sgtest import mask_bits, rel_linf
from workload import batched_mix, leaf_values

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def sgm():
    import paper_2012_08141_gb300 as sg
    return sg


def leaves_needed(spec):
    sg = sgm()
    R = spec.N // spec.L
    p = sg.Grid(spec.N, 3, 1, max_leaves=R ** 3)
    p.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    n = p.num_leaves()
    p.close()
    return n


def make_grid(spec, n_leaves, opts=15):
    sg = sgm()
    g = sg.Grid(spec.N, 3, 3, max_leaves=max(n_leaves, 1), max_sums=4, scratch_mask=0b010)
    g.set_opts(opts)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    g.list_gen()
    g.fill_hash(0, spec.seed % (1 << 24))
    return g


def test_fill_hash_matches_host_generator():
    spec = batched_mix(3, n_grids=4, lo=1e4, hi=1e5)[2]
    g = make_grid(spec, leaves_needed(spec))
    b, m = g.read_structure()
    got = g.read_field(0)
    want = leaf_values(spec.seed % (1 << 24), spec.N, spec.L, b)
    act = mask_bits(m, 512)
    np.testing.assert_array_equal(got[act], want[act])
    assert np.all(got[~act] == 0.0)
    g.close()


def run_alone(g, steps):
    for _ in range(steps):
        g.clear(1)
        g.diffuse7(0, 1, 0.1)
        g.box27(1, 2)
        g.swap(0, 2)
        g.reduce_sum(0, 0)
    return g.read_sums(1)[0]


@pytest.mark.parametrize("staged", [False, True])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_alone_and_oracle(use_graph, staged):
    """Both halo stagings of the batched kernel (register sweep; x regions
    staged in shared memory by bulk tensor copies), with and without graphs:
    every grid's field bit-identical to the grid stepped alone, sums within
    2e-5, the two smallest grids within 2e-5 of the oracle."""
    sg = sgm()
    specs = batched_mix(7, n_grids=6, lo=1e3, hi=3e5)
    steps = 5
    batched, alone = [], []
    for s in specs:
        n = leaves_needed(s)
        batched.append(make_grid(s, n))
        alone.append(make_grid(s, n))
    bt = sg.Batch(batched, 0, 1, 2, 0.1)
    bt.set(4, use_graph)
    bt.set_staging(staged)
    assert bt.config()["staged"] == staged
    for _ in range(steps):
        bt.step()
    bsums = bt.read_sums()
    assert bt.info()["launches"] == steps
    bt.close()
    for i, s in enumerate(specs):
        ref_sum = run_alone(alone[i], steps)
        assert abs(bsums[i] - ref_sum) <= TOL * abs(ref_sum)
        # the same per-voxel arithmetic in the same order: identical fields
        np.testing.assert_array_equal(batched[i].read_field(0), alone[i].read_field(0))
    # the two smallest grids also against the oracle
    for i in np.argsort([g.num_leaves() for g in batched])[:2]:
        s = specs[i]
        og = oracle.Grid(s.N, s.L, 3)
        og.activate_shell(s.lo2, s.hi2, s.lo_strict)
        ob, _ = og.structure()
        og.write_field(0, leaf_values(s.seed % (1 << 24), s.N, s.L, ob))
        cur, y = 0, 2
        for _ in range(steps):
            og.diffuse7(cur, 1, 0.1)
            og.box27(1, y)
            cur, y = y, cur
        assert rel_linf(batched[i].read_field(0), og.read_field(cur)) <= TOL
        assert abs(bsums[i] - og.sum(cur)) <= TOL * abs(og.sum(cur))
    for g in batched + alone:
        g.close()


def test_batch_autotune_picks_a_candidate():
    """The autotuner times the register sweep at 2, 4 and 8 warps per CTA and
    the staged body, and keeps one of them."""
    sg = sgm()
    specs = batched_mix(11, n_grids=5, lo=1e3, hi=1e5)
    grids = [make_grid(s, leaves_needed(s)) for s in specs]
    bt = sg.Batch(grids, 0, 1, 2, 0.1)
    w = bt.autotune(2)
    assert w in (2, 4, 8)
    cfg = bt.config()
    assert cfg["warps_per_cta"] == w
    assert cfg["staged"] in (False, True) and (not cfg["staged"] or w == 8)
    bt.step()
    sums = bt.read_sums()
    assert np.all(np.isfinite(sums)) and np.all(sums > 0)
    bt.close()
    for g in grids:
        g.close()


def test_both_stagings_on_the_64_grid_mix():
    """The 64-grid mix of the batched workload (active sizes log-uniform in
    1e3..5e6): three steps with each halo staging on separate copies of the
    grids give bit-identical fields and sums within 2e-5; the three smallest
    grids also within 2e-5 of the oracle."""
    sg = sgm()
    specs = batched_mix(0, n_grids=64, lo=1e3, hi=5e6)
    steps = 3
    sets = []
    for staged in (False, True):
        grids = [make_grid(s, leaves_needed(s)) for s in specs]
        bt = sg.Batch(grids, 0, 1, 2, 0.1)
        bt.set_staging(staged)
        for _ in range(steps):
            bt.step()
        sets.append((grids, bt.read_sums()))
        bt.close()
    (ga, sa), (gb, sb) = sets
    np.testing.assert_allclose(sb, sa, rtol=TOL)
    for a, b in zip(ga, gb):
        np.testing.assert_array_equal(b.read_field(0), a.read_field(0))
    for i in np.argsort([g.num_leaves() for g in ga])[:3]:
        s = specs[i]
        og = oracle.Grid(s.N, s.L, 3)
        og.activate_shell(s.lo2, s.hi2, s.lo_strict)
        ob, _ = og.structure()
        og.write_field(0, leaf_values(s.seed % (1 << 24), s.N, s.L, ob))
        cur, y = 0, 2
        for _ in range(steps):
            og.diffuse7(cur, 1, 0.1)
            og.box27(1, y)
            cur, y = y, cur
        assert rel_linf(gb[i].read_field(0), og.read_field(cur)) <= TOL
    for g in ga + gb:
        g.close()


def test_batch_destroy_returns_its_device_memory():
    """A batch's descriptor blocks and the staged body's tensor maps come from
    grid 0's allocator and go back to it at destroy: after the first cycle
    (which also builds the grids' own neighbour tables and run records),
    creating, stepping with both bodies and destroying a batch over the same
    grids leaves the allocated device memory unchanged."""
    import torch
    sg = sgm()
    specs = batched_mix(12, n_grids=3, lo=1e3, hi=1e5)
    grids = [make_grid(s, leaves_needed(s)) for s in specs]

    def cycle():
        bt = sg.Batch(grids, 0, 1, 2, 0.1)
        bt.set_staging(True)
        bt.step()
        bt.set_staging(False)
        bt.step()
        assert np.all(np.isfinite(bt.read_sums()))
        bt.close()
        torch.cuda.synchronize()
        return torch.cuda.memory_allocated()

    m1 = cycle()
    assert cycle() == m1
    assert cycle() == m1
    for g in grids:
        g.close()
