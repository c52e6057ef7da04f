"""GPU parity of restriction (y[i // 2] += w x[i] with activation on write) and
prolongation (x[i] += w y[i // 2]) between a grid and its half-edge grid,
against the FP64 oracle: coarse structure bit-exact, fields within 2e-5
normwise relative L-inf; the demoted repeat (activation demotion, Sec. 6.3)
gives the same result as an activating one."""
import numpy as np
import pytest

import oracle
from sgtest import rel_linf
from workload import band_bounds, leaf_values

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _pair(N, L, r0, r1, seed, opts=None):
    """A fine shell grid with seeded values in field 0 on both sides, and an
    empty coarse grid of half the edge."""
    import paper_2012_08141_gb300 as sg
    lo2, hi2 = band_bounds(r0, r1)
    lg = int(np.log2(L))
    fine, coarse = sg.Grid(N, lg, 2, max_leaves=(N // L) ** 3), sg.Grid(N // 2, lg, 2, max_leaves=(N // L) ** 3)
    if opts is not None:
        coarse.set_opts(opts)
    ofine, ocoarse = oracle.Grid(N, L, 2), oracle.Grid(N // 2, L, 2)
    fine.activate_shell(lo2, hi2, False)
    ofine.activate_shell(lo2, hi2, False)
    b, _ = fine.read_structure()
    vals = leaf_values(seed, N, L, b)
    fine.write_field(0, vals)
    ofine.write_field(0, vals)
    return fine, coarse, ofine, ocoarse


def _compare(g, og, fields):
    gb, gm = g.read_structure()
    ob, om = og.structure()
    np.testing.assert_array_equal(gb, ob)
    np.testing.assert_array_equal(gm, om)
    for f in fields:
        assert rel_linf(g.read_field(f), og.read_field(f)) <= TOL, f


@pytest.mark.parametrize("L", [8, 4])
def test_restrict_then_demoted_repeat(L):
    fine, coarse, ofine, ocoarse = _pair(64, L, 10.0, 22.0, seed=5)
    fine.restrict_to(coarse, 0, 1, 0.125)
    ofine.restrict_to(ocoarse, 0, 1, 0.125)
    _compare(coarse, ocoarse, [1])
    before = coarse.stats()["act_demoted"]
    fine.restrict_to(coarse, 0, 1, 0.125)          # fine mask unchanged: demoted
    ofine.restrict_to(ocoarse, 0, 1, 0.125)
    assert coarse.stats()["act_demoted"] == before + 1
    _compare(coarse, ocoarse, [1])
    fine.close()
    coarse.close()


@pytest.mark.parametrize("L", [8, 4])
def test_prolong(L):
    fine, coarse, ofine, ocoarse = _pair(64, L, 10.0, 22.0, seed=6)
    fine.restrict_to(coarse, 0, 1, 0.125)
    ofine.restrict_to(ocoarse, 0, 1, 0.125)
    fine.prolong_from(coarse, 1, 0, 0.5)
    ofine.prolong_from(ocoarse, 1, 0, 0.5)
    _compare(fine, ofine, [0])
    fine.close()
    coarse.close()


def test_three_level_chain_and_partial_coarse():
    """64 -> 32 -> 16 restriction chain; then prolongation from a coarse grid
    whose structure covers only part of the fine one (absent coarse voxels
    read 0)."""
    import paper_2012_08141_gb300 as sg
    f0, c1, of0, oc1 = _pair(64, 8, 6.0, 30.0, seed=7)
    c2, oc2 = sg.Grid(16, 3, 2, max_leaves=64), oracle.Grid(16, 8, 2)
    f0.restrict_to(c1, 0, 1, 0.125)
    of0.restrict_to(oc1, 0, 1, 0.125)
    c1.restrict_to(c2, 1, 1, 0.125)
    oc1.restrict_to(oc2, 1, 1, 0.125)
    _compare(c1, oc1, [1])
    _compare(c2, oc2, [1])
    # a coarse grid holding only a corner box
    part, opart = sg.Grid(32, 3, 2, max_leaves=64), oracle.Grid(32, 8, 2)
    import torch
    box = np.stack(np.meshgrid(*[np.arange(0, 16)] * 3, indexing="ij"), -1).reshape(-1, 3).astype(np.int32)
    part.activate_coords(torch.from_numpy(box).cuda())
    opart.activate_coords(box)
    pb, _ = part.read_structure()
    pv = leaf_values(8, 32, 8, pb)
    part.write_field(0, pv)
    opart.write_field(0, pv)
    f0.prolong_from(part, 0, 0, 1.0)
    of0.prolong_from(opart, 0, 0, 1.0)
    _compare(f0, of0, [0])
    for g in (f0, c1, c2, part):
        g.close()


def test_restriction_at_scale_sampled():
    """512^3 band (26,104 leaves) onto 256^3: coarse structure against the set
    of i // 2 of the fine leaves (from the fine structure), and the restricted
    sum against w * the fine sum."""
    import paper_2012_08141_gb300 as sg
    from workload import band512
    spec = band512()
    fine, coarse = sg.Grid(512, 3, 2, max_leaves=32768), sg.Grid(256, 3, 2, max_leaves=32768, max_sums=2)
    fine.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    fine.fill_hash(0, 11)
    fine.reduce_sum(0, 0)
    fs = fine.read_sums(1)[0]
    fine.restrict_to(coarse, 0, 1, 0.125)
    coarse.reduce_sum(1, 0)
    cs = coarse.read_sums(1)[0]
    assert cs == pytest.approx(0.125 * fs, rel=2e-5)
    fb, _ = fine.read_structure()
    R = 64
    bi, bj, bk = fb // (R * R), (fb // R) % R, fb % R
    want = np.unique(((bi >> 1) * 32 + (bj >> 1)) * 32 + (bk >> 1))
    cb, _ = coarse.read_structure()
    np.testing.assert_array_equal(cb, want.astype(cb.dtype))
    fine.close()
    coarse.close()


def _vcycle(levels, fmap, clear, restrict, diffuse, prolong, swap):
    """The 4-level V-cycle the multigrid benchmark times: down (clear b on the
    coarse level, restrict x into it, smooth it into x), up (prolong, smooth
    into a third field, swap).  fmap[l] maps the logical fields (x, b, t) of
    level l to storage; swap exchanges x and t."""
    for l in range(3):
        clear(l + 1, fmap[l + 1][1])
        restrict(l, fmap[l][0], fmap[l + 1][1], 0.125)
        diffuse(l + 1, fmap[l + 1][1], fmap[l + 1][0], 0.1)
    for l in (2, 1, 0):
        prolong(l, fmap[l + 1][0], fmap[l][0], 0.5)
        diffuse(l, fmap[l][0], fmap[l][2], 0.1)
        swap(l)


def test_vcycle_full_size_against_oracle():
    """Three V-cycles over the 512^3 band (26,104 leaves) and its 256^3, 128^3
    and 64^3 restrictions, with every pass on, in the launch configuration the
    benchmark times: the first cycle activates the coarse levels, the next two
    are demoted (Sec. 6.3), and from the third the finest level's smoother runs
    over the reused list's j-run records.  Every level's structure bit-exact and
    every field within 2e-5 against the oracle's three cycles."""
    import paper_2012_08141_gb300 as sg
    from workload import band512
    spec = band512()
    G = [sg.Grid(512 >> l, 3, 3, max_leaves=32768, max_sums=1) for l in range(4)]
    O = [oracle.Grid(512 >> l, 8, 3) for l in range(4)]
    for g in G:
        g.set_opts(sg.SG_OPT_ALL)
    G[0].activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    O[0].activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    ob, _ = O[0].structure()
    vals = leaf_values(3, 512, 8, ob)
    G[0].write_field(0, vals)
    O[0].write_field(0, vals)
    gmap, omap = [[0, 1, 2] for _ in G], [[0, 1, 2] for _ in O]

    def gswap(l):
        G[l].swap(0, 2)            # the grid's own field names follow the swap

    def oswap(l):
        omap[l][0], omap[l][2] = omap[l][2], omap[l][0]

    demoted0 = sum(g.stats()["act_demoted"] for g in G)
    for _ in range(3):
        _vcycle(G, gmap, lambda l, f: G[l].clear(f), lambda l, s, d, w: G[l].restrict_to(G[l + 1], s, d, w),
                lambda l, s, d, c: G[l].diffuse7(s, d, c), lambda l, s, d, w: G[l].prolong_from(G[l + 1], s, d, w),
                gswap)
        for g in G:
            g.flush()
        _vcycle(O, omap, lambda l, f: O[l].clear(f), lambda l, s, d, w: O[l].restrict_to(O[l + 1], s, d, w),
                lambda l, s, d, c: O[l].diffuse7(s, d, c), lambda l, s, d, w: O[l].prolong_from(O[l + 1], s, d, w),
                oswap)
    assert sum(g.stats()["act_demoted"] for g in G) - demoted0 == 6   # three restrictions in each of cycles 2, 3
    for l in range(4):
        gb, gm = G[l].read_structure()
        ob, om = O[l].structure()
        np.testing.assert_array_equal(gb, ob)
        np.testing.assert_array_equal(gm, om)
        for f in range(3):
            assert rel_linf(G[l].read_field(f), O[l].read_field(omap[l][f])) <= TOL, (l, f)
    for g in G:
        g.close()
