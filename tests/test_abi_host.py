"""CPU tests of the C ABI: the library loads, exports what include/sgrid.h
declares, validates arguments, and its queue optimizer makes the launch
decisions the paper describes (dry-run grids: no device work)."""
import ctypes
import os

import pytest

import paper_2012_08141_gb300 as sg
from workload import band512, tiny_shell

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_examples.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (s.strip() for s in line.split("=", 1))
            out[k] = [int(t) for t in v.split()]
    return out


def dry(res=64, lg2=3, F=3, scratch=0b010, sums=8):
    return sg.Grid(res, lg2, F, max_leaves=1024, max_sums=sums, scratch_mask=scratch, dry_run=True)


def test_library_exports_every_declared_symbol():
    lib = sg.load_library()
    names = sg.header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_library_is_in_tree():
    lib = sg.load_library()
    assert os.path.dirname(os.path.abspath(lib._name)).endswith("paper_2012_08141_gb300")


def test_invalid_arguments():
    lib = sg.load_library()
    desc = sg.SgDesc(60, 3, 2, 1, 16, 0, sg.SG_CREATE_DRY_RUN)   # 60 is not a multiple of 8
    h = ctypes.c_void_p()
    assert lib.sg_create(ctypes.byref(desc), None, ctypes.byref(h)) == sg.SG_ERR_INVALID
    assert b"multiple" in lib.sg_last_error()
    g = dry()
    with pytest.raises(sg.SgError) as e:
        g.stencil(7, 0, 1)
    assert e.value.code == sg.SG_ERR_INVALID
    with pytest.raises(sg.SgError):
        g.diffuse7(1, 1, 0.1)                      # src == dst
    with pytest.raises(sg.SgError):
        g.reduce_sum(0, 8)                         # slot out of range
    with pytest.raises(sg.SgError):
        g.set_opts(99)
    with pytest.raises(sg.SgError):
        g.read_field(0)                            # dry-run grid holds no data


def cfg1_step(g, s):
    g.activate_shell(s.lo2, s.hi2, s.lo_strict)
    g.list_gen()
    g.diffuse7(0, 1, 0.1)
    g.swap(0, 1)


def cfg2_step(g, slot):
    g.clear(1)
    g.diffuse7(0, 1, 0.1)
    g.box27(1, 2)
    g.swap(0, 2)
    g.reduce_sum(0, slot)


def launches(g, fn):
    before = g.stats()["launches"]
    fn()
    g.flush()
    return g.stats()["launches"] - before


def test_eager_is_three_tasks_per_kernel():
    """Sec. 6.1 / Fig. 8: each sparse kernel is clear list + list generation +
    struct-for; two kernels are 6 tasks."""
    gold = golden()
    g = dry()
    g.set_opts(sg.SG_OPT_EAGER)
    g.activate_shell(100, 400, False)
    g.flush()
    n = launches(g, lambda: (g.diffuse7(0, 1, 0.1), g.box27(1, 2)))
    assert n == gold["two_kernels_tasks_eager"][0] == 2 * gold["tasks_per_sparse_kernel_eager"][0]


def test_two_kernels_after_lgr_and_fusion():
    """Sec. 6.1 / Fig. 9: after list-generation removal and fusion two kernels
    need at most 3 tasks; this compaction rewrites the whole list, so it needs
    no clear-list task (one list generation + one fused kernel)."""
    gold = golden()
    g = dry()
    g.activate_shell(100, 400, False)
    g.flush()
    n = launches(g, lambda: (g.diffuse7(0, 1, 0.1), g.box27(1, 2)))
    assert n <= gold["two_kernels_tasks_optimized"][0]
    st = g.stats()
    assert st["listgen_run"] == 1 and st["ops_fused"] == 1
    # with the list current, the same pair is one launch
    assert launches(g, lambda: (g.diffuse7(0, 1, 0.1), g.box27(1, 2))) == 1


def test_fill_array_ten_clears_one_launch():
    """Supplement Sec. 1 fill_array: 10 fills of one field -> 1 task (here the
    first nine are dead stores)."""
    gold = golden()
    g = dry()
    g.activate_shell(100, 400, False)
    g.list_gen()
    g.flush()
    n = launches(g, lambda: [g.clear(0) for _ in range(gold["fill_array_kernels"][0])])
    assert n == gold["fill_array_tasks_optimized"][0]


def test_tiny_shell_launch_counts():
    s = tiny_shell(0)
    g = dry()
    g.set_opts(sg.SG_OPT_EAGER)
    per = [launches(g, lambda: cfg1_step(g, s)) for _ in range(3)]
    assert per == [6, 6, 6]             # activate + (clear list, listgen) + (clear list, listgen, diffuse)
    g2 = dry()
    per2 = [launches(g2, lambda: cfg1_step(g2, s)) for _ in range(4)]
    assert per2 == [3, 1, 1, 1]         # activation demoted and list reused after the first step
    st = g2.stats()
    assert st["act_demoted"] == 3 and st["act_launched"] == 1 and st["listgen_run"] == 1


def test_band_step_launch_counts():
    s = band512()
    e = dry(512)
    e.set_opts(sg.SG_OPT_EAGER)
    e.activate_shell(s.lo2, s.hi2, s.lo_strict)
    e.flush()
    assert [launches(e, lambda: cfg2_step(e, 0)) for _ in range(2)] == [12, 12]
    f = dry(512)
    f.activate_shell(s.lo2, s.hi2, s.lo_strict)
    f.list_gen()
    f.flush()
    # the activation's zero-fill of the scratch field t is dead: nothing in
    # its flush touches t
    assert f.stats()["stores_removed"] == 1
    # the first fused step also builds the region-mask table cached with the list
    assert [launches(f, lambda: cfg2_step(f, 0)) for _ in range(3)] == [2, 1, 1]
    st = f.stats()
    assert st["stores_removed"] == 1 + 6    # per step: the clear of t and the store of t
    assert st["ops_fused"] == 6             # per step: box27 and the sum ride in diffuse7's kernel


def test_activation_zero_fill_is_a_store():
    """Sec. 6.5 applied to activation: a new leaf's zero-fill in a field is
    dead when the field's next access in the queue is a full overwrite by a
    struct-for, or when the rest of the flush leaves a scratch field alone; a
    field read first (or a non-scratch field left alone) keeps it, and
    without DSE every fill stays.  Counted in stores_removed."""
    def removed(opts, body):
        g = dry(F=4, scratch=0b0010)
        g.set_opts(opts)
        s0 = g.stats()["stores_removed"]
        g.deactivate_all()
        g.activate_shell(100, 400, False)
        body(g)
        g.flush()
        return g.stats()["stores_removed"] - s0
    # field 1 scratch: t of the fused step; 2 fully written; 0 read; 3 untouched
    fused = lambda g: (g.diffuse7(0, 1, 0.1), g.box27(1, 2))
    assert removed(sg.SG_OPT_ALL, fused) == 2 + 1      # fills of 1 and 2; t's store
    assert removed(sg.SG_OPT_ALL, lambda g: None) == 1  # only the scratch field's fill
    assert removed(sg.SG_OPT_ALL, lambda g: g.ew(2, 2, alpha=2.0)) == 1   # 2 read first: kept
    assert removed(sg.SG_OPT_ALL, lambda g: g.ew(2, 0, alpha=2.0)) == 2   # 2 overwritten
    assert removed(sg.SG_OPT_ALL & ~sg.SG_OPT_DSE, fused) == 0
    assert removed(sg.SG_OPT_ALL, lambda g: g.reduce_sum(2, 0)) == 1       # 2 read first (a sum): kept
    assert removed(sg.SG_OPT_ALL, lambda g: g.clear(2)) == 2               # a clear overwrites 2 in full
    # a device fill sets every voxel of its field: 2 overwritten, the scratch field untouched
    assert removed(sg.SG_OPT_ALL, lambda g: g.fill_hash(2, 5)) == 2
    assert removed(sg.SG_OPT_ALL, lambda g: (g.ew(2, 0, alpha=1.0), g.fill_hash(0, 5))) == 2   # 0 read first
    # any other op before a field's first listed access keeps every fill (conservative)
    assert removed(sg.SG_OPT_ALL, lambda g: g.deactivate_all()) == 0
    # an advection reads its source and the velocity, and writes its output in full
    g = dry(F=8, scratch=0b01000000)
    s0 = g.stats()["stores_removed"]
    g.activate_shell(100, 400, False)
    g.advect(5, 3, 0, 1e-3)
    g.flush()
    assert g.stats()["stores_removed"] - s0 == 2      # 5 overwritten, 6 scratch and untouched
    # the MacCormack correction also reads q^ and q~; its output is written in full
    g = dry(F=8, scratch=0b01000000)
    s0 = g.stats()["stores_removed"]
    g.activate_shell(100, 400, False)
    g.maccormack(7, 3, 4, 5, 0, 1e-3)
    g.flush()
    assert g.stats()["stores_removed"] - s0 == 2      # 7 overwritten, 6 scratch; 0-5 read first
    g = dry(F=8, scratch=0b01010000)                  # 4 scratch too, but read as q^: kept
    s0 = g.stats()["stores_removed"]
    g.activate_shell(100, 400, False)
    g.maccormack(7, 3, 4, 5, 0, 1e-3)
    g.flush()
    assert g.stats()["stores_removed"] - s0 == 2


@pytest.mark.parametrize("opts,expect", [
    (sg.SG_OPT_ALL & ~sg.SG_OPT_DSE, 2),                         # clear kept (+ t stored)
    (sg.SG_OPT_ALL & ~sg.SG_OPT_FUSE, 3),                        # diffuse, box27, sum apart
    (sg.SG_OPT_ALL & ~sg.SG_OPT_LGR, 9),                         # no fusion without LGR; lists per op; clear dead
    (sg.SG_OPT_ALL & ~sg.SG_OPT_AD, 1),                          # still fused, stores checked
])
def test_ablation_launch_counts(opts, expect):
    s = band512()
    g = dry(512)
    g.set_opts(opts)
    g.activate_shell(s.lo2, s.hi2, s.lo_strict)
    g.list_gen()
    g.flush()
    launches(g, lambda: cfg2_step(g, 0))
    assert launches(g, lambda: cfg2_step(g, 1)) == expect


def test_fusion_negative_cases():
    """Supplement Sec. 2 criterion (3): tasks that read what another wrote at a
    different address are not fused unless a fused kernel recomputes it; a
    chain whose last output overwrites the first input is not fused."""
    g = dry()
    g.activate_shell(100, 400, False)
    g.list_gen()
    g.flush()
    assert launches(g, lambda: (g.diffuse7(0, 1, 0.1), g.diffuse7(1, 2, 0.1))) == 2
    assert launches(g, lambda: (g.diffuse7(0, 1, 0.1), g.box27(1, 0))) == 2
    assert launches(g, lambda: (g.box27(0, 1), g.diffuse7(1, 2, 0.1))) == 2


def test_deactivation_resets_demotion_and_list():
    g = dry()
    for _ in range(2):
        g.activate_shell(100, 400, False)
    g.list_gen()
    g.flush()
    st = g.stats()
    assert st["act_launched"] == 1 and st["act_demoted"] == 1
    g.deactivate_all()
    g.activate_shell(100, 400, False)
    g.diffuse7(0, 1, 0.1)
    g.flush()
    st2 = g.stats()
    assert st2["act_launched"] == 2 and st2["listgen_run"] == 2


def test_lgr_persists_across_flushes():
    """Sec. 7.1: the latest owner of the list survives a flush, so a later
    flush still removes list generation."""
    g = dry()
    g.activate_shell(100, 400, False)
    g.list_gen()
    g.flush()
    g.sync()
    assert launches(g, lambda: g.diffuse7(0, 1, 0.1)) == 1
    assert g.stats()["listgen_removed"] >= 1


def test_scratch_read_later_keeps_store():
    """DSE may drop the scratch intermediate only if nothing reads it later in
    the flush window."""
    g = dry()
    g.activate_shell(100, 400, False)
    g.list_gen()
    g.flush()
    before = g.stats()["stores_removed"]
    launches(g, lambda: (g.diffuse7(0, 1, 0.1), g.box27(1, 2), g.reduce_sum(1, 0)))
    assert g.stats()["stores_removed"] == before


def test_sort_particles_needs_the_current_binning():
    """sg_sort_particles reorders the arrays of the last binned P2G on the
    grid: without one (or for other arrays) the flush fails; with it, one
    gather per array (x, v, the ids) and the order's reset."""
    lib = sg.load_library()
    g = dry(64, 2, 4)
    x, v, ids, n = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), ctypes.c_void_p(0x40000), 1000
    assert lib.sg_sort_particles(g.h, x, v, None, None, -1) == sg.SG_ERR_INVALID
    assert lib.sg_sort_particles(g.h, x, v, None, None, n) == 0          # queued
    assert lib.sg_flush(g.h) == sg.SG_ERR_INVALID                        # nothing binned yet
    assert b"binned" in lib.sg_last_error()
    assert lib.sg_p2g(g.h, x, v, n, 1.0, 0, 1) == 0
    assert lib.sg_flush(g.h) == 0
    l0 = g.stats()["launches"]
    assert lib.sg_sort_particles(g.h, x, v, None, ids, n) == 0
    assert lib.sg_flush(g.h) == 0
    assert g.stats()["launches"] - l0 == 4
    assert lib.sg_sort_particles(g.h, ctypes.c_void_p(0x50000), v, None, None, n) == 0
    assert lib.sg_flush(g.h) == sg.SG_ERR_INVALID                        # other arrays


def test_g2p2g_argument_checks_and_launches():
    """sg_g2p2g: distinct grids of the same geometry, momentum/velocity fields
    consecutive, a binned P2G over the same particles on src or dst; it flushes
    src and launches one kernel on dst."""
    lib = sg.load_library()
    a, b = dry(64, 2, 4), dry(64, 2, 4)
    c8 = dry(64, 3, 4)
    x, v, n = 0x10000, 0x20000, 1000
    args = (ctypes.c_void_p(x), ctypes.c_void_p(v), n, 1e-4, 1, 1.0, 0, 1)
    assert lib.sg_g2p2g(a.h, a.h, *args) == sg.SG_ERR_INVALID          # src == dst
    assert lib.sg_g2p2g(a.h, c8.h, *args) == sg.SG_ERR_INVALID         # leaf sizes differ
    assert lib.sg_g2p2g(a.h, b.h, *args) == sg.SG_ERR_INVALID          # no bins for these particles
    assert b"binned" in lib.sg_last_error()
    bad = (ctypes.c_void_p(x), ctypes.c_void_p(v), n, 1e-4, 1, 1.0, 1, 1)   # mass inside momentum
    assert lib.sg_g2p2g(a.h, b.h, *bad) == sg.SG_ERR_INVALID
    assert lib.sg_p2g_apic(a.h, ctypes.c_void_p(x), ctypes.c_void_p(v), ctypes.c_void_p(0x30000), n, 1.0, 0, 1) == 0
    assert lib.sg_flush(a.h) == 0
    la, lb = a.stats()["launches"], b.stats()["launches"]
    a.grid_update(0, 1, 1e-4, 9.8, 3)
    b.deactivate_all()
    assert lib.sg_g2p2g(a.h, b.h, *args) == 0
    assert a.stats()["launches"] > la                                   # src flushed (list + update)
    assert b.stats()["launches"] == lb + 2                              # dst: deactivate + the fused kernel
    c = dry(64, 2, 4)
    assert lib.sg_p2g_apic(c.h, ctypes.c_void_p(x), ctypes.c_void_p(v), ctypes.c_void_p(0x30000), n, 1.0, 0, 1) == 0
    assert lib.sg_g2p2g(c.h, a.h, *args) == 0                           # src's queued P2G counts
    assert lib.sg_g2p2g(b.h, a.h, *args) == 0                           # bins held by dst (a) also work


def test_restriction_activation_demotion():
    """sg_restrict activates on the coarse grid the first time (mark, allocate,
    restrict); with SG_OPT_AD a repeat from an unchanged fine grid is demoted
    to one launch and leaves the coarse structure, so the coarse list is not
    generated again (Sec. 6.3).  Without AD every restriction activates."""
    fine, coarse = dry(64, 3, 2), dry(32, 3, 2)
    fine.activate_shell(100, 400, False)
    fine.list_gen()
    coarse.list_gen()
    fine.flush()
    coarse.flush()
    base = coarse.stats()
    fine.restrict_to(coarse, 0, 1, 0.125)
    s1 = coarse.stats()
    assert s1["launches"] - base["launches"] == 3 and s1["act_launched"] == base["act_launched"] + 1
    coarse.list_gen()
    coarse.flush()
    s2 = coarse.stats()
    assert s2["listgen_run"] == s1["listgen_run"] + 1          # structure changed: list made again
    fine.restrict_to(coarse, 0, 1, 0.125)
    coarse.list_gen()
    coarse.flush()
    s3 = coarse.stats()
    assert s3["launches"] - s2["launches"] == 1                # demoted: the restriction alone
    assert s3["act_demoted"] == s2["act_demoted"] + 1
    assert s3["listgen_run"] == s2["listgen_run"]              # list generation removed
    fine.activate_shell(500, 900, False)                       # the fine structure changes
    fine.restrict_to(coarse, 0, 1, 0.125)
    assert coarse.stats()["act_launched"] == s3["act_launched"] + 1
    coarse.deactivate_all()
    coarse.flush()
    fine.restrict_to(coarse, 0, 1, 0.125)                      # deactivation forgets the restriction
    assert coarse.stats()["act_launched"] == s3["act_launched"] + 2
    # activation demotion off: every restriction activates
    f2, c2 = dry(64, 3, 2), dry(32, 3, 2)
    c2.set_opts(sg.SG_OPT_ALL & ~sg.SG_OPT_AD)
    f2.activate_shell(100, 400, False)
    for _ in range(3):
        f2.restrict_to(c2, 0, 1, 0.125)
    st = c2.stats()
    assert st["act_launched"] == 3 and st["act_demoted"] == 0


def test_restriction_argument_checks():
    lib = sg.load_library()
    a, b = dry(64, 3, 2), dry(32, 3, 2)
    assert lib.sg_restrict(a.h, a.h, 0, 1, 1.0) == sg.SG_ERR_INVALID       # same grid
    assert lib.sg_restrict(b.h, a.h, 0, 1, 1.0) == sg.SG_ERR_INVALID       # coarse is not half of fine
    assert lib.sg_restrict(a.h, dry(32, 2, 2).h, 0, 1, 1.0) == sg.SG_ERR_INVALID   # leaf sizes differ
    assert lib.sg_restrict(a.h, b.h, 0, 5, 1.0) == sg.SG_ERR_INVALID       # field out of range
    assert lib.sg_prolong(b.h, a.h, 0, 1, 1.0) == 0
    assert lib.sg_prolong(a.h, b.h, 0, 1, 1.0) == sg.SG_ERR_INVALID        # arguments swapped


# ---------------------------------------------------------------------------
# The paper's microbenchmarks (Supp. Sec. 1) as launch counts on element-wise
# struct-fors: each case runs once to make the list, then its ops are counted.
# ---------------------------------------------------------------------------

def _micro(opts=sg.SG_OPT_ALL, scratch=0b1000, F=5):
    g = dry(64, 3, F, scratch=scratch)
    g.set_opts(opts)
    g.activate_shell(100, 900, False)
    g.list_gen()
    g.flush()
    return g


def _launches(g, fn):
    s0 = g.stats()
    fn(g)
    g.flush()
    s1 = g.stats()
    return {k: s1[k] - s0[k] for k in s1}


def test_micro_chain_copy():
    d = _launches(_micro(), lambda g: (g.ew(1, 0, alpha=1.0, delta=1.0), g.ew(2, 1, alpha=1.0, delta=4.0)))
    assert d["launches"] == 1 and d["ops_fused"] == 1


def test_micro_increments_and_max_fuse():
    d = _launches(_micro(), lambda g: [g.ew(0, 0, alpha=1.0, delta=1.0) for _ in range(10)])
    assert d["launches"] == 1 and d["ops_fused"] == 9
    g = _micro()
    g.set_max_fuse(4)
    d = _launches(g, lambda g: [g.ew(0, 0, alpha=1.0, delta=1.0) for _ in range(10)])
    assert d["launches"] == 3                      # 4 + 4 + 2


def test_micro_fill_array():
    d = _launches(_micro(), lambda g: [g.ew(2, delta=float(k)) for k in range(10)])
    assert d["launches"] == 1 and d["stores_removed"] == 9


def test_micro_sparse_saxpy():
    def body(g):
        g.ew(2, 0, 1, 2.0, 1.0)                     # z = 2x + y
        g.ew(1, 2, 0, 3.0, 1.0)                     # y = 3z + x
        g.ew(2, 2, 1, 1.0, 1.0)                     # z = z + y
    assert _launches(_micro(), body)["launches"] == 1
    e = _launches(_micro(sg.SG_OPT_EAGER), body)
    assert e["launches"] == 9 and e["listgen_run"] == 3     # clear-list + list + kernel per op


def test_micro_autodiff_dead_forward_passes():
    """Ten iterations of: tmp = x * x (scratch), loss = sum(tmp), grad += 2x.
    Only the last loss is read, so nine reductions are dead; the element-wise
    ops fuse into two launches (16 ops per launch)."""
    def body(g):
        for _ in range(10):
            g.ew(3, 0, 0, gamma=1.0)
            g.reduce_sum(3, 0)
            g.ew(4, 4, 0, 1.0, 2.0)
    d = _launches(_micro(), body)
    assert d["launches"] == 2 and d["stores_removed"] >= 9
    e = _launches(_micro(sg.SG_OPT_EAGER), body)
    assert e["launches"] == 90


def test_micro_not_fusible_across_a_stencil():
    """An element-wise op, a neighbour-reading stencil, an element-wise op: the
    stencil depends on the first and the second on the stencil (criterion 1),
    so three launches; the list is still made only once (Sec. 6.2)."""
    def body(g):
        g.ew(1, 0, alpha=2.0)
        g.diffuse7(1, 2, 0.1)
        g.ew(0, 2, alpha=1.0, delta=1.0)
    d = _launches(_micro(), body)
    assert d["launches"] == 3 and d["listgen_run"] == 0


def test_advection_channel_fusion_launches():
    """Three channels written channel by channel (forward advect, backward
    advect, correction each): the queue reorders by field dependencies into
    one velocity packing, one forward launch for all channels and one fused
    backward+correction launch (q~ scratch, not stored) -- against 9 launches
    without fusion and 27 eager (clear-list + list + kernel each), neither of
    which packs the velocity."""
    def step(g):
        for c in range(3):
            q, qh, qt, qn = 3 + 4 * c, 4 + 4 * c, 5 + 4 * c, 6 + 4 * c
            g.advect(qh, q, 0, 1e-3)
            g.advect(qt, qh, 0, -1e-3)
            g.maccormack(qn, q, qh, qt, 0, 1e-3)
    scratch = sum(1 << (5 + 4 * c) for c in range(3))
    counts = {}
    for name, opts in (("all", sg.SG_OPT_ALL), ("nofuse", sg.SG_OPT_ALL & ~sg.SG_OPT_FUSE), ("eager", 0)):
        g = sg.Grid(64, 3, 15, max_leaves=1024, scratch_mask=scratch, dry_run=True)
        g.set_opts(opts)
        g.activate_tube(4 * 64 * 64 * 0.32 ** 2, 4 * 64 * 64 * 0.45 ** 2)
        g.list_gen()
        g.flush()
        s0 = g.stats()
        step(g)
        g.flush()
        s1 = g.stats()
        counts[name] = {k: s1[k] - s0[k] for k in s1}
    assert counts["all"]["launches"] == 3 and counts["all"]["stores_removed"] == 3
    assert counts["all"]["velocity_packs"] == 1
    assert counts["all"]["ops_fused"] == 7
    assert counts["all"]["bounds_reused"] == 3      # each correction reads its forward clamp bounds
    assert counts["nofuse"]["launches"] == 9 and counts["nofuse"]["bounds_reused"] == 0
    assert counts["eager"]["launches"] == 27 and counts["eager"]["bounds_reused"] == 0
    assert counts["nofuse"]["velocity_packs"] == 0 and counts["eager"]["velocity_packs"] == 0


def test_advection_bounds_not_reused_after_a_write():
    """The clamp bounds of a forward advection are not reused when an op of
    the run writes the velocity, nor by a correction of another step; the
    velocity is not packed for a run that writes one of its fields."""
    g = sg.Grid(64, 3, 12, max_leaves=1024, dry_run=True)
    g.activate_tube(1000, 3000)
    g.list_gen()
    g.flush()
    b0 = g.stats()["bounds_reused"]
    g.advect(4, 3, 0, 1e-3)
    g.advect(5, 4, 0, -1e-3)
    g.maccormack(6, 3, 4, 5, 0, 2e-3)          # another step: computes its own bounds
    g.flush()
    assert g.stats()["bounds_reused"] == b0
    g.advect(4, 3, 0, 1e-3)
    g.advect(5, 4, 0, -1e-3)
    p0 = g.stats()["velocity_packs"]
    g.advect(1, 7, 9, 1e-3)                    # writes a velocity component in the same run
    g.maccormack(6, 3, 4, 5, 0, 1e-3)
    g.flush()
    assert g.stats()["bounds_reused"] == b0
    assert g.stats()["velocity_packs"] == p0
    g.advect(4, 3, 0, 1e-3)
    g.advect(5, 4, 0, -1e-3)
    g.maccormack(6, 3, 4, 5, 0, 1e-3)
    g.flush()
    assert g.stats()["bounds_reused"] == b0 + 1


def test_advection_dependencies_respected():
    """A correction whose output a later advection reads is issued before it;
    a second forward advection of the corrected field waits for the first
    channel's correction (no fusion across that dependency)."""
    g = sg.Grid(64, 3, 8, max_leaves=1024, dry_run=True)
    g.activate_tube(1000, 3000)
    g.list_gen()
    g.flush()
    s0 = g.stats()["launches"]
    g.advect(4, 3, 0, 1e-3)          # a: q^ = A(q)
    g.advect(5, 4, 0, -1e-3)         # b: q~ = A(q^, -dt)
    g.maccormack(6, 3, 4, 5, 0, 1e-3)  # m: q' from q, q^, q~
    g.advect(7, 6, 0, 1e-3)          # c: reads q' -> after m
    g.flush()
    assert g.stats()["launches"] - s0 == 4      # velocity packing | a | b+m fused | c
    lib = sg.load_library()
    assert lib.sg_advect(g.h, 3, 3, 0, 1e-3) == sg.SG_ERR_INVALID            # dst == src
    assert lib.sg_advect(g.h, 1, 3, 0, 1e-3) == sg.SG_ERR_INVALID            # dst is a velocity field
    assert lib.sg_maccormack(g.h, 4, 3, 4, 5, 0, 1e-3) == sg.SG_ERR_INVALID  # dst == qhat


def test_flush_period():
    """With a flush period of 1 every op is issued as it is queued, so nothing
    can be fused; a period covering the whole step keeps the fused form."""
    def body(g):
        for c in range(3):
            g.ew(0, 0, alpha=1.0, delta=1.0)
        g.diffuse7(0, 1, 0.1)
        g.box27(1, 2)
    res = {}
    for period in (0, 1, 5):
        g = _micro()
        g.set_flush_period(period)
        _launches(g, body)                      # the first fused stencil pair also builds region masks
        res[period] = _launches(g, body)["launches"]
    assert res[0] == 2 and res[5] == 2          # increments fused; diffuse7 + box27 fused
    assert res[1] == 5                          # one launch per op
    with pytest.raises(sg.SgError):
        _micro().set_flush_period(-1)


def test_write_structure_argument_checks():
    """Order, range and capacity of a saved structure are checked on the host
    before any device work; a dry-run grid holds no data to restore into."""
    import numpy as np
    g = dry()                                   # 64^3, 8^3 leaves: R^3 = 512, max_leaves 1024
    lib = g.lib
    m = np.zeros((3, g.W), dtype=np.uint32)
    cases = [
        (np.array([5, 5, 9], np.int32), sg.SG_ERR_INVALID),        # not strictly ascending
        (np.array([9, 5, 7], np.int32), sg.SG_ERR_INVALID),
        (np.array([-1, 5, 7], np.int32), sg.SG_ERR_INVALID),       # out of [0, R^3)
        (np.array([1, 5, 512], np.int32), sg.SG_ERR_INVALID),
        (np.array([1, 5, 511], np.int32), sg.SG_ERR_INVALID),      # valid, but a dry-run grid
    ]
    for b, rc in cases:
        assert lib.sg_write_structure(g.h, 3, b.ctypes.data, m.ctypes.data) == rc, b
    assert lib.sg_write_structure(g.h, 3, None, m.ctypes.data) == sg.SG_ERR_INVALID
    assert lib.sg_write_structure(g.h, -1, None, None) == sg.SG_ERR_INVALID
    small = sg.Grid(64, 3, 1, max_leaves=2, dry_run=True)
    b = np.array([1, 5, 7], np.int32)
    assert lib.sg_write_structure(small.h, 3, b.ctypes.data, m.ctypes.data) == sg.SG_ERR_POOL_EXHAUSTED
    assert b"max_leaves" in lib.sg_last_error()


def test_staged_upload_tickets():
    """Tickets name one of two upload slots; a ticket whose slot was refilled,
    or that was never issued, is refused; a staged write is one queued op."""
    import numpy as np
    g = dry(F=2)
    v = np.zeros(10, np.float32)
    lib = g.lib
    t1 = g.stage_active(v)
    t2 = g.stage_active(v)
    assert (t1 & 1) != (t2 & 1)
    g.write_field_staged(0, t2)
    t3 = g.stage_active(v)                                 # refills t1's slot
    assert (t3 & 1) == (t1 & 1)
    assert lib.sg_write_field_staged(g.h, 0, t1) == sg.SG_ERR_INVALID
    assert lib.sg_write_field_staged(g.h, 0, 12345) == sg.SG_ERR_INVALID
    assert lib.sg_write_field_staged(g.h, 0, 0) == sg.SG_ERR_INVALID
    assert lib.sg_write_field_staged(g.h, 7, t3) == sg.SG_ERR_INVALID   # no such field
    q0 = g.stats()["ops_enqueued"]
    g.write_field_staged(1, t3)
    assert g.stats()["ops_enqueued"] == q0 + 1
    g.flush()


def test_stencil_variants_and_their_launch_counts():
    """Every stencil kernel family keeps the fused band step at one launch;
    the grouped sweeps build their run records in the region-mask launch,
    once per list and axis; the TMA-staged kernel also lays out its task
    descriptors once per list."""
    with pytest.raises(sg.SgError):
        dry().set_stencil_variant(5)
    with pytest.raises(sg.SgError):
        dry().set_stencil_variant(-1)
    s = band512()
    axis = {sg.SG_VARIANT_SWEEP_COLUMNS: "i", sg.SG_VARIANT_SWEEP_JRUNS: "j", sg.SG_VARIANT_SWEEP_TMA: "j"}
    for variant, first in ((sg.SG_VARIANT_SWEEP, 2), (sg.SG_VARIANT_SWEEP_COLUMNS, 2), (sg.SG_VARIANT_SMEM, 1),
                           (sg.SG_VARIANT_SWEEP_JRUNS, 2), (sg.SG_VARIANT_SWEEP_TMA, 3)):
        g = dry(512)
        g.set_stencil_variant(variant)
        g.activate_shell(s.lo2, s.hi2, s.lo_strict)
        g.list_gen()
        g.flush()
        assert [launches(g, lambda: cfg2_step(g, 0)) for _ in range(3)] == [first, 1, 1], variant
        # to the leaf sweep: the region masks are made current once, unless a
        # sweep already built them for the unchanged list
        g.set_stencil_variant(sg.SG_VARIANT_SWEEP)
        assert launches(g, lambda: cfg2_step(g, 0)) == (2 if variant == sg.SG_VARIANT_SMEM else 1), variant
        # to each grouped sweep: records along a new axis are built once, the
        # TMA task descriptors once per list
        built = axis.get(variant)
        tma_built = variant == sg.SG_VARIANT_SWEEP_TMA
        for v in axis:
            g.set_stencil_variant(v)
            first = 1 + (built != axis[v]) + (v == sg.SG_VARIANT_SWEEP_TMA and not tma_built)
            assert [launches(g, lambda: cfg2_step(g, 0)) for _ in range(2)] == [first, 1], (variant, v)
            built = axis[v]
            tma_built = tma_built or v == sg.SG_VARIANT_SWEEP_TMA

def test_serving_and_batch_calls_reject_null_handles():
    """The serving and batch entry points validate their handles before any
    device work (no GPU needed): a null server or batch is SG_ERR_INVALID,
    and destroying a null handle is a no-op."""
    lib = ctypes.CDLL(sg.load_library()._name)   # own handle: the signatures below stay local
    P, I64 = ctypes.c_void_p, ctypes.c_int64
    lib.sg_server_release.argtypes = [P, I64]
    lib.sg_server_job.argtypes = [P, I64, P]
    lib.sg_server_tick.argtypes = [P]
    lib.sg_server_destroy.argtypes = [P]
    lib.sg_batch_step.argtypes = [P]
    lib.sg_batch_destroy.argtypes = [P]
    for fn in (lib.sg_server_release, lib.sg_server_job, lib.sg_server_tick, lib.sg_server_destroy,
               lib.sg_batch_step, lib.sg_batch_destroy):
        fn.restype = ctypes.c_int
    assert lib.sg_server_release(None, 1) == sg.SG_ERR_INVALID
    assert lib.sg_server_job(None, 1, None) == sg.SG_ERR_INVALID
    assert lib.sg_server_tick(None) == sg.SG_ERR_INVALID
    assert lib.sg_server_destroy(None) == sg.SG_OK
    assert lib.sg_batch_step(None) != sg.SG_OK
    assert lib.sg_batch_destroy(None) == sg.SG_OK
