"""GPU parity of the fused element-wise struct-fors against the FP64 oracle run
op by op: the same program fused (all passes), unfused (eager) and with a
small fusion limit gives the oracle's fields within 1e-6 normwise relative
L-inf (FP32 arithmetic on O(1) values) and its reductions within 2e-5."""
import numpy as np
import pytest

import oracle
from sgtest import rel_linf
from workload import leaf_values, tiny_shell

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


# (dst, a, b, alpha, beta, gamma, delta); ("sum", field, slot) is a reduction
PROGRAM = [
    (1, 0, -1, 1.0, 0.0, 0.0, 1.0),        # chain copy: y = x + 1
    (2, 1, -1, 1.0, 0.0, 0.0, 4.0),        #             z = y + 4
    (0, 0, -1, 1.0, 0.0, 0.0, 1.0),        # increments
    (0, 0, -1, 1.0, 0.0, 0.0, 1.0),
    (3, 0, 0, 0.0, 0.0, 1.0, 0.0),         # tmp = x * x (scratch)
    ("sum", 3, 0),
    (4, 4, 0, 1.0, 2.0, 0.0, 0.0),         # grad += 2x
    (2, 2, 1, -0.5, 1.0, 0.25, 0.0),       # z = -0.5 z + y + 0.25 z y
    (1, -1, -1, 0.0, 0.0, 0.0, 0.125),     # fill y
    (1, 1, 2, 1.0, 1.0, 0.0, 0.0),         # y = y + z (in place)
    ("sum", 2, 1),
]


def run(g, prog):
    for op in prog:
        if op[0] == "sum":
            if hasattr(g, "reduce_sum"):
                g.reduce_sum(op[1], op[2])
        else:
            d, a, b, al, be, ga, de = op
            g.ew(d, a, b, al, be, ga, de)


def oracle_run(og, prog):
    sums = {}
    for op in prog:
        if op[0] == "sum":
            sums[op[2]] = og.sum(op[1])
        else:
            og.ew(*op)
    return sums


def setup(L, opts, max_fuse=None, seed=3):
    import paper_2012_08141_gb300 as sg
    spec = tiny_shell(seed, N=64, L=L)
    g = sg.Grid(spec.N, int(np.log2(L)), 5, max_leaves=(64 // L) ** 3, max_sums=2, scratch_mask=0b01000)
    g.set_opts(opts)
    if max_fuse:
        g.set_max_fuse(max_fuse)
    og = oracle.Grid(spec.N, spec.L, 5)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    og.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    b, _ = g.read_structure()
    for f, s in ((0, seed), (4, seed + 100)):
        v = leaf_values(s, spec.N, spec.L, b)
        g.write_field(f, v)
        og.write_field(f, v)
    return g, og


@pytest.mark.parametrize("L", [8, 4])
@pytest.mark.parametrize("mode", ["all", "eager", "max_fuse_3"])
def test_program_parity(L, mode):
    import paper_2012_08141_gb300 as sg
    opts = sg.SG_OPT_EAGER if mode == "eager" else sg.SG_OPT_ALL
    g, og = setup(L, opts, 3 if mode == "max_fuse_3" else None)
    run(g, PROGRAM)
    want = oracle_run(og, PROGRAM)
    got = g.read_sums(2)
    for f in (0, 1, 2, 4):                 # field 3 is scratch: undefined after the flush
        assert rel_linf(g.read_field(f), og.read_field(f)) <= TOL, (mode, f)
    for slot, v in want.items():
        assert got[slot] == pytest.approx(v, rel=2e-5), (mode, slot)
    g.close()


def test_fused_run_stores_only_live_fields():
    """The scratch product is not stored when nothing later reads it, and is
    stored (equal to the oracle) when a later op does."""
    import paper_2012_08141_gb300 as sg
    g, og = setup(8, sg.SG_OPT_ALL)
    s0 = g.stats()["stores_removed"]
    g.ew(3, 0, 0, gamma=1.0)
    g.ew(1, 3, 0, 1.0, 1.0)
    g.flush()
    assert g.stats()["stores_removed"] == s0 + 1
    g.ew(3, 0, 0, gamma=1.0)
    g.ew(1, 3, -1, 1.0)
    g.diffuse7(3, 2, 0.1)                  # a later reader of the scratch field
    og.ew(3, 0, 0, gamma=1.0)
    og.ew(1, 3, 0, 1.0, 1.0)
    og.ew(3, 0, 0, gamma=1.0)
    og.ew(1, 3, -1, 1.0)
    og.diffuse7(3, 2, 0.1)
    for f in (1, 2, 3):
        assert rel_linf(g.read_field(f), og.read_field(f)) <= 2e-5, f
    g.close()


DEAD = [
    (1, 0, -1, 2.0, 0.0, 0.0, 1.0),        # y = 2x + 1: overwritten before any read (dead)
    (1, 0, 0, 0.0, 0.0, 1.0, 0.0),         # y = x * x
    (2, 1, 0, 1.0, 1.0, 0.0, 0.0),         # z = y + x: overwritten before any read (dead)
    (2, -1, -1, 0.0, 0.0, 0.0, 3.0),       # z = 3
    (4, 2, 1, 1.0, 1.0, 0.0, 0.0),         # grad = z + y
    (1, -1, 0, 0.0, 0.5, 0.0, 0.0),        # y = 0.5 x (an op reading only its second operand)
]


@pytest.mark.parametrize("L", [8, 4])
@pytest.mark.parametrize("mode", ["all", "eager"])
def test_dead_ops_in_a_run(L, mode):
    """Ops whose results are overwritten unread are dropped from the fused
    run; the fields equal the oracle's op-by-op results."""
    import paper_2012_08141_gb300 as sg
    g, og = setup(L, sg.SG_OPT_EAGER if mode == "eager" else sg.SG_OPT_ALL)
    run(g, DEAD)
    oracle_run(og, DEAD)
    for f in (0, 1, 2, 4):
        assert rel_linf(g.read_field(f), og.read_field(f)) <= TOL, (mode, f)
    g.close()
