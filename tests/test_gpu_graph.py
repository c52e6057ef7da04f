"""GPU tests of recorded steady-state steps (sg_graph_*): replays of a
recorded multigrid V-cycle (four levels, restrictions demoted) and of a
recorded band step give bit-identical fields and sums to the same cycles and
steps issued call by call; recording a structure change or a host read fails
cleanly and leaves the stream usable."""
import numpy as np
import pytest

from workload import band_bounds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def _levels(sg, stream, N=128):
    lo2, hi2 = band_bounds(0.3 * N, 0.42 * N)
    G = [sg.Grid(N >> l, 3, 3, max_leaves=(N // 8) ** 3, max_sums=1, stream=stream) for l in range(4)]
    G[0].activate_shell(lo2, hi2, False)
    G[0].fill_hash(0, 3)
    return G


def _cycle(G):
    for l in range(3):
        G[l + 1].clear(1)
        G[l].restrict_to(G[l + 1], 0, 1, 0.125)
        G[l + 1].diffuse7(1, 0, 0.1)
    for l in (2, 1, 0):
        G[l].prolong_from(G[l + 1], 0, 0, 0.5)
        G[l].diffuse7(0, 2, 0.1)
        G[l].swap(0, 2)
    for g in G:
        g.flush()


def test_vcycle_graph_equals_call_by_call():
    import torch
    import paper_2012_08141_gb300 as sg
    s = torch.cuda.Stream()
    A, B = _levels(sg, s), _levels(sg, s)
    for G in (A, B):
        _cycle(G)            # activates the coarse levels
        _cycle(G)            # the other swap parity, lists current
        for g in G:
            g.sync()
    launches = sum(g.stats()["launches"] for g in A)
    gr = sg.StepGraph(stream=s)
    with gr:                 # two cycles: every swap is undone, so replays chain
        _cycle(A)
        _cycle(A)
    assert sum(g.stats()["launches"] for g in A) - launches == 30   # recorded once, 15 launches a cycle
    for _ in range(3):
        gr.launch()
    for _ in range(6):
        _cycle(B)
    for a, b in zip(A, B):
        for f in range(3):
            np.testing.assert_array_equal(a.read_field(f), b.read_field(f))
    gr.close()
    for g in A + B:
        g.close()


def test_band_step_graph_with_sums():
    import torch
    import paper_2012_08141_gb300 as sg
    s = torch.cuda.Stream()
    lo2, hi2 = band_bounds(40.0, 56.0)

    def make():
        g = sg.Grid(128, 3, 3, max_leaves=4096, max_sums=2, scratch_mask=0b010, stream=s)
        g.activate_shell(lo2, hi2, True)
        g.fill_hash(0, 5)
        return g

    def step(g, slot):
        g.clear(1)
        g.diffuse7(0, 1, 0.1)
        g.box27(1, 2)
        g.swap(0, 2)
        g.reduce_sum(0, slot)
        g.flush()

    a, b = make(), make()
    for g in (a, b):
        step(g, 0)
        step(g, 1)
        g.sync()
    gr = sg.StepGraph(stream=s)
    with gr:
        step(a, 0)
        step(a, 1)
    for _ in range(5):
        gr.launch()
    for _ in range(5):
        step(b, 0)
        step(b, 1)
    np.testing.assert_array_equal(a.read_field(0), b.read_field(0))
    np.testing.assert_array_equal(a.read_sums(2), b.read_sums(2))
    gr.close()
    a.close()
    b.close()


def test_recording_refuses_structure_changes_and_reads():
    import torch
    import paper_2012_08141_gb300 as sg
    s = torch.cuda.Stream()
    g = sg.Grid(64, 3, 2, max_leaves=512, stream=s)
    g.activate_shell(*band_bounds(10.0, 20.0), False)
    g.fill_hash(0, 1)
    g.sync()
    with pytest.raises(sg.SgError):
        with sg.StepGraph(stream=s):
            g.activate_shell(*band_bounds(5.0, 25.0), False)
            g.flush()
    g2 = sg.Grid(64, 3, 2, max_leaves=512, stream=s)    # the stream is usable again
    g2.activate_shell(*band_bounds(10.0, 20.0), False)
    g2.fill_hash(0, 1)
    assert g2.num_leaves() > 0
    with pytest.raises(sg.SgError):
        with sg.StepGraph(stream=s):
            g2.diffuse7(0, 1, 0.1)
            g2.read_field(1)                             # a host read inside the recording
    g3 = sg.Grid(64, 3, 2, max_leaves=512, stream=s)
    g3.activate_shell(*band_bounds(10.0, 20.0), False)
    assert g3.num_leaves() == g2.num_leaves()
    for x in (g, g2, g3):
        x.close()
    with pytest.raises(sg.SgError):
        sg.StepGraph(stream=torch.cuda.default_stream()).begin()   # the legacy default stream
