"""sg_list_gen_noalloc: list generation for callers that cannot allocate.

Such callers (a process whose device memory belongs to another allocator, or
a time-critical loop where cudaMalloc/cudaFree would synchronize the device)
get the active-list compaction without any allocation by the library; its
scratch is a static device array.  These tests call the entry point through
the C ABI and check its list against the definition computed on the host
(np.flatnonzero(root >= 0) and the values at those cells), on random pointer
arrays from one look-back tile up to the largest size the scratch allows, on
two calls in a row, so that the second call also shows the shared scratch is
cleared.  One case also compares with the regular grid API's list for a shell.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from workload import band_bounds, tiny_shell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_08141_gb300 as sg
    lib = sg.load_library()
    return torch, sg, lib


def reference_list(sg, N, lo2, hi2, strict):
    """Active leaves of a shell grid from the regular entry points."""
    g = sg.Grid(N, 3, 1, max_leaves=(N // 8) ** 3)
    g.activate_shell(lo2, hi2, strict)
    g.list_gen()
    b, _ = g.read_structure()
    g.close()
    return b


def noalloc_list(torch, lib, root_np, cap):
    root = torch.from_numpy(root_np).cuda()
    slot = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    lb = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.sg_list_gen_noalloc(root.data_ptr(), root.numel(), slot.data_ptr(), lb.data_ptr(), cap,
                                 cnt.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.sg_last_error()
    torch.cuda.synchronize()
    return slot.cpu().numpy(), lb.cpu().numpy(), int(cnt.item())


def check_twice(torch, lib, root):
    want_b = np.flatnonzero(root >= 0)
    for _ in range(2):                                  # the second call reuses the scratch
        got_slot, got_b, n = noalloc_list(torch, lib, root, len(want_b))
        assert n == len(want_b)
        np.testing.assert_array_equal(got_b[:n], want_b)
        np.testing.assert_array_equal(got_slot[:n], root[want_b])


@pytest.mark.parametrize("n_cells, density", [(1024, 0.5), (32768, 0.2), (1500 * 1024, 0.01),
                                              (4194304, 0.03), (4194304 - 1000, 0.6)])
def test_noalloc_list_is_the_active_cells_in_order(env, n_cells, density):
    """Random pointer arrays (one tile; 32 tiles; 1,500 tiles, so each tile's
    look-back walks past many predecessors; the full 4,194,304 cells (4,096
    tiles); a ragged last tile): the list is exactly the cells with a value
    >= 0, in ascending order, with their values."""
    torch, sg, lib = env
    rng = np.random.default_rng(n_cells)
    root = np.full(n_cells, -1, dtype=np.int32)
    act = rng.random(n_cells) < density
    root[act] = rng.integers(0, 2 ** 31 - 1, size=int(act.sum()), dtype=np.int32)
    root[0] = 5                                          # first and last cells active
    root[-1] = 6
    check_twice(torch, lib, root)


def test_noalloc_all_inactive_and_all_active(env):
    torch, sg, lib = env
    check_twice(torch, lib, np.full(70000, -1, dtype=np.int32))
    check_twice(torch, lib, np.arange(70000, dtype=np.int32))


def test_noalloc_list_matches_regular_list_two_calls(env):
    torch, sg, lib = env
    rng = np.random.default_rng(0)
    cases = []
    s = tiny_shell(0)                                   # 64^3: 512 pointer cells, one tile
    cases.append((s.N, s.lo2, s.hi2, s.lo_strict))
    lo2, hi2 = band_bounds(90.0, 110.0)                 # 256^3: 32,768 cells, 32 tiles
    cases.append((256, lo2, hi2, True))
    for N, lo2, hi2, strict in cases:
        want_b = reference_list(sg, N, lo2, hi2, strict)
        R = N // 8
        root = np.full(R ** 3, -1, dtype=np.int32)
        slots = rng.permutation(len(want_b)).astype(np.int32)
        root[want_b] = slots
        got_slot, got_b, n = noalloc_list(torch, lib, root, len(want_b))
        assert n == len(want_b)
        np.testing.assert_array_equal(got_b[:n], want_b)
        np.testing.assert_array_equal(got_slot[:n], slots)


def test_noalloc_count_beyond_capacity_and_limits(env):
    """A list longer than cap: the first cap entries and the full count; a
    size beyond SG_NOALLOC_MAX_CELLS is rejected before any device work."""
    torch, sg, lib = env
    root = np.full(5000, -1, dtype=np.int32)
    root[[3, 17, 1024, 4999]] = [9, 8, 7, 6]
    slot, lb, n = noalloc_list(torch, lib, root, 2)
    assert n == 4
    np.testing.assert_array_equal(lb[:2], [3, 17])
    np.testing.assert_array_equal(slot[:2], [9, 8])
    dummy = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.sg_list_gen_noalloc(dummy.data_ptr(), 4194305, dummy.data_ptr(), dummy.data_ptr(), 1,
                                 dummy.data_ptr(), None)
    assert rc == sg.SG_ERR_INVALID
