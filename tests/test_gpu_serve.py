"""GPU tests of the continuous-batching request loop: jobs admitted while
others run share the batched launch, and every job's result (its final field
and its sums) equals the same job run alone."""
import numpy as np
import pytest

from workload import batched_mix

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    yield


def alone(spec, steps):
    """The job run alone through the grid API: its last sum and its final x
    at the active voxels (packed)."""
    import paper_2012_08141_gb300 as sg
    R = spec.N // 8
    g = sg.Grid(spec.N, 3, 3, max_leaves=R ** 3, max_sums=1, scratch_mask=0b010)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    g.list_gen()
    g.fill_hash(0, spec.seed % (1 << 24))
    for _ in range(steps):
        g.clear(1)
        g.diffuse7(0, 1, 0.1)
        g.box27(1, 2)
        g.swap(0, 2)
        g.reduce_sum(0, 0)
    s = g.read_sums(1)[0]
    x = g.read_field_active(0).copy()
    g.close()
    return s, x


def alone_sum(spec, steps):
    return alone(spec, steps)[0]


def test_jobs_in_the_mix_equal_jobs_alone():
    """Jobs of 1e4 to 5e6 active voxels, some admitted while others run: each
    job's final field is bit-identical to the same job run alone (the batched
    kernel runs the single-grid kernel's per-lane arithmetic) and its last sum
    agrees within 2e-5 (FP64 accumulation of FP32 partials in another order)."""
    from paper_2012_08141_gb300.serve import SG_JOB_DONE, Server
    specs = batched_mix(21, n_grids=7, lo=1e4, hi=5e6)
    rng = np.random.default_rng(2)
    steps = [int(rng.integers(3, 13)) for _ in specs]
    refs = [alone(s, k) for s, k in zip(specs, steps)]
    outs = [np.full(len(r[1]) + 5, np.nan, dtype=np.float32) for r in refs]
    srv = Server(max_jobs=4, warps_per_cta=4, hbm_reserve=1 << 30)
    ids = [srv.submit(s, k, o) for s, k, o in zip(specs[:3], steps[:3], outs[:3])]
    max_resident = 0
    for _ in range(2):
        srv.tick()
        max_resident = max(max_resident, srv.stats()["resident"])
    ids += [srv.submit(s, k, o) for s, k, o in zip(specs[3:], steps[3:], outs[3:])]   # arrive while others run
    for _ in range(200):
        st = srv.stats()
        if st["completed"] + st["failed"] == len(specs):
            break
        srv.tick()
        max_resident = max(max_resident, srv.stats()["resident"])
    st = srv.stats()
    assert st["completed"] == len(specs) and st["failed"] == 0
    assert max_resident >= 2                      # work of several jobs shared launches
    jobs = [srv.job(i) for i in ids]
    assert any(jobs[k]["t_admit"] < jobs[0]["t_done"] for k in range(3, len(jobs)))  # admitted while job 0 ran
    assert max(j["n_active"] for j in jobs) >= 1e6
    for (ref_sum, ref_x), k, jb, out in zip(refs, steps, jobs, outs):
        assert jb["state"] == SG_JOB_DONE and jb["steps_done"] == k
        n = jb["n_active"]
        assert n == len(ref_x)
        np.testing.assert_array_equal(out[:n], ref_x)
        assert np.all(np.isnan(out[n:]))          # nothing written past the job's values
        assert abs(jb["sum"] - ref_sum) <= TOL * abs(ref_sum)
        assert jb["t_submit"] <= jb["t_admit"] <= jb["t_done"]
    assert st["voxel_steps"] == pytest.approx(sum(j["n_active"] * k for j, k in zip(jobs, steps)))
    srv.close()


def test_result_buffer_too_small_fails_the_job():
    from paper_2012_08141_gb300.serve import SG_JOB_FAILED, Server
    spec = batched_mix(5, n_grids=1, lo=1e4, hi=2e4)[0]
    srv = Server(max_jobs=2, hbm_reserve=0)
    out = np.zeros(10, dtype=np.float32)
    jid = srv.submit(spec, 2, out)
    for _ in range(4):
        srv.tick()
    assert srv.job(jid)["state"] == SG_JOB_FAILED
    assert np.all(out == 0)
    srv.close()


def test_job_that_cannot_fit_fails_and_server_continues():
    import torch
    from paper_2012_08141_gb300.serve import SG_JOB_DONE, SG_JOB_FAILED, Server
    free, total = torch.cuda.mem_get_info()
    srv = Server(max_jobs=2, hbm_reserve=int(total) * 2)   # reserve more than the device has
    spec = batched_mix(5, n_grids=1, lo=1e3, hi=2e3)[0]
    jid = srv.submit(spec, 3)
    srv.tick()
    assert srv.job(jid)["state"] == SG_JOB_FAILED
    srv.close()
    srv = Server(max_jobs=2, hbm_reserve=0)
    jid = srv.submit(spec, 3)
    for _ in range(5):
        srv.tick()
    assert srv.job(jid)["state"] == SG_JOB_DONE
    srv.close()


def test_injected_allocation_failure_fails_one_job_only():
    """Host-side fault injection: the fifth device allocation of one job's
    admission fails.  That job is failed with its partial allocations freed;
    the jobs around it run to the same results as alone; after close nothing
    the server allocated is left."""
    from paper_2012_08141_gb300.serve import SG_JOB_DONE, SG_JOB_FAILED, Server
    target = {}

    def fail_alloc(i, nbytes):
        return "at" in target and i == target["at"]

    srv = Server(max_jobs=4, hbm_reserve=0, fail_alloc=fail_alloc)
    specs = batched_mix(11, n_grids=3, lo=1e3, hi=4e3)
    a = srv.submit(specs[0], 3)
    srv.tick()
    assert srv.job(a)["state"] != SG_JOB_FAILED
    live_a = dict(srv.live)
    target["at"] = srv.alloc_calls + 4          # inside the next admission's grid creation
    b = srv.submit(specs[1], 3)
    c = srv.submit(specs[2], 2)
    srv.tick()
    assert srv.job(b)["state"] == SG_JOB_FAILED
    assert srv.job(c)["state"] != SG_JOB_FAILED
    for _ in range(6):
        srv.tick()
    st = srv.stats()
    assert st["failed"] == 1 and st["completed"] == 2
    for jid, spec, k in ((a, specs[0], 3), (c, specs[2], 2)):
        jb = srv.job(jid)
        assert jb["state"] == SG_JOB_DONE and jb["steps_done"] == k
        ref = alone_sum(spec, k)
        assert abs(jb["sum"] - ref) <= TOL * abs(ref)
    assert set(srv.live) <= set(live_a)         # b's partial grid and finished jobs freed
    srv.close()
    assert not srv.live


def test_close_with_work_in_flight():
    """A tick returns with its step running and the next admissions queued
    behind it; closing the server then waits for that work and frees every
    grid (each allocation goes through the server's callbacks)."""
    from paper_2012_08141_gb300.serve import SG_JOB_RUNNING, Server
    srv = Server(max_jobs=4, hbm_reserve=0, fail_alloc=lambda i, n: False)
    specs = batched_mix(13, n_grids=3, lo=1e4, hi=5e4)
    a = srv.submit(specs[0], 5)
    b = srv.submit(specs[1], 5)
    srv.tick()                                   # a and b admitted: their work queued
    srv.tick()                                   # their first step launched, not waited for
    c = srv.submit(specs[2], 5)
    srv.tick()                                   # the next step launched, c's admission behind it
    assert all(srv.job(j)["state"] == SG_JOB_RUNNING for j in (a, b, c))
    assert srv.stats()["resident"] == 3
    srv.close()
    assert not srv.live


def test_release_forgets_finished_jobs_only():
    """sg_server_release frees a done job's record (its id becomes unknown and
    its result buffer is no longer held); a pending or running job, an
    unknown id and a second release are refused; the other jobs and the
    server's counters are unaffected."""
    from paper_2012_08141_gb300 import SgError
    from paper_2012_08141_gb300.serve import SG_JOB_DONE, Server
    specs = batched_mix(6, n_grids=2, lo=1e4, hi=2e4)
    srv = Server(max_jobs=1, hbm_reserve=0)           # one slot: the second job waits
    out = np.zeros(10 ** 6, dtype=np.float32)
    a = srv.submit(specs[0], 2, out)
    b = srv.submit(specs[1], 2)
    with pytest.raises(SgError):
        srv.release(b)                                # pending
    srv.tick()
    with pytest.raises(SgError):
        srv.release(a)                                # running
    for _ in range(8):
        srv.tick()
    ja, jb = srv.job(a), srv.job(b)
    assert ja["state"] == SG_JOB_DONE and jb["state"] == SG_JOB_DONE
    assert ja["sum"] == pytest.approx(alone_sum(specs[0], 2), rel=TOL)
    srv.release(a)
    assert a not in srv._outs
    with pytest.raises(SgError):
        srv.job(a)
    with pytest.raises(SgError):
        srv.release(a)
    with pytest.raises(SgError):
        srv.release(10 ** 9)
    assert srv.job(b)["sum"] == jb["sum"]
    st = srv.stats()
    assert st["completed"] == 2 and st["failed"] == 0
    srv.release(b)
    srv.close()
