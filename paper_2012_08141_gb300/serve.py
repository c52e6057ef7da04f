"""Python binding of the serving loop (sg_server_*).

Argument marshalling only; the scheduler (admission by free device memory,
continuous batching of every resident job's step into one launch,
retirement) runs in libsgrid.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import SgError, load_library

SG_JOB_PENDING, SG_JOB_RUNNING, SG_JOB_DONE, SG_JOB_FAILED = 0, 1, 2, 3

_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class ServerDesc(ctypes.Structure):
    _fields_ = [("max_jobs", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32), ("hbm_reserve", ctypes.c_int64),
                ("coef", ctypes.c_float), ("alloc", _ALLOC), ("free", _FREE), ("alloc_ctx", ctypes.c_void_p)]


class JobDesc(ctypes.Structure):
    _fields_ = [("res", ctypes.c_int32), ("lo_strict", ctypes.c_int32), ("lo2", ctypes.c_int64),
                ("hi2", ctypes.c_int64), ("steps", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("seed", ctypes.c_int64), ("out_values", ctypes.c_void_p), ("out_cap", ctypes.c_int64)]


class JobStatus(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("steps_done", ctypes.c_int32), ("n_active", ctypes.c_int64),
                ("sum", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("ticks", ctypes.c_int64), ("launches", ctypes.c_int64), ("admission_waits", ctypes.c_int64),
                ("resident", ctypes.c_int32), ("pending", ctypes.c_int32), ("voxel_steps", ctypes.c_double)]


def _lib():
    lib = load_library()
    if not getattr(lib, "_serve_sigs", False):
        P = ctypes.c_void_p
        sigs = {
            "sg_server_create": [ctypes.POINTER(ServerDesc), P, ctypes.POINTER(P)],
            "sg_server_submit": [P, ctypes.POINTER(JobDesc), ctypes.POINTER(ctypes.c_int64)],
            "sg_server_tick": [P],
            "sg_server_job": [P, ctypes.c_int64, ctypes.POINTER(JobStatus)],
            "sg_server_release": [P, ctypes.c_int64],
            "sg_server_get_stats": [P, ctypes.POINTER(ServerStats)],
            "sg_server_destroy": [P],
        }
        for name, args in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib._serve_sigs = True
    return lib


class Server:
    """Continuous-batching request loop over resident sparse diffusion jobs."""

    def __init__(self, max_jobs: int = 256, warps_per_cta: int = 4, hbm_reserve: int = 4 << 30, coef: float = 0.1,
                 stream=None, fail_alloc=None):
        """fail_alloc: optional fault-injection hook, called as
        fail_alloc(call_index, nbytes) before each device allocation the
        server or its jobs make; a true result makes that allocation fail
        (return NULL) as an out-of-memory device would."""
        import torch
        self.lib = _lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        dev, st = torch.cuda.current_device(), self.stream
        self.alloc_calls = 0
        self.live = {}  # device address -> bytes, for leak checks
        self._outs = {}  # job id -> result buffer borrowed by that job

        def _alloc(nbytes, ctx):
            i = self.alloc_calls
            self.alloc_calls += 1
            if fail_alloc is not None and fail_alloc(i, int(nbytes)):
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, ctx):
            self.live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

        self._cb = (_ALLOC(_alloc), _FREE(_free))
        d = ServerDesc(int(max_jobs), int(warps_per_cta), int(hbm_reserve), float(coef), self._cb[0], self._cb[1],
                       None)
        h = ctypes.c_void_p()
        rc = self.lib.sg_server_create(ctypes.byref(d), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc:
            raise SgError(rc, "sg_server_create failed")
        self.h = h

    def submit(self, spec, steps: int, out=None) -> int:
        """spec: a workload.ShellSpec with 8^3 leaves.  out: optional float32
        numpy array that receives the job's final x at its active voxels
        (packed, as Grid.read_field_active returns them) when it completes;
        it must stay alive until then."""
        ptr, cap = None, 0
        if out is not None:
            assert out.dtype == np.float32 and out.flags.c_contiguous
            ptr, cap = out.ctypes.data, out.size
        j = JobDesc(int(spec.N), int(bool(spec.lo_strict)), int(spec.lo2), int(spec.hi2), int(steps), 0,
                    int(spec.seed) % (1 << 24), ptr, cap)
        jid = ctypes.c_int64()
        rc = self.lib.sg_server_submit(self.h, ctypes.byref(j), ctypes.byref(jid))
        if rc:
            raise SgError(rc, "sg_server_submit failed")
        if out is not None:
            self._outs[jid.value] = out
        return jid.value

    def tick(self):
        rc = self.lib.sg_server_tick(self.h)
        if rc:
            raise SgError(rc, "sg_server_tick failed")

    def job(self, job_id: int) -> dict:
        st = JobStatus()
        rc = self.lib.sg_server_job(self.h, int(job_id), ctypes.byref(st))
        if rc:
            raise SgError(rc, "unknown job")
        return {name: getattr(st, name) for name, _ in JobStatus._fields_}

    def release(self, job_id: int):
        """Forget a finished (done or failed) job: its record is freed and
        its result buffer no longer held."""
        rc = self.lib.sg_server_release(self.h, int(job_id))
        if rc:
            raise SgError(rc, "sg_server_release: unknown or unfinished job")
        self._outs.pop(int(job_id), None)

    def stats(self) -> dict:
        st = ServerStats()
        self.lib.sg_server_get_stats(self.h, ctypes.byref(st))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            self.lib.sg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
