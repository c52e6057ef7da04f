"""Python binding of libsgrid, the GB300 sparse-grid time-stepping library.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch provides the device memory (through the library's allocator
callback) and the stream.  There is no CPU fallback: if libsgrid.so is missing
or cannot be loaded, importing the library raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "sgrid.h")

SG_OK, SG_ERR_INVALID, SG_ERR_OOM, SG_ERR_POOL_EXHAUSTED, SG_ERR_TIMEOUT, SG_ERR_CUDA, SG_ERR_CHECK = range(7)
SG_OPT_LGR, SG_OPT_AD, SG_OPT_FUSE, SG_OPT_DSE = 1, 2, 4, 8
SG_OPT_ALL, SG_OPT_EAGER = 15, 0
SG_CLEAR, SG_DIFFUSE7, SG_BOX27 = 0, 1, 2
SG_CREATE_DRY_RUN, SG_CREATE_CHECK = 1, 2
SG_VARIANT_SWEEP, SG_VARIANT_SMEM, SG_VARIANT_SWEEP_COLUMNS, SG_VARIANT_SWEEP_JRUNS, SG_VARIANT_SWEEP_TMA = 0, 1, 2, 3, 4
SG_MAX_FIELDS = 16

_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class SgDesc(ctypes.Structure):
    _fields_ = [("res", ctypes.c_int32), ("leaf_log2", ctypes.c_int32), ("n_fields", ctypes.c_int32),
                ("max_sums", ctypes.c_int32), ("max_leaves", ctypes.c_int64), ("scratch_mask", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("alloc", _ALLOC), ("free", _FREE), ("alloc_ctx", ctypes.c_void_p)]


class SgStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("listgen_run", ctypes.c_int64), ("listgen_removed", ctypes.c_int64),
                ("act_launched", ctypes.c_int64), ("act_demoted", ctypes.c_int64), ("ops_enqueued", ctypes.c_int64),
                ("ops_fused", ctypes.c_int64), ("stores_removed", ctypes.c_int64), ("flushes", ctypes.c_int64),
                ("bytes_model", ctypes.c_double), ("bounds_reused", ctypes.c_int64),
                ("velocity_packs", ctypes.c_int64)]


class SgCheckReport(ctypes.Structure):
    _fields_ = [("root_bad", ctypes.c_int64), ("slot_shared", ctypes.c_int64), ("list_bad", ctypes.c_int64),
                ("nbr_bad", ctypes.c_int64), ("zero_leaf_bad", ctypes.c_int64), ("inactive_nonzero", ctypes.c_int64),
                ("leaves", ctypes.c_int64), ("ctrl_bad", ctypes.c_int64)]


class SgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sgrid error {code}: {msg}")
        self.code = code


_lib = None


def header_functions() -> list[str]:
    """Names of the functions include/sgrid.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(?:int|const char \*|void)\s+\**(sg_\w+)\s*\(", text, flags=re.M)


def load_library(build: bool = True) -> ctypes.CDLL:
    """Load libsgrid.so (building it first if its sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libsgrid.so not found at {_build.LIB}; run build() first")
    lib = ctypes.CDLL(_build.LIB)
    P, I32, I64, U32, F, D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                             ctypes.c_float, ctypes.c_double)
    sigs = {
        "sg_create": [ctypes.POINTER(SgDesc), P, ctypes.POINTER(P)],
        "sg_destroy": [P],
        "sg_set_opts": [P, U32],
        "sg_activate_shell": [P, I64, I64, I32],
        "sg_activate_coords": [P, P, I64],
        "sg_deactivate_all": [P],
        "sg_list_gen": [P],
        "sg_launch_stencil": [P, I32, I32, I32, F],
        "sg_reduce_sum": [P, I32, I64],
        "sg_p2g": [P, P, P, I64, F, I32, I32],
        "sg_grid_update": [P, I32, I32, F, F, I32],
        "sg_g2p": [P, P, P, I64, F, I32],
        "sg_p2g_apic": [P, P, P, P, I64, F, I32, I32],
        "sg_g2p_apic": [P, P, P, P, I64, F, I32],
        "sg_g2p2g": [P, P, P, P, I64, F, I32, F, I32, I32],
        "sg_sort_particles": [P, P, P, P, P, I64],
        "sg_restrict": [P, P, I32, I32, F],
        "sg_launch_ew": [P, I32, I32, I32, F, F, F, F],
        "sg_activate_tube": [P, I64, I64],
        "sg_advect": [P, I32, I32, I32, F],
        "sg_maccormack": [P, I32, I32, I32, I32, I32, F],
        "sg_set_max_fuse": [P, I32],
        "sg_set_flush_period": [P, I32],
        "sg_prolong": [P, P, I32, I32, F],
        "sg_swap": [P, I32, I32],
        "sg_flush": [P],
        "sg_sync": [P],
        "sg_num_leaves": [P, ctypes.POINTER(I64)],
        "sg_read_structure": [P, I64, ctypes.POINTER(I64), P, P],
        "sg_read_field": [P, I32, I64, P],
        "sg_write_field": [P, I32, P, I64],
        "sg_write_structure": [P, I64, P, P],
        "sg_write_field_active": [P, I32, P, I64],
        "sg_read_field_active": [P, I32, I64, ctypes.POINTER(I64), P],
        "sg_stage_active": [P, P, I64, ctypes.POINTER(I32)],
        "sg_write_field_staged": [P, I32, I32],
        "sg_read_sums": [P, P, I64],
        "sg_get_stats": [P, ctypes.POINTER(SgStats)],
        "sg_debug_wait_test": [P],
        "sg_set_stencil_variant": [P, I32],
        "sg_list_gen_noalloc": [P, I64, P, P, I64, P, P],
        "sg_fill_hash": [P, I32, I64],
        "sg_batch_create": [P, I32, I32, I32, I32, F, P, ctypes.POINTER(P)],
        "sg_batch_step": [P],
        "sg_batch_read_sums": [P, P, I32],
        "sg_batch_set": [P, I32, I32],
        "sg_batch_autotune": [P, I32, ctypes.POINTER(I32)],
        "sg_batch_set_staging": [P, I32],
        "sg_batch_config": [P, ctypes.POINTER(I32), ctypes.POINTER(I32)],
        "sg_batch_info": [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I32)],
        "sg_batch_destroy": [P],
        "sg_num_active": [P, ctypes.POINTER(I64)],
        "sg_check": [P, ctypes.POINTER(SgCheckReport)],
        "sg_graph_begin": [P],
        "sg_graph_end": [P, ctypes.POINTER(P)],
        "sg_graph_launch": [P],
        "sg_graph_destroy": [P],
        "sg_debug_poke": [P, I32, I64, U32],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.sg_last_error.argtypes = []
    lib.sg_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(lib, rc: int):
    if rc != SG_OK:
        raise SgError(rc, lib.sg_last_error().decode())


def _ptr(t) -> int:
    """Device or host address of a torch tensor / numpy array."""
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


class Grid:
    """One sparse grid: a pointer root over bitmasked 2^leaf_log2 leaves, with
    n_fields FP32 fields, living on one CUDA stream.

    Device memory comes from PyTorch's caching allocator; the stream is
    torch's current stream unless one is given.  Device tensors passed to
    queued calls are kept referenced until the next sync."""

    def __init__(self, res: int, leaf_log2: int = 3, n_fields: int = 2, max_leaves: int = 4096,
                 max_sums: int = 1, scratch_mask: int = 0, stream=None, dry_run: bool = False,
                 device: int | None = None, checking: bool | None = None):
        """checking: run the invariant checks at every sync (SG_CREATE_CHECK);
        by default on when the environment variable SG_CHECK is set to 1."""
        self.lib = load_library()
        self.res, self.leaf_log2, self.n_fields = int(res), int(leaf_log2), int(n_fields)
        self.L = 1 << self.leaf_log2
        self.V = self.L ** 3
        self.W = self.V // 32
        self.max_leaves, self.max_sums = int(max_leaves), int(max_sums)
        self._borrowed = []
        self.h = None
        if checking is None:
            checking = os.environ.get("SG_CHECK", "0") == "1"
        flags = (SG_CREATE_DRY_RUN if dry_run else 0) | (SG_CREATE_CHECK if checking else 0)
        desc = SgDesc(self.res, self.leaf_log2, self.n_fields, self.max_sums, self.max_leaves, int(scratch_mask),
                      flags)
        stream_ptr = None
        if not dry_run:
            import torch
            self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            stream_ptr = self.stream.cuda_stream
            dev_index, torch_stream = self.device.index, self.stream

            def _alloc(nbytes, ctx):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev_index, torch_stream)

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (_ALLOC(_alloc), _FREE(_free))
            desc.alloc, desc.free = self._cb
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.sg_create(ctypes.byref(desc), stream_ptr, ctypes.byref(h)))
        self.h = h

    # ---- lifetime ----
    def close(self):
        if self.h:
            rc = self.lib.sg_destroy(self.h)
            self.h = None
            self._borrowed.clear()
            _check(self.lib, rc)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, rc):
        _check(self.lib, rc)

    # ---- queued calls ----
    def set_opts(self, opts: int):
        self._c(self.lib.sg_set_opts(self.h, int(opts)))

    def set_stencil_variant(self, variant: int):
        self._c(self.lib.sg_set_stencil_variant(self.h, int(variant)))

    def activate_shell(self, lo2: int, hi2: int, lo_strict: bool):
        self._c(self.lib.sg_activate_shell(self.h, int(lo2), int(hi2), int(bool(lo_strict))))

    def activate_coords(self, xyz):
        """xyz: int32 CUDA tensor (n, 3), borrowed until the next sync."""
        assert xyz.is_cuda and str(xyz.dtype) == "torch.int32" and xyz.is_contiguous()
        self._borrowed.append(xyz)
        self._c(self.lib.sg_activate_coords(self.h, _ptr(xyz), xyz.numel() // 3))

    def deactivate_all(self):
        self._c(self.lib.sg_deactivate_all(self.h))

    def list_gen(self):
        self._c(self.lib.sg_list_gen(self.h))

    def stencil(self, op: int, src: int, dst: int, coef: float = 0.0):
        self._c(self.lib.sg_launch_stencil(self.h, int(op), int(src), int(dst), float(coef)))

    def clear(self, dst: int):
        self.stencil(SG_CLEAR, dst, dst)

    def diffuse7(self, src: int, dst: int, coef: float):
        self.stencil(SG_DIFFUSE7, src, dst, coef)

    def box27(self, src: int, dst: int):
        self.stencil(SG_BOX27, src, dst)

    def ew(self, dst: int, a: int = -1, b: int = -1, alpha: float = 0.0, beta: float = 0.0, gamma: float = 0.0,
           delta: float = 0.0):
        """Queue dst = alpha a + beta b + gamma a b + delta on the active voxels (-1: absent field)."""
        self._c(self.lib.sg_launch_ew(self.h, int(dst), int(a), int(b), float(alpha), float(beta), float(gamma),
                                      float(delta)))

    def activate_tube(self, lo2: int, hi2: int):
        """Queue activation of the tube lo2 <= (2i+1-N)^2 + (2j+1-N)^2 < hi2 along k."""
        self._c(self.lib.sg_activate_tube(self.h, int(lo2), int(hi2)))

    def advect(self, dst: int, src: int, v0: int, dt: float):
        """Queue dst = src at the RK3 backtrace over dt through velocity fields v0..v0+2."""
        self._c(self.lib.sg_advect(self.h, int(dst), int(src), int(v0), float(dt)))

    def maccormack(self, dst: int, q: int, qhat: int, qtilde: int, v0: int, dt: float):
        """Queue dst = clamp(qhat + (q - qtilde) / 2) to the forward sample's values of q."""
        self._c(self.lib.sg_maccormack(self.h, int(dst), int(q), int(qhat), int(qtilde), int(v0), float(dt)))

    def set_flush_period(self, ops: int):
        """Flush automatically once `ops` ops are queued (0: only on flush / sync)."""
        self._c(self.lib.sg_set_flush_period(self.h, int(ops)))

    def set_max_fuse(self, max_ops: int):
        self._c(self.lib.sg_set_max_fuse(self.h, int(max_ops)))

    def reduce_sum(self, src: int, slot: int):
        self._c(self.lib.sg_reduce_sum(self.h, int(src), int(slot)))

    def p2g(self, x, v, pmass: float, f_mass: int, f_mom0: int):
        for t in (x, v):
            assert t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()
        self._borrowed += [x, v]
        self._c(self.lib.sg_p2g(self.h, _ptr(x), _ptr(v), x.numel() // 3, float(pmass), int(f_mass), int(f_mom0)))

    def grid_update(self, f_mass: int, f_mom0: int, dt: float, gz: float, bound: int):
        self._c(self.lib.sg_grid_update(self.h, int(f_mass), int(f_mom0), float(dt), float(gz), int(bound)))

    def p2g_apic(self, x, v, C, pmass: float, f_mass: int, f_mom0: int):
        """APIC P2G; C is (n, 9) FP32 on the device (row-major 3x3 per particle)."""
        for t in (x, v, C):
            assert t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()
        assert C.numel() == 3 * x.numel()
        self._borrowed += [x, v, C]
        self._c(self.lib.sg_p2g_apic(self.h, _ptr(x), _ptr(v), _ptr(C), x.numel() // 3, float(pmass), int(f_mass),
                                     int(f_mom0)))

    def g2p_apic(self, x, v, C, dt: float, f_mom0: int):
        """APIC G2P: overwrites x, v and C (n, 9)."""
        for t in (x, v, C):
            assert t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()
        assert C.numel() == 3 * x.numel()
        self._borrowed += [x, v, C]
        self._c(self.lib.sg_g2p_apic(self.h, _ptr(x), _ptr(v), _ptr(C), x.numel() // 3, float(dt), int(f_mom0)))

    def g2p2g(self, dst: "Grid", x, v, dt: float, f_vel0: int, pmass: float, f_mass: int, f_mom0: int):
        """Fused APIC G2P from this grid and APIC P2G into dst (C never stored)."""
        for t in (x, v):
            assert t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()
        self._borrowed += [x, v]
        dst._borrowed += [x, v]
        self._c(self.lib.sg_g2p2g(self.h, dst.h, _ptr(x), _ptr(v), x.numel() // 3, float(dt), int(f_vel0),
                                  float(pmass), int(f_mass), int(f_mom0)))

    def restrict_to(self, coarse: "Grid", f_src: int, f_dst: int, w: float):
        """coarse[f_dst][i // 2] += w * self[f_src][i] over this grid's active
        voxels, activating i // 2 on coarse (res half of this grid's)."""
        self._c(self.lib.sg_restrict(self.h, coarse.h, int(f_src), int(f_dst), float(w)))

    def prolong_from(self, coarse: "Grid", f_src: int, f_dst: int, w: float):
        """self[f_dst][i] += w * coarse[f_src][i // 2] over this grid's active voxels."""
        self._c(self.lib.sg_prolong(coarse.h, self.h, int(f_src), int(f_dst), float(w)))

    def g2p(self, x, v, dt: float, f_mom0: int):
        for t in (x, v):
            assert t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()
        self._borrowed += [x, v]
        self._c(self.lib.sg_g2p(self.h, _ptr(x), _ptr(v), x.numel() // 3, float(dt), int(f_mom0)))

    def sort_particles(self, x, v, C=None, ids=None):
        """Queue the reordering of the particle arrays (and C, ids when given:
        n x 9 float32, n int64) into the order of the last binned P2G of x."""
        for t in (x, v) + tuple(a for a in (C,) if a is not None):
            assert t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()
        if ids is not None:
            assert ids.is_cuda and str(ids.dtype) == "torch.int64" and ids.is_contiguous()
        self._borrowed += [t for t in (x, v, C, ids) if t is not None]
        self._c(self.lib.sg_sort_particles(self.h, _ptr(x), _ptr(v), _ptr(C) if C is not None else None,
                                           _ptr(ids) if ids is not None else None, x.numel() // 3))

    def swap(self, a: int, b: int):
        self._c(self.lib.sg_swap(self.h, int(a), int(b)))

    def debug_wait_test(self):
        self._c(self.lib.sg_debug_wait_test(self.h))

    # ---- flush / sync ----
    def flush(self):
        self._c(self.lib.sg_flush(self.h))

    def sync(self):
        rc = self.lib.sg_sync(self.h)
        self._borrowed.clear()
        self._c(rc)

    # ---- host reads / writes (implicit sync) ----
    def num_leaves(self) -> int:
        n = ctypes.c_int64()
        self._c(self.lib.sg_num_leaves(self.h, ctypes.byref(n)))
        self._borrowed.clear()
        return n.value

    def read_structure(self):
        """(leaf_b int32[n] ascending, masks uint32[n, W])."""
        n = self.num_leaves()
        b = np.empty(n, dtype=np.int32)
        m = np.empty((n, self.W), dtype=np.uint32)
        got = ctypes.c_int64()
        self._c(self.lib.sg_read_structure(self.h, n, ctypes.byref(got), _ptr(b), _ptr(m)))
        assert got.value == n
        return b, m

    def read_field(self, f: int, out: np.ndarray | None = None) -> np.ndarray:
        n = self.num_leaves()
        if out is None:
            out = np.empty((n, self.V), dtype=np.float32)
        self._c(self.lib.sg_read_field(self.h, int(f), n, _ptr(out)))
        return out

    def write_field(self, f: int, vals):
        """vals: (n_leaves, L^3) FP32 host array (numpy or pinned torch CPU
        tensor) in list order."""
        if isinstance(vals, np.ndarray):
            a = np.ascontiguousarray(vals, dtype=np.float32)
            n = a.size // self.V
            self._c(self.lib.sg_write_field(self.h, int(f), _ptr(a), n))
        else:
            assert not vals.is_cuda and vals.is_contiguous()
            self._c(self.lib.sg_write_field(self.h, int(f), _ptr(vals), vals.numel() // self.V))

    def write_field_active(self, f: int, vals):
        """vals: FP32 host array (numpy or torch CPU tensor, pinned is
        fastest) of the active voxels' values, in list order and mask-bit
        order within a leaf; inactive voxels become 0."""
        if isinstance(vals, np.ndarray):
            a = np.ascontiguousarray(vals, dtype=np.float32).reshape(-1)
            self._c(self.lib.sg_write_field_active(self.h, int(f), _ptr(a), a.size))
        else:
            assert not vals.is_cuda and vals.is_contiguous()
            self._c(self.lib.sg_write_field_active(self.h, int(f), _ptr(vals), vals.numel()))

    def stage_active(self, vals) -> int:
        """Start copying the active voxels' values (a pinned torch CPU tensor
        or numpy array, borrowed until its write has run) into an upload
        slot; returns the ticket for write_field_staged."""
        t = ctypes.c_int32()
        if isinstance(vals, np.ndarray):
            vals = np.ascontiguousarray(vals, dtype=np.float32).reshape(-1)
            self._c(self.lib.sg_stage_active(self.h, _ptr(vals), vals.size, ctypes.byref(t)))
        else:
            assert not vals.is_cuda and vals.is_contiguous()
            self._c(self.lib.sg_stage_active(self.h, _ptr(vals), vals.numel(), ctypes.byref(t)))
        if not hasattr(self, "_staged"):
            self._staged = [None, None]
        self._staged[t.value & 1] = vals   # kept until the slot is staged again
        return t.value

    def write_field_staged(self, f: int, ticket: int):
        """Queue: field f = the values staged under ticket."""
        self._c(self.lib.sg_write_field_staged(self.h, int(f), int(ticket)))

    def read_field_active(self, f: int, out: np.ndarray | None = None) -> np.ndarray:
        """The active voxels' values of field f (FP32, list and mask-bit
        order); out, if given, is a contiguous FP32 array of at least that
        many values."""
        if out is None:
            out = np.empty(self.num_active(), dtype=np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous
        got = ctypes.c_int64()
        self._c(self.lib.sg_read_field_active(self.h, int(f), out.size, ctypes.byref(got), _ptr(out)))
        return out.reshape(-1)[:got.value]

    def write_structure(self, leaf_b, masks):
        """Replace the structure with (leaf_b int32[n] ascending, masks
        uint32[n, W]) as read_structure returns them; every field of the
        restored leaves is zero afterwards."""
        b = np.ascontiguousarray(leaf_b, dtype=np.int32)
        m = np.ascontiguousarray(masks, dtype=np.uint32)
        assert m.shape == (b.size, self.W), (m.shape, b.size, self.W)
        self._c(self.lib.sg_write_structure(self.h, b.size, _ptr(b), _ptr(m)))
        self._borrowed.clear()

    def read_sums(self, n: int | None = None) -> np.ndarray:
        n = self.max_sums if n is None else int(n)
        out = np.zeros(n, dtype=np.float64)
        self._c(self.lib.sg_read_sums(self.h, _ptr(out), n))
        self._borrowed.clear()
        return out

    def check(self) -> dict:
        """Invariant-violation counts of the structure and stored values
        (implicit sync; all zero for a sound grid) and the leaves found."""
        r = SgCheckReport()
        self._c(self.lib.sg_check(self.h, ctypes.byref(r)))
        self._borrowed.clear()
        return {name: getattr(r, name) for name, _ in SgCheckReport._fields_}

    def stats(self) -> dict:
        s = SgStats()
        self._c(self.lib.sg_get_stats(self.h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in SgStats._fields_}


def leaf_coords(leaf_b: np.ndarray, N: int, L: int) -> np.ndarray:
    """Global voxel coordinates (n, L^3, 3) of listed leaves (int64)."""
    R = N // L
    b = np.asarray(leaf_b, dtype=np.int64)
    l = np.arange(L ** 3)
    out = np.empty((b.size, L ** 3, 3), dtype=np.int64)
    out[:, :, 0] = (b // (R * R))[:, None] * L + (l // (L * L))[None, :]
    out[:, :, 1] = ((b // R) % R)[:, None] * L + ((l // L) % L)[None, :]
    out[:, :, 2] = (b % R)[:, None] * L + (l % L)[None, :]
    return out


def _grid_fill_hash(self, f: int, seed: int):
    """Queue: field f = counter-based uniform [0,1) values at active voxels."""
    self._c(self.lib.sg_fill_hash(self.h, int(f), int(seed)))


def _grid_num_active(self) -> int:
    """Active voxels of the listed leaves (implicit sync)."""
    n = ctypes.c_int64()
    self._c(self.lib.sg_num_active(self.h, ctypes.byref(n)))
    self._borrowed.clear()
    return n.value


Grid.fill_hash = _grid_fill_hash
Grid.num_active = _grid_num_active


class StepGraph:
    """A CUDA graph of the device work that flushes issue on one stream
    between begin() and end() (sg_graph_*): steady-state steps only -- no
    structure change, list generation or host read while recording."""

    def __init__(self, stream=None):
        import torch
        self.lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = None

    def begin(self):
        _check(self.lib, self.lib.sg_graph_begin(self.stream.cuda_stream))
        return self

    def end(self):
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.sg_graph_end(self.stream.cuda_stream, ctypes.byref(h)))
        self.h = h
        return self

    def __enter__(self):
        return self.begin()

    def __exit__(self, exc_type, exc, tb):
        if exc_type is None:
            self.end()
        else:
            h = ctypes.c_void_p()
            self.lib.sg_graph_end(self.stream.cuda_stream, ctypes.byref(h))
            if h.value:
                self.lib.sg_graph_destroy(h)
        return False

    def launch(self):
        _check(self.lib, self.lib.sg_graph_launch(self.h))

    def close(self):
        if self.h:
            self.lib.sg_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many grids stepped by one persistent launch per step (see
    sg_batch_create in include/sgrid.h)."""

    def __init__(self, grids, src: int, tmp: int, dst: int, coef: float, stream=None):
        import torch
        self.lib = load_library()
        self.grids = list(grids)            # keep the grids alive
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (ctypes.c_void_p * len(self.grids))(*[g.h.value for g in self.grids])
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.sg_batch_create(arr, len(self.grids), int(src), int(tmp), int(dst), float(coef),
                                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    def step(self):
        _check(self.lib, self.lib.sg_batch_step(self.h))

    def set(self, warps_per_cta: int, use_graph: bool = True):
        _check(self.lib, self.lib.sg_batch_set(self.h, int(warps_per_cta), int(bool(use_graph))))

    def set_staging(self, staged: bool):
        """Halo staging: False the register sweep, True the body staged in
        shared memory by bulk tensor copies."""
        _check(self.lib, self.lib.sg_batch_set_staging(self.h, int(bool(staged))))

    def config(self) -> dict:
        w, st = ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib, self.lib.sg_batch_config(self.h, ctypes.byref(w), ctypes.byref(st)))
        return {"warps_per_cta": w.value, "staged": bool(st.value)}

    def autotune(self, trial_steps: int = 3) -> int:
        """Time every (halo staging, warps per CTA) choice and keep the
        fastest; returns its warps per CTA (config() gives both)."""
        w = ctypes.c_int32()
        _check(self.lib, self.lib.sg_batch_autotune(self.h, int(trial_steps), ctypes.byref(w)))
        return w.value

    def read_sums(self) -> np.ndarray:
        out = np.zeros(len(self.grids), dtype=np.float64)
        _check(self.lib, self.lib.sg_batch_read_sums(self.h, out.ctypes.data, len(self.grids)))
        return out

    def info(self) -> dict:
        tl, la, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(self.lib, self.lib.sg_batch_info(self.h, ctypes.byref(tl), ctypes.byref(la), ctypes.byref(w)))
        return {"total_leaves": tl.value, "launches": la.value, "warps_per_cta": w.value}

    def close(self):
        if self.h:
            rc = self.lib.sg_batch_destroy(self.h)
            self.h = None
            _check(self.lib, rc)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
