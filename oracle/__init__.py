"""FP64 CPU oracle of the sparse-grid time-stepping path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product library never
imports, loads or calls anything here, and this package imports nothing from
the product package.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over independent
voxels or particles); this module compiles it with gcc on first use and wraps
it with ctypes.  Each function's docstring names the passage of the paper it
follows (AsyncTaichi, Hu et al. 2021).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, OpenMP). Returns the path."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)
                 or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                   "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "og_create": (P, [I32, I32, I32]),
        "og_destroy": (None, [P]),
        "og_activate_shell": (I64, [P, I64, I64, I32]),
        "og_activate_coords": (I64, [P, P, I64]),
        "og_deactivate_all": (None, [P]),
        "og_num_leaves": (I64, [P]),
        "og_num_active": (I64, [P]),
        "og_read_structure": (None, [P, P, P]),
        "og_read_field": (None, [P, I32, P]),
        "og_write_field": (None, [P, I32, P]),
        "og_write_field64": (None, [P, I32, P]),
        "og_clear": (None, [P, I32]),
        "og_diffuse7": (None, [P, I32, I32, D]),
        "og_box27": (None, [P, I32, I32]),
        "og_sum": (D, [P, I32]),
        "og_p2g": (None, [P, P, P, I64, D, I32, I32]),
        "og_grid_update": (None, [P, I32, I32, D, D, I32]),
        "og_g2p": (None, [P, P, P, I64, D, I32]),
        "og_p2g_apic": (None, [P, P, P, P, I64, D, I32, I32]),
        "og_restrict": (None, [P, P, I32, I32, D]),
        "og_ew": (None, [P, I32, I32, I32, D, D, D, D]),
        "og_activate_tube": (I64, [P, I64, I64]),
        "og_advect": (None, [P, I32, I32, I32, D]),
        "og_maccormack": (None, [P, I32, I32, I32, I32, I32, D]),
        "og_prolong": (None, [P, P, I32, I32, D]),
        "og_g2p_apic": (None, [P, P, P, P, I64, D, I32]),
        "og_get_voxel": (D, [P, I32, I64, I64, I64]),
        "og_voxel_active": (I32, [P, I64, I64, I64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Grid:
    """A two-level sparse grid: pointer root over bitmasked leaves of edge L
    (Sec. 3.1, Fig. 3), holding F scalar fields in FP64."""

    def __init__(self, N: int, L: int, F: int):
        self.lib = _load()
        self.N, self.L, self.F = int(N), int(L), int(F)
        self.R = self.N // self.L
        self.V = self.L ** 3
        self.W = (self.V + 31) // 32
        h = self.lib.og_create(self.N, self.L, self.F)
        if not h:
            raise ValueError("invalid grid description")
        self.h = h

    def close(self):
        if self.h:
            self.lib.og_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- structure ---------------------------------------------------------
    def activate_shell(self, lo2: int, hi2: int, lo_strict: bool) -> int:
        """Activate voxels with lo2 <= D < hi2 (lo2 < D if lo_strict), where
        D = sum_a (2 i_a + 1 - N)^2.  Activation on write, Sec. 3.2 item 3."""
        return int(self.lib.og_activate_shell(self.h, int(lo2), int(hi2), int(bool(lo_strict))))

    def activate_coords(self, xyz) -> int:
        """Activate explicit voxels (n x 3 int32); out-of-domain ones ignored."""
        a = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
        return int(self.lib.og_activate_coords(self.h, _ptr(a), a.shape[0]))

    def deactivate_all(self):
        self.lib.og_deactivate_all(self.h)

    def num_leaves(self) -> int:
        return int(self.lib.og_num_leaves(self.h))

    def num_active(self) -> int:
        return int(self.lib.og_num_active(self.h))

    def structure(self):
        """(leaf_b int32[n] ascending, masks uint32[n, W]) -- the list state."""
        n = self.num_leaves()
        b = np.empty(n, dtype=np.int32)
        m = np.empty((n, self.W), dtype=np.uint32)
        if n:
            self.lib.og_read_structure(self.h, _ptr(b), _ptr(m))
        return b, m

    # --- values ------------------------------------------------------------
    def read_field(self, f: int) -> np.ndarray:
        """FP64 values in list order, shape (n, L^3); 0 at inactive voxels."""
        n = self.num_leaves()
        out = np.empty((n, self.V), dtype=np.float64)
        if n:
            self.lib.og_read_field(self.h, int(f), _ptr(out))
        return out

    def write_field(self, f: int, vals):
        """Set values from FP32 data in list order (n, L^3)."""
        a = np.ascontiguousarray(vals, dtype=np.float32)
        assert a.size == self.num_leaves() * self.V
        self.lib.og_write_field(self.h, int(f), _ptr(a))

    def write_field64(self, f: int, vals):
        """Set values from FP64 data in list order (n, L^3)."""
        a = np.ascontiguousarray(vals, dtype=np.float64)
        assert a.size == self.num_leaves() * self.V
        self.lib.og_write_field64(self.h, int(f), _ptr(a))

    def get(self, f: int, i: int, j: int, k: int) -> float:
        return float(self.lib.og_get_voxel(self.h, int(f), int(i), int(j), int(k)))

    def is_active(self, i: int, j: int, k: int) -> bool:
        return bool(self.lib.og_voxel_active(self.h, int(i), int(j), int(k)))

    # --- operations ----------------------------------------------------------
    def clear(self, f: int):
        self.lib.og_clear(self.h, int(f))

    def diffuse7(self, src: int, dst: int, coef: float):
        """dst = src + coef * (sum_6 src_n - 6 src) on active voxels."""
        self.lib.og_diffuse7(self.h, int(src), int(dst), float(coef))

    def box27(self, src: int, dst: int):
        """dst = (1/27) * sum over the 3^3 neighbourhood of src, on active voxels."""
        self.lib.og_box27(self.h, int(src), int(dst))

    def sum(self, f: int) -> float:
        return float(self.lib.og_sum(self.h, int(f)))

    def p2g(self, x, v, pmass: float, f_mass: int, f_mom0: int):
        xa = np.ascontiguousarray(x, dtype=np.float32)
        va = np.ascontiguousarray(v, dtype=np.float32)
        n = xa.size // 3
        self.lib.og_p2g(self.h, _ptr(xa), _ptr(va), n, float(pmass), int(f_mass), int(f_mom0))

    def grid_update(self, f_mass: int, f_mom0: int, dt: float, gz: float, bound: int):
        self.lib.og_grid_update(self.h, int(f_mass), int(f_mom0), float(dt), float(gz), int(bound))

    def g2p(self, x: np.ndarray, v: np.ndarray, dt: float, f_mom0: int):
        """Updates the FP32 particle arrays x, v (n x 3, C-contiguous) in place."""
        assert x.dtype == np.float32 and v.dtype == np.float32
        assert x.flags.c_contiguous and v.flags.c_contiguous
        self.lib.og_g2p(self.h, _ptr(x), _ptr(v), x.size // 3, float(dt), int(f_mom0))

    def activate_tube(self, lo2: int, hi2: int) -> int:
        """Activate the voxels with lo2 <= (2i+1-N)^2 + (2j+1-N)^2 < hi2 (a tube along k)."""
        return int(self.lib.og_activate_tube(self.h, int(lo2), int(hi2)))

    def advect(self, dst: int, src: int, v0: int, dt: float):
        """dst = src at the RK3 backtrace over dt (trilinear, through the mask).
        dst must differ from src and the velocity fields v0..v0+2 (the loop
        writes dst while it reads them)."""
        if dst == src or v0 <= dst <= v0 + 2:
            raise ValueError("advect: dst aliases src or a velocity field")
        self.lib.og_advect(self.h, int(dst), int(src), int(v0), float(dt))

    def maccormack(self, dst: int, q: int, qhat: int, qtilde: int, v0: int, dt: float):
        """dst = clamp(qhat + (q - qtilde) / 2) to the forward sample's 8 values of q.
        dst must differ from q, qhat, qtilde and the velocity fields."""
        if dst in (q, qhat, qtilde) or v0 <= dst <= v0 + 2:
            raise ValueError("maccormack: dst aliases an input or a velocity field")
        self.lib.og_maccormack(self.h, int(dst), int(q), int(qhat), int(qtilde), int(v0), float(dt))

    def ew(self, dst: int, a: int = -1, b: int = -1, alpha: float = 0.0, beta: float = 0.0, gamma: float = 0.0,
           delta: float = 0.0):
        """dst = alpha a + beta b + gamma a b + delta on the active voxels (-1: absent field)."""
        self.lib.og_ew(self.h, int(dst), int(a), int(b), float(alpha), float(beta), float(gamma), float(delta))

    def restrict_to(self, coarse: "Grid", f_src: int, f_dst: int, w: float):
        """coarse[f_dst][i // 2] += w * self[f_src][i] over the active voxels i,
        activating i // 2 on the coarse grid (its edge is half of this one's)."""
        assert coarse.N * 2 == self.N
        self.lib.og_restrict(self.h, coarse.h, int(f_src), int(f_dst), float(w))

    def prolong_from(self, coarse: "Grid", f_src: int, f_dst: int, w: float):
        """self[f_dst][i] += w * coarse[f_src][i // 2] over the active voxels i."""
        assert coarse.N * 2 == self.N
        self.lib.og_prolong(coarse.h, self.h, int(f_src), int(f_dst), float(w))

    def p2g_apic(self, x, v, C, pmass: float, f_mass: int, f_mom0: int):
        """APIC P2G: C is (n, 9) FP32, row-major 3x3 per particle."""
        xa = np.ascontiguousarray(x, dtype=np.float32)
        va = np.ascontiguousarray(v, dtype=np.float32)
        ca = np.ascontiguousarray(C, dtype=np.float32)
        n = xa.size // 3
        assert ca.size == 9 * n
        self.lib.og_p2g_apic(self.h, _ptr(xa), _ptr(va), _ptr(ca), n, float(pmass), int(f_mass), int(f_mom0))

    def g2p_apic(self, x: np.ndarray, v: np.ndarray, C: np.ndarray, dt: float, f_mom0: int):
        """APIC G2P; updates x, v (n x 3) and C (n x 9), FP32 C-contiguous, in place."""
        for a in (x, v, C):
            assert a.dtype == np.float32 and a.flags.c_contiguous
        assert C.size == 3 * x.size
        self.lib.og_g2p_apic(self.h, _ptr(x), _ptr(v), _ptr(C), x.size // 3, float(dt), int(f_mom0))


def leaf_coords(leaf_b: np.ndarray, N: int, L: int) -> np.ndarray:
    """Global voxel coordinates (n, L^3, 3) of the leaves in list order, local
    index l = (li*L + lj)*L + lk.  Pure indexing, used to sample inputs."""
    R = N // L
    b = leaf_b.astype(np.int64)
    bi, bj, bk = b // (R * R), (b // R) % R, b % R
    l = np.arange(L ** 3)
    li, lj, lk = l // (L * L), (l // L) % L, l % L
    out = np.empty((b.size, L ** 3, 3), dtype=np.int64)
    out[:, :, 0] = bi[:, None] * L + li[None, :]
    out[:, :, 1] = bj[:, None] * L + lj[None, :]
    out[:, :, 2] = bk[:, None] * L + lk[None, :]
    return out
