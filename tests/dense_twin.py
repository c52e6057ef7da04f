"""Dense brute-force twin of the sparse grid, for pinning the oracle on tiny
domains.

Everything here works on plain dense numpy arrays (an N^3 value array plus an
N^3 boolean activity array) and uses library routines (scipy.ndimage filters,
numpy.add.at) for the arithmetic, so that it shares neither data structure nor
code path with the C oracle.  Only tests import it.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage


def shell_active(N: int, lo2: int, hi2: int, lo_strict: bool) -> np.ndarray:
    """Boolean N^3 array of voxels whose D = sum_a (2 i_a + 1 - N)^2 lies in
    the band."""
    c = (2 * np.arange(N, dtype=np.int64) + 1 - N) ** 2
    D = c[:, None, None] + c[None, :, None] + c[None, None, :]
    lo_ok = (D > lo2) if lo_strict else (D >= lo2)
    return lo_ok & (D < hi2)


def structure(active: np.ndarray, L: int):
    """Leaves containing at least one allocated voxel, in ascending root index,
    with the packed bitmask (bit l of word l // 32, k fastest).  `active` here
    must already be the full set of active voxels; leaves are exactly those
    with an active voxel (valid when nothing was deactivated bit-wise)."""
    N = active.shape[0]
    R = N // L
    blocks = active.reshape(R, L, R, L, R, L).transpose(0, 2, 4, 1, 3, 5).reshape(R ** 3, L ** 3)
    has = blocks.any(axis=1)
    leaf_b = np.nonzero(has)[0].astype(np.int32)
    bits = blocks[has]
    nbits = L ** 3
    W = (nbits + 31) // 32
    padded = np.zeros((bits.shape[0], W * 32), dtype=np.uint8)
    padded[:, :nbits] = bits
    masks = np.packbits(padded.reshape(-1, W, 32), axis=2, bitorder="little").view("<u4").reshape(-1, W)
    return leaf_b, masks.astype(np.uint32)


def to_leaves(dense: np.ndarray, leaf_b: np.ndarray, L: int) -> np.ndarray:
    """Values of a dense N^3 array gathered per leaf in list order, (n, L^3)."""
    N = dense.shape[0]
    R = N // L
    blocks = dense.reshape(R, L, R, L, R, L).transpose(0, 2, 4, 1, 3, 5).reshape(R ** 3, L ** 3)
    return blocks[leaf_b]


def from_leaves(vals: np.ndarray, leaf_b: np.ndarray, N: int, L: int) -> np.ndarray:
    """Inverse of to_leaves: scatter (n, L^3) leaf values into a dense array."""
    R = N // L
    blocks = np.zeros((R ** 3, L ** 3), dtype=vals.dtype)
    blocks[leaf_b] = vals
    return blocks.reshape(R, R, R, L, L, L).transpose(0, 3, 1, 4, 2, 5).reshape(N, N, N)


_LAPLACE = np.zeros((3, 3, 3))
_LAPLACE[1, 1, 0] = _LAPLACE[1, 1, 2] = _LAPLACE[1, 0, 1] = _LAPLACE[1, 2, 1] = 1.0
_LAPLACE[0, 1, 1] = _LAPLACE[2, 1, 1] = 1.0
_LAPLACE[1, 1, 1] = -6.0


def diffuse7(x: np.ndarray, active: np.ndarray, coef: float) -> np.ndarray:
    """Dense 7-point step with zero outside the active set and the domain."""
    xm = np.where(active, x, 0.0)
    lap = ndimage.convolve(xm, _LAPLACE, mode="constant", cval=0.0)
    return np.where(active, xm + coef * lap, 0.0)


def box27(t: np.ndarray, active: np.ndarray) -> np.ndarray:
    """Dense 27-point box mean with zero outside the active set and domain."""
    tm = np.where(active, t, 0.0)
    return np.where(active, ndimage.uniform_filter(tm, size=3, mode="constant", cval=0.0), 0.0)


def bspline_weights(X: np.ndarray):
    """Quadratic B-spline base node and weights per axis; X = x * N (FP32)."""
    base = np.floor(X - np.float32(0.5)).astype(np.int64)
    fx = X.astype(np.float64) - base
    w = np.stack([0.5 * (1.5 - fx) ** 2, 0.75 - (fx - 1.0) ** 2, 0.5 * (fx - 0.5) ** 2], axis=-1)
    return base, w


def p2g(x: np.ndarray, v: np.ndarray, N: int, pmass: float):
    """Dense P2G with numpy.add.at: returns (active, mass, mom[3]) N^3 arrays.
    Stencil nodes outside the domain are dropped."""
    X = (x.astype(np.float32) * np.float32(N)).astype(np.float32)
    base, w = bspline_weights(X)
    active = np.zeros((N, N, N), dtype=bool)
    mass = np.zeros((N, N, N))
    mom = np.zeros((3, N, N, N))
    for a in range(3):
        for b in range(3):
            for c in range(3):
                i, j, k = base[:, 0] + a, base[:, 1] + b, base[:, 2] + c
                ok = (i >= 0) & (j >= 0) & (k >= 0) & (i < N) & (j < N) & (k < N)
                wt = w[ok, 0, a] * w[ok, 1, b] * w[ok, 2, c] * pmass
                idx = (i[ok], j[ok], k[ok])
                active[idx] = True
                np.add.at(mass, idx, wt)
                for d in range(3):
                    np.add.at(mom[d], idx, wt * v[ok, d].astype(np.float64))
    return active, mass, mom


def restrict(x: np.ndarray, active: np.ndarray, w: float):
    """Dense restriction onto the half-edge grid: coarse activity = any active
    child (the 2x2x2 block), coarse value = w * sum of the active children
    (block sums by reshape)."""
    N = x.shape[0]
    n = N // 2
    xa = np.where(active, x, 0.0).reshape(n, 2, n, 2, n, 2)
    act = active.reshape(n, 2, n, 2, n, 2).any(axis=(1, 3, 5))
    return w * xa.sum(axis=(1, 3, 5)), act
