"""Seeded synthetic inputs for the sparse-grid workloads.

This module is shared by the CUDA path's callers and by the oracle's callers,
so it holds none of the method's arithmetic: no activation, no list
generation, no stencil or transfer.  It only produces the numbers a workload
starts from:

* the integer band bounds (lo2, hi2) of a spherical shell or ball, given its
  radii (the predicate that uses them is implemented separately on each side);
* initial field values, as a counter-based hash of (seed, global voxel index),
  so that each side can sample the same value at any voxel it holds without a
  dense N^3 array;
* particle positions and velocities;
* the size mix of the batched and serving workloads.

Every generator is deterministic in its seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Shell / band bounds
# ---------------------------------------------------------------------------


def band_bounds(r_inner: float, r_outer: float) -> tuple[int, int]:
    """Integer bounds (lo2, hi2) for r_inner <= dist < r_outer, where a voxel's
    D = sum_a (2 i_a + 1 - N)^2 equals 4 * dist^2.  For integer D,
    D >= 4 r0^2  <=>  D >= ceil(4 r0^2), and D < 4 r1^2 <=> D < ceil(4 r1^2)."""
    lo2 = math.ceil(4.0 * r_inner * r_inner) if r_inner > 0 else 0
    hi2 = math.ceil(4.0 * r_outer * r_outer)
    return int(lo2), int(hi2)


@dataclass
class ShellSpec:
    N: int            # domain edge
    L: int            # leaf edge
    lo2: int
    hi2: int
    lo_strict: bool   # lo2 < D instead of lo2 <= D
    seed: int         # value seed
    note: str = ""


def tiny_shell(seed: int = 0, N: int = 64, L: int = 8) -> ShellSpec:
    """Shell of radius 24 +- U(-2, 2) (seed-jittered), thickness 4, centred in
    a 64^3 domain: active iff r - 2 <= dist < r + 2."""
    rng = np.random.default_rng(seed)
    r = 24.0 + rng.uniform(-2.0, 2.0)
    lo2, hi2 = band_bounds(r - 2.0, r + 2.0)
    return ShellSpec(N, L, lo2, hi2, False, seed, f"shell r={r:.6f} h=2")


def band512(seed: int = 0, N: int = 512, L: int = 8, r: float = 200.0, h: float = 8.0) -> ShellSpec:
    """Narrow band |dist - r| < h of a sphere centred in the domain:
    (2(r-h))^2 < D < (2(r+h))^2 (both bounds strict)."""
    lo2 = int(round(4.0 * (r - h) ** 2))
    hi2 = int(round(4.0 * (r + h) ** 2))
    return ShellSpec(N, L, lo2, hi2, True, seed, f"band r={r} h={h}")


# ---------------------------------------------------------------------------
# Initial values: counter-based hash (splitmix64 finaliser) -> uniform [0,1)
# ---------------------------------------------------------------------------

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function (Steele, Lea & Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (z + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        z = z ^ (z >> np.uint64(31))
    return z


def voxel_values(seed: int, N: int, i, j, k) -> np.ndarray:
    """Uniform [0,1) FP32 value of voxel (i, j, k) of an N^3 domain: the top 24
    bits of splitmix64(seed * 2^40 + linear index) times 2^-24 (exact in FP32)."""
    i = np.asarray(i, dtype=np.uint64)
    j = np.asarray(j, dtype=np.uint64)
    k = np.asarray(k, dtype=np.uint64)
    lin = (i * np.uint64(N) + j) * np.uint64(N) + k
    with np.errstate(over="ignore"):
        key = (np.uint64(seed) << np.uint64(40)) + lin
    h = _splitmix64(key)
    return ((h >> np.uint64(40)).astype(np.float64) * (1.0 / (1 << 24))).astype(np.float32)


def leaf_values(seed: int, N: int, L: int, leaf_b: np.ndarray) -> np.ndarray:
    """voxel_values sampled at every voxel of the given leaves, in the given
    order; shape (n, L^3), local index l = (li*L + lj)*L + lk."""
    R = N // L
    b = np.asarray(leaf_b, dtype=np.int64)
    bi, bj, bk = b // (R * R), (b // R) % R, b % R
    l = np.arange(L ** 3)
    li, lj, lk = l // (L * L), (l // L) % L, l % L
    gi = bi[:, None] * L + li[None, :]
    gj = bj[:, None] * L + lj[None, :]
    gk = bk[:, None] * L + lk[None, :]
    return voxel_values(seed, N, gi, gj, gk)


# ---------------------------------------------------------------------------
# Particles: uniform in 3 seed-placed spheres
# ---------------------------------------------------------------------------


@dataclass
class ParticleSpec:
    N: int                  # grid edge (unit cube, dx = 1/N)
    L: int                  # leaf edge
    n: int                  # particle count
    centers: np.ndarray     # (3, 3)
    radii: np.ndarray       # (3,)
    x: np.ndarray           # (n, 3) float32
    v: np.ndarray           # (n, 3) float32
    dt: float = 1e-4
    gravity: float = 9.8
    bound: int = 3
    pmass: float = 1.0
    note: str = ""


def spheres_particles(seed: int = 0, n: int = 2_000_000, N: int = 256, L: int = 4,
                      r_min: float = 0.05, r_max: float = 0.15,
                      v_sigma: float = 0.1, margin_cells: int = 3) -> ParticleSpec:
    """n particles uniform in 3 spheres with radii U(r_min, r_max) whose
    centres are placed so every sphere lies within [margin, 1 - margin]^3
    (margin = margin_cells / N).  Each particle picks a sphere with probability
    proportional to its volume, then a uniform point inside it; velocities are
    N(0, v_sigma) per component.  Returned as float32 (n, 3) arrays."""
    rng = np.random.default_rng(seed)
    margin = margin_cells / N
    radii = rng.uniform(r_min, r_max, size=3)
    centers = np.stack([rng.uniform(margin + r, 1.0 - margin - r, size=3) for r in radii])
    vol = radii ** 3
    which = rng.choice(3, size=n, p=vol / vol.sum())
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = radii[which] * rng.uniform(0.0, 1.0, size=n) ** (1.0 / 3.0)
    x = (centers[which] + d * rad[:, None]).astype(np.float32)
    v = rng.normal(0.0, v_sigma, size=(n, 3)).astype(np.float32)
    return ParticleSpec(N, L, n, centers, radii, np.ascontiguousarray(x), np.ascontiguousarray(v),
                        note="3 spheres, split by volume")


def cube_particles(seed: int, n: int, N: int, L: int, pad_cells: float = 3.0,
                   v_sigma: float = 0.1) -> ParticleSpec:
    """n particles uniform in the cube [-pad, 1 + pad]^3 (pad = pad_cells / N):
    every face of the domain is crossed, and some particles have no stencil
    node inside it.  Velocities N(0, v_sigma) per component; float32 (n, 3)."""
    rng = np.random.default_rng(seed)
    pad = pad_cells / N
    x = rng.uniform(-pad, 1.0 + pad, size=(n, 3)).astype(np.float32)
    v = rng.normal(0.0, v_sigma, size=(n, 3)).astype(np.float32)
    return ParticleSpec(N, L, n, np.zeros((3, 3)), np.zeros(3), np.ascontiguousarray(x), np.ascontiguousarray(v),
                        note="uniform over the domain and a band around it")


# ---------------------------------------------------------------------------
# Advection over a tube (MacCormack workload): bounds and initial fields
# ---------------------------------------------------------------------------


@dataclass
class TubeSpec:
    N: int
    L: int
    lo2: int          # (2i+1-N)^2 + (2j+1-N)^2 >= lo2
    hi2: int          # ... < hi2
    omega: float      # swirl rate about the tube axis (radians per unit time)
    axial: float      # velocity along k (domain units per unit time)
    dt: float


def tube(N: int = 256, L: int = 8, r_in: float = 0.32, r_out: float = 0.45, omega: float = 2.0,
         axial: float = 0.3) -> TubeSpec:
    """The tube inner radius r_in <= r < r_out (domain units) around the k axis
    through the domain centre: integer bounds on D = 4 N^2 r^2 (ceil, so that
    D >= ceil(4 N^2 r_in^2) <=> r >= r_in for integer D), a solid-body swirl
    plus an axial drift, and dt = 1 / N (under a cell per step)."""
    lo2 = math.ceil(4.0 * N * N * r_in * r_in)
    hi2 = math.ceil(4.0 * N * N * r_out * r_out)
    return TubeSpec(N, L, int(lo2), int(hi2), omega, axial, 1.0 / N)


def tube_fields(spec: TubeSpec, cells: np.ndarray):
    """Initial velocity (3 arrays) and three scalar channels at cell centres
    `cells` (..., 3) in cell units: the swirl u = omega (-(y - 1/2), x - 1/2,
    0) + (0, 0, axial) in domain units, and smooth channels (temperature,
    colour, density) as products of sines; float32."""
    x = (cells[..., 0] + 0.5) / spec.N
    y = (cells[..., 1] + 0.5) / spec.N
    z = (cells[..., 2] + 0.5) / spec.N
    vel = [(-spec.omega * (y - 0.5)), spec.omega * (x - 0.5), np.full_like(x, spec.axial)]
    ch = [0.5 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y),
          0.5 + 0.4 * np.sin(4 * np.pi * z + 1.0) * np.sin(2 * np.pi * (x + y)),
          np.exp(-((x - 0.5) ** 2 + (y - 0.88) ** 2 + (z - 0.5) ** 2) / 0.01)]
    return [v.astype(np.float32) for v in vel], [c.astype(np.float32) for c in ch]


# ---------------------------------------------------------------------------
# Batched and serving size mixes
# ---------------------------------------------------------------------------


def band_for_count(count: float, h: float = 8.0, L: int = 8) -> tuple[int, int, int, bool]:
    """Domain edge and band bounds whose active count is near `count`: a band of
    half-width h around radius r with 4*pi*r^2*2h ~= count, or, when that would
    put r below 2h, a ball with (4/3)*pi*r^3 ~= count.  Returns
    (N, lo2, hi2, lo_strict); the true count is whatever the predicate gives."""
    r_band = math.sqrt(count / (8.0 * math.pi * h))
    if r_band > 2.0 * h:
        r_out = r_band + h
        lo2, hi2 = int(round(4.0 * (r_band - h) ** 2)), int(round(4.0 * (r_band + h) ** 2))
        strict = True
    else:
        r_out = (3.0 * count / (4.0 * math.pi)) ** (1.0 / 3.0)
        lo2, hi2 = 0, int(math.ceil(4.0 * r_out * r_out))
        strict = False
    N = int(L * math.ceil((2.0 * r_out + 4.0) / L))
    return N, lo2, hi2, strict


def batched_mix(seed: int = 0, n_grids: int = 64, lo: float = 1e3, hi: float = 5e6) -> list[ShellSpec]:
    """n_grids shells whose target active counts are log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_grids))
    out = []
    for g, c in enumerate(counts):
        N, lo2, hi2, strict = band_for_count(float(c))
        out.append(ShellSpec(N, 8, lo2, hi2, strict, seed * 1000 + g, f"target {c:.0f}"))
    return out


@dataclass
class Job:
    arrival_s: float
    spec: ShellSpec
    steps: int


def serving_arrivals(seed: int, rate: float, duration_s: float,
                     lo: float = 1e4, hi: float = 1e7, steps_lo: int = 10, steps_hi: int = 200) -> list[Job]:
    """Poisson arrivals at `rate` per second over `duration_s`, each a diffusion
    job with a log-uniform active size in [lo, hi] and U{steps_lo..steps_hi}
    steps."""
    rng = np.random.default_rng(seed)
    jobs, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        c = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        N, lo2, hi2, strict = band_for_count(c)
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        jobs.append(Job(t, ShellSpec(N, 8, lo2, hi2, strict, int(rng.integers(1 << 30)), f"target {c:.0f}"), steps))
    return jobs
