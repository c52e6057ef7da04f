"""Benchmark of the sparse-grid hot path on GB300.  Prints ONE JSON line.

Headline workload: the 512^3 narrow band |dist - 200| < 8 over 8^3 leaves
(26,104 leaves, 8,047,608 active voxels); one step = clear(t), diffuse7(x->t),
box27(t->y), swap(x,y), sum(x), through the library's queue with every
inter-kernel pass on (one fused launch).  The eager form (list regenerated
and activation checked in every kernel, 12 launches per step) is timed beside
it.  Further legs (skipped with --only fused or on more than one rank):
  tiny      the 64^3 shell, 20 steps of activate, list generation, diffuse7
            and swap, all passes against eager: launches per step;
  batched   64 independent band/ball grids, active sizes log-uniform in
            1e3..5e6, one persistent launch per step in a CUDA graph
            (autotuned warps per CTA), against the same grids stepped one
            after another, fused and eager;
  particles 2M particles in 3 spheres, 256^3 grid of 4^3 leaves: deactivate,
            P2G with activation, grid update, G2P per step;
  mpm_apic  the same particles with APIC transfers on two grids in turn:
            separate G2P (C stored) + P2G against the fused G2P2G (C on chip);
  multigrid a 4-level V-cycle (restrict, smooth, prolong) from the 512^3 band,
            with and without activation demotion, and eager;
  micro     the paper's microbenchmarks (chain_copy, increments, fill_array,
            sparse_saxpy, autodiff, stencil_reduction) on the 512^3 band;
  advection MacCormack/RK3 advection of 3 channels over the 256^3 tube, all
            passes against no fusion and eager;
  ablation  the band step with each of the four passes switched off in turn;
  serving   Poisson arrivals of band jobs (1e4..1e7 voxels, 10..200 steps)
            into the continuous-batching server: p50/p99 job latency;
  band1024  the 1024^3 band |dist - 400| < 8, far larger than L2;
  restructure the 1024^3 band with its structure changed before every step.

Timing: W untimed warm-up steps, then K timed steps, each bracketed by CUDA
events on the launching stream; before every timed step of the band
workloads a 512 MB buffer is written to flush L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on the headline
workload (each step one full oracle step) and prints its line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from workload import (ShellSpec, band512, batched_mix, leaf_values, serving_arrivals, spheres_particles,  # noqa: E402
                      tiny_shell,
                      tube, tube_fields)

METRIC = "active voxel-steps/s"
BYTES_PER_LEAF_FUSED = 2 * 2048 + 27 * 4 + 64 + 4  # x read, x' written, nbr row, mask, list entry
BYTES_PER_LEAF_EAGER = 6 * 2048                    # clear W, diffuse R+W, box27 R+W, sum R (leaf passes)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def aggregate_max(values, dist=None, device="cpu"):
    """Per-quantity maximum over ranks (the slowest rank bounds the job's
    time); identity on one rank."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(world: int, units_per_rank: float, steps: int, seconds: float) -> float:
    """Whole-job throughput: every rank processes its own replica of the
    workload (weak scaling), so the units of all ranks over the slowest time."""
    return world * units_per_rank * steps / seconds


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the fused band step's kernel for each stencil variant
KERNEL_NAMES = {0: "k_sweep_diffuse_box<false,false,true>", 1: "k_diffuse_box<false,false,true>",
                2: "k_sweep_columns<false,false,true>", 3: "k_sweep_jruns<false,false,true>",
                4: "k_sweep_tma<true>"}


def code_sha1(path: str) -> str:
    """sha1 of a C/CUDA source with its comments and blank lines removed: it
    changes with the code, not with the comments."""
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return hashlib.sha1("\n".join(l.rstrip() for l in src.splitlines() if l.strip()).encode()).hexdigest()


# sources that shape each variant's fused-step access order: the kernel and
# the list generation / region-mask / run-record kernels (sg_structure.cu)
KERNEL_SRCS = {0: ["sg_sweep.cu", "sg_structure.cu"], 1: ["sg_stencil.cu", "sg_structure.cu"],
               2: ["sg_sweep.cu", "sg_structure.cu"], 3: ["sg_sweep.cu", "sg_structure.cu"],
               4: ["sg_sweep_tma.cu", "sg_structure.cu"]}


def sources_sha1(variant: int) -> str:
    """Combined code sha1 (code_sha1 of each source, in order) of the sources
    that shape the variant's fused kernel and its access order."""
    csrc = os.path.join(ROOT, "paper_2012_08141_gb300", "csrc")
    return hashlib.sha1("".join(code_sha1(os.path.join(csrc, f)) for f in KERNEL_SRCS[variant]).encode()).hexdigest()


def traffic_record(variant: int, workload: str = "512^3 band", path: str | None = None):
    """DRAM bytes per launch of the fused kernel on the workload from the
    committed ncu summary, or None when that summary is of another kernel or
    any source that shapes the kernel's access order changed since it was
    captured."""
    p = path or os.path.join(ROOT, "profiles", "traffic.json")
    try:
        recs = json.load(open(p))
        for rec in (recs if isinstance(recs, list) else [recs]):
            if (rec.get("sources_sha1") == sources_sha1(variant) and rec.get("kernel") == KERNEL_NAMES[variant]
                    and rec.get("workload", "").startswith(workload)):
                return rec.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during a timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm: band workloads
# ---------------------------------------------------------------------------

def setup_band(sg, spec, opts, x_host, variant=3, cap=32768):
    g = sg.Grid(spec.N, 3, 3, max_leaves=cap, max_sums=1, scratch_mask=0b010)
    g.set_opts(opts)
    g.set_stencil_variant(variant)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    g.list_gen()
    if x_host is None:
        g.fill_hash(0, spec.seed % (1 << 24))
    else:
        assert g.num_leaves() == x_host.shape[0]
        g.write_field(0, x_host)
    return g


def band_step(g):
    g.clear(1)
    g.diffuse7(0, 1, 0.1)
    g.box27(1, 2)
    g.swap(0, 2)
    g.reduce_sum(0, 0)
    g.flush()


def time_steps(torch, step_fn, steps, warmup, flush_buf, stream, launches_fn=None):
    for _ in range(warmup):
        step_fn()
    torch.cuda.synchronize()
    l0 = launches_fn() if launches_fn else 0
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            if flush_buf is not None:
                flush_buf.zero_()                      # evict L2 between timed steps
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step_fn()
            b.record(stream)
            evs.append((a, b))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    launches = (launches_fn() - l0) if launches_fn else 0
    return ms, launches


def leaves_of(sg, spec):
    R = spec.N // spec.L
    p = sg.Grid(spec.N, 3, 1, max_leaves=R ** 3)
    p.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    n = p.num_leaves()
    p.close()
    return n


def bench_band1024(torch, sg, steps, warmup, flush_buf, stream, variant=3):
    """The 1024^3 band (442 MB of fields, 3.4x L2): timed with L2 flushed before
    every step as the headline is, and back to back without the flush (the
    inputs alone exceed L2, so no step finds its x in L2: it reads the list from
    the start while L2 holds the end of the previous step's output)."""
    spec = ShellSpec(1024, 8, int(4 * 392 ** 2), int(4 * 408 ** 2), True, 5, "band r=400 h=8")
    n = leaves_of(sg, spec)
    g = setup_band(sg, spec, sg.SG_OPT_ALL, None, variant=variant, cap=n)
    act = g.num_active()
    peak, kind = peaks()
    out = {"workload": "1024^3 band |dist-400|<8, 8^3 leaves", "active_voxels": act, "leaves": n,
           "kernel": KERNEL_NAMES[variant], "bytes_per_launch": n * BYTES_PER_LEAF_FUSED,
           "traffic": traffic_record(variant, "1024^3 band")}
    for key, fb in (("flushed", flush_buf), ("unflushed", None)):
        ms, _ = time_steps(torch, lambda: band_step(g), steps, warmup, fb, stream)
        t = sum(ms) / 1e3
        ach = n * BYTES_PER_LEAF_FUSED / (t / steps) / 1e9
        r = {"value": act * steps / t, "ms_per_step": t * 1e3 / steps, "achieved_gbs": ach, "frac": ach / peak,
             "l2": "flushed before every timed step (512 MB write)" if fb is not None
             else "not flushed: inputs (442 MB) larger than L2"}
        if key == "flushed":
            out.update(r)
        else:
            out["unflushed"] = r
    g.close()
    return out


def bench_tiny(torch, sg, steps, warmup, flush_buf, stream):
    """The tiny eager workload: the 64^3 shell of radius 24 +- 2 (seed 0),
    8^3 leaves; each step activates the shell, regenerates the list, diffuses
    into a second field (dt k = 0.1) and swaps, with every pass on and in
    the eager form.  Launch-bound: the figure of merit is launches per step."""
    spec = tiny_shell(0)
    out = {"workload": "64^3 shell r=24+-2 h=2, 8^3 leaves: activate, list generation, diffuse7, swap per step",
           "l2": "flushed before every timed step (512 MB write)"}
    for mode, opts in (("all", sg.SG_OPT_ALL), ("eager", sg.SG_OPT_EAGER)):
        g = sg.Grid(spec.N, 3, 2, max_leaves=512)
        g.set_opts(opts)
        g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
        g.list_gen()
        b, _ = g.read_structure()
        g.write_field(0, leaf_values(spec.seed, spec.N, spec.L, b))
        act = g.num_active()

        def step():
            g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
            g.list_gen()
            g.diffuse7(0, 1, 0.1)
            g.swap(0, 1)
            g.flush()

        ms, launches = time_steps(torch, step, steps, warmup, flush_buf, stream, lambda: g.stats()["launches"])
        t = sum(ms) / 1e3
        out[mode] = {"ms_per_step": t * 1e3 / steps, "launches_per_step": launches / steps,
                     "value": act * steps / t, "active_voxels": act}
        g.close()
    out["unit"] = "voxel-steps/s"
    return out


def bench_restructure(torch, sg, steps, warmup, flush_buf, stream):
    """The 1024^3 band with its structure changed before every fused step:
    deactivate all, activate one of two bands (radius 400 or 401, h = 8) in
    turn, so every step regenerates the list and rebuilds the region masks and
    run records before its fused step.  Times the whole step."""
    specs = [ShellSpec(1024, 8, int(4 * (r - 8) ** 2), int(4 * (r + 8) ** 2), True, 5, f"band r={r} h=8")
             for r in (400, 401)]
    n = max(leaves_of(sg, s) for s in specs)
    g = sg.Grid(1024, 3, 3, max_leaves=n, max_sums=1, scratch_mask=0b010)
    k = [0]

    def step():
        s = specs[k[0] & 1]
        k[0] += 1
        g.deactivate_all()
        g.activate_shell(s.lo2, s.hi2, s.lo_strict)
        g.list_gen()
        g.clear(1)
        g.diffuse7(0, 1, 0.1)
        g.box27(1, 2)
        g.swap(0, 2)
        g.reduce_sum(0, 0)
        g.flush()

    ms, launches = time_steps(torch, step, steps, warmup, flush_buf, stream, lambda: g.stats()["launches"])
    g.close()
    return {"workload": "1024^3 band, structure changed every step (deactivate, activate r = 400 / 401, list, "
                        "region masks and run records, fused step)", "leaves": n,
            "ms_per_step": sum(ms) / len(ms), "launches_per_step": launches / steps,
            "l2": "flushed before every timed step (512 MB write)"}


def bench_ablation(torch, sg, x_host, steps, warmup, flush_buf, stream):
    """The four passes switched off one at a time (Table 3's ablation, on the
    512^3 band).  The step re-activates the band first, as the paper's steps
    do, so that activation demotion has an activation to remove: activate,
    clear, diffuse7, box27, swap, sum."""
    spec = band512()
    out = {"workload": "512^3 band, per step: activate (same band), clear, diffuse7, box27, swap, sum",
           "l2": "flushed before every timed step (512 MB write)"}
    base = None
    for name, opts in (("all", sg.SG_OPT_ALL), ("no_lgr", sg.SG_OPT_ALL & ~sg.SG_OPT_LGR),
                       ("no_ad", sg.SG_OPT_ALL & ~sg.SG_OPT_AD), ("no_fusion", sg.SG_OPT_ALL & ~sg.SG_OPT_FUSE),
                       ("no_dse", sg.SG_OPT_ALL & ~sg.SG_OPT_DSE), ("eager", sg.SG_OPT_EAGER)):
        g = setup_band(sg, spec, opts, x_host)

        def step():
            g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
            band_step(g)

        st0 = g.stats()
        ms, _ = time_steps(torch, step, steps, warmup, flush_buf, stream)
        st1 = g.stats()
        n = steps + warmup
        row = {"ms_per_step": sum(ms) / len(ms), "launches_per_step": (st1["launches"] - st0["launches"]) / n,
               "listgen_per_step": (st1["listgen_run"] - st0["listgen_run"]) / n,
               "activations_per_step": (st1["act_launched"] - st0["act_launched"]) / n}
        if base is None:
            base = row["ms_per_step"]
        row["slowdown"] = row["ms_per_step"] / base
        out[name] = row
        g.close()
    return out


def bench_batched(torch, sg, steps, warmup, flush_buf, stream):
    specs = batched_mix(0, n_grids=64, lo=1e3, hi=5e6)
    grids = []
    for s in specs:
        g = sg.Grid(s.N, 3, 3, max_leaves=max(1, leaves_of(sg, s)), max_sums=1, scratch_mask=0b010)
        g.activate_shell(s.lo2, s.hi2, s.lo_strict)
        g.list_gen()
        g.fill_hash(0, s.seed % (1 << 24))
        grids.append(g)
    active = sum(g.num_active() for g in grids)
    leaves = sum(g.num_leaves() for g in grids)
    bt = sg.Batch(grids, 0, 1, 2, 0.1)
    # every (halo staging, warps per CTA) choice of the autotuner, timed here too
    cands = {}
    for staged, wc in ((False, 2), (False, 4), (False, 8), (True, 8)):
        bt.set_staging(staged)
        bt.set(wc, True)
        msc, _ = time_steps(torch, bt.step, max(3, steps // 2), 2, flush_buf, stream)
        cands[("staged" if staged else "register") + f"_w{wc}"] = sum(msc) / len(msc)
    w = bt.autotune(3)
    cfg = bt.config()
    l0 = bt.info()["launches"]
    ms, _ = time_steps(torch, bt.step, steps, warmup, flush_buf, stream)
    launches = (bt.info()["launches"] - l0) / (steps + warmup)
    t_b = sum(ms) / 1e3
    bt.close()

    def seq_step():
        for g in grids:
            band_step(g)

    k2 = max(3, steps // 3)
    res = {}
    for name, opts in (("sequential_fused", sg.SG_OPT_ALL), ("sequential_eager", sg.SG_OPT_EAGER)):
        for g in grids:
            g.set_opts(opts)
        l0 = sum(g.stats()["launches"] for g in grids)
        ms2, _ = time_steps(torch, seq_step, k2, 2, flush_buf, stream)
        l1 = sum(g.stats()["launches"] for g in grids)
        t2 = sum(ms2) / 1e3
        res[name] = {"value": active * k2 / t2, "ms_per_step": t2 * 1e3 / k2, "launches_per_step": (l1 - l0) / (k2 + 2)}
    for g in grids:
        g.close()
    return {"workload": "64 band/ball grids, active sizes log-uniform 1e3..5e6 (seed 0)", "grids": len(grids),
            "active_voxels": active, "leaves": leaves, "value": active * steps / t_b,
            "ms_per_step": t_b * 1e3 / steps, "launches_per_step": launches, "warps_per_cta": w,
            "halo_staging": "shared memory (bulk tensor copies)" if cfg["staged"] else "registers",
            "autotune_candidates_ms": cands, "cuda_graph": True, **res,
            "over_sequential_eager": (active * steps / t_b) / res["sequential_eager"]["value"]}


def bench_particles(torch, sg, steps, warmup, flush_buf, stream):
    spec = spheres_particles(0)
    g = sg.Grid(spec.N, 2, 4, max_leaves=(spec.N // 4) ** 3, max_sums=1)
    x = torch.from_numpy(spec.x).cuda()
    v = torch.from_numpy(spec.v).cuda()

    def step():
        g.deactivate_all()
        g.p2g(x, v, spec.pmass, 0, 1)
        g.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        g.g2p(x, v, spec.dt, 1)
        g.flush()

    ms, launches = time_steps(torch, step, steps, warmup, flush_buf, stream, lambda: g.stats()["launches"])
    t = sum(ms) / 1e3
    g.sync()
    leaves = g.num_leaves()
    g.close()
    # the same step with the particle arrays (and the caller's ids) reordered
    # into bin order every 10 steps (sg_sort_particles), the sort inside the
    # timed steps that run it
    gs = sg.Grid(spec.N, 2, 4, max_leaves=(spec.N // 4) ** 3, max_sums=1)
    xs = torch.from_numpy(spec.x).cuda()
    vs = torch.from_numpy(spec.v).cuda()
    ids = torch.arange(spec.n, dtype=torch.int64, device="cuda")
    k = [0]

    def sorted_step():
        gs.deactivate_all()
        gs.p2g(xs, vs, spec.pmass, 0, 1)
        gs.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        gs.g2p(xs, vs, spec.dt, 1)
        if k[0] % 10 == 0:
            gs.sort_particles(xs, vs, ids=ids)
        gs.flush()
        k[0] += 1

    ms_s, _ = time_steps(torch, sorted_step, max(steps, 20), warmup, flush_buf, stream)
    gs.sync()
    gs.close()
    t_s = sum(ms_s) / 1e3
    return {"workload": "2M particles in 3 spheres, 256^3 grid of 4^3 leaves, P2G+grid update+G2P",
            "particles": spec.n, "leaves": leaves, "value": spec.n * steps / t, "unit": "particle-steps/s",
            "ms_per_step": t * 1e3 / steps, "launches_per_step": launches / steps,
            "l2": "flushed before every timed step (512 MB write)",
            "stream_bytes_per_particle": 72,
            "stream_hbm_frac": spec.n * 72 * steps / t / 1e9 / peaks()[0],
            "grid_atomics_per_s": spec.n * 27 * 4 * steps / t,
            "sorted_every_10": {"ms_per_step": t_s * 1e3 / len(ms_s), "value": spec.n * len(ms_s) / t_s,
                                "unit": "particle-steps/s", "steps": len(ms_s),
                                "note": "arrays and int64 ids reordered into bin order every 10th step"}}


def bench_mpm_apic(torch, sg, steps, warmup, flush_buf, stream):
    """2M particles, APIC transfers, two grids used in turn.  Separate form:
    deactivate, APIC G2P (C stored), APIC P2G (binned again), grid update.
    Fused form: deactivate, G2P2G (C kept on chip), grid update; and the same
    with the particle arrays sorted once into the order of the binning the
    fused steps reuse (sg_sort_particles)."""
    spec = spheres_particles(0)
    C0 = np.zeros((spec.n, 9), np.float32)
    out = {"workload": "2M particles in 3 spheres, 256^3 grid of 4^3 leaves, APIC transfers (MLS-MPM, Sec. 8.3)",
           "particles": spec.n}
    for form in ("separate", "fused", "fused_sorted"):
        A = sg.Grid(spec.N, 2, 4, max_leaves=(spec.N // 4) ** 3, max_sums=1)
        B = sg.Grid(spec.N, 2, 4, max_leaves=(spec.N // 4) ** 3, max_sums=1)
        x = torch.from_numpy(spec.x).cuda()
        v = torch.from_numpy(spec.v).cuda()
        C = torch.from_numpy(C0).cuda()
        A.p2g_apic(x, v, C, spec.pmass, 0, 1)
        A.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
        if form == "fused_sorted":
            # the arrays (and the caller's ids) into the order of the binning
            # the fused steps reuse, once, before the timed steps
            ids = torch.arange(spec.n, dtype=torch.int64, device="cuda")
            A.sort_particles(x, v, C, ids)
            A.flush()
        st = {"src": A, "dst": B}

        def step():
            src, dst = st["src"], st["dst"]
            dst.deactivate_all()
            if form != "separate":
                src.g2p2g(dst, x, v, spec.dt, 1, spec.pmass, 0, 1)
            else:
                src.g2p_apic(x, v, C, spec.dt, 1)
                src.flush()
                dst.p2g_apic(x, v, C, spec.pmass, 0, 1)
            dst.grid_update(0, 1, spec.dt, spec.gravity, spec.bound)
            dst.flush()
            st["src"], st["dst"] = dst, src

        launches = lambda: A.stats()["launches"] + B.stats()["launches"]
        ms, nl = time_steps(torch, step, steps, warmup, flush_buf, stream, launches)
        t = sum(ms) / 1e3
        A.sync()
        B.sync()
        out[form] = {"value": spec.n * steps / t, "unit": "particle-steps/s", "ms_per_step": t * 1e3 / steps,
                     "launches_per_step": nl / steps}
        A.close()
        B.close()
    out["fused_over_separate"] = out["fused"]["value"] / out["separate"]["value"]
    out["fused_sorted"]["note"] = "arrays and int64 ids sorted once into the reused binning's order"
    out["C_bytes_not_moved_per_step"] = spec.n * 72
    out["l2"] = "flushed before every timed step (512 MB write)"
    return out


def vcycle(G):
    """One V-cycle over the levels G (down: clear, restrict, smooth; up:
    prolong, smooth, swap), flushed."""
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


def bench_multigrid(torch, sg, steps, warmup, flush_buf, stream):
    """V-cycle pattern over four levels (the 512^3 band, then 256^3, 128^3,
    64^3, 8^3 leaves): down, clear b on the coarse level, restrict, smooth;
    up, prolong and smooth.  The coarse levels' structure comes only from the
    restrictions, so with activation demotion (Sec. 6.3) the repeated
    restrictions leave it unchanged and their list generations are removed.
    Timed with all passes, without activation demotion, and eager."""
    spec = band512()
    out = {"workload": "4-level V-cycle: 512^3 band |dist-200|<8 and its 256^3, 128^3, 64^3 restrictions, 8^3 leaves",
           "l2": "flushed before every timed step (512 MB write)"}
    for name, opts in (("all_passes", sg.SG_OPT_ALL), ("no_demotion", sg.SG_OPT_ALL & ~sg.SG_OPT_AD),
                       ("eager", sg.SG_OPT_EAGER)):
        G = [sg.Grid(512 >> l, 3, 3, max_leaves=32768, max_sums=1) for l in range(4)]
        for g in G:
            g.set_opts(opts)
        G[0].activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
        G[0].fill_hash(0, 3)

        stat = lambda key: sum(g.stats()[key] for g in G)
        vcycle(G)                                  # the first cycle activates the coarse levels
        for g in G:
            g.sync()
        l0, g0 = stat("launches"), stat("listgen_run")
        ms, _ = time_steps(torch, lambda: vcycle(G), steps, warmup, flush_buf, stream)
        l1, g1 = stat("launches"), stat("listgen_run")
        n = steps + warmup
        out[name] = {"ms_per_cycle": sum(ms) / len(ms), "launches_per_cycle": (l1 - l0) / n,
                     "listgen_per_cycle": (g1 - g0) / n, "leaves": [g.num_leaves() for g in G]}
        for g in G:
            g.close()
    # all passes, the cycle recorded as CUDA graphs on a stream of their own:
    # one graph per swap parity, replayed alternately (one cycle per timed step)
    gs = torch.cuda.Stream()
    G = [sg.Grid(512 >> l, 3, 3, max_leaves=32768, max_sums=1, stream=gs) for l in range(4)]
    G[0].activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    G[0].fill_hash(0, 3)
    vcycle(G)
    vcycle(G)
    for g in G:
        g.sync()
    graphs = [sg.StepGraph(stream=gs), sg.StepGraph(stream=gs)]
    for gr in graphs:
        with gr:
            vcycle(G)
    turn = [0]

    def replay():
        graphs[turn[0] & 1].launch()
        turn[0] += 1

    ms, _ = time_steps(torch, replay, steps, warmup + (warmup & 1), flush_buf, gs)
    out["all_passes_graph"] = {"ms_per_cycle": sum(ms) / len(ms), "graph_launches_per_cycle": 1,
                               "kernels_per_cycle": 15}
    for gr in graphs:
        gr.close()
    for g in G:
        g.close()
    out["graph_over_all_passes"] = out["all_passes"]["ms_per_cycle"] / out["all_passes_graph"]["ms_per_cycle"]
    out["no_demotion_over_all_passes"] = out["no_demotion"]["ms_per_cycle"] / out["all_passes"]["ms_per_cycle"]
    out["eager_over_all_passes"] = out["eager"]["ms_per_cycle"] / out["all_passes"]["ms_per_cycle"]
    return out


MICRO = {
    # the paper's microbenchmarks (Supp. Sec. 1) as element-wise struct-fors on
    # fields 0 (x), 1 (y), 2 (z), 3 (scratch), 4 (grad)
    "chain_copy": lambda g: (g.ew(1, 0, alpha=1.0, delta=1.0), g.ew(2, 1, alpha=1.0, delta=4.0)),
    "increments": lambda g: [g.ew(0, 0, alpha=1.0, delta=1.0) for _ in range(10)],
    "fill_array": lambda g: [g.ew(2, delta=float(k)) for k in range(10)],
    "sparse_saxpy": lambda g: (g.ew(2, 0, 1, 2.0, 1.0), g.ew(1, 2, 0, 3.0, 1.0), g.ew(2, 2, 1, 1.0, 1.0)),
    "autodiff": lambda g: [(g.ew(3, 0, 0, gamma=1.0), g.reduce_sum(3, 0), g.ew(4, 4, 0, 1.0, 2.0))
                           for _ in range(10)],
    "stencil_reduction": lambda g: (g.diffuse7(0, 1, 0.1), g.reduce_sum(1, 0)),
}


def bench_micro(torch, sg, steps, warmup, flush_buf, stream):
    """The microbenchmarks on the 512^3 band (26,104 leaves, 5 fields), each
    case flushed as one program: all passes against eager."""
    spec = band512()
    out = {"workload": "paper microbenchmarks as element-wise struct-fors on the 512^3 band",
           "l2": "flushed before every timed step (512 MB write)"}
    for name, body in MICRO.items():
        row = {}
        for mode, opts in (("all_passes", sg.SG_OPT_ALL), ("eager", sg.SG_OPT_EAGER)):
            g = sg.Grid(512, 3, 5, max_leaves=32768, max_sums=1, scratch_mask=0b01000)
            g.set_opts(opts)
            g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
            g.fill_hash(0, 1)
            g.fill_hash(1, 2)
            g.sync()

            def step():
                body(g)
                g.flush()

            ms, nl = time_steps(torch, step, steps, warmup, flush_buf, stream, lambda: g.stats()["launches"])
            row[mode] = {"ms": sum(ms) / len(ms), "launches": nl / len(ms)}
            g.close()
        row["speedup"] = row["eager"]["ms"] / row["all_passes"]["ms"]
        out[name] = row
    return out


def bench_advection(torch, sg, steps, warmup, flush_buf, stream):
    """MacCormack / RK3 advection of three channels over the 256^3 tube
    (inner radius 0.32, outer 0.45; Sec. 8.2, Supp. Sec. 4.2), written channel
    by channel (forward advection, backward advection, correction, swap):
    all passes, without task fusion, and eager."""
    spec = tube(256, 8)
    out = {"workload": "MacCormack/RK3 advection of 3 channels, 256^3 tube r in [0.32, 0.45), 8^3 leaves",
           "l2": "flushed before every timed step (512 MB write)"}
    scratch = sum(1 << (5 + 4 * c) for c in range(3))
    for name, opts in (("all_passes", sg.SG_OPT_ALL), ("no_fusion", sg.SG_OPT_ALL & ~sg.SG_OPT_FUSE),
                       ("eager", sg.SG_OPT_EAGER)):
        g = sg.Grid(256, 3, 15, max_leaves=32768, scratch_mask=scratch)
        g.set_opts(opts)
        g.activate_tube(spec.lo2, spec.hi2)
        b, _ = g.read_structure()
        R = 256 // 8
        bi, bj, bk = b // (R * R), (b // R) % R, b % R
        l = np.arange(512)
        cells = np.stack([bi[:, None] * 8 + l[None, :] // 64, bj[:, None] * 8 + (l[None, :] // 8) % 8,
                          bk[:, None] * 8 + l[None, :] % 8], -1).astype(np.float64)
        vel, ch = tube_fields(spec, cells)
        for a in range(3):
            g.write_field(a, vel[a])
        for c in range(3):
            g.write_field(3 + 4 * c, ch[c])
        n_active = g.num_active()

        def step():
            for c in range(3):
                q, qh, qt, qn = 3 + 4 * c, 4 + 4 * c, 5 + 4 * c, 6 + 4 * c
                g.advect(qh, q, 0, spec.dt)
                g.advect(qt, qh, 0, -spec.dt)
                g.maccormack(qn, q, qh, qt, 0, spec.dt)
                g.swap(q, qn)
            g.flush()

        ms, nl = time_steps(torch, step, steps, warmup, flush_buf, stream, lambda: g.stats()["launches"])
        t = sum(ms) / 1e3
        out[name] = {"ms_per_step": t * 1e3 / steps, "launches_per_step": nl / steps,
                     "value": 3 * n_active * steps / t, "unit": "channel voxel-steps/s"}
        out["active_voxels"] = n_active
        out["leaves"] = len(b)
        g.close()
    out["all_over_no_fusion"] = out["no_fusion"]["ms_per_step"] / out["all_passes"]["ms_per_step"]
    out["all_over_eager"] = out["eager"]["ms_per_step"] / out["all_passes"]["ms_per_step"]
    return out


def bench_serving(torch, sg, rates=(50, 100, 200, 500, 1000, 2000), duration=2.0, cap_s=60.0):
    from paper_2012_08141_gb300.serve import Server
    out = []
    for rate in rates:
        jobs = serving_arrivals(1000 + rate, rate, duration)
        srv = Server(max_jobs=256, warps_per_cta=4, hbm_reserve=8 << 30)
        ids, k = [], 0
        max_pending = max_resident = 0
        t0 = time.perf_counter()
        while True:
            now = time.perf_counter() - t0
            while k < len(jobs) and jobs[k].arrival_s <= now:
                ids.append(srv.submit(jobs[k].spec, jobs[k].steps))
                k += 1
            st = srv.stats()
            max_pending = max(max_pending, st["pending"])
            max_resident = max(max_resident, st["resident"])
            if k == len(jobs) and st["completed"] + st["failed"] == len(jobs):
                break
            if now > duration + cap_s:
                break
            if st["resident"] or st["pending"]:
                srv.tick()
            else:
                time.sleep(min(1e-4, max(0.0, jobs[k].arrival_s - now)) if k < len(jobs) else 0)
        elapsed = time.perf_counter() - t0
        st = srv.stats()
        lat = sorted(srv.job(i)["t_done"] - srv.job(i)["t_submit"] for i in ids if srv.job(i)["state"] == 2)
        out.append({"rate_per_s": rate, "jobs": len(jobs), "completed": st["completed"], "failed": st["failed"],
                    "p50_ms": 1e3 * lat[len(lat) // 2] if lat else None,
                    "p99_ms": 1e3 * lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)] if lat else None,
                    "voxel_steps_per_s": st["voxel_steps"] / elapsed, "ticks": st["ticks"],
                    "admission_waits": st["admission_waits"], "max_queued": max_pending, "max_resident": max_resident,
                    "wall_s": elapsed})
        srv.close()
    return {"workload": "Poisson arrivals of band jobs, 1e4..1e7 voxels, 10..200 steps", "duration_s": duration,
            "rates": out}


def run_ours(args):
    import torch
    import paper_2012_08141_gb300 as sg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    sg.load_library()

    spec = band512()
    probe = sg.Grid(spec.N, 3, 1, max_leaves=32768)
    probe.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    leaf_b, masks = probe.read_structure()
    probe.close()
    n_leaves = len(leaf_b)
    n_active = int(np.unpackbits(masks.view(np.uint8)).sum())
    x_host = leaf_values(spec.seed, spec.N, spec.L, leaf_b)
    flush_buf = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    if args.skip_headline:  # profiling runs of one extra leg
        ms_f, launches_f, ms_e, launches_e, e2e_steps, e2e_s = [float("nan")], 0, [float("nan")], 0, 0, 1.0
        clk = None
    else:
        fused = setup_band(sg, spec, sg.SG_OPT_ALL, x_host, args.variant)
        eager = setup_band(sg, spec, sg.SG_OPT_EAGER, x_host, args.variant)

        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev) as clk:
            ms_f, launches_f = time_steps(torch, lambda: band_step(fused), args.steps, args.warmup, flush_buf, stream,
                                          lambda: fused.stats()["launches"])
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        if args.only != "all":
            ms_e, launches_e = [float("nan")], 0
        else:
            ms_e, launches_e = time_steps(torch, lambda: band_step(eager), max(args.steps // 2, 5), max(args.warmup, 3),
                                          flush_buf, stream, lambda: eager.stats()["launches"])
        torch.cuda.synchronize()

        # end-to-end through the public API: every step uploads the active
        # voxels' x values from pinned host memory (two buffers, alternating)
        # and reads the step's sum back; the next step's upload is staged while
        # the current step runs (sg_stage_active / sg_write_field_staged)
        bits = np.unpackbits(masks.view(np.uint8), bitorder="little").reshape(n_leaves, -1).astype(bool)
        x_packed = np.ascontiguousarray(x_host[bits])
        bufs = [torch.from_numpy(x_packed).pin_memory(), torch.from_numpy(x_packed.copy()).pin_memory()]
        e2e_steps = 0 if args.only != "all" else max(3, min(args.steps, 20))

        def e2e_run(nsteps):
            ticket = fused.stage_active(bufs[0])
            for s in range(nsteps):
                fused.write_field_staged(0, ticket)
                band_step(fused)
                if s + 1 < nsteps:
                    ticket = fused.stage_active(bufs[(s + 1) & 1])
                fused.read_sums(1)

        if e2e_steps:
            e2e_run(3)
        t0 = time.perf_counter()
        if e2e_steps:
            e2e_run(e2e_steps)
        e2e_s = max(time.perf_counter() - t0, 1e-9)
        fused.close()
        eager.close()

    t_f = sum(ms_f) / 1e3
    t_e = sum(ms_e) / 1e3
    t_f, t_e, e2e_s = aggregate_max([t_f, t_e, e2e_s], dist, "cuda")
    value = job_throughput(world, n_active, args.steps, t_f)
    eager_value = job_throughput(world, n_active, len(ms_e), t_e)
    avg_ms = t_f * 1e3 / args.steps
    peak, peak_kind = peaks()
    achieved = n_leaves * BYTES_PER_LEAF_FUSED / (avg_ms / 1e3) / 1e9
    achieved_eager = n_leaves * BYTES_PER_LEAF_EAGER / (t_e / len(ms_e)) / 1e9
    traffic = traffic_record(args.variant)

    extra = {}
    if world == 1 and args.only != "fused":
        k = max(5, min(args.steps, 20))
        for name, fn in (("tiny", lambda: bench_tiny(torch, sg, 20, 3, flush_buf, stream)),
                         ("band1024", lambda: bench_band1024(torch, sg, k, 3, flush_buf, stream, args.variant)),
                         ("restructure", lambda: bench_restructure(torch, sg, k, 3, flush_buf, stream)),
                         ("batched", lambda: bench_batched(torch, sg, k, 3, flush_buf, stream)),
                         ("particles", lambda: bench_particles(torch, sg, k, 3, flush_buf, stream)),
                         ("mpm_apic", lambda: bench_mpm_apic(torch, sg, k, 3, flush_buf, stream)),
                         ("multigrid", lambda: bench_multigrid(torch, sg, k, 3, flush_buf, stream)),
                         ("micro", lambda: bench_micro(torch, sg, k, 3, flush_buf, stream)),
                         ("advection", lambda: bench_advection(torch, sg, k, 3, flush_buf, stream)),
                         ("ablation", lambda: bench_ablation(torch, sg, x_host, k, 3, flush_buf, stream)),
                         ("serving", lambda: bench_serving(torch, sg, duration=args.serving_duration))):
            if args.only not in ("all", name):
                continue
            try:
                t0 = time.perf_counter()
                extra[name] = fn()
                extra[name]["bench_wall_s"] = time.perf_counter() - t0
            except Exception as exc:  # report, keep the headline line
                extra[name] = {"error": repr(exc)}
            torch.cuda.synchronize()

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline and args.only == "all":
            cpu = cpu_baseline(spec, leaf_b, x_host, n_active, budget_s=args.cpu_budget)
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "voxel-steps/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": avg_ms,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "fused sparse diffusion at scale: 512^3 band |dist-200|<8, 8^3 leaves, "
                                   "clear+diffuse7+box27+swap+sum per step",
                       "active_voxels": n_active, "leaves": n_leaves, "parallelism": f"replicas x{world}",
                       "l2": "flushed before every timed step (512 MB write)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "achieved_active_only": n_active * 8 / (avg_ms / 1e3) / 1e9,
                         "kernel": KERNEL_NAMES[args.variant],
                         "bytes_per_launch": n_leaves * BYTES_PER_LEAF_FUSED},
            "e2e": {"value": world * n_active * e2e_steps / e2e_s if e2e_steps else None, "unit": "voxel-steps/s",
                    "h2d_bytes_per_step": 4 * n_active, "d2h_bytes_per_step": 8},
            "gpu_launches": int(launches_f),
            "launches_per_step": launches_f / args.steps,
            "eager": {"value": eager_value, "ms_per_step": t_e * 1e3 / len(ms_e),
                      "launches_per_step": launches_e / len(ms_e), "achieved_gbs": achieved_eager},
            "fused_over_eager": value / eager_value,
            "clocks": clk.summary() if clk else None,
            "cpu_baseline": cpu,
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# oracle (CPU) arm and baseline
# ---------------------------------------------------------------------------

def oracle_band(spec, leaf_b=None, x_host=None):
    import oracle
    og = oracle.Grid(spec.N, spec.L, 3)
    og.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    b, m = og.structure()
    og.write_field(0, leaf_values(spec.seed, spec.N, spec.L, b) if x_host is None else x_host)
    return og, b, m


def oracle_step(og, cur, y):
    og.clear(1)
    og.diffuse7(cur, 1, 0.1)
    og.box27(1, y)
    og.sum(y)
    return y, cur


def cpu_baseline(spec, leaf_b, x_host, n_active, budget_s=15.0):
    og, _, _ = oracle_band(spec, leaf_b, x_host)
    cur, y = 0, 2
    steps, t0 = 0, time.perf_counter()
    while steps < 2 or time.perf_counter() - t0 < budget_s:
        cur, y = oracle_step(og, cur, y)
        steps += 1
        if steps >= 50:
            break
    dt = time.perf_counter() - t0
    return {"value": n_active * steps / dt, "unit": "voxel-steps/s", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle", "sample": f"{steps} full steps of the 512^3 band workload (FP64, OpenMP)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec = band512()
    og, b, m = oracle_band(spec)
    n_active = int(np.unpackbits(m.view(np.uint8)).sum())
    cur, y = 0, 2
    for _ in range(args.warmup):
        cur, y = oracle_step(og, cur, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cur, y = oracle_step(og, cur, y)
    dt = time.perf_counter() - t0
    value = n_active * args.steps / dt
    cores = len(os.sched_getaffinity(0))
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": "voxel-steps/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fused sparse diffusion at scale: 512^3 band |dist-200|<8, 8^3 leaves, "
                               "clear+diffuse7+box27+swap+sum per step", "active_voxels": n_active,
                   "leaves": len(b), "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": "voxel-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} full oracle steps of the workload"},
        "e2e": {"value": value, "unit": "voxel-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--variant", type=int, default=3, choices=[0, 1, 2, 3, 4],
                    help="stencil kernel family (0 sweep, 1 smem, 2 sweep over i-columns, 3 sweep over j-runs, "
                         "4 j-runs staged in shared memory by bulk tensor copies)")
    ap.add_argument("--serving-duration", type=float, default=2.0,
                    help="seconds of Poisson arrivals per rate in the serving leg")
    ap.add_argument("--only", choices=["all", "fused", "tiny", "band1024", "restructure", "batched", "particles", "mpm_apic", "multigrid",
                                       "micro", "advection", "ablation", "serving"],
                    default="all",
                    help="fused: only the fused headline step; a leg name: the headline step and that leg "
                         "(for profiling runs)")
    ap.add_argument("--skip-headline", action="store_true",
                    help="with --only <leg>: time that leg alone (profiling runs; the headline keys are NaN)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
