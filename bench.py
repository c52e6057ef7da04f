"""Benchmark of the fused sparse-grid step on GB300.

Workload (default): the 512^3 narrow band |dist - 200| < 8 over 8^3 leaves
(26,104 leaves, 8,047,608 active voxels); one step = clear(t), diffuse7(x->t),
box27(t->y), swap(x,y), sum(x), through the library's queue with every
inter-kernel pass on (one fused launch).  The eager form (list regenerated and
activation checked in every kernel, 12 launches) is timed beside it.

Timing: W untimed warm-up steps, then K timed steps; before every timed step
a 512 MB buffer is written to flush L2 (the band's fields fit in L2), and each
step is bracketed by CUDA events on the grid's stream.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores on the same
workload (each step one full oracle step) and prints its line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from workload import band512, leaf_values, spheres_particles  # noqa: E402

METRIC = "active voxel-steps/s"
BYTES_PER_LEAF_FUSED = 2 * 2048 + 27 * 4 + 64 + 4  # x read, y written, nbr row, mask, list entry
BYTES_PER_LEAF_EAGER = 6 * 2048                    # clear W, diffuse R+W, box27 R+W, sum R (leaf passes)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_record(kernel_src: str):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    or None when the kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p))
        h = hashlib.sha1(open(kernel_src, "rb").read()).hexdigest()
        if rec.get("kernel_sha1") == h:
            return rec.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

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
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def setup_band(sg, spec, opts, x_host, variant=0):
    g = sg.Grid(spec.N, 3, 3, max_leaves=32768, max_sums=1, scratch_mask=0b010)
    g.set_opts(opts)
    g.set_stencil_variant(variant)
    g.activate_shell(spec.lo2, spec.hi2, spec.lo_strict)
    g.list_gen()
    n = g.num_leaves()
    assert n == x_host.shape[0]
    g.write_field(0, x_host)
    return g


def band_step(g):
    g.clear(1)
    g.diffuse7(0, 1, 0.1)
    g.box27(1, 2)
    g.swap(0, 2)
    g.reduce_sum(0, 0)
    g.flush()


def time_steps(torch, g, steps, warmup, flush_buf, stream):
    for _ in range(warmup):
        band_step(g)
    torch.cuda.synchronize()
    l0 = g.stats()["launches"]
    evs = []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            flush_buf.zero_()                      # evict L2 between timed steps
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            band_step(g)
            b.record(stream)
            evs.append((a, b))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in evs]
    launches = g.stats()["launches"] - l0
    return ms, launches


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

    fused = setup_band(sg, spec, sg.SG_OPT_ALL, x_host, args.variant)
    eager = setup_band(sg, spec, sg.SG_OPT_EAGER, x_host, args.variant)

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        ms_f, launches_f = time_steps(torch, fused, args.steps, args.warmup, flush_buf, stream)
    torch.cuda.synchronize()
    if args.only == "fused":
        ms_e, launches_e = [float("nan")], 0
    else:
        ms_e, launches_e = time_steps(torch, eager, max(args.steps // 2, 5), max(args.warmup, 3), flush_buf, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    # end-to-end through the public API: pinned host x in, sum out, every step
    x_pinned = torch.from_numpy(x_host).pin_memory()
    e2e_steps = 0 if args.only == "fused" else max(3, min(args.steps, 20))
    for _ in range(2 if e2e_steps else 0):
        fused.write_field(0, x_pinned)
        band_step(fused)
        fused.read_sums(1)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        fused.write_field(0, x_pinned)
        band_step(fused)
        fused.read_sums(1)
    e2e_s = max(time.perf_counter() - t0, 1e-9)

    t_f = sum(ms_f) / 1e3
    t_e = sum(ms_e) / 1e3
    if dist:
        tt = torch.tensor([t_f, t_e, e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_f, t_e, e2e_s = tt.tolist()
    value = world * n_active * args.steps / t_f
    eager_value = world * n_active * len(ms_e) / t_e
    avg_ms = t_f * 1e3 / args.steps
    peak, peak_kind = peaks()
    achieved = n_leaves * BYTES_PER_LEAF_FUSED / (avg_ms / 1e3) / 1e9
    achieved_eager = n_leaves * BYTES_PER_LEAF_EAGER / (t_e / len(ms_e)) / 1e9
    kernel_src = os.path.join(ROOT, "paper_2012_08141_gb300", "csrc",
                              "sg_sweep.cu" if args.variant == 0 else "sg_stencil.cu")
    traffic = traffic_record(kernel_src)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline and args.only != "fused":
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
                         "kernel": ("k_sweep_diffuse_box<false,false,true>" if args.variant == 0
                                    else "k_diffuse_box<false,false,true>"),
                         "bytes_per_launch": n_leaves * BYTES_PER_LEAF_FUSED},
            "e2e": {"value": world * n_active * e2e_steps / e2e_s, "unit": "voxel-steps/s",
                    "h2d_bytes_per_step": int(x_host.nbytes), "d2h_bytes_per_step": 8},
            "gpu_launches": int(launches_f),
            "launches_per_step": launches_f / args.steps,
            "eager": {"value": eager_value, "ms_per_step": t_e * 1e3 / len(ms_e),
                      "launches_per_step": launches_e / len(ms_e), "achieved_gbs": achieved_eager},
            "fused_over_eager": value / eager_value,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    fused.close()
    eager.close()
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
    ap.add_argument("--variant", type=int, default=0, help="stencil kernel family (0 sweep, 1 smem)")
    ap.add_argument("--only", choices=["all", "fused"], default="all",
                    help="fused: time only the fused step (for profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
