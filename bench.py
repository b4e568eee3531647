"""Benchmark: full BSCCS MAP fits by cyclic coordinate descent on one GB300.

Workload (one "step" = one whole MAP fit from beta = 0 to convergence, i.e. every step of
the hot path for every coordinate of every cycle): 1M subjects, ~10M eras (geometric, mean
10), 1,000 binary drug columns with Zipf(1.2) sizes from 10 to 2M, offsets uniform 1-365,
20 true effects, Normal prior variance 0.1, FP64, stop at relative |dP| < 1e-12.

Prints one JSON line.  `--impl reference` times the CPU oracle instead (rank 0 only).
With torchrun (N > 1) every rank fits its own replica (no collective on the data path;
weak scaling) and the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coord-updates/s (full SCCS MAP fit, FP64)"
UNIT = "coord-updates/s"


def workload_config(d, fit):
    return {
        "workload": "mid SCCS MAP fit: 1M subjects, ~10M eras (geometric mean 10), 1000 binary drugs "
                    "Zipf(1.2) sizes 10..2M, offsets U{1..365}, 20 true effects, Normal prior var 0.1, "
                    "FP64, rel |dP| < 1e-12",
        "subjects": int(d.N), "eras": int(d.K), "drugs": int(d.J), "nnz": int(d.nnz),
        "prior": f"{fit['prior']} var={fit['variance']}", "tol": f"{fit['tol_mode']} {fit['tol']}",
        "seed": d.recipe["seed"],
        "l2": "256 MB buffer written between timed steps (L2 flushed)",
    }


def recorded_traffic():
    """DRAM bytes per fit-kernel launch from the committed ncu record, if it was taken on the
    kernel source that is built now (else None: the counters are stale)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "fit_kernel_traffic_mid_1M_subjects.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["kernel_source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        if sha != rec["kernel_source_sha256"]:
            return None
        return rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]
    except Exception:
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(d, cycles, nonzero_frac=1.0):
    """Bytes the fit must move per launch (see the design notes): per coordinate step
    20 B per nonzero (4 index + 8 E read + 8 E write) and 28 B per touched subject
    (8 segment descriptor + 8 D read + 4 n_i + 8 D write); per cycle end 8 K + 28 N for
    the denominator refresh; plus one refresh at the start."""
    nnz = d["nnz_kept"]
    segs = d["segments"]
    K, N = d["rows_kept"], d["subjects_kept"]
    per_cycle = 12 * nnz + 20 * segs + nonzero_frac * (8 * nnz + 8 * segs) + 8 * K + 28 * N
    return cycles * per_cycle + 8 * K + 28 * N


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_reference(args, rank, world):
    """The CPU oracle on bounded samples of the same workload: each step is full CCD cycles
    of the serial FP64 oracle on one host core."""
    if rank != 0:
        return 0
    import oracle
    from synth import mid_fit_config
    d, fit = mid_fit_config()
    prob = oracle.Problem.from_data(d)
    cycles_per_step = 1
    for _ in range(args.warmup):
        prob.fit(prior=fit["prior"], variance=fit["variance"], fixed_cycles=cycles_per_step)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        prob.fit(prior=fit["prior"], variance=fit["variance"], fixed_cycles=cycles_per_step)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = d.J * cycles_per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(d, fit),
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": 1,
                         "sample": f"serial FP64 oracle (C, gcc -O2), {cycles_per_step} full CCD cycle "
                                   f"({d.J} coordinate updates incl. set-up of the cycle) per step on "
                                   "the benchmarked workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import torch
    import paper_1208_0945_gb300 as sccs
    from synth import mid_fit_config

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    d, fit = mid_fit_config(scale=args.scale)
    stream = torch.cuda.current_stream(dev)
    model = sccs.SCCSModel(d, device=local, stream=__import__("ctypes").c_void_p(stream.cuda_stream))
    model.set_prior(fit["prior"], fit["variance"])
    info = model.info
    fkw = dict(tol_mode=fit["tol_mode"], tol=fit["tol"], max_cycles=fit["max_cycles"])

    for _ in range(args.warmup):
        model.fit(**fkw)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    results = []
    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            r = model.fit(**fkw)
            ev[k][1].record(stream)
            results.append(r)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - wall0
    barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms_max = reduce_max(total_ms, world, dev)
    cycles = [r["cycles"] for r in results]
    units_local = float(sum(d.J * c for c in cycles))
    units = reduce_sum(units_local, world, dev)
    value = units / (total_ms_max / 1e3)

    # roofline of the dominant kernel (the persistent fit kernel; one launch per fit)
    kern_ms = statistics.mean(r["kernel_ms"] for r in results)
    nz_frac = statistics.mean(r["nonzero_steps"] / max(1, r["steps"]) for r in results)
    bytes_launch = algorithmic_bytes(info, statistics.mean(cycles), nz_frac)
    peak, peak_kind = load_peaks()
    achieved = bytes_launch / (kern_ms / 1e3) / 1e9
    clocks = clk.summary()

    # end to end through the C ABI from host arrays: create (validate, lay out, upload),
    # fit, read beta back, destroy
    e2e_ms = []
    h2d = d2h = 0
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        m2 = sccs.SCCSModel(d, device=local, stream=__import__("ctypes").c_void_p(stream.cuda_stream))
        m2.set_prior(fit["prior"], fit["variance"])
        r2 = m2.fit(**fkw)
        h2d = m2.info["upload_bytes"]
        m2.close()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        d2h = 8 * d.J + 128
    e2e_ms_max = reduce_max(statistics.mean(e2e_ms), world, dev)
    e2e_value = reduce_sum(float(d.J * r2["cycles"]), world, dev) / (e2e_ms_max / 1e3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(d, fit)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator; stands in for the licensed claims data)",
            "config": workload_config(d, fit),
            "fit": {"cycles": cycles[0], "nonzero_steps": results[0]["nonzero_steps"],
                    "logpost": results[0]["logpost"], "fit_ms": total_ms_max / args.steps,
                    "kernel_ms": kern_ms, "nnz_steps_per_s": info["nnz_kept"] * cycles[0] / (kern_ms / 1e3),
                    "shards": info["num_shards"], "threads_per_block": info["threads_per_block"],
                    "wall_s": wall},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": recorded_traffic() if args.scale == 1.0 else None,
                         "kernel": "fit_kernel (one persistent launch per fit)",
                         "algorithmic_bytes_per_launch": bytes_launch, "peak_source": peak_kind},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": e2e_ms_max,
                    "what": "sccs_create from host arrays (validate, lay out, upload) + sccs_fit + beta D2H + destroy"},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    model.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def cpu_baseline(d, fit):
    """The serial oracle, as it stands, on a bounded sample: 2 full CCD cycles (~5 s)."""
    import oracle
    prob = oracle.Problem.from_data(d)
    t0 = time.perf_counter()
    r = prob.fit(prior=fit["prior"], variance=fit["variance"], fixed_cycles=2)
    dt = time.perf_counter() - t0
    return {"value": d.J * r["cycles"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"2 full CCD cycles ({2 * d.J} coordinate updates) of the benchmarked workload, "
                      f"serial FP64 C oracle, {dt:.1f} s"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the workload's subjects")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
