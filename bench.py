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
    kernel source that is built now (else None: the counters are stale), and how it was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "fit_kernel_traffic_mid_1M_subjects.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, rec["kernel_source"]), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        if sha != rec["kernel_source_sha256"]:
            return None, None
        return rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"], rec.get("config_note")
    except Exception:
        return None, None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_fp64_peak():
    """FP64 FMA throughput of the GPU in GFLOP/s (measured on this machine, profiles/fp64_fma_peak.json)."""
    try:
        with open(os.path.join(ROOT, "profiles", "fp64_fma_peak.json")) as f:
            return float(json.load(f)["fp64_gflops"]), "measured"
    except Exception:
        return 1000.0, "fallback"


def fp64_flops(d, cycles, nonzero_frac=1.0):
    """FP64 flops the fit must execute per launch (FMA = 2): per coordinate step, phase A's
    nnz + 13 P (per segment the quotient 9, n w 1, n w (1 - w) 2, the two running sums 2; one add
    per further row of a segment) and, when db != 0, phase C's nnz + 2 P (E e^db per row, the
    D update by FMA per segment); per cycle end K adds and about 21 per subject for n_i log D_i."""
    nnz, segs = d["nnz_kept"], d["segments"]
    K, N = d["rows_kept"], d["subjects_kept"]
    per_cycle = (nnz + 13 * segs) + nonzero_frac * (nnz + 2 * segs) + K + 21 * N
    return cycles * per_cycle + K + 21 * N


def roofline(bytes_launch, flops_launch, kern_ms, kernel, traffic=None, fp64=True):
    """Both roofs of the dominant kernel: HBM (algorithmic bytes / time against the measured copy
    bandwidth) and, for FP64 arithmetic, the FP64 ALU (algorithmic flops / time against the
    measured FP64 FMA rate); the one closer to its peak is reported as the bound."""
    peak, peak_kind = load_peaks()
    hbm = bytes_launch / (kern_ms / 1e3) / 1e9
    out = {"bound": "hbm", "achieved": hbm, "peak": peak, "unit": "GB/s", "frac": hbm / peak, "traffic": traffic,
           "kernel": kernel, "algorithmic_bytes_per_launch": bytes_launch, "peak_source": peak_kind}
    if fp64 and flops_launch:
        fpk, fpk_kind = load_fp64_peak()
        alu = flops_launch / (kern_ms / 1e3) / 1e12
        out["hbm"] = {"achieved": hbm, "peak": peak, "unit": "GB/s", "frac": hbm / peak, "peak_source": peak_kind}
        out["fp64"] = {"achieved": alu, "peak": fpk / 1e3, "unit": "TFLOP/s", "frac": alu / (fpk / 1e3),
                       "algorithmic_flops_per_launch": flops_launch, "peak_source": fpk_kind}
        if alu / (fpk / 1e3) > hbm / peak:
            out.update({"bound": "alu", "achieved": alu, "peak": fpk / 1e3, "unit": "TFLOP/s",
                        "frac": alu / (fpk / 1e3), "peak_source": fpk_kind})
    return out


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
    model = sccs.SCCSModel(d, device=local, stream=__import__("ctypes").c_void_p(stream.cuda_stream),
                           cluster_ctas=args.cluster_ctas)
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
    flops_launch = fp64_flops(info, statistics.mean(cycles), nz_frac)
    clocks = clk.summary()

    traffic, traffic_note = recorded_traffic() if args.scale == 1.0 else (None, None)
    # end to end through the C ABI from host arrays: create (validate, lay out, upload),
    # fit, read beta back, destroy
    e2e_ms = []
    h2d = d2h = 0
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        m2 = sccs.SCCSModel(d, device=local, stream=__import__("ctypes").c_void_p(stream.cuda_stream),
                            cluster_ctas=args.cluster_ctas)
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
            "roofline": roofline(bytes_launch, flops_launch, kern_ms, "fit_kernel (one persistent launch per fit)",
                                 traffic),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "ms_per_step": e2e_ms_max,
                    "what": "sccs_create from host arrays (validate, lay out, upload) + sccs_fit + beta D2H + destroy"},
            "gpu_launches": 2 * args.steps,
            "clocks": clocks,
        }
        if traffic_note:
            line["roofline"]["traffic_note"] = traffic_note
        if cpu is not None:
            line["cpu_baseline"] = cpu
    model.close()
    if rank == 0 and world == 1 and not args.no_legs and args.scale == 1.0:
        line.update(run_legs(args, local))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _leg(full, keep):
    return {k: full[k] for k in keep if k in full}


def run_legs(args, local):
    """The other workloads at their full shapes, run after the headline fit in the same process
    (one GPU): the paper-scale FP32 + polish fit with its per-coefficient error against the oracle
    (which runs in a separate process meanwhile), the 256-fit batched launch against one fit at a
    time, and the served fits per arrival rate against one fit at a time.  Each carries its own
    clock record and roofline."""
    import copy
    legs = {}
    a = copy.copy(args)
    a.steps, a.warmup = 2, 3
    t0 = time.perf_counter()
    paper, pending = run_paper(a, 0, 1, local, emit=False, oracle_check=True)
    paper["wall_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    batched = run_batched(a, 0, 1, local, emit=False)
    batched["wall_s"] = time.perf_counter() - t0
    a2 = copy.copy(a)
    a2.rates, a2.requests = "2,10,50,200", -1
    t0 = time.perf_counter()
    serving = run_serving(a2, 0, 1, local, emit=False)
    serving["wall_s"] = time.perf_counter() - t0
    paper["error_vs_oracle"] = paper_oracle_error(pending)
    keep = ("metric", "value", "unit", "ms_per_step", "higher_is_better", "dtype", "config", "roofline", "clocks",
            "wall_s")
    legs["paper_scale"] = _leg(paper, keep + ("fit", "fp64_throughout", "error_vs_fp64", "error_vs_oracle"))
    legs["batched"] = _leg(batched, keep + ("batch", "one_at_a_time", "e2e", "cpu_baseline"))
    legs["serving"] = _leg(serving, keep + ("sweep", "one_at_a_time", "p50_ms", "p99_ms"))
    return legs


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


# ------------------------------------------------------------------ batched and served fits

def _spawn_pool(workers: int):
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    return ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def _oracle_sample_batched(plan, f, cycles):
    """Pool worker: draw fit f of the batch and time `cycles` cycles of the serial oracle on it."""
    import oracle
    from synth import batched_fit_one
    d, fit = batched_fit_one(plan, f)
    prob = oracle.Problem.from_data(d)
    t0 = time.perf_counter()
    prob.fit(prior=fit["prior"], variance=fit["variance"], fixed_cycles=cycles)
    return f, int(d.nnz), time.perf_counter() - t0


def _est_nnz_batched(plan, f):
    return float(plan["sizes"][f]) * 8.0 * float(np.sum(plan["dens"]))


def run_batched(args, rank, world, local, emit=True):
    """One step = one batched launch of all the batch's fits from beta = 0 to convergence."""
    import ctypes
    from synth import batched_fit_plan, batched_fit_one
    import oracle

    plan = batched_fit_plan(n_fits=args.fits, max_subjects=args.max_subjects)
    n = args.fits
    cores = _host_cores()
    # oracle sample first (host cores only, before the GPU is touched): one fit per core,
    # spread over the size range, 2 cycles each
    cpu_sample = []
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oracle.build()
        by_size = np.argsort(plan["sizes"])
        pick = sorted(set(int(by_size[int(round(q))]) for q in np.linspace(0, n - 1, min(cores, n))))
        t0 = time.perf_counter()
        with _spawn_pool(min(cores, len(pick))) as ex:
            cpu_sample = list(ex.map(_oracle_sample_batched, [plan] * len(pick), pick, [2] * len(pick)))
        cpu_wall = time.perf_counter() - t0

    import torch
    import paper_1208_0945_gb300 as sccs
    from paper_1208_0945_gb300 import autotune

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    model = autotune.measure(local)
    est = [(int(plan["J"]), _est_nnz_batched(plan, f), 0.9 * _est_nnz_batched(plan, f)) for f in range(n)]
    teams = autotune.assign(est, model)

    # draw the fits in parallel and keep two resident copies of each: the autotuned team for
    # the batch, and the library's default shard count for one-at-a-time fits
    stream = torch.cuda.current_stream(dev)
    cst = ctypes.c_void_p(stream.cuda_stream)
    batch_m, plain_m, infos, fits = [], [], [], []
    t_gen = time.perf_counter()
    with _spawn_pool(min(cores, 16)) as ex:
        for f, (d, fit) in enumerate(ex.map(batched_fit_one, [plan] * n, range(n))):
            mb = sccs.SCCSModel(d, device=local, stream=cst, num_shards=teams[f])
            mb.set_prior(fit["prior"], fit["variance"])
            mp_ = sccs.SCCSModel(d, device=local, stream=cst)
            mp_.set_prior(fit["prior"], fit["variance"])
            batch_m.append(mb)
            plain_m.append(mp_)
            infos.append(mb.info)
            fits.append(fit)
    t_gen = time.perf_counter() - t_gen
    fkw = dict(tol_mode="rel_logpost", tol=1e-12, max_cycles=1000)
    handles = [m.handle for m in batch_m]
    Js = [m.J for m in batch_m]

    for _ in range(args.warmup):
        sccs.sccs_fit_batch(handles, Js, **fkw)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    step_ms, walls, res = [], [], None
    barrier(world)
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            res = sccs.sccs_fit_batch(handles, Js, **fkw)
            walls.append(1e3 * (time.perf_counter() - t0))
            step_ms.append(res[0]["kernel_ms"])
    barrier(world)
    clocks = clk.summary()
    ms = reduce_max(statistics.mean(step_ms), world, dev)
    value = reduce_sum(float(n), world, dev) / (ms / 1e3)

    # the same fits one at a time (plain sccs_fit, default shards), once
    plain_m[0].fit(**fkw)
    seq_ms, seq_wall, seq_res = 0.0, 0.0, []
    torch.cuda.synchronize(dev)
    for m in plain_m:
        t0 = time.perf_counter()
        r = m.fit(**fkw)
        seq_wall += time.perf_counter() - t0
        seq_ms += r["kernel_ms"]
        seq_res.append(r)
    seq_ms = reduce_max(seq_ms, world, dev)
    same_cycles = sum(1 for a, b in zip(res, seq_res) if a["cycles"] == b["cycles"])
    max_dlogpost = max(abs(a["logpost"] - b["logpost"]) / max(1.0, abs(b["logpost"])) for a, b in zip(res, seq_res))

    total_bytes = total_flops = 0.0
    for info, r in zip(infos, res):
        nz = r["nonzero_steps"] / max(1, r["steps"])
        total_bytes += algorithmic_bytes(info, r["cycles"], nz)
        total_flops += fp64_flops(info, r["cycles"], nz)

    cpu = None
    if cpu_sample:
        # oracle seconds per nonzero-cycle on the sample, applied to every fit's nonzeros and
        # the cycles the GPU needed, spread over the host cores
        rate = sum(2.0 * nz for _, nz, _ in cpu_sample) / sum(dt for _, _, dt in cpu_sample)
        cpu_s = sum(info["nnz_kept"] * r["cycles"] for info, r in zip(infos, res)) / rate / cores
        cpu = {"value": n / cpu_s, "unit": "fits/s", "cores": cores, "kind": "oracle",
               "sample": f"serial FP64 C oracle, 2 cycles on each of {len(cpu_sample)} fits spread over the "
                         f"size range, one fit per process on {min(cores, len(cpu_sample))} cores "
                         f"({cpu_wall:.1f} s wall); extrapolated to all {n} fits by nonzeros x the cycles "
                         f"each fit needed, divided over {cores} cores"}
    if rank == 0:
        line = {
            "metric": "batched SCCS MAP fits/s (FP64, one persistent graph-captured launch)",
            "value": value, "unit": "fits/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator)", "workload": "batched",
            "config": {"workload": f"batched: {n} independent SCCS fits, subjects log-uniform 2k-"
                                   f"{args.max_subjects // 1000}k, eras geometric mean 8, {plan['J']} drugs "
                                   "with shared densities U[0.5%,5%], Normal prior var 0.01/0.1/1 in turn, "
                                   "FP64, rel |dP| < 1e-12; team sizes from the autotuner",
                       "fits": n, "subjects": int(sum(i["subjects_kept"] for i in infos)),
                       "eras": int(sum(i["rows_kept"] for i in infos)),
                       "nnz": int(sum(i["nnz_kept"] for i in infos)),
                       "teams": {"min": int(min(teams)), "max": int(max(teams)), "sum": int(sum(teams))},
                       "seed": int(plan["seed"]), "l2": "256 MB buffer written between timed steps (L2 flushed)"},
            "batch": {"kernel_ms": statistics.mean(step_ms), "wall_ms": statistics.mean(walls),
                      "cycles_total": int(sum(r["cycles"] for r in res)),
                      "setup_s": t_gen},
            "one_at_a_time": {"fits_per_s": n / (seq_ms / 1e3), "kernel_ms": seq_ms, "wall_s": seq_wall,
                              "speedup_of_batch": seq_ms / ms,
                              "same_cycles": f"{same_cycles}/{n}",
                              "max_rel_logpost_diff": max_dlogpost},
            "roofline": roofline(total_bytes, total_flops, statistics.mean(step_ms),
                                 "fit_queue_kernel (one launch per batch)"),
            "e2e": {"value": n / (statistics.mean(walls) / 1e3), "unit": "fits/s",
                    "h2d_bytes_per_step": None, "d2h_bytes_per_step": int(sum(8 * J for J in Js)),
                    "what": "sccs_fit_batch wall time: per-fit entries staged, graph launched, results and betas "
                            "copied back (datasets resident)"},
            "gpu_launches": 3 * args.steps,
            "clocks": clocks,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if emit:
            print(json.dumps(line), flush=True)
    for m in batch_m + plain_m:
        m.close()
    if not emit:
        return line if rank == 0 else None
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _serve_sweep(sccs, device, handles_of, Js, rates, n_per_rate, max_inflight, budget, seed0, folds_of=None,
                 alts_of=None):
    """Submit each rate's Poisson arrivals to a fresh server and collect latencies.  With
    folds_of (per outcome, the fold of each input subject), a request with fold k fits on the
    other folds and returns the held-out predictive log-likelihood of fold k."""
    from synth import fold_weights, serving_requests
    nf = 0 if folds_of is None else int(max(f.max() for f in folds_of)) + 1
    rows = []
    for ri, rate in enumerate(rates):
        if n_per_rate > 0:
            n_req = n_per_rate
        elif n_per_rate < 0:          # a short sweep: about 3 s of arrivals, 12 to 64 requests
            n_req = int(max(12, min(64, 3.0 * rate)))
        else:
            n_req = int(min(192, max(32, 3.0 * rate)))
        reqs = serving_requests(n_req, rate, len(Js), seed=seed0 + ri, folds=nf)
        masks = [fold_weights(folds_of[o], k - 1) if k > 0 else (None, None) for (_t, o, _p, _v, k) in reqs]
        with sccs.FitServer(device=device, max_inflight=max_inflight, hbm_budget_bytes=budget) as srv:
            tickets = []
            t0 = time.perf_counter()
            for (ta, o, prior, var, _fold), (wt, wh) in zip(reqs, masks):
                dt = t0 + ta - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets.append(sccs.sccs_submit(srv.server, handles_of[o], prior=prior, variance=var,
                                                tol_mode="rel_logpost", tol=1e-12, max_cycles=1000,
                                                weights=wt, heldout_weights=wh,
                                                dataset_alt=None if alts_of is None else alts_of[o]))
            out = []
            for t, (ta, o, *_rest) in zip(tickets, reqs):
                while True:
                    r = sccs.sccs_poll(srv.server, t, Js[o])
                    if r is not None:
                        break
                    time.sleep(0.0005)
                out.append(r)
            t_end = time.perf_counter()
        lat = np.array([r["latency_ms"] for r in out])
        done_span = (t_end - t0)
        rows.append({"rate_per_s": rate, "requests": n_req,
                     "fits_per_s": n_req / done_span,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_queue_ms": float(np.mean([r["queue_ms"] for r in out])),
                     "failed": int(sum(1 for r in out if r["status"] < 0)),
                     "heldout_evaluated": int(sum(1 for r in out if np.isfinite(r["heldout_loglik"]))),
                     "on_full_device_team": int(sum(1 for r in out if r["team"] >= 100))})
    return rows


def run_serving(args, rank, world, local, emit=True):
    """Poisson-arrival fit requests over a pool of resident outcomes, served with continuous
    batching, beside the same arrivals served one fit at a time."""
    import ctypes
    from synth import serving_pool_plan, serving_outcome
    import torch
    import paper_1208_0945_gb300 as sccs
    from paper_1208_0945_gb300 import autotune

    plan = serving_pool_plan(n_outcomes=args.outcomes, max_eras=args.max_eras)
    cores = _host_cores()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    model = autotune.measure(local)
    stream = torch.cuda.current_stream(dev)
    cst = ctypes.c_void_p(stream.cuda_stream)
    served, plain, infos = [], [], []
    t_gen = time.perf_counter()
    with _spawn_pool(min(cores, 16)) as ex:
        ds = list(ex.map(serving_outcome, [plan] * args.outcomes, range(args.outcomes)))
    from synth import cv_folds
    folds_of = [cv_folds(int(1 + np.count_nonzero(d.patient_id[1:] != d.patient_id[:-1])), folds=10, seed=1300 + o)
                for o, d in enumerate(ds)]
    est = [(d.J, d.nnz, 0.9 * d.nnz) for d in ds]
    teams = autotune.assign(est, model)
    for d, S in zip(ds, teams):
        served.append(sccs.SCCSModel(d, device=local, stream=cst, num_shards=S))
        plain.append(sccs.SCCSModel(d, device=local, stream=cst))
        infos.append(served[-1].info)
    del ds
    t_gen = time.perf_counter() - t_gen
    Js = [m.J for m in served]
    rates = [float(x) for x in args.rates.split(",")]
    budget = int(args.hbm_budget_gb * (1 << 30))
    # warm-up: three rounds of requests through each arm
    for arm in (served, plain):
        for w in range(3):
            _serve_sweep(sccs, local, [m.handle for m in arm], Js, [1000.0], min(args.outcomes, 8), 64, budget,
                         999 + w, folds_of)
    with ClockSampler(local) as clk:
        ours = _serve_sweep(sccs, local, [m.handle for m in served], Js, rates, args.requests, 64, budget, 2000,
                            folds_of, alts_of=[m.handle for m in plain])
    clocks = clk.summary()
    one = _serve_sweep(sccs, local, [m.handle for m in plain], Js, rates, args.requests, 1, 0, 2000, folds_of)
    top = ours[-1]
    if rank == 0:
        line = {
            "metric": "served SCCS MAP fits/s and p50/p99 latency (FP64, Poisson arrivals, continuous batching)",
            "value": top["fits_per_s"], "unit": "fits/s", "n_gpus": world, "steps": len(rates),
            "warmup": 3, "ms_per_step": 1e3 / top["fits_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)", "workload": "serving",
            "config": {"workload": f"serving: {args.outcomes} resident outcomes, eras log-uniform 20k-"
                                   f"{args.max_eras / 1e6:g}M, 1000-5000 drugs, Zipf(1.2) columns up to eras/5; "
                                   "requests = outcome x Normal/Laplace x variance grid "
                                   "{0.01..1} x fold 1..10 (fit on 9 folds, held-out predictive log-likelihood "
                                   "of the 10th returned), FP64 to rel |dP| < 1e-12; each outcome resident with "
                                   "an autotuned team and a full-device team, the server choosing per request; "
                                   + (f"{args.requests} Poisson arrivals per rate" if args.requests > 0 else
                                      ("about 3 s of Poisson arrivals per rate (12 to 64 requests)" if args.requests < 0
                                       else "3 s of Poisson arrivals per rate (32 to 192 requests)")),
                       "outcomes": args.outcomes, "eras": int(sum(i["rows_kept"] for i in infos)),
                       "nnz": int(sum(i["nnz_kept"] for i in infos)), "rates_per_s": rates,
                       "teams": {"min": int(min(teams)), "max": int(max(teams))},
                       "max_inflight": 64, "hbm_budget_gb": args.hbm_budget_gb, "setup_s": t_gen},
            "sweep": ours,
            "one_at_a_time": one,
            "p50_ms": top["p50_ms"], "p99_ms": top["p99_ms"],
            "roofline": None,
            "e2e": {"value": top["fits_per_s"], "unit": "fits/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(8 * np.mean(Js)),
                    "what": "submit -> poll through the C ABI, datasets resident; the value itself is end to end"},
            "clocks": clocks,
        }
        if emit:
            print(json.dumps(line), flush=True)
    for m in served + plain:
        m.close()
    if not emit:
        return line if rank == 0 else None
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def algorithmic_bytes32(d, cycles, nonzero_frac=1.0):
    """FP32 mode: E is 4 bytes and D an 8-byte (hi, lo) pair."""
    nnz = d["nnz_kept"]
    segs = d["segments"]
    K, N = d["rows_kept"], d["subjects_kept"]
    per_cycle = 8 * nnz + 20 * segs + nonzero_frac * (4 * nnz + 8 * segs) + 4 * K + 28 * N
    return cycles * per_cycle + 4 * K + 28 * N


def _oracle_paper_fit(scale, cycles):
    """Pool worker: the serial FP64 oracle's Algorithm 1 on the paper-scale data (drawn again
    from its seed), for a fixed number of cycles."""
    import oracle
    from synth import paper_scale_config
    t0 = time.perf_counter()
    d, fit = paper_scale_config(scale=scale)
    prob = oracle.Problem.from_data(d)
    t1 = time.perf_counter()
    r = prob.fit(prior=fit["prior"], variance=fit["variance"], fixed_cycles=cycles)
    return r["beta"], r["logpost"], time.perf_counter() - t1, t1 - t0


def paper_oracle_error(pending, timeout_s=1500.0):
    """Per-coefficient error of the GPU's FP32 + polish fit against the oracle's FP64 fit after the
    same number of cycles (the oracle ran in a separate process meanwhile)."""
    pool, fut, beta, logpost, cycles = pending
    try:
        ob, olp, fit_s, setup_s = fut.result(timeout=timeout_s)
        db = np.abs(beta - ob)
        out = {"max_abs_dbeta": float(db.max()), "mean_abs_dbeta": float(db.mean()),
               "rel_logpost": abs(logpost - olp) / abs(olp),
               "zero_pattern_identical": bool(np.array_equal(beta == 0, ob == 0)),
               "nonzero_coefficients": int(np.count_nonzero(ob)), "cycles": int(cycles),
               "oracle_fit_s": fit_s, "oracle_setup_s": setup_s,
               "reference": "serial FP64 C oracle, Algorithm 1 for the same number of cycles as the GPU fit "
                            "(FP32 phase + FP64 polish) on the same data"}
    except Exception as e:  # a timeout or a failed worker is reported, not hidden
        out = {"unavailable": f"oracle comparison did not finish: {type(e).__name__}: {e}"[:200]}
    pool.shutdown(wait=False, cancel_futures=True)
    return out


def run_paper(args, rank, world, local, emit=True, oracle_check=False):
    """The paper-scale fit (4M subjects, ~40M eras, 5,000 drugs, Laplace): FP32 with compensated
    per-subject sums then an FP64 polish, beside the same fit in FP64 throughout.  With
    oracle_check the oracle's fit for the same number of cycles starts in a separate process;
    returns (line, pending) for paper_oracle_error."""
    import ctypes
    import torch
    import paper_1208_0945_gb300 as sccs
    from synth import paper_scale_config

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    d, fit = paper_scale_config(scale=args.scale)
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    model = sccs.SCCSModel(d, device=local, stream=ctypes.c_void_p(stream.cuda_stream))
    t_create = time.perf_counter() - t0
    model.set_prior(fit["prior"], fit["variance"])
    info = model.info
    fkw = dict(tol_mode=fit["tol_mode"], tol=fit["tol"], max_cycles=fit["max_cycles"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    with ClockSampler(local) as clk:
        for prec in ("fp32_polish", "fp64"):
            for _ in range(args.warmup):
                model.fit(precision=prec, **fkw)
            rs = []
            for k in range(args.steps):
                flush.fill_(float(k))
                torch.cuda.synchronize(dev)
                rs.append(model.fit(precision=prec, **fkw))
            res[prec] = rs
    clocks = clk.summary()
    r32, r64 = res["fp32_polish"][-1], res["fp64"][-1]
    ms32 = statistics.mean(r["kernel_ms"] for r in res["fp32_polish"])
    ms64 = statistics.mean(r["kernel_ms"] for r in res["fp64"])
    ms32 = reduce_max(ms32, world, dev)
    ms64 = reduce_max(ms64, world, dev)
    value = reduce_sum(float(d.J * r32["cycles"]), world, dev) / (ms32 / 1e3)
    dbeta = np.abs(r32["beta"] - r64["beta"])
    zero_same = bool(np.array_equal(r32["beta"] == 0, r64["beta"] == 0))
    nz32 = r32["nonzero_steps"] / max(1, r32["steps"])
    fp32_c = r32["fp32_cycles"]
    bytes32 = algorithmic_bytes32(info, fp32_c, nz32) + algorithmic_bytes(info, r32["cycles"] - fp32_c, nz32)
    flops_polish = fp64_flops(info, r32["cycles"] - fp32_c, nz32)
    pending = None
    if oracle_check and rank == 0:
        pool = _spawn_pool(1)
        pending = (pool, pool.submit(_oracle_paper_fit, args.scale, int(r32["cycles"])), r32["beta"].copy(),
                   r32["logpost"], r32["cycles"])
    line = None
    if rank == 0:
        line = {
            "metric": "coord-updates/s (paper-scale SCCS MAP fit, FP32 compensated + FP64 polish)",
            "value": value, "unit": "coord-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic (seeded generator)", "workload": "paper",
            "config": {"workload": "paper-scale SCCS MAP fit: 4M subjects, ~40M eras (geometric mean 10), 5000 "
                                   "binary drugs Zipf(1.1) sizes 10..5M, 50 true effects, Laplace prior var 0.05, "
                                   "FP32 (Kahan per-subject sums, exact cross-subject sums, FP64 step) to rel 1e-6 "
                                   "then FP64 to rel |dP| < 1e-12",
                       "subjects": int(info["subjects_kept"]), "eras": int(info["rows_kept"]), "drugs": int(d.J),
                       "nnz": int(info["nnz_kept"]), "narrow_columns": int(info["narrow_columns"]),
                       "seed": d.recipe["seed"], "scale": args.scale,
                       "l2": "256 MB buffer written between timed steps (L2 flushed)",
                       "setup_s": {"generate": t_gen, "create": t_create}},
            "fit": {"fp32_cycles": fp32_c, "fp64_polish_cycles": r32["cycles"] - fp32_c, "kernel_ms": ms32,
                    "logpost": r32["logpost"]},
            "fp64_throughout": {"value": d.J * r64["cycles"] / (ms64 / 1e3), "unit": "coord-updates/s",
                                "cycles": r64["cycles"], "kernel_ms": ms64, "logpost": r64["logpost"],
                                "speedup_of_fp32_polish": ms64 / ms32},
            "error_vs_fp64": {"max_abs_dbeta": float(dbeta.max()), "mean_abs_dbeta": float(dbeta.mean()),
                              "rel_logpost": abs(r32["logpost"] - r64["logpost"]) / abs(r64["logpost"]),
                              "zero_pattern_identical": zero_same,
                              "reference": "the same fit in FP64 on the GPU (which matches the oracle to 1e-8 "
                                           "at reduced scale in the tests)"},
            "roofline": roofline(bytes32, flops_polish, ms32, "fit_kernel (FP32 phase then FP64 polish)"),
            "e2e": {"value": None, "unit": "coord-updates/s", "h2d_bytes_per_step": int(info["upload_bytes"]),
                    "d2h_bytes_per_step": 8 * d.J, "what": f"create {t_create:.1f} s, not repeated per step"},
            "gpu_launches": 6 * args.steps,
            "clocks": clocks,
        }
    model.close()
    if not emit:
        return line, pending
    if rank == 0:
        if pending is not None:
            line["error_vs_oracle"] = paper_oracle_error(pending)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_large_columns(args, rank, world, local):
    """The regime where HBM or the FP64 ALU can bind a coordinate step: 1M subjects and 16 drug
    columns of 1M to 2M nonzeros each.  FP64 fits (against the FP64-ALU and HBM roofs) and FP32
    cycles (against HBM), a fixed number of cycles per step."""
    import ctypes
    import torch
    import paper_1208_0945_gb300 as sccs
    from synth import large_columns_config

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    d, fit = large_columns_config(scale=args.scale)
    stream = torch.cuda.current_stream(dev)
    model = sccs.SCCSModel(d, device=local, stream=ctypes.c_void_p(stream.cuda_stream), cluster_ctas=args.cluster_ctas)
    model.set_prior(fit["prior"], fit["variance"])
    info = model.info
    cycles = fit["cycles"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    with ClockSampler(local) as clk:
        for prec in ("fp64", "fp32"):
            for _ in range(args.warmup):
                model.fit(precision=prec, tol=-1.0, max_cycles=cycles)
            rs = []
            for k in range(args.steps):
                flush.fill_(float(k))
                torch.cuda.synchronize(dev)
                rs.append(model.fit(precision=prec, tol=-1.0, max_cycles=cycles))
            res[prec] = rs
    clocks = clk.summary()
    out = {}
    for prec, rs in res.items():
        ms = reduce_max(statistics.mean(r["kernel_ms"] for r in rs), world, dev)
        nz = statistics.mean(r["nonzero_steps"] / max(1, r["steps"]) for r in rs)
        if prec == "fp64":
            rl = roofline(algorithmic_bytes(info, cycles, nz), fp64_flops(info, cycles, nz), ms,
                          "fit_kernel (FP64, 16 columns of 1-2M nonzeros)")
        else:
            rl = roofline(algorithmic_bytes32(info, cycles, nz), 0.0, ms, "fit_kernel (FP32, 16 columns of 1-2M nonzeros)",
                          fp64=False)
        out[prec] = {"kernel_ms": ms, "us_per_step": 1e3 * ms / (cycles * d.J),
                     "value": reduce_sum(float(d.J * cycles), world, dev) / (ms / 1e3), "roofline": rl}
    if rank == 0:
        r64 = out["fp64"]
        line = {
            "metric": "coord-updates/s (large-column SCCS fit, FP64)", "value": r64["value"], "unit": "coord-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r64["kernel_ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator)", "workload": "large-columns",
            "config": {"workload": f"large columns: {int(info['subjects_kept'])} subjects, {int(info['rows_kept'])} eras, "
                                   f"{d.J} drugs of 1M-2M nonzeros, Normal prior var {fit['variance']}, "
                                   f"{cycles} cycles per step", "nnz": int(info["nnz_kept"]),
                       "segments": int(info["segments"]), "seed": d.recipe["seed"],
                       "l2": "256 MB buffer written between timed steps (L2 flushed)"},
            "roofline": r64["roofline"], "us_per_step": r64["us_per_step"], "fp32": out["fp32"],
            "e2e": None, "gpu_launches": 2 * args.steps, "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    model.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the workload's subjects")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true",
                    help="fit workload: only the headline fit (no paper-scale, batched and serving results)")
    ap.add_argument("--oracle-check", action="store_true",
                    help="paper workload: also run the oracle for the same cycles and report the per-beta error")
    ap.add_argument("--workload", default="fit", choices=["fit", "batched", "serving", "paper", "large-columns"],
                    help="fit: one full MAP fit per step (default); batched: all fits of a batch in one "
                         "launch per step; serving: Poisson-arrival requests over resident outcomes")
    ap.add_argument("--cluster-ctas", type=int, default=0,
                    help="fit workload: CTAs per thread-block cluster of the cluster columns (0: the library's "
                         "default, -1: none; ncu drops the cluster shape of a launch, so captures use -1)")
    ap.add_argument("--fits", type=int, default=256, help="batched: fits per batch")
    ap.add_argument("--max-subjects", type=int, default=500_000, help="batched: largest fit's subjects")
    ap.add_argument("--outcomes", type=int, default=32, help="serving: resident outcomes")
    ap.add_argument("--max-eras", type=float, default=20e6, help="serving: largest outcome's eras")
    ap.add_argument("--rates", default="1,2,5,10,20,50,100,200", help="serving: arrival rates per second")
    ap.add_argument("--requests", type=int, default=0,
                    help="serving: requests per rate (0: 3 s of arrivals, at least 32 and at most 192)")
    ap.add_argument("--hbm-budget-gb", type=float, default=48.0, help="serving: fit-slot memory budget")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if args.workload != "fit":
            if rank == 0:
                print(json.dumps({"impl": "reference", "workload": args.workload,
                                  "unavailable": "the oracle arm times the single-fit workload; batched and "
                                                 "serving lines carry their own oracle sample"}), flush=True)
            return 0
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched(args, rank, world, local)
    if args.workload == "serving":
        return run_serving(args, rank, world, local)
    if args.workload == "paper":
        return run_paper(args, rank, world, local, oracle_check=args.oracle_check)
    if args.workload == "large-columns":
        return run_large_columns(args, rank, world, local)
    return run_ours(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
