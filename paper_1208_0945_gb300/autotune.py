"""Autotuners: launch parameters of one fit, and team sizes for batched fits.

`tune_launch` picks the launch parameters of a dataset's handle by timed probe fits through the
library on the caller's own data: the thread-block cluster that takes the small and mid-size
columns (its size, and the column size up to which a column runs there: the column tile of the
cluster path), or without a cluster the narrow-column size and group limits, and the threads
(warps) per CTA.  A coordinate search: each knob in turn, keeping the fastest setting so far.

Team sizes for batched fits:

A fit run by a team of S CTAs costs, per CCD cycle, about

    t(S) = J * lat(S) + nnz * c / S

where lat(S) is the per-coordinate latency of a team of S CTAs (phase A on a tiny slice, the
team's all-reduce, the FP64 step, phase C) and c the device time per nonzero on one CTA.  Both
are measured on the device with probe fits through the library (`measure`).  `assign` then
gives every fit of a batch a team size by greedy makespan minimisation against a simulation of
the library's batched launch (a ticket queue: fits handed out longest first, each starting
when its team's CTAs are free): start from one CTA per fit and keep growing the team of the
fit that runs longest while the simulated makespan drops.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import sccs as _s


@dataclasses.dataclass
class CostModel:
    lat_us: dict          # team size -> microseconds per coordinate step
    c_us_per_nnz: float   # microseconds per nonzero on one CTA
    capacity: int         # CTAs the device holds at once

    def latency(self, S: int) -> float:
        ks = sorted(self.lat_us)
        if S <= ks[0]:
            return self.lat_us[ks[0]]
        if S >= ks[-1]:
            return self.lat_us[ks[-1]]
        hi = next(k for k in ks if k >= S)
        lo = max(k for k in ks if k <= S)
        if hi == lo:
            return self.lat_us[lo]
        w = (np.log(S) - np.log(lo)) / (np.log(hi) - np.log(lo))
        return (1 - w) * self.lat_us[lo] + w * self.lat_us[hi]

    def cycle_us(self, J: int, nnz: int, S: int) -> float:
        return J * self.latency(S) + nnz * self.c_us_per_nnz / S


def _probe(data, S, device, cycles):
    with _s.SCCSModel(data, device=device, num_shards=S) as m:
        m.set_prior("normal", 1.0)
        m.fit(tol=-1.0, max_cycles=1)                       # warm-up
        r = m.fit(tol=-1.0, max_cycles=cycles)
        return r["kernel_ms"] * 1e3 / cycles, m.info


def measure(device: int = 0, team_sizes=(1, 2, 4, 8, 16, 32, 64, 128), cycles: int = 3) -> CostModel:
    from synth import make_dataset
    import ctypes

    # latency: many tiny columns (one or two nonzeros per shard)
    tiny = make_dataset(n_patients=3000, eras=("uniform", 1, 4), J=64, columns=("density", 0.01), n_true=0,
                        beta_sd=0.0, seed=5150)
    # throughput: a few dense columns
    dense = make_dataset(n_patients=150_000, eras=("geometric", 8), J=4, columns=("density", 0.3), n_true=0,
                         beta_sd=0.0, seed=5151)
    cap = _capacity(device)
    lat = {}
    for S in team_sizes:
        if S > cap:
            continue
        us, _ = _probe(tiny, S, device, cycles)
        lat[S] = us / tiny.J
    S_big = max(k for k in lat)
    us, info = _probe(dense, S_big, device, cycles)
    c = max(us - dense.J * lat[S_big], 1e-3) * S_big / max(info["nnz_kept"], 1)
    return CostModel(lat_us=lat, c_us_per_nnz=c, capacity=cap)


def _capacity(device: int) -> int:
    import torch

    props = torch.cuda.get_device_properties(device)
    return int(props.multi_processor_count)   # one CTA per SM (512 threads, ~134 KB shared memory)


def library_order(fits, S) -> list:
    """The order in which the library's batched launch hands out tickets: longest first by its
    own estimate (8192 per coordinate plus (nnz + 2 segments) per CTA of the team)."""
    cost = [8192.0 * J + (nnz + 2.0 * segs) / s for (J, nnz, segs), s in zip(fits, S)]
    return sorted(range(len(fits)), key=lambda k: -cost[k])


def makespan(fits, S, model: CostModel, capacity: int | None = None) -> float:
    """Device time per cycle of the batch under the queue launch: fits in library order, each
    starting when its S CTAs are free (the S earliest-free CTAs), per-cycle cost from the model."""
    import heapq

    cap = capacity or model.capacity
    free = [0.0] * min(cap, sum(S))
    heapq.heapify(free)
    end = 0.0
    for k in library_order(fits, S):
        J, nnz, _ = fits[k]
        got = [heapq.heappop(free) for _ in range(S[k])]
        t1 = max(got) + model.cycle_us(J, nnz, S[k])
        for _ in range(S[k]):
            heapq.heappush(free, t1)
        end = max(end, t1)
    return end


def assign(fits, model: CostModel, capacity: int | None = None, max_rounds: int = 4000) -> list:
    """fits: [(J, nnz per cycle, segments)]; returns a team size per fit.

    Starts from one CTA per fit and repeatedly doubles (then grows by one) the team of the fit
    that ends last in the simulated schedule, keeping a change only when the makespan drops."""
    cap = capacity or model.capacity
    fits = [tuple(f) + (0,) * (3 - len(f)) for f in fits]
    S = [1] * len(fits)
    best = makespan(fits, S, model, cap)
    frozen = set()
    for _ in range(max_rounds):
        cand = [k for k in range(len(fits)) if k not in frozen]
        if not cand:
            break
        f = max(cand, key=lambda k: model.cycle_us(fits[k][0], fits[k][1], S[k]))
        improved = False
        for new in (min(cap, 2 * S[f]), min(cap, S[f] + 1)):
            if new <= S[f]:
                continue
            trial = list(S)
            trial[f] = new
            t = makespan(fits, trial, model, cap)
            if t < best:
                S, best, improved = trial, t, True
                break
        if not improved:
            frozen.add(f)
    return S


# ------------------------------------------------------------------ launch parameters of one fit

@dataclasses.dataclass
class LaunchChoice:
    options: dict         # sccs_create keyword options of the fastest probe
    kernel_ms: float      # its device time for the probe cycles
    trials: list          # every probe: (options, kernel_ms), in the order taken


def _knob_stages(best: dict) -> list:
    """The settings tried for each knob in turn, given the choices made so far."""
    on = best.get("cluster_ctas", 16) > 0
    return [
        [dict(cluster_ctas=16), dict(cluster_ctas=8), dict(cluster_ctas=-1)],
        ([dict(cluster_max_nnz=v) for v in (8192, 16384, 65536)] if on
         else [dict(narrow_max_nnz=v) for v in (512, 1024, 2048)]),
        [] if on else [dict(narrow_group_max=g) for g in (1, 4, 8)],
        [dict(threads_per_block=t) for t in (512, 384, 256)],
    ]


def _probe_launch(data, options, device, prior, variance, cycles) -> float:
    with _s.SCCSModel(data, device=device, **options) as m:
        m.set_prior(prior, variance)
        m.fit(tol=-1.0, max_cycles=1)                       # warm-up
        return min(m.fit(tol=-1.0, max_cycles=cycles)["kernel_ms"] for _ in range(2))


def tune_launch(data, device: int = 0, prior: str = "normal", variance: float = 1.0, cycles: int = 2,
                timer=None) -> LaunchChoice:
    """Timed probe fits (`cycles` fixed cycles from beta = 0, best of two) on `data` for each knob
    in turn; returns the fastest options.  `timer(data, options)` replaces the probe (tests)."""
    probe = timer or (lambda d, o: _probe_launch(d, o, device, prior, variance, cycles))
    best, best_ms, trials, seen = {}, float("inf"), [], {}
    for stage in range(4):
        cands = _knob_stages(best)[stage]
        if not cands:
            continue
        stage_best = None
        for c in cands:
            opts = {**best, **c}
            key = tuple(sorted(opts.items()))
            if key not in seen:
                seen[key] = probe(data, opts)
                trials.append((opts, seen[key]))
            if stage_best is None or seen[key] < stage_best[1]:
                stage_best = (opts, seen[key])
        best, best_ms = stage_best
    return LaunchChoice(options=best, kernel_ms=best_ms, trials=trials)
