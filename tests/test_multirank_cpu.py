"""Two CPU ranks over gloo (127.0.0.1): the multi-rank paths without a GPU.

* the benchmark's cross-rank reductions and barrier (the N > 1 bench path: replicas, max time
  over ranks, units summed over ranks);
* subject shards on separate ranks: L, g_j and h_j are sums over subjects (M is block
  diagonal), so each rank's partial sums, all-reduced, must give the unsharded values; and a
  cyclic coordinate descent that all-reduces (g_j, h_j) once per coordinate — the exchange a
  subject-sharded multi-GPU fit would make — must follow the single-process oracle's trajectory.
"""
import os
import socket
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path[:0] = [ROOT, HERE]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    import bench
    import oracle
    from sccs_testlib import from_dense, random_tiny, to_dense

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {"max": bench.reduce_max(rank + 1.0, world), "sum": bench.reduce_sum(rank + 1.0, world)}
        bench.barrier(world)

        d = random_tiny(12, n_patients=60, J=4, beta_scale=0.6)
        X = to_dense(d)
        mask = (d.patient_id % world) == rank          # this rank's subjects
        part = oracle.Problem.from_data(from_dense(d.patient_id[mask], d.y[mask], d.L[mask], X[mask]))
        full = oracle.Problem.from_data(d)
        beta_probe = np.array([0.3, -0.2, 0.5, -0.1])
        t = torch.tensor([part.loglik(beta_probe)] + [v for j in range(d.J) for v in part.grad_hess(j, beta_probe)],
                         dtype=torch.float64)
        dist.all_reduce(t)
        ref = [full.loglik(beta_probe)] + [v for j in range(d.J) for v in full.grad_hess(j, beta_probe)]
        res["shard_sums_err"] = float(np.max(np.abs(t.numpy() - np.array(ref)) / np.maximum(1.0, np.abs(ref))))

        # CCD with one (g_j, h_j) all-reduce per coordinate; Normal prior, trust region as the oracle's
        var, cycles = 0.5, 3
        beta = np.zeros(d.J)
        trust = np.ones(d.J)
        for _ in range(cycles):
            for j in range(d.J):
                g, h = part.grad_hess(j, beta)
                gh = torch.tensor([g, h], dtype=torch.float64)
                dist.all_reduce(gh)
                g, h = gh.tolist()
                dv = (g - beta[j] / var) / (-h + 1.0 / var)
                db = min(max(dv, -trust[j]), trust[j])
                trust[j] = max(2.0 * abs(db), 0.5 * trust[j])
                beta[j] += db
        oref = full.fit(prior="normal", variance=var, fixed_cycles=cycles)
        res["ccd_err"] = float(np.max(np.abs(beta - oref["beta"])))
        res["ccd_nontrivial"] = float(np.max(np.abs(oref["beta"])))
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def results():
    import oracle
    import torch.multiprocessing as mp
    oracle.build()
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        return dict(out)


def test_bench_reductions_over_two_ranks(results):
    for r in (0, 1):
        assert results[r]["max"] == 2.0 and results[r]["sum"] == 3.0


def test_subject_shards_on_two_ranks_add_up(results):
    for r in (0, 1):
        assert results[r]["shard_sums_err"] <= 1e-12


def test_ccd_with_one_allreduce_per_coordinate_follows_the_oracle(results):
    for r in (0, 1):
        assert results[r]["ccd_nontrivial"] > 0.05
        assert results[r]["ccd_err"] <= 1e-10
