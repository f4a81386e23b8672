"""The N > 1 path of the benchmark on CPU: two gloo ranks.  Walks are
independent, so the ranks are replicas with disjoint walk ids (no data-path
collective); only the whole-job time (max over ranks) and evaluation count
(sum) are combined."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, W, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2307_11248_gb300 import instances
    w = instances.workload_asym50()
    base = bench.replica_walk_base(rank, W)
    o = oracle.run_walks(w["F"], w["D"], W, seed=w["seed"], iters=40, tenure=w["tenure"],
                         walk_ids=np.arange(base, base + W), threads=1)
    evals = float(o["iters_done"].sum()) * 50 * 49 / 2
    ms, total = bench.combine_ranks(10.0 + rank, evals, torch.device("cpu"))
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), best=o["best_cost"], hash=o["hash"],
             ms=ms, total=total, evals=evals)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_are_disjoint_replicas(tmp_path):
    world, W = 2, 3
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, W, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / f"rank{k}.npz") for k in range(world)]
    # max over ranks and sum of evaluations, seen identically by both ranks
    for k in range(world):
        assert float(r[k]["ms"]) == 11.0
        assert float(r[k]["total"]) == float(r[0]["evals"]) + float(r[1]["evals"])
    # the union of the replicas is the one-process search of world * W walks
    import oracle
    from paper_2307_11248_gb300 import instances
    w = instances.workload_asym50()
    one = oracle.run_walks(w["F"], w["D"], world * W, seed=w["seed"], iters=40,
                           tenure=w["tenure"])
    assert np.array_equal(np.concatenate([r[0]["best"], r[1]["best"]]), one["best_cost"])
    assert np.array_equal(np.concatenate([r[0]["hash"], r[1]["hash"]]), one["hash"])
