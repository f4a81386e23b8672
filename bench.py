"""Benchmark: swap-delta evaluations/s of the tabu-search hot path on GB300.

One step = one whole search of the n=50 asymmetric uniform instance: 256
independent tabu walks x 5000 iterations (tenure [45, 55] redrawn every 100
iterations, aspiration on), every walk evaluating all 1225 pairwise
exchanges per iteration, in one persistent launch of the CUDA library.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  value = swap-delta evaluations per second over all
ranks (walks x iterations x n(n-1)/2 / time), inputs already resident on the
device; e2e = the same metric through the blocking C-ABI call with host
buffers (instance upload, search, result download, teardown per step).
With N > 1 (torchrun) every rank runs its own walks (replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "swap-delta evals/sec and tabu iters/sec vs SMEM roofline; batched vs plain"
UNIT = "evals/s"
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2
SMEM_BYTES_PER_CLK_PER_SM = 128


def workload():
    from paper_2307_11248_gb300 import instances
    w = instances.workload_asym50()
    n = w["F"].shape[0]
    return dict(w, n=n, pairs=n * (n - 1) // 2)


def algorithmic_bytes_per_iteration(n, delta_bytes, sym):
    """Bytes one tabu iteration of one walk must touch on chip: every delta
    read and written once (2w per pair), a 2-byte tabu stamp read per pair,
    and the rows (and, asymmetric, columns) of F and P read for the 2(n-2)
    recomputed pairs (2n^2 or 4n^2 one-byte elements)."""
    T = n * (n - 1) // 2
    return T * (2 * delta_bytes + 2) + (2 if sym else 4) * n * n


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu_id)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# the sources of the kernels' code (the qap_walk_* / qap_batch_* units only
# list which template instances exist)
KERNEL_SOURCES = ("qap_kernels.cuh", "qap_philox.cuh")


def kernel_source_hash():
    """Hash of the kernel sources' code: comments and blank lines are left
    out, so a change of wording does not orphan a profile."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2307_11248_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name)) as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def ncu_traffic(kernel_hash):
    """DRAM bytes per launch of the walk kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "walk_kernel_asym50.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if m_hash and m_bytes and m_hash.group(1) == kernel_hash:
        return float(m_bytes.group(1))
    return None


def peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(w, walks, iters, threads):
    import oracle
    t0 = time.perf_counter()
    out = oracle.run_walks(w["F"], w["D"], walks, seed=w["seed"], iters=iters,
                           tenure=w["tenure"], aspiration=True, threads=threads)
    dt = time.perf_counter() - t0
    evals = float(out["iters_done"].sum()) * w["pairs"]
    return evals / dt, dt, out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def replica_walk_base(rank, walks_per_rank):
    """Walk ids of rank r are r*W .. r*W + W - 1: replicas search disjoint
    walks whose union is the one-process search of N*W walks."""
    return rank * walks_per_rank


def combine_ranks(total_ms, evals_rank, device):
    """Whole-job figures: the slowest rank's time and the sum of all ranks'
    evaluations (torch.distributed when it is initialised, else this rank's)."""
    import torch
    tmax = torch.tensor([total_ms], dtype=torch.float64, device=device)
    evals = torch.tensor([evals_rank], dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(evals, op=torch.distributed.ReduceOp.SUM)
    return tmax.item(), evals.item()


def run_reference(args, world, rank):
    """The oracle (CPU), timed on the host cores: each step is a bounded
    sample of the workload (the first `ref_walks` walks, full iterations)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = workload()
    threads = os.cpu_count() or 1
    walks = args.ref_walks
    for _ in range(args.warmup):
        cpu_baseline(w, max(1, threads), min(w["iters"], 200), threads)
    times, evals = [], 0.0
    for _ in range(args.steps):
        v, dt, out = cpu_baseline(w, walks, w["iters"], threads)
        times.append(dt)
        evals += float(out["iters_done"].sum()) * w["pairs"]
    total = sum(times)
    value = evals / total
    sample = f"{walks} of {w['walks']} walks x {w['iters']} iterations per step, OpenMP over walks"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": "tabu n=50 asym uniform[0,99], 256 walks x 5000 iters",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-walks", type=int, default=64)
    ap.add_argument("--cpu-walks", type=int, default=128, help="oracle sample for cpu_baseline")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-walk-per-launch form")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--threads-per-walk", type=int, default=0)
    ap.add_argument("--iters", type=int, default=0,
                    help="override the iteration count (smaller cases for profiling)")
    ap.add_argument("--walks", type=int, default=0, help="override the walk count")
    ap.add_argument("--workload", choices=["asym50", "sym12", "grid100", "batch512", "serve",
                                           "sweep"],
                    default="asym50",
                    help="asym50 is the benchmark line; the others measure the remaining "
                         "workloads (one JSON line each)")
    ap.add_argument("--requests", type=int, default=600, help="serve: requests per run")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload != "asym50" and args.impl == "ours":
        return other_workloads(args)

    if args.impl == "reference":
        # rank 0 alone times the oracle on the host cores; no process group
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")),
                      int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_setup()

    import torch
    import paper_2307_11248_gb300 as q
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload()
    if args.iters:
        w["iters"] = args.iters
    if args.walks:
        w["walks"] = args.walks
    n, T, W, iters = w["n"], w["pairs"], w["walks"], w["iters"]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    inst = q.Instance(w["F"], w["D"])
    prm = q.make_params(W, seed=w["seed"], iters=iters, tenure=w["tenure"], aspiration=True,
                        walk_base=replica_walk_base(rank, W),
                        threads_per_walk=args.threads_per_walk)
    plan = inst.plan(prm)
    outs = inst.device_outputs(W, device=dev)

    def step():
        inst.search_async(prm, outs, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()

    # ---- timed region: K steps, L2 flushed between them (not timed)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    gpu_uuid = str(torch.cuda.get_device_properties(dev).uuid)
    gpu_id = gpu_uuid if gpu_uuid.startswith("GPU-") else f"GPU-{gpu_uuid}"
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(gpu_id) as clocks:
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(k & 0xff)
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    iters_done = outs["iters_done"].sum().item()
    evals_rank = float(iters_done) * T * args.steps
    max_ms, evals_all = combine_ranks(total_ms, evals_rank, dev)
    total_s = max_ms / 1e3
    value = evals_all / total_s
    clk = clocks.summary()

    # ---- plain form: one launch per walk (same kernel body), one step
    plain = None
    if not args.no_plain and rank == 0:
        pprm = q.make_params(W, seed=w["seed"], iters=iters, tenure=w["tenure"],
                             aspiration=True, walk_base=replica_walk_base(rank, W),
                             launch=q.LAUNCH_PLAIN,
                             threads_per_walk=args.threads_per_walk)
        pouts = inst.device_outputs(W, device=dev)
        with torch.cuda.stream(stream):
            inst.search_async(pprm, pouts, stream=stream)  # warm-up
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            inst.search_async(pprm, pouts, stream=stream)
            b.record(stream)
        torch.cuda.synchronize(dev)
        pms = a.elapsed_time(b)
        same = all(torch.equal(pouts[k], outs[k]) for k in outs)
        plain = {"value": float(pouts["iters_done"].sum().item()) * T / (pms / 1e3), "unit": UNIT,
                 "ms_per_step": pms, "launches_per_step": W, "results_identical": same}

    # ---- end to end through the blocking C-ABI call with host buffers
    e2e_times = []
    h2d = d2h = 0
    for k in range(max(2, min(args.steps, 3)) + 1):
        t0 = time.perf_counter()
        h = q.qap_create(w["F"], w["D"])
        res = q.qap_search(h, prm, n=n)
        q.qap_destroy(h)
        dt = time.perf_counter() - t0
        if k > 0:
            e2e_times.append(dt)
        info_dbytes = 2 * n * ((n + 7) // 8 * 8) * (1 if inst.info["sym_flow"] else 2)
        h2d = info_dbytes + n * n
        d2h = sum(v.nbytes for v in res.values())
    e2e_value = float(res["iters_done"].sum()) * T / float(np.mean(e2e_times)) * world

    # ---- roofline of the walk kernel (one launch per step)
    launch_s = float(np.mean(step_ms)) / 1e3
    dbytes = inst.info["delta_bytes"]
    sym = bool(inst.info["sym_flow"] and inst.info["sym_dist"])
    bytes_per_unit = algorithmic_bytes_per_iteration(n, dbytes, sym)
    units_per_launch = float(iters_done)
    achieved = bytes_per_unit * units_per_launch / launch_s / 1e9
    sm_max = clk["sm_max_mhz"] or 2070.0
    peak = SMEM_BYTES_PER_CLK_PER_SM * plan["sms"] * sm_max * 1e6 / 1e9
    khash = kernel_source_hash()
    traffic = ncu_traffic(khash)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32" if dbytes == 4 else "int64",
        "data": "synthetic",
        "config": {"workload": f"tabu n=50 asym uniform[0,99], {W} walks x {iters} iters",
                   "n": n, "walks_per_gpu": W, "iters": iters, "tenure": list(w["tenure"]),
                   "aspiration": True, "launch": "persistent, one launch per step",
                   "threads_per_walk": plan["threads_per_walk"], "grid": plan["grid"],
                   "l2": "flushed between timed steps (256 MiB write); working set on chip",
                   "parallelism": f"replicas x{world}"},
        "tabu_iters_per_s": value / T,
        "roofline": {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_note": "derived: 128 B/clk/SM x SMs x max SM clock",
                     "bytes_per_unit": bytes_per_unit, "unit_def": "one tabu iteration of one walk",
                     "units_per_launch": units_per_launch},
        "gpu_launches": args.steps,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
                   "reasons": clk["reasons"], "samples": clk["samples"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "call": "qap_create + qap_search (host outputs) + qap_destroy"},
        "plain": plain,
        "batched_over_plain": (value / world / plain["value"]) if plain else None,
        "kernel_sources": khash,
    }

    if rank == 0 and world == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        cw = min(args.cpu_walks, W)
        v, dt, _ = cpu_baseline(w, cw, iters, threads)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"{cw} of {W} walks x {iters} iterations, "
                                          f"{dt:.1f} s wall on {threads} threads"}
    if rank == 0:
        print(json.dumps(line))
    inst.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def timed_steps(step, steps, stream, flush, dev):
    """Device time of `steps` calls of step(), L2 flushed between them."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    gpu_uuid = str(torch.cuda.get_device_properties(dev).uuid)
    gpu_id = gpu_uuid if gpu_uuid.startswith("GPU-") else f"GPU-{gpu_uuid}"
    torch.cuda.synchronize(dev)
    with ClockSampler(gpu_id) as clocks:
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.fill_(k & 0xff)
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    return [a.elapsed_time(b) for a, b in ev], clocks.summary()


def sampled_plain(q, inst, prm_kw, walks, stream, dev):
    """The one-walk-per-launch form on a bounded sample of walks: evals/s
    (2opt moves and tabu iterations, n(n-1)/2 evaluations each)."""
    import torch
    n = inst.n
    prm = q.make_params(walks, launch=q.LAUNCH_PLAIN, **prm_kw)
    outs = inst.device_outputs(walks, device=dev)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        a.record(stream)
        inst.search_async(prm, outs, stream=stream)
        b.record(stream)
    stream.synchronize()
    moves = float(outs["iters_done"].sum().item() + outs["descent_moves"].sum().item())
    return moves * n * (n - 1) / 2 / (a.elapsed_time(b) / 1e3)


def sampled_oracle(F, D, walks, **kw):
    """The oracle (O(1)-update mode, all host cores) on a bounded sample."""
    import oracle
    oracle.build()
    n = F.shape[0]
    t0 = time.perf_counter()
    o = oracle.run_walks(F, D, walks, **kw)
    dt = time.perf_counter() - t0
    moves = float(o["iters_done"].sum() + o["descent_moves"].sum())
    return moves * n * (n - 1) / 2 / dt, dt, oracle.num_threads()


def other_workloads(args):
    """The remaining workloads, one JSON line each (N = 1)."""
    import torch
    import paper_2307_11248_gb300 as q
    from paper_2307_11248_gb300 import instances
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    line = {"unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic"}

    if args.workload == "grid100":
        w = instances.workload_grid100()
        n = w["F"].shape[0]
        T = n * (n - 1) // 2
        W = args.walks or w["walks"]
        iters = args.iters or w["iters"]
        inst = q.Instance(w["F"], w["D"])
        prm = q.make_params(W, seed=w["seed"], iters=iters, tenure=w["tenure"], descend=True)
        outs = inst.device_outputs(W, device=dev)
        with torch.cuda.stream(stream):
            inst.search_async(prm, outs, stream=stream)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()  # the whole search as one graph launch
        with torch.cuda.graph(graph, stream=stream):
            inst.search_async(prm, outs, stream=stream)
        for _ in range(args.warmup):
            graph.replay()
        ms, clk = timed_steps(graph.replay, args.steps, stream, flush, dev)
        moves = float(outs["iters_done"].sum().item() + outs["descent_moves"].sum().item())
        plan = inst.plan(prm)
        kw = dict(seed=w["seed"], iters=iters, tenure=w["tenure"], descend=True)
        if not args.no_plain:
            plain = sampled_plain(q, inst, kw, 16, stream, dev)
            line.update(plain={"value": plain, "unit": "evals/s", "sample": f"16 walks x "
                               f"{iters} iterations, one launch per walk"})
        if not args.no_cpu:
            cpu, cpu_s, cores = sampled_oracle(w["F"], w["D"], 32, seed=w["seed"], iters=1000,
                                               tenure=w["tenure"], descend=True)
            line.update(cpu_baseline={"value": cpu, "unit": "evals/s", "cores": cores,
                                      "kind": "oracle", "sample": "32 walks x (2opt + 1000 "
                                      f"iterations), {cpu_s:.1f} s wall"})
        line.update(metric=METRIC, value=moves * T / (sum(ms) / 1e3 / args.steps),
                    ms_per_step=sum(ms) / args.steps, steps=args.steps, warmup=args.warmup,
                    dtype="int32" if inst.info["delta_bytes"] == 4 else "int64",
                    tabu_iters_per_s=float(outs["iters_done"].sum().item()) /
                    (sum(ms) / 1e3 / args.steps),
                    config={"workload": f"2opt then tabu, n=100 grid, {W} walks x {iters} iters",
                            "launch": "persistent, replayed as one CUDA graph",
                            "threads_per_walk": plan["threads_per_walk"], "grid": plan["grid"],
                            "evals": "2opt moves and tabu iterations, n(n-1)/2 each",
                            "l2": "flushed between timed steps"},
                    gpu_launches=args.steps, clocks=clk)
    elif args.workload == "batch512":
        w = instances.workload_batch512()
        insts = w["instances"]
        W = args.walks or w["walks"]
        iters = args.iters or w["iters"]
        b = q.Batch([i.F for i in insts], [i.D for i in insts], force_int64=True)
        prm = q.make_params(W, seed=w["seed"], iters=iters, tenure=(90, 110, 200), tenure_per_n=True)
        # plans per size class picked by the library's autotuner (outside the timed region)
        tune = b.autotune(prm, trial_iters=max(50, iters // 20))
        outs = b.device_outputs(W, device=dev)
        step = lambda: b.search_async(prm, outs, stream=stream)  # noqa: E731
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
        ms, clk = timed_steps(step, args.steps, stream, flush, dev)
        it = outs["iters_done"].cpu().numpy().reshape(len(insts), W)
        evals = sum(float(it[i].sum()) * insts[i].n * (insts[i].n - 1) / 2
                    for i in range(len(insts)))
        plan = b.plan(prm)
        # bounded samples: the plain form on 4 walks of 8 instances, the oracle on
        # 8 walks x 500 iterations of the same 8 instances
        sample = insts[::64]
        pl_e = pl_t = cpu_e = cpu_t = 0.0
        cores = 0
        for inst_ in sample:
            if not args.no_plain:
                with q.Instance(inst_.F, inst_.D, force_int64=True) as one:
                    tn = instances.periodic_tenure(inst_.n)
                    e = sampled_plain(q, one, dict(seed=w["seed"], iters=iters, tenure=tn), 4,
                                      stream, dev)
                    pl_e += 4 * iters * inst_.n * (inst_.n - 1) / 2
                    pl_t += 4 * iters * inst_.n * (inst_.n - 1) / 2 / e
            if not args.no_cpu:
                v, dt, cores = sampled_oracle(inst_.F, inst_.D, 8, seed=w["seed"], iters=500,
                                              tenure=instances.periodic_tenure(inst_.n))
                cpu_e += v * dt
                cpu_t += dt
        if not args.no_plain:
            line.update(plain={"value": pl_e / pl_t, "unit": "evals/s",
                               "sample": "4 walks of every 64th instance, one launch per walk"})
        if not args.no_cpu:
            line.update(cpu_baseline={"value": cpu_e / cpu_t, "unit": "evals/s",
                                      "cores": cores, "kind": "oracle",
                                      "sample": "8 walks x 500 iterations of every 64th "
                                      f"instance, {cpu_t:.1f} s wall"})
        line.update(metric=METRIC, value=evals / (sum(ms) / 1e3 / args.steps),
                    ms_per_step=sum(ms) / args.steps, steps=args.steps, warmup=args.warmup,
                    dtype="int64", tabu_iters_per_s=float(it.sum()) / (sum(ms) / 1e3 / args.steps),
                    config={"workload": f"{len(insts)} lognormal instances, n in [20,150], "
                                        f"{W} walks x {iters} iters each",
                            "launch": "one persistent launch per size class, classes concurrent "
                                      "on forked streams, device work queues, largest n first",
                            "classes": plan["classes"],
                            "autotuned": [{"n": [r["nmin"], r["nmax"]],
                                           "plan": [r["threads_per_walk"], r["pairs_per_thread"]],
                                           "workspace": bool(r["workspace"]),
                                           "products": bool(r["products"]),
                                           "trial_ms": round(r["trial_ms"], 3),
                                           "rule_ms": round(r["rule_ms"], 3)} for r in tune],
                            "l2": "flushed between timed steps"},
                    gpu_launches=args.steps * plan["classes"], clocks=clk)
    elif args.workload == "sym12":
        line.update(sym12(args, q, instances, stream, flush, dev))
    elif args.workload == "sweep":
        line.update(sweep(args, q, instances, stream, dev))
    else:
        line.update(serve(args, q, instances))
    print(json.dumps(line))


def sym12(args, q, instances, stream, flush, dev):
    """n = 12 symmetric, 2opt to local minima from 32 starts: the latency
    case.  One persistent launch (batched) against one launch per walk
    (plain), and the oracle on the host cores."""
    import torch
    import oracle
    w = instances.workload_sym12()
    n, W = w["F"].shape[0], w["walks"]
    T = n * (n - 1) // 2
    inst = q.Instance(w["F"], w["D"])
    res = {}
    for form, launch in (("batched", q.LAUNCH_PERSISTENT), ("plain", q.LAUNCH_PLAIN)):
        prm = q.make_params(W, seed=w["seed"], descend=True, launch=launch)
        outs = inst.device_outputs(W, device=dev)
        step = lambda: inst.search_async(prm, outs, stream=stream)  # noqa: E731
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
        ms, clk = timed_steps(step, args.steps, stream, flush, dev)
        moves = float(outs["descent_moves"].sum().item())
        res[form] = dict(ms=sum(ms) / args.steps, moves=moves, clk=clk)
    oracle.build()
    t0 = time.perf_counter()
    o = oracle.run_walks(w["F"], w["D"], W, seed=w["seed"], descend=True)
    cpu_s = time.perf_counter() - t0
    b = res["batched"]
    return dict(metric="2opt to local minima, 32 starts: latency and swap-delta evals/s",
                value=b["moves"] * T / (b["ms"] / 1e3), ms_per_step=b["ms"], steps=args.steps,
                warmup=args.warmup, dtype="int32",
                plain={"ms_per_step": res["plain"]["ms"], "launches_per_step": W},
                batched_over_plain=res["plain"]["ms"] / b["ms"],
                cpu_baseline={"kind": "oracle", "ms": cpu_s * 1e3, "cores": oracle.num_threads(),
                              "identical_moves": int(o["descent_moves"].sum()) == int(b["moves"])},
                config={"workload": "sym12: n=12 symmetric uniform[0,99], 2opt from 32 starts",
                        "launch": "persistent, one launch per step", "l2": "flushed between steps"},
                gpu_launches=args.steps, clocks=b["clk"])


def sweep(args, q, instances, stream, dev):
    """Tabu sensitivity to the iteration budget, the walk count and the seed
    (the paper's Section 6.6, Figs. 7-9), on the asym50 stand-in and on one
    int64 lognormal instance of the batch family, plus 2opt on the GPU
    against the oracle on the host cores (Fig. 4).  Gap = (best of the walks
    - best known) / best known, the best known being the lowest cost any run
    here found (including a 1024 x 20000 reference run)."""
    import torch
    import oracle

    def run(inst, W, iters, seed, tn, descend=False):
        prm = q.make_params(W, seed=seed, iters=iters, tenure=tn, descend=descend)
        outs = inst.device_outputs(W, device=dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            inst.search_async(prm, outs, stream=stream)
            b.record(stream)
        stream.synchronize()
        return int(outs["best_cost"].min().item()), a.elapsed_time(b)

    out = {}
    lognormal = instances.lognormal_instance(100, 77, symmetric=False)
    for name, (F, D), f64 in (("asym50", (instances.workload_asym50()["F"],
                                          instances.workload_asym50()["D"]), False),
                              ("lognormal100", lognormal, True)):
        n = F.shape[0]
        tn = instances.periodic_tenure(n)
        inst = q.Instance(F, D, force_int64=f64)
        run(inst, 64, 100, 1, tn)  # warm-up
        rows = []
        ref, _ = run(inst, 1024, 20000, 999, tn)
        for iters in (500, 1000, 2000, 5000, 10000, 20000):
            for seed in (1, 2, 3):
                c, ms = run(inst, 256, iters, seed, tn)
                rows.append(("iters", iters, 256, seed, c, ms))
        for W in (32, 64, 128, 256, 512, 1024):
            for seed in (1, 2, 3):
                c, ms = run(inst, W, 5000, seed, tn)
                rows.append(("walks", 5000, W, seed, c, ms))
        for seed in range(10, 18):
            c, ms = run(inst, 256, 5000, seed, tn)
            rows.append(("seeds", 5000, 256, seed, c, ms))
        best = min([ref] + [r[4] for r in rows])
        table = {}
        for kind, iters, W, seed, c, ms in rows:
            key = f"{kind}:{iters}x{W}"
            t = table.setdefault(key, {"iters": iters, "walks": W, "gaps_pct": [], "ms": []})
            t["gaps_pct"].append(round(100.0 * (c - best) / best, 4))
            t["ms"].append(round(ms, 2))
        out[name] = {"n": n, "best_known": best, "reference_run": "1024 walks x 20000 iters",
                     "tenure": list(tn), "rows": table}
        inst.close()
    # 2opt: GPU (32 starts, one launch) against the oracle on all host cores
    fig4 = []
    oracle.build()
    for n in (30, 50, 80, 100):
        F, D = instances.uniform_instance(n, 300 + n, symmetric=False)
        inst = q.Instance(F, D)
        run(inst, 32, 0, 5, (1, 1, 0), descend=True)
        _, ms = run(inst, 32, 0, 5, (1, 1, 0), descend=True)
        inst.close()
        t0 = time.perf_counter()
        oracle.run_walks(F, D, 32, seed=5, descend=True)
        cpu_ms = (time.perf_counter() - t0) * 1e3
        fig4.append({"n": n, "gpu_ms": round(ms, 3), "cpu_oracle_ms": round(cpu_ms, 2),
                     "cpu_threads": oracle.num_threads()})
    return dict(metric="tabu solution-quality gap vs iterations, walks and seeds; 2opt GPU vs CPU",
                value=None, unit="gap %", higher_is_better=False, dtype="int32/int64",
                sweeps=out, two_opt_vs_cpu=fig4,
                config={"workload": "asym50 and a lognormal n=100 instance (int64); "
                                    "2opt on uniform n in {30,50,80,100}"},
                gpu_launches=None)


def serve(args, q, instances):
    """Poisson stream of 32-walk x 2000-iteration tabu requests, n in
    [12, 256], through the serving loop: solves/s and latency percentiles,
    at the offered 2000 req/s and at 0.8x the measured capacity."""
    count = args.requests
    reqs = instances.poisson_requests(count, seed=4, rate_per_s=2000.0)
    prms = [q.make_params(32, seed=r.rid, iters=2000, tenure=instances.periodic_tenure(r.inst.n))
            for r in reqs]
    warm = instances.poisson_requests(20, seed=99)

    def run(rate, sv):
        t0 = time.perf_counter()
        tickets = []
        for r, p in zip(reqs, prms):
            due = t0 + (r.arrival_s * 2000.0 / rate if rate else 0.0)
            now = time.perf_counter()
            if due > now:
                time.sleep(due - now)
            tickets.append(sv.submit(r.inst.F, r.inst.D, p))
        lat = []
        for t in tickets:
            _, tm = sv.wait(t, timeout_ms=600000)
            lat.append(tm["total_us"] / 1e3)
        wall = time.perf_counter() - t0
        lat = np.array(lat)
        return {"solves_per_s": count / wall, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "wall_s": wall}

    # baselines on bounded samples: the same requests one at a time through
    # qap_search (no overlap), and the plain one-walk-per-launch form
    t0 = time.perf_counter()
    for r, p in list(zip(reqs, prms))[:60]:
        with q.Instance(r.inst.F, r.inst.D) as one:
            one.search(p)
    sequential = 60 / (time.perf_counter() - t0)
    t0 = time.perf_counter()
    for r in reqs[:6]:
        with q.Instance(r.inst.F, r.inst.D) as one:
            one.search(q.make_params(32, seed=r.rid, iters=2000,
                                     tenure=instances.periodic_tenure(r.inst.n),
                                     launch=q.LAUNCH_PLAIN))
    plain = 6 / (time.perf_counter() - t0)
    with q.Server(slots=64, mem_bytes=2 << 30) as sv:
        for r in warm:
            sv.wait(sv.submit(r.inst.F, r.inst.D, q.make_params(
                32, seed=r.rid, iters=200, tenure=instances.periodic_tenure(r.inst.n))))
        run(0, sv)                        # grows every slot's pinned buffers and the arena
        saturated = run(0, sv)            # all at once: capacity
        offered = run(2000.0, sv)         # the offered Poisson rate
        rate80 = 0.8 * saturated["solves_per_s"]
        at80 = run(rate80, sv)
    evals = sum(32 * 2000 * r.inst.n * (r.inst.n - 1) / 2 for r in reqs)
    return {"metric": "solves/s (serving, 32-walk x 2000-iteration tabu requests)",
            "value": offered["solves_per_s"], "unit": "solves/s", "steps": 1, "warmup": 1,
            "ms_per_step": offered["wall_s"] * 1e3, "dtype": "int32",
            "p50_ms": offered["p50_ms"], "p99_ms": offered["p99_ms"],
            "overloaded": offered["solves_per_s"] < 0.95 * 2000.0,
            "capacity_solves_per_s": saturated["solves_per_s"],
            "at_0.8_capacity": {"rate": rate80, **at80},
            "swap_evals_per_s_at_capacity": evals / saturated["wall_s"],
            "sequential": {"solves_per_s": sequential,
                           "sample": "first 60 requests one at a time through qap_search"},
            "plain": {"solves_per_s": plain,
                      "sample": "first 6 requests, one launch per walk, one at a time"},
            "capacity_over_sequential": saturated["solves_per_s"] / sequential,
            "capacity_over_plain": saturated["solves_per_s"] / plain,
            "config": {"workload": f"{count} Poisson requests (2000/s offered), n in [12,256], "
                                   "generators sym uniform / asym uniform / grid",
                       "server": "64 slots, 2 GiB arena, FIFO admission by slot and memory"},
            "gpu_launches": 4 * count}


if __name__ == "__main__":
    main()
