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


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2307_11248_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(f.read())
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
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

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
                        walk_base=rank * W, threads_per_walk=args.threads_per_walk)
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
    tmax = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    evals_all = torch.tensor([evals_rank], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(tmax, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(evals_all, op=torch.distributed.ReduceOp.SUM)
    total_s = tmax.item() / 1e3
    value = evals_all.item() / total_s
    clk = clocks.summary()

    # ---- plain form: one launch per walk (same kernel body), one step
    plain = None
    if not args.no_plain and rank == 0:
        pprm = q.make_params(W, seed=w["seed"], iters=iters, tenure=w["tenure"],
                             aspiration=True, walk_base=rank * W, launch=q.LAUNCH_PLAIN,
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


if __name__ == "__main__":
    main()
