"""Benchmark: swap-delta evaluations/s of the tabu-search hot path on GB300.

The headline step is the batched form over uneven instances: 512 QAP
instances (n uniform in [20, 150], half symmetric, lognormal flows, int64
deltas), 64 tabu walks x 5000 iterations each, one persistent launch per size
class of the library's autotuned plans, the classes concurrent on forked
streams.  Every walk evaluates all n(n-1)/2 pairwise exchanges per
iteration.  The same line carries the n=50 asymmetric workload (256 walks x
5000 tabu iterations, one persistent launch) and the n=100 grid workload
(1024 walks x (2opt + 10^4 tabu iterations), one CUDA graph) as nested
lines, each with its own roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batch512|asym50|grid100|sym12|serve|sweep]

Prints one JSON line.  value = swap-delta evaluations per second over all
ranks (walks x iterations x n(n-1)/2 / device time), inputs already resident
on the device; e2e = the same metric through the blocking C-ABI calls with
host buffers (instance upload, search, result download, teardown per step).
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
WARP_ISSUE_PER_CLK_PER_SM = 4  # four schedulers, one warp instruction each per cycle


def unit_bytes(n, delta_bytes, flow_bytes, dist_bytes, sym):
    """Bytes one tabu iteration of one walk must touch on chip: every delta
    read and written once (2w per pair), a 2-byte tabu stamp read per pair,
    and the rows (and, asymmetric, columns) of F and P read for the 2(n-2)
    recomputed pairs: n^2 elements of each (symmetric) or 2n^2 (asymmetric),
    F elements of flow_bytes and P elements of dist_bytes."""
    T = n * (n - 1) // 2
    return T * (2 * delta_bytes + 2) + (1 if sym else 2) * n * n * (flow_bytes + dist_bytes)


def smem_peak_gbs(sms, sm_mhz):
    """Shared-memory bandwidth from the unit counts and clock: 128 B per
    clock per SM."""
    return SMEM_BYTES_PER_CLK_PER_SM * sms * sm_mhz * 1e6 / 1e9


def issue_peak(sms, sm_mhz):
    """Warp instructions per second: four schedulers per SM issue one each
    per clock."""
    return WARP_ISSUE_PER_CLK_PER_SM * sms * sm_mhz * 1e6


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


def gpu_uuid_of(dev):
    import torch
    u = str(torch.cuda.get_device_properties(dev).uuid)
    return u if u.startswith("GPU-") else f"GPU-{u}"


# the sources of the kernels' code and of the rules that pick a launch's
# plan (the qap_walk_* / qap_batch_* units only list which template
# instances exist)
KERNEL_SOURCES = ("qap_kernels.cuh", "qap_philox.cuh", "qap_host.cuh")


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


def profile_figures(name, kernel_hash):
    """Numbers recorded in a committed ncu summary (profiles/<name>.md) as
    `key: value` lines, if the summary was taken on the current kernel
    sources; else {}.  Keys: dram_bytes_per_launch (per launch, or per step
    for a batch of class launches) and warp_insts_per_unit (warp
    instructions per walk-iteration)."""
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return {}
    text = open(path).read()
    m_hash = re.search(r"kernel_sources_sha256_16:\s*([0-9a-f]+)", text)
    if not m_hash or m_hash.group(1) != kernel_hash:
        return {}
    out = {}
    for key in ("dram_bytes_per_launch", "warp_insts_per_unit"):
        m = re.search(key + r":\s*([0-9.eE+]+)", text)
        if m:
            out[key] = float(m.group(1))
    return out


def phase_x_of(q, args):
    return q.PHASE_X_DOTS if args.phase_x == "dots" else q.PHASE_X_AUTO


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


def barrier():
    import torch
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()


def timed_steps(step, steps, stream, flush, dev, after_step=None):
    """Device time of `steps` calls of step() (CUDA events on `stream`), L2
    flushed between them; clocks sampled meanwhile.  after_step(k), if
    given, runs on the host after step k has finished (outside its events)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(gpu_uuid_of(dev)) as clocks:
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.fill_(k & 0xff)
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
                if after_step is not None:
                    stream.synchronize()
                    after_step(k)
        torch.cuda.synchronize(dev)
    barrier()
    return [a.elapsed_time(b) for a, b in ev], clocks.summary()


def clock_fields(clk):
    return {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"],
            "reasons": clk["reasons"], "samples": clk["samples"]}


def rooflines(bytes_per_launch, units_per_launch, launch_s, sms, sm_mhz, figs, kernel):
    """Shared-memory roofline (primary) and integer-issue bound (secondary)
    of a launch: algorithmic bytes / launch time against 128 B/clk/SM, and
    warp instructions (per unit, from the committed ncu capture of the same
    kernel sources) / launch time against 4 per clk per SM."""
    achieved = bytes_per_launch / launch_s / 1e9
    peak = smem_peak_gbs(sms, sm_mhz)
    roof = {"bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": figs.get("dram_bytes_per_launch"),
            "peak_note": f"derived: 128 B/clk/SM x {sms} SMs x {sm_mhz:.0f} MHz (max SM clock)",
            "kernel": kernel, "bytes_per_launch": bytes_per_launch,
            "units_per_launch": units_per_launch, "unit_def": "one tabu iteration of one walk"}
    ipu = figs.get("warp_insts_per_unit")
    issue = None
    if ipu:
        ach = ipu * units_per_launch / launch_s
        pk = issue_peak(sms, sm_mhz)
        issue = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "warp inst/s",
                 "frac": ach / pk, "warp_insts_per_unit": ipu,
                 "peak_note": f"derived: 4 warp instructions/clk/SM x {sms} SMs x "
                              f"{sm_mhz:.0f} MHz; warp_insts_per_unit from the committed ncu "
                              "capture of these kernel sources"}
    return roof, issue


# ---------------------------------------------------------------------------
# baselines on bounded samples
# ---------------------------------------------------------------------------

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


def plain_streams(q, inst, prm_kw, walks, dev, nstreams=32, walk_base=0):
    """The one-walk-per-launch form with its launches spread over `nstreams`
    streams, so that walks run on many SMs at once: (evals/s, device ms).
    Launch k runs walk walk_base + k and writes row k of the outputs."""
    import torch
    n = inst.n
    outs = inst.device_outputs(walks, device=dev)
    streams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)]
    prms = [q.make_params(1, walk_base=walk_base + k, **prm_kw) for k in range(walks)]
    rows = [{key: t[k:k + 1] for key, t in outs.items()} for k in range(walks)]
    main = torch.cuda.current_stream(dev)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rep in range(2):  # a warm-up pass, then the timed one
        torch.cuda.synchronize(dev)
        start.record(main)
        for st in streams:
            st.wait_event(start)
        for k in range(walks):
            inst.search_async(prms[k], rows[k], stream=streams[k % nstreams])
        for st in streams:
            ev = torch.cuda.Event()
            ev.record(st)
            main.wait_event(ev)
        stop.record(main)
        torch.cuda.synchronize(dev)
    ms = start.elapsed_time(stop)
    moves = float(outs["iters_done"].sum().item() + outs["descent_moves"].sum().item())
    return moves * n * (n - 1) / 2 / (ms / 1e3), ms


def sampled_oracle(F, D, walks, **kw):
    """The oracle (O(1)-update mode, all host cores) on a bounded sample:
    (evals/s, wall seconds, threads used)."""
    import oracle
    oracle.build()
    n = F.shape[0]
    t0 = time.perf_counter()
    o = oracle.run_walks(F, D, walks, **kw)
    dt = time.perf_counter() - t0
    moves = float(o["iters_done"].sum() + o["descent_moves"].sum())
    return moves * n * (n - 1) / 2 / dt, dt, min(oracle.num_threads(), walks)


def image_bytes(n, flow_bytes, dist_bytes, sym_flow):
    """Bytes of one instance's device images that the library uploads: F
    (and F^T when asymmetric) with rows padded to an odd number of 16-byte
    chunks, and D."""
    per = 16 // flow_bytes
    ldF = per * (((n * flow_bytes + 15) // 16) | 1)
    return n * ldF * flow_bytes * (1 if sym_flow else 2) + n * n * dist_bytes


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def measure_asym50(args, q, stream, flush, dev, world, rank, khash, baselines=True):
    """n=50 asymmetric uniform, 256 tabu walks x 5000 iterations per rank in
    one persistent launch per step."""
    from paper_2307_11248_gb300 import instances
    w = instances.workload_asym50()
    n = w["F"].shape[0]
    T = n * (n - 1) // 2
    W = args.walks or w["walks"]
    iters = args.iters or w["iters"]
    inst = q.Instance(w["F"], w["D"])
    prm = q.make_params(W, seed=w["seed"], iters=iters, tenure=w["tenure"], aspiration=True,
                        walk_base=replica_walk_base(rank, W),
                        threads_per_walk=args.threads_per_walk, phase_x=phase_x_of(q, args))
    plan = inst.plan(prm)
    outs = inst.device_outputs(W, device=dev)
    step = lambda: inst.search_async(prm, outs, stream=stream)  # noqa: E731
    import torch
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    ms, clk = timed_steps(step, args.steps, stream, flush, dev)
    total_ms = sum(ms)
    iters_done = float(outs["iters_done"].sum().item())
    max_ms, evals_all = combine_ranks(total_ms, iters_done * T * args.steps, dev)
    value = evals_all / (max_ms / 1e3)
    info = inst.info
    sym = bool(info["sym_flow"] and info["sym_dist"])
    bpu = unit_bytes(n, info["delta_bytes"], info["flow_bytes"], info["dist_bytes"], sym)
    sm_mhz = clk["sm_max_mhz"] or 2070.0
    roof, issue = rooflines(bpu * iters_done, iters_done, float(np.mean(ms)) / 1e3, plan["sms"],
                            sm_mhz, profile_figures("walk_kernel_asym50", khash),
                            f"walk_kernel (int32 deltas, int{8 * info['flow_bytes']} flows, "
                            f"{plan['threads_per_walk']} x {plan['pairs_per_thread']}, "
                            f"products {plan['products']})")
    roof["bytes_per_unit"] = bpu
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": total_ms / args.steps,
        "steps": args.steps, "warmup": args.warmup,
        "dtype": "int32" if info["delta_bytes"] == 4 else "int64",
        "config": {"workload": f"asym50: tabu n=50 asym uniform[0,99], {W} walks x {iters} iters",
                   "n": n, "walks_per_gpu": W, "iters": iters, "tenure": list(w["tenure"]),
                   "aspiration": True, "launch": "persistent, one launch per step",
                   "phase_x": args.phase_x, "products": int(plan["products"]),
                   "threads_per_walk": plan["threads_per_walk"],
                   "pairs_per_thread": plan["pairs_per_thread"], "grid": plan["grid"],
                   "l2": "flushed between timed steps (256 MiB write); working set on chip"},
        "tabu_iters_per_s": value / T, "roofline": roof, "issue": issue,
        "gpu_launches": args.steps, "clocks": clock_fields(clk),
    }
    if baselines and rank == 0 and not args.no_plain:
        # plain form: one launch per walk (same kernel body), one step
        pprm = q.make_params(W, seed=w["seed"], iters=iters, tenure=w["tenure"],
                             aspiration=True, walk_base=replica_walk_base(rank, W),
                             launch=q.LAUNCH_PLAIN, threads_per_walk=args.threads_per_walk,
                             phase_x=phase_x_of(q, args))
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
        pv = float(pouts["iters_done"].sum().item()) * T / (pms / 1e3)
        line["plain"] = {"value": pv, "unit": UNIT, "ms_per_step": pms, "launches_per_step": W,
                         "results_identical": same, "form": "one launch per walk, one stream"}
        line["batched_over_plain"] = value / world / pv
        ps, pms = plain_streams(q, inst, dict(seed=w["seed"], iters=iters, tenure=w["tenure"],
                                              aspiration=True), W, dev,
                                walk_base=replica_walk_base(rank, W))
        line["plain_streams"] = {"value": ps, "unit": UNIT, "ms_per_step": pms,
                                 "launches_per_step": W,
                                 "form": "one launch per walk, launches over 32 streams"}
        line["batched_over_plain_streams"] = value / world / ps
    if baselines and rank == 0:
        # end to end through the blocking C-ABI call with host buffers
        e2e_times = []
        for k in range(3):
            t0 = time.perf_counter()
            h = q.qap_create(w["F"], w["D"])
            res = q.qap_search(h, prm, n=n)
            q.qap_destroy(h)
            if k > 0:
                e2e_times.append(time.perf_counter() - t0)
        line["e2e"] = {"value": float(res["iters_done"].sum()) * T / float(np.mean(e2e_times)),
                       "unit": UNIT,
                       "h2d_bytes_per_step": image_bytes(n, info["flow_bytes"], info["dist_bytes"],
                                                         info["sym_flow"]),
                       "d2h_bytes_per_step": sum(v.nbytes for v in res.values()),
                       "call": "qap_create + qap_search (host outputs) + qap_destroy"}
        if not args.no_cpu and world == 1:
            cw = min(args.cpu_walks, W)
            v, dt, cores = sampled_oracle(w["F"], w["D"], cw, seed=w["seed"], iters=iters,
                                          tenure=w["tenure"], aspiration=True)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"{cw} of {W} walks x {iters} iterations, "
                                              f"{dt:.1f} s wall"}
    inst.close()
    return line


def measure_grid100(args, q, stream, flush, dev, world, rank, khash, baselines=True):
    """n=100 grid, 1024 walks x (2opt + 10^4 tabu iterations) per rank in one
    persistent launch, replayed as one CUDA graph per step."""
    import torch
    from paper_2307_11248_gb300 import instances
    w = instances.workload_grid100()
    n = w["F"].shape[0]
    T = n * (n - 1) // 2
    W = args.walks or w["walks"]
    iters = args.iters or w["iters"]
    inst = q.Instance(w["F"], w["D"])
    prm = q.make_params(W, seed=w["seed"], iters=iters, tenure=w["tenure"], descend=True,
                        walk_base=replica_walk_base(rank, W), phase_x=phase_x_of(q, args))
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
    max_ms, evals_all = combine_ranks(sum(ms), moves * T * args.steps, dev)
    value = evals_all / (max_ms / 1e3)
    plan = inst.plan(prm)
    info = inst.info
    sym = bool(info["sym_flow"] and info["sym_dist"])
    bpu = unit_bytes(n, info["delta_bytes"], info["flow_bytes"], info["dist_bytes"], sym)
    sm_mhz = clk["sm_max_mhz"] or 2070.0
    roof, issue = rooflines(bpu * moves, moves, float(np.mean(ms)) / 1e3, plan["sms"], sm_mhz,
                            profile_figures("walk_kernel_grid100", khash),
                            f"walk_kernel (int32 deltas, int{8 * info['flow_bytes']} flows, "
                            f"{plan['threads_per_walk']} x {plan['pairs_per_thread']})")
    roof["bytes_per_unit"] = bpu
    roof["unit_def"] = "one 2opt move or tabu iteration of one walk"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": sum(ms) / args.steps,
        "steps": args.steps, "warmup": args.warmup,
        "dtype": "int32" if info["delta_bytes"] == 4 else "int64",
        "tabu_iters_per_s": float(outs["iters_done"].sum().item()) * world /
        (max_ms / 1e3 / args.steps),
        "config": {"workload": f"grid100: 2opt then tabu, n=100 grid, {W} walks x {iters} iters",
                   "launch": "persistent, replayed as one CUDA graph", "phase_x": args.phase_x,
                   "threads_per_walk": plan["threads_per_walk"],
                   "pairs_per_thread": plan["pairs_per_thread"], "grid": plan["grid"],
                   "ctas_per_sm": plan["ctas_per_sm"], "products": int(plan["products"]),
                   "evals": "2opt moves and tabu iterations, n(n-1)/2 each",
                   "l2": "flushed between timed steps"},
        "roofline": roof, "issue": issue, "gpu_launches": args.steps, "clocks": clock_fields(clk),
    }
    if baselines and rank == 0:
        kw = dict(seed=w["seed"], iters=iters, tenure=w["tenure"], descend=True)
        if not args.no_plain:
            pv = sampled_plain(q, inst, kw, 16, stream, dev)
            line["plain"] = {"value": pv, "unit": UNIT, "sample": f"16 walks x (2opt + {iters} "
                             "iterations), one launch per walk"}
            line["batched_over_plain"] = value / world / pv
        if not args.no_cpu and world == 1:
            cpu, cpu_s, cores = sampled_oracle(w["F"], w["D"], 32, seed=w["seed"], iters=1000,
                                               tenure=w["tenure"], descend=True)
            line["cpu_baseline"] = {"value": cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                                    "sample": f"32 walks x (2opt + 1000 iterations), "
                                              f"{cpu_s:.1f} s wall"}
    inst.close()
    return line


def batch512_sample(insts, every=64):
    return insts[::every]


def measure_batch512(args, q, stream, flush, dev, world, rank, khash, baselines=True):
    """512 lognormal instances (n in [20, 150], int64 deltas), 64 walks x
    5000 tabu iterations each per rank: one persistent launch per size class
    (the autotuner's plans), classes concurrent on forked streams."""
    import torch
    from paper_2307_11248_gb300 import instances
    w = instances.workload_batch512()
    insts = w["instances"]
    W = args.walks or w["walks"]
    iters = args.iters or w["iters"]
    Fs, Ds = [i.F for i in insts], [i.D for i in insts]
    b = q.Batch(Fs, Ds, force_int64=True)
    tenure = (90, 110, 200)  # [0.9n, 1.1n] every 2n, per instance
    prm = q.make_params(W, seed=w["seed"], iters=iters, tenure=tenure, tenure_per_n=True,
                        walk_base=replica_walk_base(rank, W), phase_x=phase_x_of(q, args))
    t0 = time.perf_counter()
    tune = [] if args.no_tune else b.autotune(prm, trial_iters=max(50, iters // 20))
    tune_s = time.perf_counter() - t0
    outs = b.device_outputs(W, device=dev)
    step = lambda: b.search_async(prm, outs, stream=stream)  # noqa: E731
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    classes, inst_class = b.classes(prm)
    nc = len(classes)
    class_ms = np.zeros(nc)
    b.set_timing(True)

    def read_classes(k):
        cl, _ = b.classes(prm)
        for i, c in enumerate(cl):
            class_ms[i] += c["last_ms"]

    ms, clk = timed_steps(step, args.steps, stream, flush, dev, after_step=read_classes)
    b.set_timing(False)
    class_ms /= args.steps
    it = outs["iters_done"].cpu().numpy().reshape(len(insts), W).astype(np.float64)
    ns = np.array([i.n for i in insts])
    evals_rank = float(sum(it[i].sum() * ns[i] * (ns[i] - 1) / 2 for i in range(len(insts))))
    max_ms, evals_all = combine_ranks(sum(ms), evals_rank * args.steps, dev)
    value = evals_all / (max_ms / 1e3)
    step_s = float(np.mean(ms)) / 1e3
    # algorithmic bytes per step, per class and in total
    syms = [bool((i.F == i.F.T).all() and (i.D == i.D.T).all()) for i in insts]
    cls_bytes = np.zeros(nc)
    cls_units = np.zeros(nc)
    for i, inst in enumerate(insts):
        c = classes[inst_class[i]]
        bpu = unit_bytes(inst.n, c["delta_bytes"], c["flow_bytes"], c["dist_bytes"], syms[i])
        cls_bytes[inst_class[i]] += bpu * it[i].sum()
        cls_units[inst_class[i]] += it[i].sum()
    sms = b.plan(prm)["sms"]
    sm_mhz = clk["sm_max_mhz"] or 2070.0
    figs = profile_figures("batch_kernel_batch512", khash)
    roof, issue = rooflines(float(cls_bytes.sum()), float(cls_units.sum()), step_s, sms, sm_mhz,
                            figs, f"batch_kernel: {nc} class launches per step, concurrent")
    roof["bytes_per_unit"] = "T(2w+2) + (1 sym | 2 asym) n^2 (eF + eP) per instance, " \
                             "w = 8, eF = 2, eP = 1"
    peak = roof["peak"]
    dom = int(np.argmax(class_ms))

    def class_entry(i):
        c = classes[i]
        ach = cls_bytes[i] / (class_ms[i] / 1e3) / 1e9 if class_ms[i] > 0 else None
        return {"n": [c["nmin"], c["nmax"]], "instances": c["instances"], "walks": c["walks"],
                "plan": [c["threads_per_walk"], c["pairs_per_thread"]],
                "products": int(c["products"]), "workspace": bool(c["workspace"]),
                "grid": c["grid"], "ctas_per_sm": c["ctas_per_sm"],
                "kernel_ms": round(float(class_ms[i]), 3),
                "share_of_step": round(float(class_ms[i]) / (step_s * 1e3), 4),
                "bytes": float(cls_bytes[i]), "achieved_gbs": ach,
                "frac": (ach / peak) if ach else None}

    roof["classes"] = [class_entry(i) for i in range(nc)]
    roof["dominant_class"] = class_entry(dom)
    roof["dominant_class"]["note"] = ("the class kernel with the longest launch, timed by CUDA "
                                      "events on the stream it runs on; classes overlap, so "
                                      "shares add up to more than 1 and a launch's time "
                                      "includes waiting for SMs the other classes hold")
    heavy = int(np.argmax(cls_bytes))
    roof["heaviest_class"] = class_entry(heavy)
    roof["heaviest_class"]["note"] = "the class with the most algorithmic bytes per step"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": sum(ms) / args.steps,
        "steps": args.steps, "warmup": args.warmup, "dtype": "int64",
        "tabu_iters_per_s": float(it.sum()) * world / (max_ms / 1e3 / args.steps),
        "config": {"workload": f"batch512: {len(insts)} lognormal QAP instances, n in [20,150], "
                               f"half symmetric, {W} tabu walks x {iters} iters each, int64",
                   "launch": "one persistent launch per size class, classes concurrent on "
                             "forked streams, device work queues, largest n first",
                   "classes": nc, "tenure": "[0.9n, 1.1n] redrawn every 2n",
                   "phase_x": args.phase_x,
                   "autotune_s": round(tune_s, 2),
                   "autotuned": [{"n": [r["nmin"], r["nmax"]],
                                  "plan": [r["threads_per_walk"], r["pairs_per_thread"]],
                                  "workspace": bool(r["workspace"]),
                                  "products": int(r["products"]),
                                  "trial_ms": round(r["trial_ms"], 3),
                                  "rule_ms": round(r["rule_ms"], 3)} for r in tune],
                   "l2": "flushed between timed steps (256 MiB write)"},
        "roofline": roof, "issue": issue, "gpu_launches": args.steps * nc,
        "clocks": clock_fields(clk),
    }
    if baselines and rank == 0:
        sample = batch512_sample(insts)
        if not args.no_plain:
            pl_e = pl_t = 0.0
            for inst_ in sample:
                with q.Instance(inst_.F, inst_.D, force_int64=True) as one:
                    tn = instances.periodic_tenure(inst_.n)
                    e = sampled_plain(q, one, dict(seed=w["seed"], iters=iters, tenure=tn), 4,
                                      stream, dev)
                    ev = 4 * iters * inst_.n * (inst_.n - 1) / 2
                    pl_e += ev
                    pl_t += ev / e
            line["plain"] = {"value": pl_e / pl_t, "unit": UNIT,
                             "sample": f"4 walks x {iters} iterations of every 64th instance, "
                                       "one launch per walk, one stream"}
            line["batched_over_plain"] = value / world / line["plain"]["value"]
            ps_e = ps_t = 0.0
            for inst_ in sample:
                with q.Instance(inst_.F, inst_.D, force_int64=True) as one:
                    tn = instances.periodic_tenure(inst_.n)
                    e, ms_ = plain_streams(q, one, dict(seed=w["seed"], iters=iters, tenure=tn),
                                           W, dev)
                    ps_e += e * ms_ / 1e3
                    ps_t += ms_ / 1e3
            line["plain_streams"] = {"value": ps_e / ps_t, "unit": UNIT,
                                     "sample": f"all {W} walks of every 64th instance, one "
                                               "instance at a time, one launch per walk over "
                                               "32 streams"}
            line["batched_over_plain_streams"] = value / world / line["plain_streams"]["value"]
        # end to end: qap_batch_create + qap_batch_search (host outputs) +
        # qap_batch_destroy per step, the rule's plans (no autotuning)
        e2e_t, res = [], None
        for k in range(3):
            t0 = time.perf_counter()
            bb = q.Batch(Fs, Ds, force_int64=True)
            res = bb.search(prm)
            bb.close()
            if k > 0:
                e2e_t.append(time.perf_counter() - t0)
        it2 = res["iters_done"].reshape(len(insts), W).astype(np.float64)
        e2e_evals = float(sum(it2[i].sum() * ns[i] * (ns[i] - 1) / 2 for i in range(len(insts))))
        fb = classes[0]["flow_bytes"]
        db = classes[0]["dist_bytes"]
        line["e2e"] = {"value": e2e_evals / float(np.mean(e2e_t)), "unit": UNIT,
                       "h2d_bytes_per_step": int(sum(image_bytes(i.n, fb, db,
                                                                 bool((i.F == i.F.T).all()))
                                                     for i in insts)),
                       "d2h_bytes_per_step": int(sum(v.nbytes for v in res.values())),
                       "call": "qap_batch_create + qap_batch_search (host outputs) + "
                               "qap_batch_destroy, the rule's plans"}
        if not args.no_cpu and world == 1:
            cpu_e = cpu_t = 0.0
            cores = 0
            for inst_ in sample:
                v, dt, cores = sampled_oracle(inst_.F, inst_.D, 16, seed=w["seed"], iters=iters,
                                              tenure=instances.periodic_tenure(inst_.n))
                cpu_e += v * dt
                cpu_t += dt
            line["cpu_baseline"] = {"value": cpu_e / cpu_t, "unit": UNIT, "cores": cores,
                                    "kind": "oracle",
                                    "sample": f"16 walks x {iters} iterations of every 64th "
                                              f"instance ({len(sample)}), {cpu_t:.1f} s wall"}
    b.close()
    return line


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    """The oracle (the paper's method in plain C, O(1)-update mode, OpenMP
    over walks), timed on the host cores by rank 0 alone, each step a bounded
    sample of the same workload as this bench's own line."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle
    from paper_2307_11248_gb300 import instances
    oracle.build()
    threads = oracle.num_threads()
    wl = args.workload
    if wl == "asym50":
        w = instances.workload_asym50()
        n = w["F"].shape[0]
        walks = args.ref_walks

        def one(k, warm):
            return sampled_oracle(w["F"], w["D"], walks, seed=w["seed"],
                                  iters=200 if warm else w["iters"], tenure=w["tenure"],
                                  aspiration=True, walk_ids=np.arange(walks) + (k * walks) % 256)
        sample = f"{walks} of {w['walks']} walks x {w['iters']} iterations per step"
        cfg = f"asym50: tabu n=50 asym uniform[0,99], {w['walks']} walks x {w['iters']} iters"
    elif wl == "grid100":
        w = instances.workload_grid100()

        def one(k, warm):
            return sampled_oracle(w["F"], w["D"], 16, seed=w["seed"],
                                  iters=100 if warm else 1000, tenure=w["tenure"], descend=True,
                                  walk_ids=np.arange(16) + 16 * k)
        sample = "16 walks x (2opt + 1000 iterations) per step"
        cfg = f"grid100: 2opt then tabu, n=100 grid, {w['walks']} walks x {w['iters']} iters"
    else:
        w = instances.workload_batch512()
        insts = batch512_sample(w["instances"], 16)  # 32 instances, 4 per step in turn

        def one(k, warm):
            e = t = 0.0
            for j in range(4):
                inst = insts[(4 * k + j) % len(insts)]
                v, dt, _ = sampled_oracle(inst.F, inst.D, 16, seed=w["seed"],
                                          iters=100 if warm else 1000,
                                          tenure=instances.periodic_tenure(inst.n))
                e += v * dt
                t += dt
            return e / t, t, threads
        sample = ("4 instances (of every 16th, in turn) x 16 walks x 1000 iterations per step")
        cfg = (f"batch512: {len(w['instances'])} lognormal QAP instances, n in [20,150], half "
               f"symmetric, {w['walks']} tabu walks x {w['iters']} iters each, int64")
    for k in range(args.warmup):
        one(k, True)
    evals = total = 0.0
    for k in range(args.steps):
        v, dt, _ = one(k, False)
        evals += v * dt
        total += dt
    value = evals / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": cfg, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# main
# ---------------------------------------------------------------------------

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
    ap.add_argument("--no-nested", action="store_true",
                    help="batch512 only: skip the nested asym50 and grid100 lines")
    ap.add_argument("--no-tune", action="store_true",
                    help="batch512: the rule's plans, without the autotuner (profiling)")
    ap.add_argument("--threads-per-walk", type=int, default=0)
    ap.add_argument("--phase-x", choices=["auto", "dots"], default="auto",
                    help="phase X from maintained products where they apply (auto) or by "
                         "dot products")
    ap.add_argument("--iters", type=int, default=0,
                    help="override the iteration count (smaller cases for profiling)")
    ap.add_argument("--walks", type=int, default=0, help="override the walk count")
    ap.add_argument("--workload", choices=["batch512", "asym50", "grid100", "sym12", "serve",
                                           "sweep"],
                    default="batch512",
                    help="batch512 is the benchmark line (with asym50 and grid100 nested); "
                         "the others measure one workload each")
    ap.add_argument("--requests", type=int, default=600, help="serve: requests per run")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        # rank 0 alone times the oracle on the host cores; no process group
        run_reference(args)
        return
    if args.workload in ("sym12", "serve", "sweep"):
        return other_workloads(args)

    world, rank, local = dist_setup()
    import copy
    import torch
    import paper_2307_11248_gb300 as q
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    khash = kernel_source_hash()
    measure = {"batch512": measure_batch512, "asym50": measure_asym50,
               "grid100": measure_grid100}[args.workload]
    line = measure(args, q, stream, flush, dev, world, rank, khash)
    if args.workload == "batch512" and not args.no_nested:
        nested_args = copy.copy(args)
        nested_args.walks = nested_args.iters = 0
        line["workloads"] = {
            "asym50": measure_asym50(nested_args, q, stream, flush, dev, world, rank, khash),
            "grid100": measure_grid100(nested_args, q, stream, flush, dev, world, rank, khash),
        }
    line.update(n_gpus=world, higher_is_better=True, scaling="weak", vs_baseline=None,
                data="synthetic", kernel_sources=khash)
    line["config"]["parallelism"] = f"replicas x{world}"
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def other_workloads(args):
    """The latency case, the sweeps and the serving loop (N = 1)."""
    import torch
    import paper_2307_11248_gb300 as q
    from paper_2307_11248_gb300 import instances
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    line = {"unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic"}
    if args.workload == "sym12":
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
    [12, 256], through the serving loop: capacity as a closed loop with K
    requests outstanding, then p50/p99 latency at the offered 2000 req/s and
    at 0.8x the measured capacity, with the requests' kernel intervals on
    the device clock showing how many ran at once."""
    count = args.requests
    reqs = instances.poisson_requests(count, seed=4, rate_per_s=2000.0)
    prms = [q.make_params(32, seed=r.rid, iters=2000, tenure=instances.periodic_tenure(r.inst.n))
            for r in reqs]
    warm = instances.poisson_requests(20, seed=99)
    slots = 64

    def summary(lat, kt, wall):
        lat = np.array(lat)
        ks = np.array([t["kernel_start_us"] for t in kt])
        ke = np.array([t["kernel_end_us"] for t in kt])
        span = float(ke.max() - ks.min())
        ev = sorted([(a, 1) for a in ks] + [(b, -1) for b in ke])
        depth = peak = 0
        for _, d in ev:
            depth += d
            peak = max(peak, depth)
        return {"solves_per_s": count / wall, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "wall_s": wall,
                "kernels_mean_concurrent": float((ke - ks).sum() / span),
                "kernels_peak_concurrent": peak}

    def open_loop(rate, sv):
        t0 = time.perf_counter()
        tickets = []
        for r, p in zip(reqs, prms):
            due = t0 + r.arrival_s * 2000.0 / rate
            now = time.perf_counter()
            if due > now:
                time.sleep(due - now)
            tickets.append(sv.submit(r.inst.F, r.inst.D, p))
        lat, kt = [], []
        for t in tickets:
            _, tm = sv.wait(t, timeout_ms=600000)
            lat.append(tm["total_us"] / 1e3)
            kt.append(tm)
        return summary(lat, kt, time.perf_counter() - t0)

    def closed_loop(k, sv):
        """k requests outstanding: a new one is submitted as each finishes."""
        t0 = time.perf_counter()
        pending = []
        lat, kt = [], []
        it = iter(zip(reqs, prms))
        for r, p in it:
            pending.append(sv.submit(r.inst.F, r.inst.D, p))
            if len(pending) == k:
                break
        while pending:
            _, tm = sv.wait(pending.pop(0), timeout_ms=600000)
            lat.append(tm["total_us"] / 1e3)
            kt.append(tm)
            nxt = next(it, None)
            if nxt is not None:
                pending.append(sv.submit(nxt[0].inst.F, nxt[0].inst.D, nxt[1]))
        return summary(lat, kt, time.perf_counter() - t0)

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
    with q.Server(slots=slots, mem_bytes=2 << 30) as sv:
        for r in warm:
            sv.wait(sv.submit(r.inst.F, r.inst.D, q.make_params(
                32, seed=r.rid, iters=200, tenure=instances.periodic_tenure(r.inst.n))))
        closed_loop(slots, sv)                    # warms every code path and plan
        capacity = closed_loop(2 * slots, sv)     # K = 2 x slots outstanding
        offered = open_loop(2000.0, sv)           # the offered Poisson rate
        rate80 = 0.8 * capacity["solves_per_s"]
        at80 = open_loop(rate80, sv)
        stats = sv.stats()
    evals = sum(32 * 2000 * r.inst.n * (r.inst.n - 1) / 2 for r in reqs)
    return {"metric": "solves/s (serving, 32-walk x 2000-iteration tabu requests)",
            "value": offered["solves_per_s"], "unit": "solves/s", "steps": 1, "warmup": 1,
            "ms_per_step": offered["wall_s"] * 1e3, "dtype": "int32",
            "p50_ms": offered["p50_ms"], "p99_ms": offered["p99_ms"],
            "offered": offered,
            "overloaded": offered["solves_per_s"] < 0.95 * 2000.0,
            "capacity": {"solves_per_s": capacity["solves_per_s"], "outstanding": 2 * slots,
                         **{k: v for k, v in capacity.items() if k != "solves_per_s"}},
            "at_0.8_capacity": {"rate": rate80, **at80},
            "swap_evals_per_s_at_capacity": evals / capacity["wall_s"],
            "peak_in_flight": stats["peak_in_flight"],
            "sequential": {"solves_per_s": sequential,
                           "sample": "first 60 requests one at a time through qap_search"},
            "plain": {"solves_per_s": plain,
                      "sample": "first 6 requests, one launch per walk, one at a time"},
            "capacity_over_sequential": capacity["solves_per_s"] / sequential,
            "capacity_over_plain": capacity["solves_per_s"] / plain,
            "config": {"workload": f"{count} Poisson requests (2000/s offered), n in [12,256], "
                                   "generators sym uniform / asym uniform / grid",
                       "server": f"{slots} slots, 2 GiB arena, FIFO admission by slot and "
                                 "memory, images built at submit into a pinned slab"},
            "gpu_launches": 4 * count}


if __name__ == "__main__":
    main()
