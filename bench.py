#!/usr/bin/env python
"""Benchmark of the batched EC layout-decomposition search on one GB300.

One step = the whole search path over one synthetic layout (unit-disk
conflict graph, 200,000 polygons, mean degree 3, stitch p = 0.2, k = 3,
seed 2): every connected sub-graph left after simplification is searched by
the persistent batched kernel (one launch, device work queue, replayed from a
CUDA graph).  ``value`` = segments searched per second of kernel time, with
the EC matrices already resident in HBM: the segments inside the search
instances, not the ones simplification removed before the search (those are
recovered on the host afterwards and counted in ``e2e``).  ``e2e`` = all
segments of the layout per second through the C ABI from host graph arrays
to host masks (build + upload + search + copy back + recovery + counts), for
K layouts submitted together to the serving API so that the host work of one
overlaps the search of another (``e2e.serial``: one layout at a time through
mpld_build_matrix and mpld_solve_batch).  ``cpu_baseline`` is the oracle's
search phase on the same instances, same metric; its whole decomposition is
reported beside it.  Every search instance has the same node budget on the
GPU and in the CPU oracle, so both compute the same answer.

Also in the line: ``serving`` (Poisson streams of whole layouts at 10, 100
and 1000 requests/s through the server, p50 / p99 latency) and ``configs``
(the other workloads: 24-segment instance searched exactly, the 506-segment
single instance, the k = 4 layout), each with its oracle time and whether
the GPU result matches the oracle element by element.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank decomposes its own layout (seed + 1000 *
rank): the units are independent, no data-path collective; the max over
ranks of the timed region is used (weak scaling).
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

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

METRIC = "EC search nodes/s & segments/s (batched vs plain GPU vs CPU DLX); p99 latency"

# DRAM bytes of one step (the budgeted split search's three launches: first
# searches, the lanes' subtrees, the warps' subtrees) from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum per launch) on the workload
# scaled down by 10 (23,960 segments: 439,296 + 256, 597,504 + 59,648 and
# 68,352 + 0 bytes), per segment; traffic grows with the instances, i.e. with
# the segments.  Valid only for the kernel source and search mode it was
# measured on.
TRAFFIC = {"k3_n200k_p02_batched": {"bytes_per_segment": (103680 + 0 + 5041920 + 1678080 + 1773568 +
                                                          498944 + 113664 + 1536) / 59953,
                                    "kernel_sha256_16": "a4d89a7b061515b5",
                                    "split_budget": True,
                                    "profile": "profiles/split_step_traffic_k3_n50k_budget64k.md"}}
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="k3_n200k_p02_batched")
    ap.add_argument("--budget", type=int, default=1 << 16)
    ap.add_argument("--time-limit-ms", type=int, default=0,
                    help="per-instance search time limit (0 = the library's 60 s)")
    ap.add_argument("--parallel-exact", action="store_true",
                    help="exact search (node budget 0) with the warps of a CTA splitting each "
                         "instance of 16+ segments (for single-instance workloads)")
    ap.add_argument("--sequential-budget", action="store_true",
                    help="spend each instance's node budget in one depth-first search instead "
                         "of the budgeted split search (a first search, then independent "
                         "subtree searches on every lane and warp)")
    ap.add_argument("--biconnected", action="store_true",
                    help="search the biconnected blocks of each sub-graph and join them at cut "
                         "segments")
    ap.add_argument("--clique-bound", action="store_true",
                    help="second bound mode: also count untouched edge-disjoint (k+1)-cliques")
    ap.add_argument("--column-rule", choices=["mrv", "bfs"], default="mrv",
                    help="column to branch on: fewest rows (mrv) or the paper's rule "
                         "(a single-row column, else breadth-first order)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--scale", type=int, default=1,
                    help="divide the workload's polygon count (same density and degree); "
                         "for small profiling cases")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving loop (10, 100 and 1000 requests/s)")
    ap.add_argument("--serve-seconds", type=float, nargs=3, default=[8.0, 4.0, 2.0],
                    help="arrival span of the 10, 100 and 1000 requests/s streams")
    ap.add_argument("--serve-budget", type=int, default=1 << 12)
    ap.add_argument("--serve-pool", type=int, default=24,
                    help="distinct pre-generated requests the Poisson streams cycle through")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the legs of the other workloads")
    ap.add_argument("--shard", choices=["layouts", "instances"], default="layouts",
                    help="several GPUs: every rank decomposes its own layout (weak scaling), or "
                         "one layout's instances are shared over the ranks, longest processing "
                         "time first, and their results gathered (strong scaling)")
    ap.add_argument("--plain-scale", type=int, default=20,
                    help="the plain one-launch-per-instance path runs on the same workload with "
                         "polygons / plain-scale (same density and degree)")
    args = ap.parse_args()
    if args.parallel_exact:
        args.budget = 0      # the split exact search is exact only
    args.split_budget = not (args.sequential_budget or args.parallel_exact or args.clique_bound)
    return args


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(HERE, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def workload_layout(name: str, rank: int, scale: int = 1):
    from paper_2303_14335_gb300 import shard, synth
    cfg = dict(synth.WORKLOADS[name])
    mode = cfg.pop("mode")
    cfg["seed"] = shard.rank_seed(cfg["seed"], rank)
    if scale > 1:
        cfg["n_poly"] = max(cfg["n_poly"] // scale, 100)
    return synth.unit_disk_layout(name=name, **cfg), mode


def split_launches(mpld, prob, k, sizes=None):
    """Kernel launches of one budgeted split search step over a problem: the
    warps' first searches of the instances beyond the per-lane form and the
    lane kernel's first searches of the others (each when there are some),
    then the lanes' and the warps' subtree launches."""
    import numpy as np
    sizes = np.asarray(mpld.mpld_instance_sizes(prob) if sizes is None else sizes)
    if len(sizes) == 0:
        return 0
    n_lane = int(np.sum(sizes <= 64)) if k <= 4 else 0
    return (1 if n_lane < len(sizes) else 0) + (1 if n_lane > 0 else 0) + 2


def run_serving(args, mpld, synth):
    """Poisson streams of whole layouts through the server (continuous batching).

    Requests: 1k-200k polygons (log-uniform), k in {3, 4}, stitch p = 0.2,
    mean degree U[3, 5], seeded per request; a pool of distinct requests is
    generated first and the stream cycles through it.  Latency = result in
    host memory minus the request's scheduled arrival time.
    """
    import numpy as np
    pool = [synth.serving_request(2023, i) for i in range(args.serve_pool)]
    pool_segments = [L.n_seg for L in pool]
    out = {"budget": args.serve_budget, "pool_requests": len(pool),
           "pool_mean_segments": float(np.mean(pool_segments)), "loads": []}
    for rate, duration in zip((10, 100, 1000), args.serve_seconds):
        n = int(rate * duration)
        arrivals = synth.poisson_arrivals(777 + rate, n, rate)
        cfg = mpld.mpld_server_config(arena_bytes=8 << 30, result_pool_bytes=1 << 30,
                                      max_in_flight=256, streams=16)
        srv = mpld.mpld_server_create(cfg, mpld.make_params(
            node_budget=args.serve_budget,
            flags=(mpld.MPLD_COLUMN_BFS if args.column_rule == "bfs" else 0) |
            (mpld.MPLD_SPLIT_BUDGET if args.split_budget else 0)))
        arrival_of, lat, segs = {}, [], 0
        t0 = time.perf_counter()
        i = 0
        deadline = duration * 6 + 60
        while len(lat) < n:
            now = time.perf_counter() - t0
            while i < n and arrivals[i] <= now:
                L = pool[i % len(pool)]
                t = mpld.mpld_server_submit(
                    srv, L, flags=(mpld.MPLD_BICONNECTED if args.biconnected else 0) |
                    (mpld.MPLD_CLIQUE_BOUND if args.clique_bound else 0))
                arrival_of[t] = (arrivals[i], L.n_seg)
                i += 1
            busy = False
            for t in mpld.mpld_server_poll(srv):
                rc, mask, res = mpld.mpld_server_result(srv, t)
                a, ns = arrival_of.pop(t)
                lat.append(time.perf_counter() - t0 - a)
                segs += ns
                busy = True
            if now > deadline:
                break
            if not busy and (i >= n or arrivals[i] > now + 0.0005):
                time.sleep(0.0002)
        wall = time.perf_counter() - t0
        st = mpld.mpld_server_stats_get(srv)
        srv.close()
        lat_ms = np.array(lat) * 1000.0
        achieved = len(lat) / wall
        # the Poisson stream's own rate over its span (the offered rate is its mean)
        arrival_rate = n / max(float(arrivals[-1]), 1e-9)
        out["loads"].append({
            "offered_req_per_s": rate, "arrival_req_per_s": arrival_rate,
            "requests": n, "completed": len(lat),
            "p50_ms": float(np.percentile(lat_ms, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat) else None,
            "mean_ms": float(lat_ms.mean()) if len(lat) else None,
            "achieved_req_per_s": achieved, "segments_per_s": segs / wall,
            "saturated": bool(achieved < 0.9 * arrival_rate),
            "max_concurrent_layouts": int(st.max_concurrent),
            "arena_peak_bytes": int(st.arena_peak_bytes)})
    return out


def oracle_flags(oracle, args, mode):
    flags = (oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE) if mode == "single" else 0
    if args.column_rule == "bfs":
        flags |= oracle.COLUMN_BFS
    if args.biconnected and mode != "single":
        flags |= oracle.BICONNECTED
    if args.clique_bound:
        flags |= oracle.CLIQUE_BOUND
    if args.split_budget:
        flags |= oracle.SPLIT_BUDGET
    return flags


def run_reference(args, rank, world):
    """The CPU oracle (Knuth dancing links on all host cores) on the same workload.

    value = segments inside the search instances per second of the oracle's
    search phase (the same metric as the GPU line's value); the whole
    decomposition (simplify, split, search, recover, count) is reported
    beside it."""
    if rank != 0:
        return
    import oracle
    layout, mode = workload_layout(args.workload, 0)
    flags = oracle_flags(oracle, args, mode)
    cores = os.cpu_count() or 1
    oracle.build()
    for _ in range(args.warmup):
        oracle.decompose(layout, flags=flags, budget=args.budget, nthreads=cores)
    search_s, whole_s = [], []
    res = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        res = oracle.decompose(layout, flags=flags, budget=args.budget, nthreads=cores)
        whole_s.append(time.perf_counter() - t0)
        search_s.append(res.search_seconds)
    total = sum(search_s)
    value = res.instance_segments * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "segments/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "segments": layout.n_seg, "k": layout.k,
                   "instance_segments": res.instance_segments,
                   "node_budget": args.budget, "column_rule": args.column_rule,
                   "biconnected": bool(args.biconnected and mode != "single"),
                   "clique_bound": bool(args.clique_bound)},
        "nodes_per_s": res.nodes * args.steps / total,
        "whole_decomposition": {"segments_per_s": layout.n_seg * args.steps / sum(whole_s),
                                "ms_per_step": 1000 * sum(whole_s) / args.steps,
                                "form": "simplify, split, search, recover, count"},
        "cpu_baseline": {"value": value, "unit": "segments/s", "cores": cores, "kind": "oracle",
                         "sample": f"search phase of the whole layout ({res.instance_segments} "
                                   f"instance segments, {res.n_components} instances) per step"},
        "e2e": {"value": value, "unit": "segments/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_leg(name, budget, search_flags, label, mpld, oracle, torch, stream, flush, cores,
               reps=3):
    """One other workload: batched search timed with CUDA events (median of
    ``reps`` after one warm-up, L2 flushed before each), then the oracle on
    the same layout and budget (one thread for single-instance workloads,
    every host core for layouts), compared element by element."""
    import numpy as np
    layout, mode = workload_layout(name, 0)
    s = stream.cuda_stream
    flags = (mpld.MPLD_NO_SIMPLIFY | mpld.MPLD_SINGLE_INSTANCE) if mode == "single" else 0
    prob = mpld.mpld_build_matrix(layout, mpld.make_params(flags=flags), s)
    try:
        info = mpld.mpld_problem_info(prob)
        prm = mpld.make_params(node_budget=budget, flags=search_flags)
        if mode != "single":
            mpld.mpld_autotune([prob], prm, s)
        mpld.mpld_search_batch_async([prob], prm, s)
        stream.synchronize()
        ms = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mpld.mpld_search_batch_async([prob], prm, s)
            e1.record(stream)
            stream.synchronize()
            ms.append(e0.elapsed_time(e1))
        rc, mask, res = mpld.mpld_fetch(prob, s)
    finally:
        prob.close()
    med = statistics.median(ms) / 1000.0
    oflags = (oracle.NO_SIMPLIFY | oracle.SINGLE_INSTANCE) if mode == "single" else 0
    if search_flags & mpld.MPLD_SPLIT_BUDGET:
        oflags |= oracle.SPLIT_BUDGET
    nthreads = 1 if mode == "single" else cores
    ref = oracle.decompose(layout, flags=oflags, budget=budget, nthreads=nthreads)
    split = bool(search_flags & mpld.MPLD_PARALLEL_EXACT)
    return {
        "workload": name, "search": label, "node_budget": budget, "segments": layout.n_seg,
        "instances": info.n_components, "max_instance": info.max_component,
        "instance_segments": info.instance_segments, "ms_per_step": 1000 * med,
        "step_ms": ms, "value": info.instance_segments / med, "unit": "segments/s",
        "nodes_per_s": res.nodes / med, "nodes": res.nodes, "cost": res.cost,
        "budget_instances": res.n_budget_components, "status": rc,
        "oracle": {"value": ref.instance_segments / ref.search_seconds, "unit": "segments/s",
                   "search_ms": 1000 * ref.search_seconds, "threads": nthreads,
                   "nodes_per_s": ref.nodes / ref.search_seconds, "nodes": ref.nodes},
        "gpu_over_oracle": ref.search_seconds / med,
        # split subtrees: node counts depend on timing, the answer does not
        "matches_gpu": bool(np.array_equal(ref.mask, mask) and ref.cost == res.cost and
                            (split or ref.nodes == res.nodes)),
    }


def run_shards(args, rank, world, local_rank):
    """One layout over all ranks: every rank builds the same problem, searches
    its longest-processing-time-first share of the instances (timed on the
    device, max over ranks), the per-instance results are all-gathered and
    every rank finishes (recovery and counts) from the merged results."""
    import numpy as np
    import torch

    from paper_2303_14335_gb300 import mpld, synth

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    layout, mode = synth.workload(args.workload)      # the same layout on every rank
    flags = (mpld.MPLD_NO_SIMPLIFY | mpld.MPLD_SINGLE_INSTANCE) if mode == "single" else 0
    sflags = (mpld.MPLD_COLUMN_BFS if args.column_rule == "bfs" else 0) | \
        (mpld.MPLD_SPLIT_BUDGET if args.split_budget else 0)
    prm = mpld.make_params(node_budget=args.budget, flags=sflags, time_limit_ms=args.time_limit_ms)
    prob = mpld.mpld_build_matrix(layout, mpld.make_params(flags=flags), s)
    info = mpld.mpld_problem_info(prob)
    owner = mpld.mpld_shard_instances(prob, world)
    mine = np.flatnonzero(owner == rank).astype(np.int32)
    sizes = mpld.mpld_instance_sizes(prob)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 1)):
        mpld.mpld_search_subset_async(prob, mine, prm, s)
        stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.2)
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        mpld.mpld_search_subset_async(prob, mine, prm, s)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_s = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    if dist:
        t = torch.tensor([total_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())

    def gather_and_finish():
        nd, co, stt, ms = mpld.mpld_fetch_instances(prob, s)
        part = (mine.tolist(), nd[mine].tolist(), co[mine].tolist(), stt[mine].tolist(),
                [ms[off[c]:off[c + 1]].tobytes() for c in mine])
        parts = [part]
        if dist:
            parts = [None] * world
            dist.all_gather_object(parts, part)
        C = len(sizes)
        nodes, cost = np.zeros(C, np.int64), np.zeros(C, np.int64)
        status, masks = -np.ones(C, np.int32), np.zeros(int(off[-1]), np.int8)
        for ids, nds, cos, sts, mss in parts:
            for c, a, b, st_, m in zip(ids, nds, cos, sts, mss):
                nodes[c], cost[c], status[c] = a, b, st_
                masks[off[c]:off[c + 1]] = np.frombuffer(m, dtype=np.int8)
        return mpld.mpld_finish_from(prob, nodes, cost, status, masks)

    rc, mask, res = gather_and_finish()
    # end to end: this rank's share searched, results gathered, finished
    e2e_t = []
    for i in range(args.warmup + args.steps):
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mpld.mpld_search_subset_async(prob, mine, prm, s)
        rc2, mask2, _ = gather_and_finish()
        if i >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
        assert np.array_equal(mask2, mask)
    e2e_s = sum(e2e_t)
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    matches = None
    if rank == 0:
        # the same layout searched whole on this GPU
        rc1, masks1, res1 = mpld.mpld_solve_batch([prob], prm, s)
        matches = bool(np.array_equal(masks1[0], mask) and res1[0].cost == res.cost and
                       res1[0].nodes == res.nodes)
    prob.close()
    if rank == 0:
        searched = float(info.instance_segments)
        out = {
            "metric": METRIC, "value": searched * args.steps / total_s, "unit": "segments/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total_s / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "segments": layout.n_seg,
                       "instance_segments": info.instance_segments, "k": layout.k,
                       "node_budget": args.budget, "split_budget": bool(args.split_budget),
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"one layout's instances shared over {world} GPUs "
                                      "(longest processing time first), results all-gathered"},
            "nodes_per_s": res.nodes * args.steps / total_s,
            "search": {"nodes": res.nodes, "cost": res.cost, "status": rc,
                       "instances_rank0": int(len(mine)), "instances": int(len(sizes))},
            "gpu_launches": args.steps * (split_launches(mpld, prob, layout.k, sizes[mine])
                                          if args.split_budget else 1),
            "clocks": clk,
            "e2e": {"value": layout.n_seg * len(e2e_t) / e2e_s, "unit": "segments/s",
                    "h2d_bytes_per_step": 4 * int(len(mine)),
                    "d2h_bytes_per_step": 32 * int(len(sizes)) + int(info.instance_segments) + 4,
                    "ms_per_step": 1000 * e2e_s / len(e2e_t),
                    "form": "share searched, per-instance results copied back, all-gathered, "
                            "recovery and counts on every rank"},
            "matches_one_gpu": matches,
        }
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.shard == "instances":
        run_shards(args, rank, world, local_rank)
        return

    import numpy as np
    import torch

    from paper_2303_14335_gb300 import mpld

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    layout, mode = workload_layout(args.workload, rank, scale=args.scale)
    flags = (mpld.MPLD_NO_SIMPLIFY | mpld.MPLD_SINGLE_INSTANCE) if mode == "single" else 0
    if args.biconnected and mode != "single":
        flags |= mpld.MPLD_BICONNECTED
    if args.clique_bound:
        flags |= mpld.MPLD_CLIQUE_BOUND
    prob = mpld.mpld_build_matrix(layout, mpld.make_params(flags=flags), s)
    info = mpld.mpld_problem_info(prob)
    rule_flag = mpld.MPLD_COLUMN_BFS if args.column_rule == "bfs" else 0
    if args.parallel_exact:
        rule_flag |= mpld.MPLD_PARALLEL_EXACT
    if args.split_budget:
        rule_flag |= mpld.MPLD_SPLIT_BUDGET
    prm = mpld.make_params(node_budget=args.budget, flags=rule_flag,
                           time_limit_ms=args.time_limit_ms)
    tune = None
    if not args.no_tune:
        tune = mpld.mpld_autotune([prob], prm, s)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    # warm-up
    for _ in range(max(args.warmup, 1)):
        mpld.mpld_search_batch_async([prob], prm, s)
        stream.synchronize()

    # timed: K steps, each bracketed by events on the launching stream, L2
    # flushed between steps (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.2)
    for i in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        mpld.mpld_search_batch_async([prob], prm, s)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1000.0
    if dist:
        from paper_2303_14335_gb300 import shard
        all_segments, _ = shard.aggregate(dist, layout.n_seg, total_s, "cuda")
        searched, total_s = shard.aggregate(dist, info.instance_segments, total_s, "cuda")
    else:
        all_segments = float(layout.n_seg)
        searched = float(info.instance_segments)
    rc, mask, res = mpld.mpld_fetch(prob, s)
    seq = None
    if args.split_budget and not args.no_plain:
        # the same budget spent by one depth-first search per instance, on the
        # same matrices (L2 flushed before each run)
        prm_seq = mpld.make_params(node_budget=args.budget, flags=rule_flag & ~mpld.MPLD_SPLIT_BUDGET)
        if not args.no_tune:
            mpld.mpld_autotune([prob], prm_seq, s)
        mpld.mpld_search_batch_async([prob], prm_seq, s)
        stream.synchronize()
        seq_ms = []
        for _ in range(3):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mpld.mpld_search_batch_async([prob], prm_seq, s)
            e1.record(stream)
            stream.synchronize()
            seq_ms.append(e0.elapsed_time(e1))
        _, _, sres = mpld.mpld_fetch(prob, s)
        med = statistics.median(seq_ms) / 1000.0
        seq = {"ms_per_step": 1000 * med, "value": info.instance_segments / med,
               "nodes_per_s": sres.nodes / med, "cost": sres.cost, "nodes": sres.nodes,
               "budget_instances": sres.n_budget_components,
               "form": "the same node budget spent by one depth-first search per instance"}
        # the split search's results again for what follows (e2e checks)
        mpld.mpld_search_batch_async([prob], prm, s)
        rc, mask, res = mpld.mpld_fetch(prob, s)
    inst_status = None
    if args.parallel_exact:
        # which instances the exact search finished, and the sizes of the ones
        # it did not (time limit)
        _, icost, istat, icomp = mpld.mpld_component_results(prob)
        isize = np.bincount(icomp[icomp >= 0], minlength=len(istat))
        late = np.flatnonzero(istat != mpld.MPLD_OK)
        inst_status = {"finished": int((istat == mpld.MPLD_OK).sum()), "timed_out": int(len(late)),
                       "timed_out_sizes": sorted(isize[late].tolist(), reverse=True)[:50]}
    # segments the timed kernel searched (simplification removed the rest on
    # the host before the search; they are recovered after it)
    value = searched * args.steps / total_s
    nodes_per_s = res.nodes * world * args.steps / total_s

    out = {
        "metric": METRIC, "value": value, "unit": "segments/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": args.workload + (f"/scale{args.scale}" if args.scale > 1 else ""),
                   "segments": layout.n_seg, "polygons": layout.n_poly,
                   "k": layout.k, "node_budget": args.budget, "column_rule": args.column_rule,
                   "biconnected": bool(flags & mpld.MPLD_BICONNECTED),
                   "clique_bound": bool(flags & mpld.MPLD_CLIQUE_BOUND),
                   "parallel_exact": bool(args.parallel_exact),
                   "split_budget": bool(args.split_budget),
                   "time_limit_ms": args.time_limit_ms or 60000,
                   "instances": info.n_components,
                   "instance_segments": info.instance_segments,
                   "max_instance": info.max_component,
                   "removed_segments": info.n_removed_segments,
                   "value_counts": "segments inside the search instances (removed segments "
                                   "are recovered on the host and counted in e2e only)",
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"weak: {world} independent layouts" if world > 1 else "1 GPU",
                   "launch": ({"warps_per_cta": tune.warps_per_cta, "slot_bytes": tune.slot_bytes,
                               "ctas_per_sm": tune.ctas_per_sm,
                               "spilled_instances": tune.n_instances_spilled}
                              if tune else "default")},
        "nodes_per_s": nodes_per_s,
        "search": {"nodes": res.nodes, "cost": res.cost, "conflicts": res.n_conflicts,
                   "stitches": res.n_stitches, "budget_instances": res.n_budget_components,
                   "status": rc, "step_ms": step_ms,
                   "median_step_ms": statistics.median(step_ms) if step_ms else None,
                   "instances_exact": inst_status},
        # launches per step: the split search's (see split_launches); the
        # exact split search's queue launch before the batched one when the
        # layout has several instances, one grid launch for a single instance
        "gpu_launches": args.steps * (split_launches(mpld, prob, layout.k) if args.split_budget else
                                      2 if (args.parallel_exact and info.n_components > 1) else 1),
        "sequential_budget": seq,
        "clocks": clk,
    }

    # roofline of the dominant kernel (the persistent search kernel): integer
    # ALU work per launch / launch duration vs the SMs' 32-bit integer issue
    # rate (64 ops per SM per clock; the probe below measures it)
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(local_rank)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak_gops = props.multi_processor_count * 64 * sm_mhz * 1e6 / 1e9
    achieved = res.work / (total_s / args.steps) / 1e9
    traffic = None
    tr = TRAFFIC.get(args.workload)
    if tr is not None and tr.get("split_budget", False) == bool(args.split_budget):
        import hashlib
        src = os.path.join(HERE, "paper_2303_14335_gb300", "csrc", "mpld_search.cu")
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == tr["kernel_sha256_16"]:
            traffic = tr["bytes_per_segment"] * layout.n_seg
    out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": alu_peak_gops,
                       "unit": "Gop/s", "frac": achieved / alu_peak_gops, "traffic": traffic,
                       "traffic_source": ("ncu capture of the step's four launches at 1/4 scale, "
                                          "scaled by segments" if traffic is not None else None),
                       "peak_source": f"{props.multi_processor_count} SMs x 64 int32 ops per clock x "
                                      f"{sm_mhz:.0f} MHz (max clock from MEASURED_PEAKS.json); "
                                      "derived, see int_pipes_measured",
                       "work_ops_per_launch": res.work,
                       "covers": ("the launches of a step (the warps' and the lanes' first "
                                  "searches, side by side; the lanes' subtree searches; the warps' "
                                  "subtree searches, started beside the lanes'), timed together"
                                  if args.split_budget else "the one launch of a step")}
    # the integer pipes' measured throughput for the same op mix (context for
    # the derived peak above)
    import ctypes
    pk = (ctypes.c_double * 2)()
    fn = mpld.probe_library().mpld_probe_int_peak
    if fn(1 << 14, pk) == 0:
        out["roofline"]["int_pipes_measured"] = {
            "logic_add_gops": pk[0], "logic_popc_add_gops": pk[1],
            "frac_of_logic_popc_add": achieved / pk[1],
            "source": "mpld_probe_int_peak (libmpld_probe.so): 8 independent chains per thread, 2,048 threads "
                      "per SM, every SM"}

    if not args.no_e2e:
        if dist:
            from paper_2303_14335_gb300 import shard
        # end to end through the C ABI: host arrays in, host masks out
        e2e_t = []
        for i in range(args.warmup + args.steps):
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p2 = mpld.mpld_build_matrix(layout, mpld.make_params(flags=flags), s)
            rc2, masks2, res2 = mpld.mpld_solve_batch([p2], prm, s)
            t1 = time.perf_counter()
            inf2 = mpld.mpld_problem_info(p2)
            p2.close()
            if i >= args.warmup:
                e2e_t.append(t1 - t0)
            assert np.array_equal(masks2[0], mask)
        e2e_total = sum(e2e_t)
        if dist:
            _, e2e_total = shard.aggregate(dist, layout.n_seg, e2e_total, "cuda")
        # bytes copied per step: read-only blocks + descriptors + order up;
        # instance results + instance masks + status word down
        h2d = inf2.arena_bytes + 80 * inf2.n_components + 4 * inf2.n_components
        d2h = 32 * inf2.n_components + inf2.instance_segments + 4
        serial = {"value": all_segments * len(e2e_t) / e2e_total,
                  "ms_per_step": 1000 * e2e_total / len(e2e_t),
                  "form": "one layout at a time: mpld_build_matrix then mpld_solve_batch"}

        # the same decompositions as a stream of K layouts through the
        # server: host build, upload, search, copy-back and recovery of
        # different layouts overlap (the form a user decomposing many
        # layouts takes); every layout is still built, uploaded, searched,
        # copied back and recovered inside the timed region
        req_flags = flags & (mpld.MPLD_NO_SIMPLIFY | mpld.MPLD_SINGLE_INSTANCE |
                             mpld.MPLD_BICONNECTED | mpld.MPLD_CLIQUE_BOUND)
        # the server's own launch shape (small CTAs, so that launches of
        # different layouts share the SMs)
        cfg = mpld.mpld_server_config(arena_bytes=8 << 30, result_pool_bytes=1 << 30,
                                      max_in_flight=max(args.steps, args.warmup, 1), streams=8)
        srv = mpld.mpld_server_create(cfg, prm)

        def stream_run(n):
            t0 = time.perf_counter()
            pending = {mpld.mpld_server_submit(srv, layout, flags=req_flags) for _ in range(n)}
            got = []
            while pending:
                done = mpld.mpld_server_poll(srv)
                for t in done:
                    got.append(mpld.mpld_server_result(srv, t))
                    pending.discard(t)
                if not done:
                    time.sleep(0.0002)
            return time.perf_counter() - t0, got

        stream_run(args.warmup)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_stream, got = stream_run(args.steps)
        srv.close()
        for rc3, m3, r3 in got:
            assert rc3 == rc and np.array_equal(m3, mask) and r3.cost == res.cost
        if dist:
            _, t_stream = shard.aggregate(dist, layout.n_seg, t_stream, "cuda")
        out["e2e"] = {"value": all_segments * args.steps / t_stream, "unit": "segments/s",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                      "ms_per_step": 1000 * t_stream / args.steps,
                      "gpu_launches_per_step": (split_launches(mpld, prob, layout.k)
                                                if args.split_budget else 1),
                      "form": f"{args.steps} layouts submitted together to the server API "
                              "(mpld_server_submit / poll / result)",
                      "serial": serial}

    if rank == 0 and not args.no_plain:
        # plain one-launch-per-instance path vs the batched one on a smaller
        # layout of the same workload (same density and degree)
        small, _ = workload_layout(args.workload, 0, scale=args.plain_scale)
        ps = mpld.mpld_build_matrix(small, mpld.make_params(flags=flags), s)
        pinfo = mpld.mpld_problem_info(ps)
        times = {}
        for name in ("plain", "batched"):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for rep in range(2):
                e0.record(stream)
                if name == "plain":
                    mpld.mpld_search_plain_async(ps, prm, s)
                else:
                    mpld.mpld_search_batch_async([ps], prm, s)
                e1.record(stream)
                stream.synchronize()
            times[name] = e0.elapsed_time(e1) / 1000.0
        ps.close()
        out["plain"] = {"segments": small.n_seg, "instances": pinfo.n_components,
                        "instance_segments": pinfo.instance_segments,
                        "plain_segments_per_s": pinfo.instance_segments / times["plain"],
                        "batched_segments_per_s": pinfo.instance_segments / times["batched"],
                        "batched_over_plain": times["plain"] / times["batched"],
                        "gpu_launches_plain": pinfo.n_components}

    if rank == 0 and not args.no_serve:
        from paper_2303_14335_gb300 import synth
        out["serving"] = run_serving(args, mpld, synth)

    cores = os.cpu_count() or 1
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        ref = oracle.decompose(layout, flags=oracle_flags(oracle, args, mode), budget=args.budget,
                               nthreads=cores)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {
            "value": ref.instance_segments / ref.search_seconds, "unit": "segments/s",
            "cores": cores, "kind": "oracle",
            "sample": f"search phase of the whole layout ({ref.instance_segments} instance "
                      f"segments, {ref.n_components} instances), one decomposition",
            "nodes_per_s": ref.nodes / ref.search_seconds,
            "search_ms": 1000 * ref.search_seconds,
            "whole_decomposition": {"segments_per_s": layout.n_seg / dt, "ms": 1000 * dt},
            # with split subtrees the node count depends on timing
            "matches_gpu": bool(np.array_equal(ref.mask, mask) and ref.cost == res.cost and
                                (args.parallel_exact or ref.nodes == res.nodes))}

    if rank == 0 and not args.no_configs:
        import oracle
        oracle.build()
        sb = mpld.MPLD_SPLIT_BUDGET if args.split_budget else 0
        mode = "budgeted split search" if args.split_budget else "one search per instance"
        legs = [("k3_n24_plain", 0, mpld.MPLD_PARALLEL_EXACT,
                 "exact, subtrees split over every warp of the grid"),
                ("k3_n400_p025_plain", args.budget, sb, f"one instance, node budget, {mode}"),
                ("k4_n100k_p03_batched", args.budget, sb, f"batched, node budget, {mode}")]
        out["configs"] = [config_leg(n, b, f, lab, mpld, oracle, torch, stream, flush, cores)
                          for n, b, f, lab in legs if n != args.workload]
    prob.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
