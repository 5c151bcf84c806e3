#!/usr/bin/env python3
"""CFR+ iteration throughput of the GB300 path (one JSON line on stdout).

A step is one full CFR+ iteration over the compiled game: forward reach of
both players, terminal values (chance folded at compile time), backward values
with the fused regret / regret-matching+ / linear-average update. The default
workload is the two-round card game (8 ranks x 4 suits, stack 2 antes, cap 3
bets per round: 264,306,001 nodes) in the FP32 mode with FP64 accumulators,
executed as per-level kernels replayed from one CUDA graph per iteration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large_card|random_tree|tiny]

Multi-GPU runs (torchrun, one rank per GPU) solve independent replicas of the
workload; value = all ranks' edges / the slowest rank's time ("weak").
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CFR iters/sec & edges/sec (HBM GB/s vs peak); batched time-to-1e-3 exploitability"
UNIT = "edges/s"
L2_BYTES = 129 * 1024 * 1024


def workloads(deal_stride: int = 1, stack: int = 2, cap: int = 3):
    import gamegen as gg

    return {
        "large_card": dict(
            make=lambda: gg.large_card_sampled(deal_stride, 8, 4, stack, cap),
            sample=lambda: (gg.large_card_sampled(200, 8, 4, 2, 3), "every 200th root deal of the same game"),
            desc="two-round card game: 8 ranks x 4 suits, two private cards, one public card, "
                 "bets {1/2 pot, pot, all-in}, cap 3 per round, stack 2 antes"),
        "random_tree": dict(
            make=lambda: gg.random_tree(0),
            sample=lambda: (gg.random_tree(0), "the full tree"),
            desc="seeded random perfect-recall tree, depth 14, branching U{2,3,4}, 20% chance, sets of 1-16"),
        "tiny": dict(
            make=lambda: gg.tiny_card(),
            sample=lambda: (gg.tiny_card(), "the full game"),
            desc="one-card poker, 5 ranks, cap 2 bets (301 nodes)"),
    }


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="large_card", choices=["large_card", "random_tree", "tiny", "serving", "warmstart"])
    p.add_argument("--train-games", type=int, default=10000, help="warmstart only: training solves")
    p.add_argument("--heldout", type=int, default=512, help="warmstart only: held-out games")
    p.add_argument("--alone-sample", type=int, default=128,
                   help="warmstart only: held-out games also solved one at a time, cold and warm")
    p.add_argument("--requests", type=int, default=512, help="serving only: number of endgame solves")
    p.add_argument("--max-iters", type=int, default=5000, help="serving only: iteration cap per solve")
    p.add_argument("--baseline-sample", type=int, default=48, help="serving only: solves timed one by one")
    p.add_argument("--batched-requests", type=int, default=128,
                   help="large_card: endgame solves of the batched-serving leg after the timed region (0: none)")
    p.add_argument("--batched-baseline", type=int, default=12,
                   help="large_card: of those, solves timed one by one for the batching speed-up")
    p.add_argument("--exec", dest="exec_form", default="graph", choices=["graph", "levels", "persistent", "auto"])
    p.add_argument("--reach-order", default="members", choices=["members", "bfs", "slots"],
                   help="layout of the internal nodes' reach (members: the forward pulls; bfs, slots: it pushes)")
    p.add_argument("--precision", default="p32", choices=["p32", "p64"])
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--deal-stride", type=int, default=1,
                   help="large_card only: keep every k-th root deal (a smaller instance for profiling)")
    p.add_argument("--stack", type=int, default=2, help="large_card only: stack behind the ante")
    p.add_argument("--cap", type=int, default=3, help="large_card only: bets per round")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-autotune", action="store_true", help="keep the lane counts picked from mean set sizes")
    p.add_argument("--lanes", type=int, default=0,
                   help="pin cfr_options.lanes_per_set (512: the streaming backward wherever it can run) and skip "
                        "the autotuner (for profiling runs whose launch shapes must not depend on timing)")
    p.add_argument("--profile-iteration", action="store_true",
                   help="set up and warm up as usual, then run exactly one iteration between profiler start and "
                        "stop (for ncu --profile-from-start off) and exit without timing")
    return p.parse_args()


# ----------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampler: median SM clock under load and throttle reasons."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    rows.append((float(parts[2]), float(parts[3]), parts[6:10]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        busy = [r for r in rows if r[0] >= 0.5 * r[1]] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in busy for i in range(4) if r[2][i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(busy)}


# -------------------------------------------------------------- cpu oracle
def cpu_oracle(wl, seconds: float, min_iters: int = 3):
    import oracle

    spec, what = wl["sample"]()
    o = oracle.Oracle(spec)
    o.iterate(1)  # warm caches
    n, t0 = 0, time.perf_counter()
    while n < min_iters or time.perf_counter() - t0 < seconds:
        o.iterate(1)
        n += 1
    dt = time.perf_counter() - t0
    return {"value": spec.n_edges * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host_cores": os.cpu_count(), "host": host_cpu(),
            "sample": "%s (%d edges), %d FP64 iterations in %.1f s, one thread" % (what, spec.n_edges, n, dt)}


def host_cpu() -> str:
    """The host's CPU model (for the record next to the oracle's timing)."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.machine()


def run_reference_serving(args):
    """The oracle solving the serving workload's requests one by one (same stop
    rule), for about --cpu-seconds of host work: solves/s."""
    import gamegen as gg
    import oracle

    t0 = time.perf_counter()
    done, edges = 0, 0
    for seed in range(args.requests):
        sp = gg.endgame(seed)
        o = oracle.Oracle(sp)
        it = 0
        while it < args.max_iters:
            o.iterate(50)
            it += 50
            if o.exploitability() <= 1e-3 * sp.pot:
                break
        done, edges = done + 1, edges + sp.n_edges
        if time.perf_counter() - t0 > args.cpu_seconds:
            break
    dt = time.perf_counter() - t0
    value = done / dt
    what = "endgame requests seeds 0-%d (%d edges), each solved alone to 1e-3 pot (checked every 50 iterations, " \
           "cap %d), one thread" % (done - 1, edges, args.max_iters)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": done, "warmup": 0, "ms_per_step": 1e3 * dt / done, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serving: endgame subgames, edges log-uniform in [1e3, 1e6]", "sample": what},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": what,
                         "host_cores": os.cpu_count(), "host": host_cpu()},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_reference_warmstart(args):
    """The warm start's yardstick on the oracle: cold-start CFR+ iterations to
    1e-3 pot on the held-out endgames, for about --cpu-seconds of host work."""
    import oracle
    from paper_2609_11923_gb300 import warmstart as ws

    t0 = time.perf_counter()
    iters = []
    for sp in ws.iter_endgame_family(range(20000, 20000 + args.heldout), 1e3, 1e6):  # the bench's held-out games
        o = oracle.Oracle(sp)
        it = 0
        while it < args.max_iters:
            o.iterate(50)
            it += 50
            if o.exploitability() <= 1e-3 * sp.pot:
                break
        iters.append(it)
        if time.perf_counter() - t0 > args.cpu_seconds:
            break
    dt = time.perf_counter() - t0
    value = sum(iters) / len(iters)
    what = "held-out endgames seeds 20000-%d, cold-start CFR+ to 1e-3 pot (checked every 50 iterations, cap %d), " \
           "one thread, %.1f s" % (20000 + len(iters) - 1, args.max_iters, dt)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iterations to 1e-3 pot (mean, cold start)",
        "n_gpus": args.gpus, "steps": len(iters), "warmup": 0, "ms_per_step": 1e3 * dt / len(iters),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "warm start yardstick: cold-start CFR+ on held-out endgames", "sample": what},
        "cpu_baseline": {"value": value, "unit": "iterations to 1e-3 pot (mean, cold start)", "cores": 1,
                         "host_cores": os.cpu_count(), "host": host_cpu(),
                         "kind": "oracle", "sample": what},
        "e2e": {"value": value, "unit": "iterations to 1e-3 pot (mean, cold start)", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload == "serving":
        return run_reference_serving(args)
    if args.workload == "warmstart":
        return run_reference_warmstart(args)
    import oracle

    wl = workloads()[args.workload]
    spec, what = wl["sample"]()
    o = oracle.Oracle(spec)
    for _ in range(args.warmup):
        o.iterate(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.iterate(1)
    dt = time.perf_counter() - t0
    value = spec.n_edges * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "description": wl["desc"],
                                        "sample": what, "edges": spec.n_edges},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "host_cores": os.cpu_count(), "host": host_cpu(),
                         "sample": "%s (%d edges), each step one FP64 iteration, one thread" % (what, spec.n_edges)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ ours
def max_over_ranks(dist, seconds: float, device) -> float:
    """The job's time: the slowest rank's, known to every rank (replicas)."""
    if dist is None:
        return seconds
    import torch

    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _code_only(text: str) -> str:
    """C++ source without comments and with whitespace collapsed (string
    literals kept as they are): what the compiler sees of the code."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":  # literal
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            i = text.find("\n", i)
            i = n if i < 0 else i
        elif text.startswith("/*", i):
            i = text.find("*/", i + 2)
            i = n if i < 0 else i + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash() -> str:
    """Hash of the kernels, the launch code and the compiler (which fixes
    the layout), comments and whitespace left out: recorded DRAM traffic
    applies while it matches."""
    h = hashlib.sha1()
    for f in ("kernels.cuh", "bwd_stream.cuh", "launch.h", "launch_impl.cuh", "k_bwd32.cu", "cfr_api.cu", "compile.cpp",
              "compiled.h"):
        with open(os.path.join(ROOT, "paper_2609_11923_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str, kernel: str):
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = rec.get(workload, {}).get(kernel)
    if ent and ent.get("source_hash") == kernel_source_hash():
        return ent.get("bytes_per_launch")
    return None


def run_ours(args):
    import torch

    from paper_2609_11923_gb300 import cfr

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()

    wl = workloads(args.deal_stride, args.stack, args.cap)[args.workload]
    spec = wl["make"]()
    forms = {"graph": cfr.EXEC_GRAPH, "levels": cfr.EXEC_LEVELS, "persistent": cfr.EXEC_PERSISTENT,
             "auto": cfr.EXEC_AUTO}
    prec = cfr.P32 if args.precision == "p32" else cfr.P64
    orders = {"members": cfr.REACH_MEMBERS, "bfs": cfr.REACH_BFS, "slots": cfr.REACH_SLOTS}
    solver = cfr.Solver(spec, precision=prec, exec_form=forms[args.exec_form], device=str(dev),
                        reach_order=orders[args.reach_order], lanes_per_set=args.lanes)
    counts = solver.counts
    E, D = counts["n_edges"], counts["depth_blocks"]
    pot, n_nodes = spec.pot, spec.n_nodes
    del spec  # the compiled copy lives in the handle
    stream = torch.cuda.current_stream(dev)
    s = int(stream.cuda_stream)
    tune = not args.no_autotune and args.lanes == 0
    lanes = solver.autotune() if tune else list(cfr.cfr_export_array(solver.h, "level_lanes"))

    # warm-up (graph capture happens on the first call)
    solver.iterate(args.warmup)
    solver.synchronize()
    if args.profile_iteration:
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.start()
        cfr.cfr_iterate(solver.h, 1, s)
        torch.cuda.synchronize(dev)
        torch.cuda.profiler.stop()
        if rank == 0:
            print(json.dumps({"profile_iteration": args.workload, "lanes_per_set_by_depth": [int(x) for x in lanes],
                              "source_hash": kernel_source_hash()}))
        return 0
    clocks = Clocks(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    cfr.cfr_iterate(solver.h, args.steps, s)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    solver.synchronize()
    dt = max_over_ranks(dist, ev0.elapsed_time(ev1) / 1e3, dev)
    iters_per_s = args.steps / dt
    value = world * E * iters_per_s
    algo_gbps = counts["algo_bytes_per_iter"] * iters_per_s / 1e9

    # per-launch times of one iteration (same kernels, same stream; outside the timed region)
    prof = [cfr.cfr_profile_iteration(solver.h, D, s) for _ in range(5)]
    fwd_ms = [statistics.median(p[0][d] for p in prof) for d in range(D)]
    bwd_ms = [statistics.median(p[1][d] for p in prof) for d in range(D)]
    launches = []
    fwd_kernel = "fwd_pull_kernel" if args.reach_order == "members" else "fwd_level_kernel"
    for d in range(D):
        fb, bb = cfr.cfr_level_bytes(solver.h, d)
        launches.append((fwd_kernel, d, fwd_ms[d], fb))
        launches.append(("bwd_stream_kernel" if int(lanes[d]) == cfr.STREAM_LANES else "bwd_level_kernel", d,
                         bwd_ms[d], bb))
    total_ms = sum(x[2] for x in launches)
    dom = max(launches, key=lambda x: x[2])
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    peak = float(peaks["hbm_gbs"])
    achieved = dom[3] / (dom[2] / 1e3) / 1e9
    kname = "%s[depth %d]" % (dom[0], dom[1])
    traffic = recorded_traffic(args.workload, kname)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "share_of_iteration": dom[2] / total_ms,
                "algo_bytes_per_launch": dom[3], "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}

    # the launch structure alone (empty kernels, same grids / same barriers), for comparison with ms_per_step
    floor_graph, floor_pers = cfr.cfr_launch_floor(solver.h, 200, s)
    launch_floor = {"graph_ms": floor_graph, "persistent_ms": floor_pers,
                    "what": "per iteration: a graph of the same %d launches (same grids) of an empty kernel; one "
                            "cooperative empty kernel with the persistent form's grid and %d grid barriers"
                            % ((D - 1 if args.reach_order == "members" else D) + D, 2 * D)}

    # end to end through the public API: upload (bind) + K iterations + average strategy to host
    e2e = None
    if not args.no_e2e:
        import numpy as np

        out = np.empty(counts["n_slots"])
        cfr.cfr_pin_host(solver.h)  # the compiled game's host arrays, page-locked once
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        cfr.cfr_bind(solver.h, solver.arena_ptr, solver.arena_bytes, s)
        cfr.cfr_iterate(solver.h, args.steps, s)
        cfr.cfr_avg_strategy(solver.h, out, False, s)
        t1 = time.perf_counter()
        et = max_over_ranks(dist, t1 - t0, dev)
        e2e = {"value": world * E * args.steps / et, "unit": UNIT,
               "h2d_bytes_per_step": counts["upload_bytes"] / args.steps,
               "d2h_bytes_per_step": 8.0 * counts["n_slots"] / args.steps,
               "what": "cfr_bind (upload of the compiled game from pinned host memory) + cfr_iterate(K) + "
                       "cfr_avg_strategy to host, wall clock"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle(wl, args.cpu_seconds)

    # the metric's second half: batched serving of endgame subgames (outside
    # the timed region; the game's arena is released first)
    batched = None
    arena_gb = solver.arena_bytes / 1e9
    if rank == 0 and args.batched_requests > 0 and args.workload == "large_card":
        solver.close()
        del solver
        torch.cuda.empty_cache()
        batched = serving_leg(args.batched_requests, args.max_iters, args.batched_baseline)
    barrier()

    # per depth one forward and one backward launch; in member order the
    # deepest depth has no forward launch (no internal node below it pulls)
    fwd_launches = D - 1 if args.reach_order == "members" else D
    per_iter_launches = {cfr.EXEC_GRAPH: fwd_launches + D, cfr.EXEC_LEVELS: fwd_launches + D}.get(counts["exec_form"], 0)
    gpu_launches = args.steps * per_iter_launches if per_iter_launches else 1
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == cfr.P32 else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload + ("" if args.deal_stride == 1 else " (every %dth deal)" % args.deal_stride)
                   + ("" if (args.stack, args.cap) == (2, 3) else " (stack %d, cap %d)" % (args.stack, args.cap)),
                   "description": wl["desc"], "nodes": n_nodes, "edges": E,
                   "infosets": counts["n_infosets"], "slots": counts["n_slots"], "depth_blocks": D,
                   "precision": args.precision + (" (FP64 regret/average accumulators)" if prec == cfr.P32 else ""),
                   "exec_form": args.exec_form, "reach_order": args.reach_order, "pot": pot, "parallelism": "replicas x%d" % world,
                   "lanes_per_set_by_depth": [int(x) for x in lanes],
                   "autotuned": tune,
                   "l2": "inputs larger than L2 (arena %.1f GB vs 129 MB L2)" % arena_gb},
        "iters_per_s": world * iters_per_s,
        "algo_gbps_per_gpu": algo_gbps,
        "algo_bytes_per_iter": counts["algo_bytes_per_iter"],
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "launch_profile_ms": {"fwd": fwd_ms, "bwd": bwd_ms},
        "launch_floor": launch_floor,
        "batched": batched,
    }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def serving_leg(n_requests: int, max_iters: int, baseline_sample: int, seed0: int = 0):
    """Batched serving of endgame subgames (seeds seed0 .. seed0 + n - 1):
    saturated solves/s (all requests at t = 0), p50/p99 latency under Poisson
    arrivals at 0.8x that rate, and a sample of the same solves run one by
    one (single-game solver per request, same stop rule) for the batching
    speed-up. Returns the figures as a dict."""
    import numpy as np
    import torch

    import gamegen as gg
    from paper_2609_11923_gb300 import cfr, serve

    n = n_requests
    specs = [gg.endgame(seed) for seed in range(seed0, seed0 + n)]
    edges = np.array([sp.n_edges for sp in specs])
    (threads, lanes), tune = serve.autotune_batch(specs[:64])
    hs = [cfr.cfr_compile(sp) for sp in specs[:8]]
    per_edge = max(cfr.cfr_plan(h) / sp.n_edges for h, sp in zip(hs, specs[:8]))
    for h in hs:
        cfr.cfr_destroy(h)
    pool_bytes = int(per_edge * edges.sum() * 1.2) + (64 << 20)

    def run(reqs):
        srv = serve.Server(pool_bytes, max_active=n, threads=threads, lanes=lanes, check_every=50,
                           max_iters=max_iters, target=1e-3)
        t = time.perf_counter()
        res = srv.serve(reqs)
        dt = time.perf_counter() - t
        rounds = srv.rounds
        srv.close()
        return res, dt, rounds

    res_b, dt_b, rounds_b = run([serve.Request(i, sp, 0.0) for i, sp in enumerate(specs)])
    rate = n / dt_b
    rng = np.random.default_rng(0)
    arrivals = np.cumsum(rng.exponential(1.0 / (0.8 * rate), size=n))
    res_p, dt_p, rounds_p = run([serve.Request(i, sp, float(a)) for i, (sp, a) in enumerate(zip(specs, arrivals))])
    lat = np.array([r.latency for r in res_p])
    conv_p = np.array([r.status == "solved" for r in res_p])
    sample = rng.choice(n, size=min(baseline_sample, n), replace=False)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for i in sample:
        serve.solve_alone(specs[i], check_every=50, max_iters=max_iters, target=1e-3)
    torch.cuda.synchronize()
    alone_rate = len(sample) / (time.perf_counter() - t)
    solved = np.array([r.status == "solved" for r in res_b])
    return {
        "requests": n, "edges_total": int(edges.sum()), "seeds": "%d-%d" % (seed0, seed0 + n - 1),
        "stop": "exploitability <= 1e-3 pot, checked every 50 iterations, cap %d" % max_iters,
        "launch_shape": {"threads": threads, "lanes": lanes,
                         "autotune_s": {"%dx%d" % k: v for k, v in tune.items()}},
        "saturated_solves_per_s": rate, "burst_seconds": dt_b, "burst_rounds": rounds_b,
        "poisson": {"rate_per_s": 0.8 * rate, "p50_s": float(np.percentile(lat, 50)),
                    "p99_s": float(np.percentile(lat, 99)),
                    "p50_s_solved": float(np.percentile(lat[conv_p], 50)) if conv_p.any() else None,
                    "p99_s_solved": float(np.percentile(lat[conv_p], 99)) if conv_p.any() else None,
                    "seconds": dt_p, "rounds": rounds_p,
                    "note": "latencies of every request; a capped request's latency is its time to the cap"},
        "per_instance_solves_per_s": alone_rate, "batching_speedup": rate / alone_rate,
        "per_instance_sample": int(len(sample)),
        "converged_fraction": float(solved.mean()), "censored_fraction": float(1.0 - solved.mean()),
        "iterations_p50": float(np.percentile([r.iterations for r in res_b], 50)),
        "gpu_launches": 2 * (rounds_b + rounds_p),
    }


def run_serving(args):
    """Batched serving of endgame subgames as its own bench line (solves/s)."""
    import torch

    torch.cuda.set_device(0)
    leg = serving_leg(args.requests, args.max_iters, args.baseline_sample)
    rate = leg["saturated_solves_per_s"]
    line = {
        "metric": METRIC, "value": rate, "unit": "solves/s", "n_gpus": 1, "steps": args.requests, "warmup": 0,
        "ms_per_step": 1e3 / rate, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving: %d endgame subgames, edges log-uniform in [1e3, 1e6] (total %d)"
                               % (args.requests, leg["edges_total"]),
                   "stop": leg["stop"], "launch_shape": leg["launch_shape"]},
        "gpu_launches": leg["gpu_launches"],
    }
    line.update({k: v for k, v in leg.items() if k not in ("stop", "launch_shape", "gpu_launches")})
    print(json.dumps(line))
    return 0


def run_warmstart(args):
    """Learned warm start: train the MLP on solved endgames, then iterations
    and wall time to 1e-3 pot exploitability, warm vs cold, on held-out seeds."""
    import numpy as np
    import torch

    from paper_2609_11923_gb300 import warmstart as ws

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    train = ws.endgame_family(list(range(10000, 10000 + args.train_games)), 1e3, 1e5)
    X, na, T = ws.make_dataset(train, iters=1000)
    t_data = time.perf_counter() - t0
    t1 = time.perf_counter()
    net = ws.train(X, na, T, epochs=6)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    val = ws.endgame_family(list(range(15000, 15064)), 1e3, 1e5)
    kappa, ktable = ws.choose_kappa(net, val)
    held = ws.endgame_family(list(range(20000, 20000 + args.heldout)), 1e3, 1e6)
    # each game on its own (a single real-time re-solve): iterations and wall
    # time to the target, on a sample of the held-out games
    alone = {"cold": [], "warm": []}
    for sp in held[:args.alone_sample]:
        alone["cold"].append(ws.time_to_target_alone(sp, max_iters=args.max_iters))
        alone["warm"].append(ws.time_to_target_alone(sp, net=net, kappa=kappa, max_iters=args.max_iters))
    alone_stats = {}
    for arm, rows in alone.items():
        it = np.array([r[0] for r in rows])
        sec = np.array([r[1] for r in rows])
        alone_stats[arm] = {"mean_iters": float(it.mean()), "mean_s": float(sec.mean()),
                            "median_s": float(np.median(sec)), "reached": float(np.mean([r[2] for r in rows]))}
    cold_t, warm_t = {}, {}
    cold, cold_fin, cold_wall = ws.iterations_to_target(held, max_iters=args.max_iters, timings=cold_t)
    # the warm start's wall time includes its features (from the compiled
    # games) and the network pass
    warm, warm_fin, warm_wall = ws.iterations_to_target(held, net=net, kappa=kappa, max_iters=args.max_iters,
                                                        timings=warm_t)
    line = {
        "metric": METRIC, "value": float(np.mean(warm)), "unit": "iterations to 1e-3 pot (mean, warm start)",
        "n_gpus": 1, "steps": args.heldout, "warmup": 0, "ms_per_step": None, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16 network / f32 CFR", "data": "synthetic",
        "config": {"workload": "warm start: MLP 3x256 on %d solved endgames (1e3-1e5 edges, 1000 iterations each), "
                               "%d held-out endgames (1e3-1e6 edges)" % (args.train_games, args.heldout),
                   "stop": "exploitability <= 1e-3 pot, checked every 50 iterations, cap %d" % args.max_iters},
        "cold": {"mean_iters": float(np.mean(cold)), "median_iters": float(np.median(cold)),
                 "finished": float(cold_fin.mean()), "wall_s": cold_wall, "breakdown_s": cold_t},
        "warm": {"mean_iters": float(np.mean(warm)), "median_iters": float(np.median(warm)),
                 "finished": float(warm_fin.mean()), "wall_s": warm_wall, "breakdown_s": warm_t,
                 "wall_includes": "compile, features from the compiled games, one network pass, the solves"},
        "wall_ratio_warm_over_cold": warm_wall / cold_wall,
        "iteration_ratio_warm_over_cold": float(np.mean(warm) / np.mean(cold)),
        "alone": dict(alone_stats, games=len(alone["cold"]),
                      what="each game solved on its own (single-game form chosen by size), warm start = "
                           "features from its compiled game + one network pass + initial regrets; wall time "
                           "from compile to the target",
                      wall_ratio_warm_over_cold=alone_stats["warm"]["mean_s"] / alone_stats["cold"]["mean_s"]),
        "kappa": kappa, "kappa_validation_mean_iters": ktable,
        "training": {"samples": int(X.shape[0]), "data_s": t_data, "train_s": t_train,
                     "loss_by_epoch": [float(x) for x in net.history]},
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
