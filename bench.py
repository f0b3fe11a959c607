"""Benchmark: neighbour evaluations per second of the plain solver at
L=121 (D=61), 131072 concurrent walks of 8192 steps, a budget of 1e11
neighbour evaluations (two whole rounds), Philox seed 1 (rank r uses seed 1+r).

One "step" = one whole solve (every round until the budget) through the C ABI.
  value   : evaluations/s with inputs resident in HBM (device buffers, workspace
            preallocated), CUDA events on the launching stream, max over ranks;
  e2e     : the same metric through labs_walks with HOST buffers (seed upload,
            workspace allocation and result download inside the timed region);
  roofline: the walk kernel against the popcount (XU) pipe: the population
            counts the bit-sliced evaluation needs per neighbour (popc_needed)
            over the kernel's per-launch time, against 152 SMs x 16 x 2070 MHz;
            the int32 ALU-pipe unit beside it;
  batched : the 64-instance workload through the persistent batch path, against
            one labs_walks per instance, with its own roofline;
  serving : a Poisson request stream through the server (p50/p99 latency),
            against one labs_walks per request, and the server's capacity with
            all of the stream's requests submitted at once;
  cpu_baseline: the CPU oracle on a bounded sample of the same walks.

`--impl reference` times the CPU oracle (the reference arm of this project)
on the same workload and prints the same JSON line with "impl": "reference".
Other workloads (--workload batched, serving, large, table1, walklen,
variants) print their own lines.

Multi-GPU (torchrun): each rank solves its own independent problem (weak
scaling, no data-path collective); the host barrier and a max-reduction of the
time are the only communication.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_L = 121
L = DEFAULT_L
WALKS = 131072
WALK_LEN = 8192
BUDGET = 10 ** 11
SEED = 1
INT_LANES_PER_SM = 64          # int32 ALU-pipe lanes per SM per clock (LOP3/SHF/IADD3 class)
POPC_LANES_PER_SM = 16         # population counts per SM per clock (XU pipe)
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


# DRAM traffic of one walk-kernel launch of the default workload, from an ncu
# capture of the walk kernel on 107008 walks x 1024 steps (20.87 GB, scaled by
# walk-steps to 131072 x 8192), valid only for the kernel code it was captured
# from (the hash below covers the sources' code, not their comments).
TRAFFIC = {"sources_sha256_prefix": "18c322da31ea710b", "bytes_per_launch": 20.868e9 * (131072 * 8192) / (107008 * 1024)}
WALK_SOURCES = ["walk_core.cuh", "walk_device.cuh", "walk_incr.cuh", "walk_class.cu", "walk_kernels.cuh"]


def walk_sources_hash():
    """sha256 prefix of the walk kernel's sources without their // comments and blank lines."""
    import hashlib
    h = hashlib.sha256()
    for f in WALK_SOURCES:
        with open(os.path.join(ROOT, "paper_2210_15962_gb300", "csrc", f)) as fh:
            code = [line.split("//", 1)[0].rstrip() for line in fh.read().splitlines()]
        h.update("\n".join(c for c in code if c).encode())
    return h.hexdigest()[:16]


def digits_for(L):
    T = 1
    while (1 << T) < L - 1:
        T += 1
    return T


def core_alu_ops_per_eval(L, planes, full=False):
    """ALU-pipe lane-ops of the bit-sliced Delta core per neighbour evaluation:
    per 32 lags and digit plane, two masked XORs and a carry-save full adder
    (4 LOP3), for the number of digit planes the scan used; the lags are the
    (L-1)/2 even ones of a skew sequence or all L-1 in the full space."""
    m = (L - 1) if full else (L - 1) // 2
    return 4.0 * planes * m / 32.0


def popc_words_per_step(L):
    """(nw, n2) of the skew scan's formulation at length L, summed over the D
    flips of one walk step: nw = 32-lag words holding any valid lag of the
    flip, n2 = words holding valid lags on both sides.  A flip j (position
    a = j, class q = a % 2, index t = a // 2) has x-side lags i = 1..t and
    y-side lags i = 1..N_q-1-t without the lag of its own mirror pair
    (c - a), N_q = D - q, and no y side at the centre a = c = D - 1."""
    D, m = (L + 1) // 2, (L - 1) // 2
    c, W = D - 1, (m + 31) // 32
    nw = n2 = 0
    for a in range(D):
        q, t = a & 1, a >> 1
        xs_hi = t                       # x lags 1..t
        ys = set() if a == c else set(range(1, D - q - t)) - {c - a}
        for w in range(W):
            lo, hi = 32 * w + 1, 32 * w + 32
            xw = xs_hi >= lo
            yw = any(lo <= i <= hi for i in ys)
            nw += xw or yw
            n2 += xw and yw
    return nw, n2


def popc_needed(L, evals, plane_steps):
    """Population counts the bit-sliced evaluation needs for `evals` neighbour
    evaluations at length L whose steps used `plane_steps` digit planes in all:
    per flip and 32-lag word, one count per digit plane over the valid lags
    (TP), plus two for a word with lags on both sides (the top digit of the
    equal-bits lags and the count of those lags).  One step evaluates D flips."""
    nw, n2 = popc_words_per_step(L)
    steps = evals / ((L + 1) // 2)
    return plane_steps * nw + 2.0 * steps * n2


def popc_peak_tops():
    """The XU pipe: POPC_LANES_PER_SM population counts per SM per clock, all SMs, at the maximum clock."""
    return SM_COUNT * POPC_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12


def popc_roofline(needed, seconds, **extra):
    achieved = needed / seconds / 1e12
    peak = popc_peak_tops()
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T popcount lane-ops/s (XU pipe)",
           "frac": achieved / peak,
           "peak_basis": "152 SMs x 16 POPC lanes/clk/SM x 2070 MHz max clock (of measured: 16.00 lanes/clk)"}
    out.update(extra)
    return out


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
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
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_seed(rank):
    """Each rank solves its own independent problem (weak scaling)."""
    return SEED + rank


def combine_ranks(times, counts, dist=None, device="cpu"):
    """Whole-job totals over ranks: the maximum of each time, the sum of each count.
    Host-side control only (no data-path collective); works with nccl or gloo."""
    import torch
    t = torch.tensor([float(x) for x in times], dtype=torch.float64, device=device)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu()], [float(x) for x in c.cpu()]


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


CPU_SAMPLE_LAG_UPDATES = 1.5e10  # about 13 s of oracle work on 16 host cores


CPU_STEP_OVERHEAD = 256  # the oracle's per-step set lookups and move, in (flip, lag) updates


def cpu_sample_walks(L, walk_len, cores, full=False, total_walks=None, lag_updates=CPU_SAMPLE_LAG_UPDATES):
    """Walks in the oracle's timed sample: a whole number of walks per core,
    enough for about `lag_updates` (flip, lag) updates (the oracle's cost per
    evaluation grows with the lag count), at least one walk per core and at
    most the workload's walks."""
    flips = L if full else (L + 1) // 2
    lags = max(1, L - 1 if full else (L - 1) // 2)
    per_walk = float(walk_len) * (flips * lags + CPU_STEP_OVERHEAD)
    per_core = max(1, -(-int(lag_updates) // max(1, int(per_walk * cores))))
    n = per_core * cores
    return min(n, total_walks) if total_walks else n


def cpu_baseline(n_walks=None, walk_len=WALK_LEN, seed=SEED, L=L, total_walks=WALKS, full=False, one_core=False):
    """The oracle on a bounded sample of the benchmark's walks, all host cores
    (with one_core, also the rate of one core on an eighth of one core's share
    of the sample, at least one walk: about 2 s)."""
    import oracle
    cores = os.cpu_count() or 1
    n = n_walks or cpu_sample_walks(L, walk_len, cores, full, total_walks)
    t0 = time.perf_counter()
    r = oracle.walk_batch(L, seed, 0, 0, n, walk_len, threads=cores, full=full)
    dt = time.perf_counter() - t0
    ev = int(r["evals"].sum())
    out = {"value": ev / dt, "unit": "neighbour_evals/s", "cores": cores, "kind": "oracle",
           "sample": "%d of the %d walks of round 0 (L=%d, %d steps each), %d evaluations in %.1f s"
                     % (n, total_walks, L, walk_len, ev, dt)}
    if one_core:
        n1 = max(1, (n // cores) // 8)
        t0 = time.perf_counter()
        r1 = oracle.walk_batch(L, seed, 0, 0, n1, walk_len, threads=1, full=full)
        dt1 = time.perf_counter() - t0
        ev1 = int(r1["evals"].sum())
        out["one_core"] = {"value": ev1 / dt1, "sample": "%d walks, %d evaluations in %.1f s" % (n1, ev1, dt1)}
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return
    steps, times = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(n_walks=args.ref_walks or 8 * (os.cpu_count() or 1))
        if i >= args.warmup:
            steps.append(cb)
            times.append(time.perf_counter() - t0)
    val = statistics.mean(s["value"] for s in steps)
    line = {
        "metric": "neighbour_evals_per_s", "value": val, "unit": "neighbour_evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic (Philox starts, seed 1)",
        "impl": "reference",
        "config": {"workload": "plain_L121_131072x8192_budget1e11", "L": L, "walks": WALKS, "walk_len": WALK_LEN,
                   "budget": BUDGET, "note": "each step: the CPU oracle on a bounded sample of the walks"},
        "cpu_baseline": {"value": val, "unit": "neighbour_evals/s", "cores": steps[0]["cores"], "kind": "oracle",
                         "sample": steps[0]["sample"]},
        "e2e": {"value": val, "unit": "neighbour_evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_batched(args, rank, steps, warmup):
    """The batched workload: args.instances instances of odd L in [101, 223],
    args.batch_walks walks each, walk length 8*D, log-uniform budgets in
    [1e8, 1e10], seed 1000+i (+1000*rank).  The persistent batch path (CUDA
    graph replay, autotuned shapes) against one labs_walks per instance on the
    same problems.  Returns the measurements as a dict."""
    import torch
    import paper_2210_15962_gb300 as pkg
    from paper_2210_15962_gb300 import workloads
    wl = workloads.batched_instances(n=args.instances, walks=args.batch_walks)
    # --batch-walk-len > 0 replaces the 8*D walk length (a smaller device footprint for profiler captures)
    probs = [(p.L, p.walks, args.batch_walk_len or p.walk_len, p.seed + 1000 * rank, p.step_budget)
             for p in wl.problems]
    stream = torch.cuda.Stream()
    # a fixed block size and table factor (both given) replace the autotuner's choice
    b = pkg.Batch(probs, use_graph=True, autotune=True, walk_mode=args.batch_walk_mode,
                  block_threads=args.batch_block, table_factor_x10=args.batch_table_factor, stream=stream)
    for _ in range(warmup):
        b.run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ev = launches = wlaunch = 0
    kms = 0.0
    for _ in range(steps):
        st = b.run()
        ev += st["evals"]
        launches += st["launches"]
        kms += st["walk_kernel_ms"]
        wlaunch += st["walk_launches"]
    e1.record(stream)
    e1.synchronize()
    dev_s = e0.elapsed_time(e1) / 1e3
    res = b.results()
    shapes = {W: b.shape(W) for W in sorted({((p[0] - 1) // 2 + 31) // 32 for p in probs})}
    b.close()
    # the algorithm's popcounts of one run, from each problem's digit planes (every run is the same)
    needed = sum(popc_needed(p[0], r["evals"], r["plane_steps"]) for p, r in zip(probs, res))
    # the plain path: one solve per instance, each its own launch sequence
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    plain_ev = 0
    same = True
    t0.record(stream)
    for i, p in enumerate(probs[:args.plain_instances]):
        r = pkg.labs_walks(p[0], [p[3]], p[1], p[2], p[4], stream=stream)
        plain_ev += int(r["evals"][0])
        same = same and int(r["best_E"][0]) == res[i]["best_E"] and int(r["evals"][0]) == res[i]["evals"] \
            and bool((r["best_seq"][0] == res[i]["best_seq"]).all())
    t1.record(stream)
    t1.synchronize()
    plain_s = t0.elapsed_time(t1) / 1e3
    Ls = [p[0] for p in probs]
    return {
        "value": ev / dev_s, "unit": "neighbour_evals/s", "steps": steps, "ms_per_step": dev_s * 1e3 / steps,
        "evals": ev, "seconds": dev_s, "launches": launches, "walk_launches": wlaunch,
        "config": {"workload": wl.name, "instances": len(probs), "walks": args.batch_walks,
                   "L_range": [min(Ls), max(Ls)], "walk_len": args.batch_walk_len or "8*D",
                   "budget_range": [min(p[4] for p in probs), max(p[4] for p in probs)],
                   "path": "batched persistent kernel, CUDA graph replay, autotuned shapes",
                   "walk_mode": ["autotuned", "lane", "warp", "CTA"][args.batch_walk_mode],
                   "shapes": {str(k): v for k, v in shapes.items()}},
        "roofline": popc_roofline(needed * steps, kms / 1e3, kernel="batch_kernel<W> (all classes, concurrent)",
                                  kernel_ms_per_run=kms / steps,
                                  popc_per_eval=needed / max(1, ev / steps)),
        "plain": {"value": plain_ev / plain_s, "unit": "neighbour_evals/s",
                  "instances": min(args.plain_instances, len(probs)),
                  "path": "labs_walks per instance (one launch sequence per L)", "same_results": bool(same)},
    }


def run_batched(args, world, rank, local):
    """The batched workload on its own (see measure_batched); weak scaling over ranks."""
    import torch
    import paper_2210_15962_gb300 as pkg
    from paper_2210_15962_gb300 import workloads
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.load()
    if dist is not None:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    m = measure_batched(args, rank, args.steps, args.warmup)
    clocks = sampler.stop()
    (dev_s, _), (tot_ev, _) = combine_ranks([m["seconds"], 0.0], [m["evals"], 0], dist, "cuda")
    if rank == 0:
        line = {
            "metric": "neighbour_evals_per_s", "value": tot_ev / dev_s, "unit": "neighbour_evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (Philox starts; instances from SplitMix64 seed %d)" % workloads.MANIFEST_SEED,
            "config": dict(m["config"], l2="visited-table pools larger than L2"),
            "roofline": m["roofline"], "plain": m["plain"], "gpu_launches": m["launches"], "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def serving_targets(pkg, Ls, budget):
    """Per-L target energies: the best the plain path reaches with `budget`
    evaluations, 2048 walks of 8*D steps, seed 99."""
    from paper_2210_15962_gb300 import workloads
    out = {}
    for L in sorted(set(Ls)):
        r = pkg.labs_walks(L, [99], 2048, workloads.paper_walk_len(L), budget)
        out[L] = int(r["best_E"][0])
    return out


def measure_serving(args, warmup):
    """Poisson request stream (mean args.rate/s for args.serve_seconds s) of odd L
    uniform in [121, 301], 2048 walks, walk length 8*D, budget args.serve_budget,
    stop at the budget or at a per-L target energy (serving_targets); continuous
    batching with memory admission.  Beside it, the plain path on the first
    requests, one labs_walks per request, one at a time.  Returns a dict."""
    import numpy as np
    import paper_2210_15962_gb300 as pkg
    from paper_2210_15962_gb300 import workloads
    wl = workloads.serving_stream(duration_s=args.serve_seconds, rate_per_s=args.rate, budget=args.serve_budget)
    reqs = wl.problems
    targets = serving_targets(pkg, [p.L for p in reqs], args.target_budget)
    sv = pkg.Server(max_L=301, max_walks=2048, max_active=args.max_active, mem_bytes=args.mem_gib << 30,
                    rounds_per_launch=args.rounds_per_launch, walk_mode=args.serve_walk_mode)
    for i in range(warmup):  # a few requests end to end
        p = reqs[i % len(reqs)]
        sv.wait(sv.submit(p.L, p.walks, p.walk_len, 10 ** 6 + i, p.walk_len * p.walks))
    st0 = sv.stats()
    tickets = []
    t0 = time.perf_counter()
    for p in reqs:
        delay = t0 + p.arrival_s - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(sv.submit(p.L, p.walks, p.walk_len, p.seed, p.step_budget, targets[p.L]))
    results = [sv.wait(t, timeout_s=3600) for t in tickets]
    t1 = time.perf_counter()
    st = sv.stats()
    # capacity: the first requests of the stream all submitted at once, so that
    # the server is never short of work (throughput is then the server's own,
    # not the stream's offered load)
    cap_reqs = reqs[:args.capacity_requests] if args.capacity_requests > 0 else reqs
    tc0 = time.perf_counter()
    cap_t = [sv.submit(p.L, p.walks, p.walk_len, p.seed, p.step_budget, targets[p.L]) for p in cap_reqs]
    cap_res = [sv.wait(t, timeout_s=3600) for t in cap_t]
    tc1 = time.perf_counter()
    stc = sv.stats()
    sv.close()
    cap_evals = sum(r["evals"] for r in cap_res)
    cap_busy = (stc["busy_ms"] - st["busy_ms"]) / 1e3
    cap_needed = sum(popc_needed(p.L, r["evals"], r["plane_steps"]) for p, r in zip(cap_reqs, cap_res))
    cap_lat = np.array([r["latency_s"] for r in cap_res])
    same_cap = all(a["best_E"] == b["best_E"] and a["evals"] == b["evals"] for a, b in zip(cap_res, results))
    lat = np.array([r["latency_s"] for r in results])
    qwait = np.array([(r["t_admit_ns"] - r["t_submit_ns"]) / 1e9 for r in results])
    evals = sum(r["evals"] for r in results)
    busy_s = (st["busy_ms"] - st0["busy_ms"]) / 1e3
    needed = sum(popc_needed(p.L, r["evals"], r["plane_steps"]) for p, r in zip(reqs, results))
    # the plain path on the first requests, one labs_walks per request
    tp0 = time.perf_counter()
    plain_ev = 0
    plain_t = []  # each request's time to its target (or budget) alone, with no queue
    same = True
    for p, r in list(zip(reqs, results))[:args.plain_requests]:
        tq = time.perf_counter()
        g = pkg.labs_walks(p.L, [p.seed], p.walks, p.walk_len, p.step_budget, target_E=targets[p.L])
        plain_t.append(time.perf_counter() - tq)
        plain_ev += int(g["evals"][0])
        same = same and int(g["best_E"][0]) == r["best_E"] and int(g["evals"][0]) == r["evals"] \
            and bool((g["best_seq"][0] == r["best_seq"]).all())
    tp1 = time.perf_counter()
    return {
        "value": evals / (t1 - t0), "unit": "neighbour_evals/s", "seconds": t1 - t0, "evals": evals,
        "config": {"workload": wl.name, "requests": len(reqs), "duration_s": args.serve_seconds,
                   "rate_per_s": args.rate, "walks": 2048, "walk_len": "8*D", "budget": args.serve_budget,
                   "targets": "per L: plain-path best with budget %g, seed 99" % args.target_budget,
                   "max_active": args.max_active, "mem_gib": args.mem_gib,
                   "rounds_per_launch": args.rounds_per_launch,
                   "walk_mode": ["chosen per launch", "lane per walk", "warp per walk"][args.serve_walk_mode]},
        "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                      "mean": float(lat.mean()), "max": float(lat.max())},
        "queue_wait_s": {"p50": float(np.percentile(qwait, 50)), "p99": float(np.percentile(qwait, 99))},
        "completed": len(results), "reached_target": int(sum(r["reached_target"] for r in results)),
        # Eq. 7 of the predictive model for each request's evaluations
        "p_optimal": {"p50": float(np.percentile([r["p_optimal"] for r in results], 50)),
                      "min": float(min(r["p_optimal"] for r in results))},
        "device_busy_frac": busy_s / (t1 - t0),
        "evals_run": st["evals_run"] - st0["evals_run"],
        "useful_frac": (st["evals"] - st0["evals"]) / max(1, st["evals_run"] - st0["evals_run"]),
        "mem_peak_bytes": st["mem_peak"],
        "class_kernels": {"lane": stc["lane_launches"], "lane_unrolled": stc["lane_unrolled_launches"],
                          "warp": stc["warp_launches"]},
        "roofline": popc_roofline(needed, busy_s, kernel="batch_kernel<W> (all classes, two launches in flight)",
                                  popc_per_eval=needed / max(1, evals),
                                  note="useful evaluations only (rounds past a request's stop not counted), "
                                       "over the device's busy time"),
        # the plain path one request at a time: its time per request with no queue, and the
        # stream's load over what it sustains (above 1 its queue, and so its latency, grows
        # without bound at the stream's rate)
        "plain": {"value": plain_ev / (tp1 - tp0), "unit": "neighbour_evals/s",
                  "requests": min(args.plain_requests, len(reqs)), "path": "labs_walks per request, one at a time",
                  "same_results": bool(same),
                  "seconds_per_request_alone": ({"p50": float(np.percentile(plain_t, 50)), "max": float(max(plain_t))}
                                                if plain_t else None),
                  "stream_load": (evals / (t1 - t0)) / max(1e-9, plain_ev / (tp1 - tp0)) if plain_t else None},
        "gpu_launches": st["launches"] - st0["launches"],
        "capacity": {
            "value": cap_evals / (tc1 - tc0), "unit": "neighbour_evals/s", "requests": len(cap_reqs),
            "seconds": tc1 - tc0, "device_busy_frac": cap_busy / (tc1 - tc0),
            "useful_frac": (stc["evals"] - st["evals"]) / max(1, stc["evals_run"] - st["evals_run"]),
            "latency_s": {"p50": float(np.percentile(cap_lat, 50)), "p99": float(np.percentile(cap_lat, 99))},
            "same_results_as_stream": bool(same_cap),
            "roofline": popc_roofline(cap_needed, cap_busy, popc_per_eval=cap_needed / max(1, cap_evals),
                                      note="useful evaluations only, over the device's busy time"),
            "note": "the stream's requests submitted at once (same seeds and targets)"},
        # the stream's useful throughput is its offered load: this share of what the
        # server sustains when saturated, so its launches keep part of the lanes busy
        "load_vs_capacity": (evals / (t1 - t0)) / max(1e-9, cap_evals / (tc1 - tc0)),
    }


def run_serving(args, world, rank, local):
    """The serving workload on its own (see measure_serving)."""
    import torch
    import paper_2210_15962_gb300 as pkg
    from paper_2210_15962_gb300 import workloads
    torch.cuda.set_device(local)
    pkg.load()
    sampler = ClockSampler(local)
    sampler.start()
    m = measure_serving(args, args.warmup)
    clocks = sampler.stop()
    line = {
        "metric": "neighbour_evals_per_s", "value": m["value"], "unit": "neighbour_evals/s",
        "n_gpus": 1, "steps": 1, "warmup": args.warmup, "ms_per_step": m["seconds"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic request stream (SplitMix64 seed %d)" % workloads.MANIFEST_SEED,
        "clocks": clocks,
    }
    line.update({k: v for k, v in m.items() if k not in ("value", "unit", "seconds", "evals")})
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_large(args, world, rank, local):
    """Time to a target energy at L=449 (D=225), 65536 walks x 16384 steps per
    round, plain path against batched path.  The target is fixed independently
    of both arms: the best energy of a calibration solve with its own seed (99)
    and --large-cal-rounds rounds.  Each arm then solves --large-seeds seeds
    (1..) to that target, each capped at --large-cap-s seconds of rounds, and
    the median and spread of the times are reported.  Plain: labs_walks (one
    walk-kernel launch per round).  Batched: the persistent batch path with the
    instance alone (--large-rpl rounds per launch, the later ones skipped on
    the device once a round reaches the target)."""
    import numpy as np
    import torch
    import paper_2210_15962_gb300 as pkg
    torch.cuda.set_device(local)
    pkg.load()
    L, walks, wl = 449, args.walks_large, args.walk_len_large
    D = (L + 1) // 2
    per_round = walks * wl * D
    stream = torch.cuda.Stream()

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    sampler = ClockSampler(local)
    sampler.start()
    cal, t_cal = timed(lambda: pkg.labs_walks(L, [99], walks, wl, args.large_cal_rounds * per_round, stream=stream))
    target = int(cal["best_E"][0])
    round_s = t_cal / args.large_cal_rounds
    max_rounds = max(1, int(args.large_cap_s / round_s))
    budget = max_rounds * per_round
    arms = {"plain": [], "batched": []}
    for sd in range(1, args.large_seeds + 1):
        seed = sd + 1000 * rank
        r, t = timed(lambda: pkg.labs_walks(L, [seed], walks, wl, budget, target_E=target, stream=stream))
        arms["plain"].append({"seed": seed, "seconds": t, "reached": int(r["best_E"][0]) <= target,
                              "rounds": int(r["rounds"][0]), "evals": int(r["evals"][0]), "best_E": int(r["best_E"][0])})
        b = pkg.Batch([(L, walks, wl, seed, budget, target)], rounds_per_launch=args.large_rpl, stream=stream)
        st, t = timed(b.run)
        res = b.result(0)
        b.close()
        arms["batched"].append({"seed": seed, "seconds": t, "reached": res["best_E"] <= target, "rounds": res["rounds"],
                                "evals": res["evals"], "best_E": res["best_E"],
                                "same_as_plain": res["best_E"] == arms["plain"][-1]["best_E"]
                                and res["rounds"] == arms["plain"][-1]["rounds"]})
    clocks = sampler.stop()

    def summary(rows):
        ts = [x["seconds"] if x["reached"] else float("inf") for x in rows]
        ok = [x for x in ts if x != float("inf")]
        return {"median_s": float(np.median(ts)), "min_s": min(ts), "max_s": max(ts),
                "quartiles_s": [float(np.percentile(ts, 25)), float(np.percentile(ts, 75))],
                "reached": len(ok), "runs": len(rows),
                "evals_per_s": sum(x["evals"] for x in rows) / sum(x["seconds"] for x in rows),
                "runs_detail": rows}

    line = {
        "metric": "time_to_target_s", "value": summary(arms["batched"])["median_s"], "unit": "s", "n_gpus": world,
        "steps": args.large_seeds, "warmup": 1, "ms_per_step": None, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (Philox starts, seeds 1..%d)" % args.large_seeds,
        "config": {"workload": "time_to_target_L449_%dx%d" % (walks, wl), "L": L, "walks": walks, "walk_len": wl,
                   "target_E": target, "target_F": L * L / (2.0 * target),
                   "target_from": "best of a %d-round calibration solve, seed 99 (%.1f s)" % (args.large_cal_rounds,
                                                                                            t_cal),
                   "cap_rounds": max_rounds, "cap_s": args.large_cap_s, "batched_rounds_per_launch": args.large_rpl},
        "plain": summary(arms["plain"]), "batched": summary(arms["batched"]),
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def table1_rows():
    """Table 1 of the paper (Section 4.2), from the test fixture that records it:
    {L: (E, F, P percent, hex)}."""
    rows = {}
    with open(os.path.join(ROOT, "tests", "golden", "table1_skew_sequences.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                r = line.split()
                rows[int(r[0])] = (int(r[1]), float(r[2]), float(r[3]), r[4])
    return rows


def symmetry_orbit(seq):
    """The sequences with the same energy under negation, reversal and
    alternating signs (s_i -> (-1)^i s_i), which keep skew symmetry."""
    import numpy as np
    s = np.asarray(seq, dtype=np.int8)
    alt = np.where(np.arange(s.size) % 2 == 0, 1, -1).astype(np.int8)
    out = []
    for a in (s, s[::-1]):
        for b in (a, (a * alt).astype(np.int8)):
            out += [b, (-b).astype(np.int8)]
    return out


def run_table1(args, world, rank, local):
    """Time for the plain path to reach the energy Table 1 prints for L
    (--table1-L, default 171): walks --table1-walks, walk length 8*D (the
    paper's rule), seed --table1-seed + rank, target E of Table 1, step budget the
    predictive model's for probability 0.999 (Eq. 6/7), capped at
    --table1-seconds of rounds.  Reports the model's probability (Eq. 7) for the
    evaluations spent and whether the sequence found is Table 1's up to the
    symmetries that keep the energy."""
    import numpy as np
    import torch
    import paper_2210_15962_gb300 as pkg
    torch.cuda.set_device(local)
    pkg.load()
    L = args.table1_L
    E_tab, F_tab, P_tab, hx = table1_rows()[L]
    D = (L + 1) // 2
    walks, wl, seed = args.table1_walks, 8 * D, args.table1_seed + rank
    per_round = walks * wl * D
    budget = pkg.labs_model_budget(L, 0.999)
    stream = torch.cuda.Stream()
    # one round to warm up (the first call also times the kernel variants and
    # allocates), then one more to size the time cap in rounds
    pkg.labs_walks(L, [seed + 7919], walks, wl, per_round, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pkg.labs_walks(L, [seed + 7919], walks, wl, per_round, stream=stream)
    torch.cuda.synchronize()
    t_round = time.perf_counter() - t0
    max_rounds = max(1, int(args.table1_seconds / t_round))
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = pkg.labs_walks(L, [seed], walks, wl, budget, target_E=E_tab, max_rounds=max_rounds, stream=stream)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    clocks = sampler.stop()
    E = int(r["best_E"][0])
    evals = int(r["evals"][0])
    tab = pkg.from_hex(hx, L)
    same = any(np.array_equal(r["best_seq"][0], o) for o in symmetry_orbit(tab))
    line = {
        "metric": "time_to_target_s", "value": t if E <= E_tab else None, "unit": "s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": t * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (Philox starts, seed %d)" % seed,
        "config": {"workload": "table1_L%d_%dx%d" % (L, walks, wl), "L": L, "walks": walks, "walk_len": wl,
                   "target_E": E_tab, "budget": budget, "max_rounds": max_rounds},
        "reached": E <= E_tab, "best_E": E, "F": L * L / (2.0 * E), "rounds": int(r["rounds"][0]),
        "evals": evals, "neighbour_evals_per_s": evals / t,
        "model": {"nses": pkg.labs_model_nses_of_evals(L, evals),
                  "p_optimal": pkg.labs_model_p_optimal(L, pkg.labs_model_nses_of_evals(L, evals)),
                  "nses_limit_99_per_run_of_100": pkg.labs_model_nses_limit(L, 0.99, 100)},
        "table1": {"E": E_tab, "F": F_tab, "P_percent": P_tab, "same_sequence_up_to_symmetry": bool(same)},
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_walklen(args, world, rank, local):
    """The walk-length rule (the paper's n = 8 D against D .. 32 D) as time to a
    target energy: L (--L, default 121), --walks walks per round, target = the
    best E of a calibration solve (walk length 8 D, seed 99, --walklen-cal-budget
    evaluations); for each walk length, --walklen-seeds solves (seeds 1..) with
    that target, each capped at about --walklen-seconds of rounds; the median
    time to target per length."""
    import numpy as np
    import torch
    import paper_2210_15962_gb300 as pkg
    torch.cuda.set_device(local)
    pkg.load()
    L, walks = args.L, args.walks
    D = (L + 1) // 2
    stream = torch.cuda.Stream()

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    cal, t_cal = timed(lambda: pkg.labs_walks(L, [99], walks, 8 * D, args.walklen_cal_budget, stream=stream))
    target = int(cal["best_E"][0])
    speed = int(cal["evals"][0]) / t_cal
    sampler = ClockSampler(local)
    sampler.start()
    rows = {}
    for mult in (1, 2, 4, 8, 16, 32):
        wl = mult * D
        per_round = walks * wl * D
        max_rounds = max(1, int(args.walklen_seconds * speed / per_round))
        times, reached, evals = [], 0, []
        for sd in range(1, args.walklen_seeds + 1):
            r, t = timed(lambda: pkg.labs_walks(L, [sd], walks, wl, 1 << 62, target_E=target, max_rounds=max_rounds,
                                                stream=stream))
            ok = int(r["best_E"][0]) <= target
            reached += ok
            times.append(t if ok else float("inf"))
            evals.append(int(r["evals"][0]))
        rows["%dD" % mult] = {"walk_len": wl, "median_s": float(np.median(times)), "reached": reached,
                              "times_s": [None if x == float("inf") else x for x in times],
                              "median_evals": float(np.median(evals))}
    clocks = sampler.stop()
    best = min(rows, key=lambda k: rows[k]["median_s"])
    line = {
        "metric": "time_to_target_s", "value": rows["8D"]["median_s"], "unit": "s", "n_gpus": world, "steps": 1,
        "warmup": 1, "ms_per_step": None, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic (Philox starts, seeds 1..%d)" % args.walklen_seeds,
        "config": {"workload": "walklen_L%d_%dwalks" % (L, walks), "L": L, "walks": walks, "target_E": target,
                   "calibration": {"walk_len": 8 * D, "seed": 99, "budget": args.walklen_cal_budget,
                                   "evals_per_s": speed}},
        "by_walk_length": rows, "fastest": best, "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_variants(args, world, rank, local):
    """One lane per walk against one warp and one CTA per walk (labs_opts.kernel
    1, 3 and 4) and the library's timed choice (kernel 0): one round of --walk-len-variants
    steps at each L of --variants-L and each walk count of --variants-walks,
    evaluations per second of each (CUDA events around the call's kernels)."""
    import torch
    import paper_2210_15962_gb300 as pkg
    torch.cuda.set_device(local)
    pkg.load()
    stream = torch.cuda.Stream()
    rows = []
    sampler = ClockSampler(local)
    sampler.start()
    for L in [int(x) for x in args.variants_L.split(",")]:
        D = (L + 1) // 2
        wl = args.walk_len_variants
        for walks in [int(x) for x in args.variants_walks.split(",")]:
            row = {"L": L, "walks": walks, "walk_len": wl}
            ref = None
            for name, k in (("lane_per_walk", 1), ("warp_per_walk", 3), ("cta_per_walk", 4), ("library_choice", 0)):
                pkg.labs_walks(L, [7], walks, min(wl, 64), walks * min(wl, 64) * D, kernel=k, stream=stream)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = pkg.labs_walks(L, [7], walks, wl, walks * wl * D, kernel=k, stream=stream)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                row[name] = {"evals_per_s": int(r["evals"][0]) / (r["stats"]["walk_kernel_ms"] / 1e3),
                             "wall_s": dt}
                got = (int(r["best_E"][0]), r["best_seq"][0].tobytes(), int(r["evals"][0]))
                ref = ref or got
                row["same_results"] = row.get("same_results", True) and got == ref
            rows.append(row)
    clocks = sampler.stop()
    line = {"metric": "neighbour_evals_per_s", "value": None, "unit": "neighbour_evals/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic (Philox starts, seed 7)",
            "config": {"workload": "variants"}, "rows": rows, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--L", type=int, default=DEFAULT_L)
    ap.add_argument("--walks", type=int, default=WALKS)
    ap.add_argument("--walk-len", type=int, default=WALK_LEN)
    ap.add_argument("--budget", type=int, default=BUDGET)
    ap.add_argument("--ref-walks", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--device-only", action="store_true", help="skip the end-to-end (host buffer) measurement")
    ap.add_argument("--plain-only", action="store_true",
                    help="the plain workload alone, without the batched and serving sub-measurements")
    ap.add_argument("--workload", default="plain",
                    choices=["plain", "batched", "serving", "large", "table1", "walklen", "variants"])
    ap.add_argument("--variants-L", default="121,301,449,511")
    ap.add_argument("--variants-walks", default="256,1024,8192,65536")
    ap.add_argument("--walk-len-variants", type=int, default=2048)
    ap.add_argument("--walklen-cal-budget", type=int, default=10 ** 12)
    ap.add_argument("--walklen-seeds", type=int, default=4)
    ap.add_argument("--walklen-seconds", type=float, default=20.0)
    ap.add_argument("--table1-L", type=int, default=171)
    ap.add_argument("--table1-walks", type=int, default=233472)  # 3 full waves of the 3-word kernel
    ap.add_argument("--table1-seconds", type=float, default=300.0)
    ap.add_argument("--table1-seed", type=int, default=SEED, help="seed of rank 0 (rank r uses seed + r)")
    ap.add_argument("--kernel", type=int, default=0, help="0 library choice, 1 full scan, 2 incremental")
    ap.add_argument("--space", default="skew", choices=["skew", "full"],
                    help="plain workload over the skew-symmetric sequences or all length-L sequences")
    ap.add_argument("--large-cal-rounds", type=int, default=2)
    ap.add_argument("--large-seeds", type=int, default=8)
    ap.add_argument("--large-cap-s", type=float, default=45.0)
    ap.add_argument("--large-rpl", type=int, default=2)
    ap.add_argument("--walks-large", type=int, default=65536)
    ap.add_argument("--walk-len-large", type=int, default=16384)
    ap.add_argument("--serve-seconds", type=float, default=15.0)
    ap.add_argument("--rate", type=float, default=20.0)
    ap.add_argument("--serve-budget", type=int, default=10 ** 10)
    ap.add_argument("--target-budget", type=int, default=2 * 10 ** 9)
    ap.add_argument("--max-active", type=int, default=256)
    ap.add_argument("--mem-gib", type=int, default=64)
    ap.add_argument("--rounds-per-launch", type=int, default=4)
    ap.add_argument("--serve-walk-mode", type=int, default=0, choices=[0, 1, 2],
                    help="0: lane or warp per walk chosen per launch, 1: lane per walk, 2: warp per walk")
    ap.add_argument("--plain-requests", type=int, default=10)
    ap.add_argument("--capacity-requests", type=int, default=0, help="0: all of the stream's requests")
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--batch-walks", type=int, default=2048)
    ap.add_argument("--batch-walk-len", type=int, default=0, help="batched workload walk length, 0: 8*D")
    ap.add_argument("--batch-walk-mode", type=int, default=0, choices=[0, 1, 2, 3],
                    help="batched workload: 0 autotuned, 1 lane, 2 warp, 3 CTA per walk")
    ap.add_argument("--batch-block", type=int, default=0, help="batched workload: threads per CTA, 0 autotuned")
    ap.add_argument("--batch-table-factor", type=int, default=0,
                    help="batched workload: visited-table slots per pivot x10, 0 autotuned")
    ap.add_argument("--plain-instances", type=int, default=64)
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.workload == "batched" and args.impl != "reference":
        run_batched(args, world, rank, local)
        return
    if args.workload == "serving" and args.impl != "reference":
        run_serving(args, world, rank, local)
        return
    if args.workload == "large" and args.impl != "reference":
        run_large(args, world, rank, local)
        return
    if args.workload == "table1" and args.impl != "reference":
        run_table1(args, world, rank, local)
        return
    if args.workload == "walklen" and args.impl != "reference":
        run_walklen(args, world, rank, local)
        return
    if args.workload == "variants" and args.impl != "reference":
        run_variants(args, world, rank, local)
        return

    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import numpy as np
    import torch
    import paper_2210_15962_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.load()
    stream = torch.cuda.Stream()
    seed = rank_seed(rank)
    L = args.L
    walks, wl, budget = args.walks, args.walk_len, args.budget
    full = args.space == "full"
    flips = L if full else (L + 1) // 2  # neighbour evaluations per walk step
    ws_bytes = pkg.labs_walks_workspace_size(L, 1, walks, wl, space=args.space)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    seeds_d = torch.tensor([seed], dtype=torch.int64, device="cuda")
    best_seq_d = torch.zeros((1, L), dtype=torch.int8, device="cuda")
    best_E_d = torch.zeros(1, dtype=torch.int64, device="cuda")

    def device_step():
        return pkg.labs_walks_device(L, seeds_d, walks, wl, budget, best_seq_d, best_E_d, stream=stream,
                                     workspace=ws, kernel=args.kernel, space=args.space)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing
    for _ in range(args.warmup):
        device_step()
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    total_evals = 0
    launches = 0
    walk_ms = 0.0
    walk_launches = 0
    planes = 0
    for _ in range(args.steps):
        st = device_step()
        total_evals += st["evals"]
        planes += st["plane_steps"]
        launches += st["launches"]
        walk_ms += st["walk_kernel_ms"]
        walk_launches += st["walk_launches"]
    e1.record(stream)
    e1.synchronize()
    clocks = sampler.stop()
    dev_s = e0.elapsed_time(e1) / 1e3
    barrier()

    # ---- end to end through the public call with host buffers
    del ws
    torch.cuda.synchronize()
    e2e_evals = 0
    t0 = t1 = 0.0
    if not args.device_only:
        pkg.labs_walks(L, [seed], walks, wl, budget, kernel=args.kernel, space=args.space)  # maps the pool
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r = pkg.labs_walks(L, [seed], walks, wl, budget, kernel=args.kernel, space=args.space)
            e2e_evals += int(r["evals"].sum())
        t1 = time.perf_counter()
        barrier()
    h2d = 8 + 8 + 8          # seed, budget, target per problem
    d2h = L + 8 + 8 + 4 + 4  # best sequence, best E, evaluations, rounds, stop flag
    e2e_s = t1 - t0

    # ---- max over ranks, totals over ranks
    (dev_s, e2e_s), (tot_evals, tot_e2e) = combine_ranks([dev_s, e2e_s], [total_evals, e2e_evals], dist, "cuda")

    if rank == 0:
        value = tot_evals / dev_s
        per_launch_ms = walk_ms / max(walk_launches, 1)
        evals_per_launch = total_evals / max(walk_launches, 1)
        avg_planes = planes / max(total_evals / flips, 1.0)
        ops_per_eval = core_alu_ops_per_eval(L, avg_planes, full)
        achieved = evals_per_launch * ops_per_eval / (per_launch_ms / 1e3) / 1e12
        peak = SM_COUNT * INT_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
        traffic = (TRAFFIC["bytes_per_launch"] if (walk_sources_hash() == TRAFFIC["sources_sha256_prefix"]
                                                  and (L, walks, wl, full) == (DEFAULT_L, WALKS, WALK_LEN, False))
                   else None)
        kernel_name = ("full_walk_kernel<W=%d,K=4>" % ((L - 1 + 31) // 32) if full
                       else "walk_kernel<W=%d,K=4>" % (((L - 1) // 2 + 31) // 32))
        alu = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (int32 ALU-pipe lane-ops)",
               "frac": achieved / peak, "ops_per_eval": ops_per_eval,
               "basis": "4 LOP3 per 32 lags and digit plane; 152 SMs x 64 lanes/clk x 2070 MHz"}
        if full:
            # the full space's formulation has its own popcount count; its roofline stays in ALU lane-ops
            roofline = dict(alu, traffic=traffic, kernel=kernel_name, kernel_ms_per_launch=per_launch_ms,
                            avg_digit_planes=avg_planes)
        else:
            needed = popc_needed(L, evals_per_launch, planes / max(walk_launches, 1))
            roofline = popc_roofline(needed, per_launch_ms / 1e3, traffic=traffic, kernel=kernel_name,
                                     kernel_ms_per_launch=per_launch_ms, popc_per_eval=needed / evals_per_launch,
                                     avg_digit_planes=avg_planes, alu_lane_ops=alu)
        line = {
            "metric": "neighbour_evals_per_s", "value": value, "unit": "neighbour_evals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic (Philox-drawn uniform +-1 starts, seed %d per rank)" % SEED,
            "config": {"workload": ("plain_L121_131072x8192_budget1e11"
                                    if (L, walks, wl, budget, full) == (121, WALKS, WALK_LEN, BUDGET, False)
                                    else "plain_%sL%d_%dx%d_budget%d" % ("full_" if full else "", L, walks, wl,
                                                                          budget)),
                       "space": args.space,
                       "L": L, "walks": walks, "walk_len": wl,
                       "budget": budget, "rounds_per_step": int(round(total_evals / args.steps /
                                                                     (walks * wl * flips))),
                       "parallelism": "independent problem per GPU" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2: %.1f GiB of visited tables per round" % (ws_bytes / 2 ** 30)},
            "roofline": roofline,
            "e2e": ({"value": tot_e2e / e2e_s, "unit": "neighbour_evals/s", "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": d2h} if e2e_s > 0 else None),
            "gpu_launches": launches,
            "clocks": clocks,
        }
        if world == 1 and not args.plain_only and not full:
            # the batched and serving paths of the same library, each against
            # the plain path on the same problems
            sampler = ClockSampler(local)
            sampler.start()
            line["batched"] = measure_batched(args, rank, max(2, min(args.steps, 5)), 1)
            line["serving"] = measure_serving(args, 2)
            line["batched_serving_clocks"] = sampler.stop()
            line["gpu_launches_batched_serving"] = line["batched"]["launches"] + line["serving"]["gpu_launches"]
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(walk_len=wl, L=L, total_walks=walks, full=full, one_core=True)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
