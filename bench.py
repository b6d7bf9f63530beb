#!/usr/bin/env python
"""Throughput benchmark of the multislice-Leiden hot path on GB300.

A step is one complete solve of the synthetic power-law temporal workload
with T=64 snapshots of n=1,000,000 nodes (64M supra-nodes, ~1.15G stored
entries; degree-corrected SBM with power-law degrees (exponent 2.3, mean 16)
and community sizes, mixing 0.4, 5% edge churn per snapshot, weights 1..16,
ordinal coupling omega=1, gamma=1): supra-graph build from device-resident
snapshots, Leiden (two passes: local moving, refinement, aggregation) and
Q_MS.  The metric is local-moving supra-edges per second: the sum over all
local-moving rounds of the level's directed entries, divided by the whole
step's device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mslice|reference]
  python bench.py --workload plain-t16        (T=16, n=100,000: the smaller power-law recipe)
  python bench.py --workload batched [--scale S]
  python bench.py --workload serving [--scale S] [--requests R] [--slots K]
  python bench.py --workload large-sweep [--scale S]   (T=64 at omega 1/10, 1, 10, plain and batched)

The batched workload (64 temporal planted-partition graphs of uneven n and
T, each solved at 6 gammas x 3 omegas = 1,152 solves) is timed twice on the
same GPU: every solve as its own call (the plain path) and the solves packed
into batches (mslice_batch_*).  Both report the plain path's local-moving
supra-edges per second of wall time, and the batched labels and Q must equal
the plain ones bit for bit.

The reference arm is the CPU oracle (single thread) on a bounded sample of
the same recipe.  With N > 1 (torchrun) every rank solves its own replica;
the timed region is bracketed by barriers and the max over ranks is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# The plain workloads: the recipe, its config and the oracle's bounded sample
# (n scaled so that one single-thread oracle solve takes ~10-30 s).
PLAIN = {
    "plain": dict(
        recipe="powerlaw_t64_n1m", oracle_n=3000,
        config={"workload": "multislice Leiden, power-law temporal DC-SBM, T=64, n=1,000,000", "T": 64,
                "n": 1000000, "deg_exp": 2.3, "mean_deg": 16, "size_exp": 1.5, "sizes": "20-5000", "mixing": 0.4,
                "churn": 0.05, "weights": "1-16", "gamma": "1/1", "omega": "1/1", "n_iterations": 2, "K": 4,
                "seed": 0, "supra_nodes": 64000000}),
    "plain-t16": dict(
        recipe="powerlaw_t16_n100k", oracle_n=20000,
        config={"workload": "multislice Leiden, power-law temporal DC-SBM", "T": 16, "n": 100000, "deg_exp": 2.5,
                "mean_deg": 20, "size_exp": 1.5, "sizes": "20-5000", "mixing": 0.3, "churn": 0.05, "weights": "1-8",
                "gamma": "1/1", "omega": "1/1", "n_iterations": 2, "K": 4, "seed": 0, "supra_nodes": 1600000}),
}
METRIC = "supra-edges/s in Leiden local-move"
UNIT = "supra-edges/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mslice", choices=["mslice", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="plain workload: skip the three-omega plain-vs-batched comparison")
    ap.add_argument("--no-serving", action="store_true",
                    help="plain workload: skip the serving measurement at n/20")
    ap.add_argument("--workload", default="plain",
                    choices=["plain", "plain-t16", "batched", "serving", "large-sweep", "school"])
    ap.add_argument("--null", default="multislice", choices=["multislice", "global", "cpm"],
                    help="plain workload: Q_MS (default), the supra-graph's plain modularity, or temporal CPM")
    ap.add_argument("--theta", default=None,
                    help="plain workload: randomised refinement theta as num/den (default: the greedy limit)")
    ap.add_argument("--coupling", default="ordinal", choices=["ordinal", "categorical", "tables"],
                    help="plain workload: ordinal omega (default), categorical coupling of every snapshot pair, "
                         "or the general form's tables (per-pair omega, per-snapshot gamma)")
    ap.add_argument("--requests", type=int, default=4, help="serving workload: timed snapshots per graph")
    ap.add_argument("--slots", type=int, default=2, help="serving workload: server workers")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="node-count scale of every graph (batched and serving workloads; plain workloads: "
                         "--profile-run only, for small profiler captures)")
    ap.add_argument("--graphs", type=int, default=None, help="batched workload: first G graphs only")
    ap.add_argument("--batch-nodes", type=int, default=BATCH_MAX_NODES,
                    help="batched workload: supra-nodes packed into one batch at most")
    ap.add_argument("--batch-entries", type=int, default=BATCH_MAX_ENTRIES,
                    help="batched workload: stored entries packed into one batch at most")
    ap.add_argument("--profile-run", action="store_true",
                    help="one solve of the workload and exit (a short target for ncu captures)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Ranks:
    """The replicas' process group: one rank per GPU, each solving its own
    copy of the workload, with no collective on the data path -- only the
    barriers around the timed region and the reductions of the reported
    numbers.  dist is torch.distributed (None for one rank); device is where
    the reduction tensors live ("cuda" under NCCL, "cpu" under gloo)."""

    def __init__(self, dist=None, device="cuda"):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def _reduce(self, x, op):
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.MAX)

    def sum(self, x):
        return self._reduce(x, None if self.dist is None else self.dist.ReduceOp.SUM)


def replica_throughput(ranks, ms, units):
    """Whole-job throughput of weak-scaled replicas: the units every rank
    processed divided by the slowest rank's time (ms).  Returns (units per
    second, slowest ms, total units)."""
    ms_max = ranks.max(ms)
    total = ranks.sum(units)
    return total / (ms_max / 1e3), ms_max, total


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Committed ncu summaries of one decision round per plain workload; each
# holds a "traffic_bytes_per_launch:" line (DRAM bytes of one sub-round's
# decision launches, null once the kernels changed after the capture).
TRAFFIC_PROFILES = {"plain": "local_move_decide_powerlaw_t64_n1m.md",
                    "plain-t16": "local_move_decide_powerlaw_t16_n100k.md"}


def decide_traffic(args):
    """DRAM bytes per launch of the decision kernel from the committed ncu
    summary of this workload (None when absent)."""
    p = os.path.join(ROOT, "profiles", TRAFFIC_PROFILES.get(args.workload, ""))
    try:
        for line in open(p):
            if line.startswith("traffic_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null") else float(v)
    except OSError:
        pass
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        # the raw samples go to MSLICE_BENCH_OUT (default: the temp directory)
        out = os.environ.get("MSLICE_BENCH_OUT") or __import__("tempfile").gettempdir()
        self.path = os.path.join(out, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for name, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# General-form tables of the plain workloads (--coupling tables): omega^(s,s+1)
# alternating 1/2 and 3/2, gamma^(s) cycling 3/4, 1, 5/4.
def table_omegas(T):
    return [1 if s % 2 == 0 else 3 for s in range(T - 1)]  # over omega_den 2


def table_gammas(T):
    return [[(3, 4), (1, 1), (5, 4)][s % 3] for s in range(T)]


def plain_spec(args):
    return PLAIN[args.workload]


def gen_kwargs(args):
    """(build kwargs, solve kwargs shared by the library and the oracle) of the
    plain workload's model."""
    build, solve = {}, {"null": args.null}
    T = plain_spec(args)["config"]["T"]
    if args.theta:
        num, den = (args.theta.split("/") + ["1"])[:2]
        solve["theta"] = (int(num), int(den))
    if args.coupling == "categorical":
        build["coupling"] = "categorical"
    elif args.coupling == "tables":
        solve.update(omega=(1, 2), omegas=table_omegas(T))
        if args.null != "global":
            solve["gammas"] = table_gammas(T)
    return build, solve


def oracle_kwargs(args):
    build, solve = gen_kwargs(args)
    return {**solve, **build}


def workload(args):
    """The plain workload's config; the null model and coupling are named when
    they are not Q_MS with ordinal omega."""
    c = dict(plain_spec(args)["config"])
    if args.null == "multislice" and args.coupling == "ordinal" and not args.theta:
        return c
    if args.theta:
        c.update(workload=c["workload"] + ", randomised refinement", theta=args.theta)
    if args.null != "multislice":
        what = {"global": "global null model (plain modularity of the supra-graph)",
                "cpm": "temporal Constant Potts Model"}[args.null]
        c.update(workload=c["workload"] + ", " + what, null_model=args.null)
    if args.coupling == "categorical":
        c.update(workload=c["workload"] + ", categorical coupling", coupling="categorical")
    elif args.coupling == "tables":
        c.update(workload=c["workload"] + ", per-pair omega and per-snapshot gamma",
                 omega="per pair: 1/2, 3/2 alternating",
                 gamma="per snapshot: 3/4, 1, 5/4 cycling" if args.null != "global" else c["gamma"])
    return c


def oracle_sample(args):
    """The oracle's bounded sample of the plain workload: the same recipe with
    n scaled down (every snapshot kept)."""
    from paper_2608_03695_gb300 import synth
    spec = plain_spec(args)
    return synth.recipe_graph(spec["recipe"], scale_n=spec["oracle_n"]), spec["oracle_n"], spec["config"]["T"]


def cpu_baseline(args):
    import oracle
    snaps, n, T = oracle_sample(args)
    t = time.perf_counter()
    _, _, st = oracle.leiden(snaps, **oracle_kwargs(args))
    el = time.perf_counter() - t
    return {"value": st["lm_edges"] / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one oracle solve of the same recipe at n={n}, T={T} "
                      f"({st['lm_edges']} local-move supra-edges in {el:.1f} s, single thread)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    snaps, n, T = oracle_sample(args)
    for _ in range(args.warmup):
        oracle.leiden(snaps, n_iterations=1, max_rounds=2, **oracle_kwargs(args))  # short warm-up (page-in)
    edges, secs = 0, 0.0
    for _ in range(args.steps):
        t = time.perf_counter()
        _, _, st = oracle.leiden(snaps, **oracle_kwargs(args))
        secs += time.perf_counter() - t
        edges += st["lm_edges"]
    v = edges / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {**workload(args), "n": n, "supra_nodes": n * T,
                       "note": "bounded sample of the same recipe (n scaled) for the single-thread CPU oracle"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} oracle solves at n={n}, T={T}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _gen_batched(spec):
    from paper_2608_03695_gb300 import synth
    return synth.batched_graph(spec)


# Packing of the batched path: a batch holds at most 2^21 supra-nodes and 2^26
# stored entries, so its randomly accessed state (labels, sizes, the hashed
# community tables: ~50 B per supra-node) stays in the 129 MB L2; a graph
# larger than that is solved as a batch of one.
BATCH_MAX_NODES = 1 << 21
BATCH_MAX_ENTRIES = 1 << 26


def run_batched(args):
    import multiprocessing as mp
    import hashlib
    from paper_2608_03695_gb300 import synth
    specs = synth.batched_specs(args.scale, args.graphs)
    t = time.perf_counter()
    # the pool starts (spawn) before this process touches CUDA
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        graphs = pool.map(_gen_batched, specs, chunksize=1)
    t_gen = time.perf_counter() - t
    import torch
    import paper_2608_03695_gb300 as pkg
    torch.cuda.set_device(0)
    handles = [pkg.mslice_build(g) for g in graphs]
    solves = [(gi, gm, om) for gi in range(len(graphs)) for gm in synth.BATCHED_GAMMAS for om in synth.BATCHED_OMEGAS]
    N_sum = sum(h.N for h in handles) * len(synth.BATCHED_GAMMAS) * len(synth.BATCHED_OMEGAS)

    def digest(lab, Q):
        return hashlib.sha1(np.ascontiguousarray(lab, dtype=np.int32).tobytes()).hexdigest(), Q

    # warm-up: one small solve each way
    handles[0].mslice_leiden()
    with pkg.Batch() as b:
        b.add(handles[0])
        b.run()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    # plain path: one call per solve
    t = time.perf_counter()
    plain, work, launches_plain, host_plain = [], 0, 0, 0
    for gi, gm, om in solves:
        lab, Q, st = handles[gi].mslice_leiden(gamma=gm, omega=om)
        plain.append(digest(lab, Q))
        work += st["lm_edges"]
        launches_plain += st["kernel_launches"]
        host_plain += st["host_launches"]
    t_plain = time.perf_counter() - t
    # batched path: solves packed in add order under the per-batch budget
    chunks, cur, cn, ce = [], [], 0, 0
    for k, (gi, gm, om) in enumerate(solves):
        h = handles[gi]
        if cur and (cn + h.N > args.batch_nodes or ce + h.nnz > args.batch_entries):
            chunks.append(cur)
            cur, cn, ce = [], 0, 0
        cur.append(k)
        cn += h.N
        ce += h.nnz
    if cur:
        chunks.append(cur)
    t = time.perf_counter()
    batched, launches_b, host_b = [None] * len(solves), 0, 0
    ms_dev = 0.0
    for ch in chunks:
        with pkg.Batch() as b:
            for k in ch:
                gi, gm, om = solves[k]
                b.add(handles[gi], gm, om)
            st = b.run()
            launches_b += st["kernel_launches"]
            host_b += st["host_launches"]
            ms_dev += st["ms_total"]
            labs, Qs = b.results()
            _, _, off = b.info()
        for j, k in enumerate(ch):
            batched[k] = digest(labs[off[j]:off[j + 1]], float(Qs[j]))
    t_batch = time.perf_counter() - t
    clk = clocks.stop()
    same = all(a == b for a, b in zip(plain, batched))
    for h in handles:
        h.close()
    v_plain, v_batch = work / t_plain, work / t_batch
    cfg = {"workload": "batched multislice Leiden: 64 temporal planted-partition graphs x 6 gamma x 3 omega",
           "graphs": len(graphs), "solves": len(solves), "n": "log-uniform 1k-200k" + (f" x {args.scale}" if args.scale != 1 else ""),
           "T": "uniform 2-32", "mean_deg": "uniform 8-32", "weights": "1-8",
           "gamma": [f"{a}/{b}" for a, b in synth.BATCHED_GAMMAS], "omega": [f"{a}/{b}" for a, b in synth.BATCHED_OMEGAS],
           "supra_nodes_per_graph_sum": sum(g[0].n * len(g) for g in graphs),
           "supra_nodes_solved": N_sum, "batches": len(chunks), "n_iterations": 2, "K": 4, "seed": 0,
           "parallelism": "single", "l2": "inputs larger than L2"}
    line = {"metric": "supra-edges/s in Leiden local-move, batched vs plain", "value": v_batch, "unit": UNIT,
            "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * t_batch, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": cfg,
            "plain": {"value": v_plain, "unit": UNIT, "seconds": t_plain, "gpu_launches": launches_plain,
                      "host_launches": host_plain},
            "batched": {"value": v_batch, "unit": UNIT, "seconds": t_batch, "gpu_launches": launches_b,
                        "host_launches": host_b, "device_ms": ms_dev,
                        "packing": {"max_nodes": args.batch_nodes, "max_entries": args.batch_entries}},
            "batched_over_plain": v_batch / v_plain, "identical_results": same,
            "work_supra_edges": work, "generate_s": t_gen, "clocks": clk}
    print(json.dumps(line), flush=True)
    if not same:
        raise SystemExit("batched results differ from the plain solves")


def _gen_serving(job):
    from paper_2608_03695_gb300 import synth
    spec, steps = job
    return synth.serving_stream(spec, steps)


def run_serving(args):
    line = serving_measurement(args)
    print(json.dumps(line), flush=True)
    if not line["identical_results"]:
        raise SystemExit("served results differ between open loop, burst and plain paths")


def serving_measurement(args):
    """Serving workload: 32 live graphs with windows of 8 slices.  The first
    8 snapshots of every graph fill the windows (untimed); then R snapshots per
    graph arrive as a Poisson process at the recipe's rate (open loop) and
    latency is taken per request (submit to done).  The same R x 32 requests
    are then timed as one burst on a fresh server (capacity) and one by one
    through mslice_build + mslice_leiden_ex (the plain per-instance path);
    all three must give the same labels."""
    import multiprocessing as mp
    import hashlib
    from paper_2608_03695_gb300 import synth
    W = synth.SERVING["window"]
    specs = synth.serving_specs(args.scale, args.graphs)
    steps = W + args.requests
    t = time.perf_counter()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        streams = pool.map(_gen_serving, [(sp, steps) for sp in specs], chunksize=1)
    t_gen = time.perf_counter() - t
    import torch
    import paper_2608_03695_gb300 as pkg
    torch.cuda.set_device(0)
    G = len(streams)
    rng = np.random.default_rng(11)

    def digest(lab):
        return hashlib.sha1(np.ascontiguousarray(lab, dtype=np.int32).tobytes()).hexdigest()

    def prefill(srv):
        ids = [srv.add_graph(s[0].n) for s in streams]
        for t in range(W):
            rids = [srv.submit(ids[g], streams[g][t]) for g in range(G)]
            for r in rids:
                srv.wait(r)
        return ids

    # timed requests: graph g's snapshots W..W+R-1 in a random interleaving
    order = [g for g in range(G) for _ in range(args.requests)]
    rng.shuffle(order)
    seq, nxt = [], [W] * G
    for g in order:
        seq.append((g, nxt[g]))
        nxt[g] += 1
    rate = synth.SERVING["rate_per_s"]
    gaps = rng.exponential(1.0 / rate, size=len(seq))
    clocks = ClockSampler(0)
    clocks.start()
    # open loop at the recipe's rate
    with pkg.Server(window=W, n_slots=args.slots) as srv:
        ids = prefill(srv)
        t0 = time.perf_counter()
        due = t0
        rids = []
        for (g, t), gap in zip(seq, gaps):
            due += gap
            d = due - time.perf_counter()
            if d > 0:
                time.sleep(d)
            rids.append(srv.submit(ids[g], streams[g][t]))
        res = [srv.wait(r) for r in rids]
        t_open = time.perf_counter() - t0
    lat = np.array([i["t_done"] - i["t_submit"] for _, i in res])
    svc = np.array([i["t_done"] - i["t_admit"] for _, i in res])
    wait = np.array([i["t_admit"] - i["t_submit"] for _, i in res])
    open_digest = [digest(l) for l, _ in res]
    batch_sizes = [i["batch_size"] for _, i in res]
    slots_used = len({i["slot"] for _, i in res})
    # overlap: total device-busy span of batches vs their summed durations
    spans = sorted({(i["slot"], i["t_batch_start"], i["t_batch_end"]) for _, i in res}, key=lambda x: x[1])
    busy = sum(e - b for _, b, e in spans)
    union, cur_b, cur_e = 0.0, None, None
    for _, b, e in spans:
        if cur_e is None or b > cur_e:
            if cur_e is not None:
                union += cur_e - cur_b
            cur_b, cur_e = b, e
        else:
            cur_e = max(cur_e, e)
    if cur_e is not None:
        union += cur_e - cur_b
    # closed loop: all requests at once (capacity of the server)
    with pkg.Server(window=W, n_slots=args.slots) as srv:
        ids = prefill(srv)
        t0 = time.perf_counter()
        rids = [srv.submit(ids[g], streams[g][t]) for g, t in seq]
        burst = [srv.wait(r) for r in rids]
        t_burst = time.perf_counter() - t0
    same = [digest(l) for l, _ in burst] == open_digest
    # plain per-instance path: window build + warm-started solve, one by one
    # (the prefill chain is replayed untimed to get the same warm starts)
    prevs = {}
    for g in range(G):
        lab, n = None, streams[g][0].n
        for t in range(W):
            lab = _plain_window_solve(pkg, streams[g], t, W, lab, n)[0]
        prevs[g] = lab
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain = []
    cyc = {"ms_total": 0.0, "ms_capped": 0.0, "capped_levels": 0, "capped_rounds": 0, "lm_rounds": 0}
    for g, t in seq:
        n = streams[g][0].n
        lab, _, st = _plain_window_solve(pkg, streams[g], t, W, prevs[g], n)
        prevs[g] = lab
        plain.append(digest(lab))
        for key in cyc:
            cyc[key] += st[key]
    t_plain = time.perf_counter() - t0
    same = same and plain == open_digest
    clk = clocks.stop()
    nreq = len(seq)
    cfg = {"workload": "serving: live temporal planted-partition graphs, sliding windows, Poisson arrivals",
           "graphs": G, "window": W, "n": "log-uniform 10k-2M" + (f" x {args.scale}" if args.scale != 1 else ""),
           "mean_deg": synth.SERVING["mean_deg"], "churn": synth.SERVING["churn"], "weights": "1-8",
           "gamma": "1/1", "omega": "1/1", "rate_per_s": rate, "timed_requests": nreq,
           "requests_per_graph": args.requests, "slots": args.slots, "n_iterations": 2, "K": 4, "seed": 0,
           "parallelism": "single", "l2": "inputs larger than L2"}
    line = {"metric": "served snapshots/s (Poisson arrivals) with p50/p99 latency", "value": nreq / t_open,
            "unit": "snapshots/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": 1e3 * t_open,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": cfg,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max()), "mean": float(lat.mean()),
                          "note": "submit to done; includes queueing when the offered rate exceeds capacity"},
            "service_s": {"p50": float(np.percentile(svc, 50)), "p99": float(np.percentile(svc, 99)),
                          "note": "admitted to done (the batch's solve)"},
            "queue_wait_s": {"p50": float(np.percentile(wait, 50)), "p99": float(np.percentile(wait, 99))},
            "offered_per_s": rate, "achieved_per_s": nreq / t_open,
            "capacity": {"value": nreq / t_burst, "unit": "snapshots/s", "note": "all timed requests at once"},
            "plain": {"value": nreq / t_plain, "unit": "snapshots/s",
                      "note": "one mslice_build + mslice_leiden_ex per request, same warm starts"},
            "served_over_plain": (nreq / t_burst) / (nreq / t_plain),
            "capped_levels": {"levels": cyc["capped_levels"], "rounds": cyc["capped_rounds"],
                              "of_rounds": cyc["lm_rounds"], "ms": cyc["ms_capped"],
                              "share_of_solve": cyc["ms_capped"] / max(cyc["ms_total"], 1e-9),
                              "note": "plain window solves: local-moving levels that stopped at max_rounds with "
                                      "nodes still moving"},
            "batching": {"mean_batch": float(np.mean(batch_sizes)), "max_batch": int(max(batch_sizes)),
                         "slots_used": slots_used, "device_busy_s": busy, "busy_union_s": union,
                         "overlap": busy / union if union > 0 else 1.0},
            "identical_results": same, "generate_s": t_gen, "clocks": clk}
    return line


def _plain_window_solve(pkg, snaps, t, W, prev, n):
    """One request through the plain path: build the window's handle and run
    mslice_leiden_ex from the warm-start labels."""
    window = snaps[max(0, t + 1 - W):t + 1]
    init = None
    if prev is not None:
        w_prev = len(prev) // n
        e = 1 if w_prev == W else 0
        src = np.minimum(np.arange(len(window)) + e, w_prev - 1)
        init = np.concatenate([prev[s * n:(s + 1) * n] for s in src]).astype(np.int32)
    with pkg.mslice_build(window) as h:
        lab, Q, st = h.mslice_leiden(init=init)
    return lab, Q, st


def run_large(args):
    """The T=64, n=1,000,000 power-law recipe (64M supra-nodes, ~1.15G stored
    entries) at omega = 1/10, 1 and 10: three plain solves on one handle, then
    the same three as one batch when the device has room for it; both must
    give the same labels and Q."""
    import hashlib
    import torch
    import paper_2608_03695_gb300 as pkg
    from paper_2608_03695_gb300 import synth
    n = int(synth.RECIPES["powerlaw_t64_n1m"]["n"] * args.scale)
    t = time.perf_counter()
    snaps = synth.recipe_graph("powerlaw_t64_n1m", scale_n=n)
    t_gen = time.perf_counter() - t
    torch.cuda.set_device(0)
    omegas = [(1, 10), (1, 1), (10, 1)]
    clocks = ClockSampler(0)
    clocks.start()
    t = time.perf_counter()
    h = pkg.mslice_build(snaps)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t
    del snaps

    def digest(lab):
        return hashlib.sha1(np.ascontiguousarray(lab, dtype=np.int32).tobytes()).hexdigest()

    plain, work, ms_plain = [], 0, 0.0
    t = time.perf_counter()
    for om in omegas:
        lab, Q, st = h.mslice_leiden(omega=om)
        plain.append((digest(lab), Q))
        work += st["lm_edges"]
        ms_plain += st["ms_total"]
    t_plain = time.perf_counter() - t
    free, _ = torch.cuda.mem_get_info()
    need = 3 * (300 * h.N + 60 * h.nnz)
    batched = None
    if free > need:
        t = time.perf_counter()
        with pkg.Batch() as b:
            for om in omegas:
                b.add(h, (1, 1), om)
            st = b.run()
            batched = [(digest(b.results(i)[0]), b.results(i)[1]) for i in range(3)]
        t_batch = time.perf_counter() - t
    clk = clocks.stop()
    same = batched is None or batched == plain
    line = {"metric": "supra-edges/s in Leiden local-move (large)", "value": work / t_plain, "unit": UNIT,
            "n_gpus": 1, "steps": 3, "warmup": 0, "ms_per_step": 1e3 * t_plain / 3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "multislice Leiden, power-law temporal DC-SBM, T=64", "n": n, "T": 64,
                       "deg_exp": 2.3, "mean_deg": 16, "mixing": 0.4, "churn": 0.05, "weights": "1-16",
                       "gamma": "1/1", "omega": ["1/10", "1/1", "10/1"], "supra_nodes": h.N, "entries": h.nnz,
                       "parallelism": "single", "l2": "inputs larger than L2"},
            "plain": {"seconds": t_plain, "device_ms": ms_plain, "Q": [q for _, q in plain]},
            "batched": (None if batched is None else
                        {"value": work / t_batch, "unit": UNIT, "seconds": t_batch, "device_ms": st["ms_total"]}),
            "batched_note": None if batched is not None else f"skipped: {free / 1e9:.0f} GB free, ~{need / 1e9:.0f} GB needed",
            "identical_results": same, "build_s": t_build, "generate_s": t_gen, "clocks": clk}
    h.close()
    print(json.dumps(line), flush=True)
    if not same:
        raise SystemExit("batched results differ from the plain solves")


def run_school(args):
    """The school-shaped contact sequence (n = 327, T = 7,375: 2.4M supra-nodes,
    4.8M coupling entries against 0.38M contact entries), the paper's
    long-sequence case: solved whole (the timed steps) and in windows of 64
    snapshots at stride 32 (mslice_leiden_windowed), whose stitched labels are
    scored by Q_MS of the whole sequence."""
    import torch
    import oracle
    import paper_2608_03695_gb300 as pkg
    from paper_2608_03695_gb300 import synth
    torch.cuda.set_device(0)
    snaps = synth.recipe_graph("school_t7375_n327")
    if args.profile_run:  # one build and one solve, for profilers
        with pkg.mslice_build(snaps) as h:
            _, Q, st = h.mslice_leiden()
        print(json.dumps({"profile_run": True, "workload": "school", "Q": Q, "kernel_launches": st["kernel_launches"],
                          "ms_total": st["ms_total"]}), flush=True)
        return
    stream = torch.cuda.Stream()

    def solve():
        h = pkg.mslice_build(snaps, stream=stream.cuda_stream)
        lab, Q, st = h.mslice_leiden()
        launches = h.kernel_launches
        h.close()
        return lab, Q, st, launches

    for _ in range(max(args.warmup, 3)):
        solve()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    work, launches = 0, 0
    for _ in range(args.steps):
        lab, Q, st, nl = solve()
        work += st["lm_edges"]
        launches += nl
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # windowed: W = 64, stride 32
    pkg.leiden_windowed(snaps, 64, 32)
    t = time.perf_counter()
    wlab, wQ, wst = pkg.leiden_windowed(snaps, 64, 32)
    t_win = time.perf_counter() - t
    clk = clocks.stop()
    with pkg.mslice_build(snaps) as h:
        Q_win_whole = h.mslice_modularity(wlab)
    N = 327 * len(snaps)
    line = {"metric": "supra-edges/s in Leiden local-move (school-shaped, T=7375)", "value": work / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "multislice Leiden, school-shaped contact sequence", "n": 327, "T": len(snaps),
                       "classes": 9, "static_pairs": 7004, "contacts": int(sum(x.nnz for x in snaps) // 2),
                       "gamma": "1/1", "omega": "1/1", "supra_nodes": N, "parallelism": "single",
                       "l2": "working set below L2 (2.4M supra-nodes); every step rebuilds from host arrays"},
            "Q": Q, "communities": int(lab.max()) + 1, "gpu_launches": launches,
            "solve": {"levels": st["levels"], "lm_rounds": st["lm_rounds"], "ms_total": st["ms_total"]},
            "windowed": {"W": 64, "stride": 32, "windows": len(wQ), "seconds": t_win,
                         "Q_whole_sequence": Q_win_whole, "communities": int(wlab.max()) + 1,
                         "lm_edges": wst["lm_edges"]},
            "clocks": clk}
    if not args.no_cpu_baseline:
        sample = synth.recipe_graph("school_t7375_n327", T=1000)
        t = time.perf_counter()
        _, _, ost = oracle.leiden(sample)
        el = time.perf_counter() - t
        line["cpu_baseline"] = {"value": ost["lm_edges"] / el, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"one oracle solve of the first 1,000 snapshots' recipe (T = 1,000) "
                                          f"({ost['lm_edges']} supra-edges in {el:.1f} s, single thread)"}
    print(json.dumps(line), flush=True)


# n scale of the serving measurement that the default run adds
SERVING_SUB_SCALE = 0.05

# Config 4's own comparison: the same graph at omega = 1/10, 1 and 10, solved
# plain (one call per omega) and as one batch of the three instances.
PLAIN_VS_BATCHED_OMEGAS = [(1, 10), (1, 1), (10, 1)]


def plain_vs_batched(pkg, dsnaps, stream, skw):
    """Times the three omegas as three plain solves and as one batch on a
    handle built from the device-resident snapshots (CUDA events on the
    library's stream), and checks that the batch gives the plain labels and Q
    bit for bit.  Not part of the timed region of the headline metric."""
    import hashlib
    import torch

    def digest(lab):
        return hashlib.sha1(np.ascontiguousarray(lab.cpu().numpy() if hasattr(lab, "cpu") else lab,
                                                 dtype=np.int32).tobytes()).hexdigest()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain, edges, st_plain = [], 0, []
    # the plain solves on a handle of their own, closed (with its solver
    # scratch) before the batch is built
    with pkg.mslice_build(dsnaps, device_ptrs=True, stream=stream.cuda_stream) as hp:
        e0.record(stream)
        for om in PLAIN_VS_BATCHED_OMEGAS:
            lab, Q, st = hp.mslice_leiden(omega=om, **skw)
            plain.append((digest(lab), Q))
            edges += st["lm_edges"]
            st_plain.append(st)
        e1.record(stream)
        torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    h = pkg.mslice_build(dsnaps, device_ptrs=True, stream=stream.cuda_stream)
    try:
        try:
            with pkg.Batch(stream=stream.cuda_stream) as b:
                for om in PLAIN_VS_BATCHED_OMEGAS:
                    b.mslice_batch_add(h, (1, 1), om)
                e0.record(stream)
                bst = b.mslice_batch_run(**skw)
                e1.record(stream)
                torch.cuda.synchronize()
                ms_batch = e0.elapsed_time(e1)
                batched = [(digest(b.results(i)[0]), b.results(i)[1]) for i in range(len(PLAIN_VS_BATCHED_OMEGAS))]
        except pkg.MsliceError as ex:  # a batch that does not fit the device
            return {"omegas": ["1/10", "1/1", "10/1"], "plain_ms": ms_plain, "batched": None,
                    "batched_note": f"not run: {ex}"}
        return {"omegas": ["1/10", "1/1", "10/1"], "plain_ms": ms_plain, "batched_ms": ms_batch,
                "speedup": ms_plain / ms_batch, "plain_value": edges / (ms_plain / 1e3),
                "batched_value": edges / (ms_batch / 1e3), "unit": UNIT, "identical_results": batched == plain,
                "Q": [q for _, q in plain],
                "kernel_launches": {"plain": sum(x["kernel_launches"] for x in st_plain),
                                    "batched": bst["kernel_launches"]},
                "host_launches": {"plain": sum(x["host_launches"] for x in st_plain),
                                  "batched": bst["host_launches"]}}
    finally:
        h.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "large-sweep":
        return run_large(args)
    if args.workload == "school":
        return run_school(args)
    import torch
    import paper_2608_03695_gb300 as pkg
    from paper_2608_03695_gb300 import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ranks = Ranks(dist, "cuda")
    barrier, max_over_ranks, sum_over_ranks = ranks.barrier, ranks.max, ranks.sum

    t_gen = time.perf_counter()
    n_full = plain_spec(args)["config"]["n"]
    snaps = synth.recipe_graph(plain_spec(args)["recipe"],
                               scale_n=None if args.scale == 1.0 else max(8, int(round(n_full * args.scale))))
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.Stream()
    if args.scale != 1.0 and not args.profile_run:
        raise SystemExit("--scale applies to a plain workload's --profile-run only")
    if args.profile_run:
        bkw, skw = gen_kwargs(args)
        with pkg.mslice_build(snaps, **bkw) as h:
            _, Q, st = h.mslice_leiden(**skw)
        print(json.dumps({"profile_run": True, "Q": Q, "kernel_launches": st["kernel_launches"],
                          "ms_total": st["ms_total"]}), flush=True)
        return

    class DevSnap:
        def __init__(self, s, pin=False, device=None):
            conv = (lambda a: torch.from_numpy(a).pin_memory()) if pin else (lambda a: torch.from_numpy(a).to(device))
            self.indptr, self.indices, self.weights = conv(s.indptr), conv(s.indices), conv(s.weights)

    dsnaps = [DevSnap(s, device="cuda") for s in snaps]
    N = snaps[0].n * len(snaps)
    # level-0 supra-CSR: int64 row pointers and 8-byte {column, weight} entries
    # (intra-snapshot entries plus two per ordinal coupling pair)
    csr_bytes = 8 * (N + 1) + 8 * (sum(s.nnz for s in snaps) + 2 * snaps[0].n * (len(snaps) - 1))
    dlabels = torch.empty(N, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def step_device(profile=False):
        h = pkg.mslice_build(dsnaps, device_ptrs=True, stream=stream.cuda_stream, **gen_kwargs(args)[0])
        _, Q, st = h.mslice_leiden(out=dlabels, profile=profile, **gen_kwargs(args)[1])
        launches = h.kernel_launches
        h.close()
        return st, launches, Q

    for _ in range(max(args.warmup, 3)):
        step_device()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    edges = launches = 0
    Qs = []
    for _ in range(args.steps):
        st, nl, Q = step_device()
        edges += st["lm_edges"]
        launches += nl
        Qs.append(Q)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    value, ms_max, total_edges = replica_throughput(ranks, ms, edges)

    # decision-kernel roofline from one profiled step (not part of the timed region)
    stp, _, _ = step_device(profile=True)
    peak, peak_kind = measured_peak()
    achieved = stp["decide_bytes"] / (stp["ms_decide"] / 1e3) / 1e9 if stp["ms_decide"] > 0 else 0.0
    # counters taken under Q_MS with ordinal omega only
    traffic = (decide_traffic(args) if args.null == "multislice" and args.coupling == "ordinal" and not args.theta
               else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (traffic if traffic is None else traffic), "peak_source": peak_kind,
                "kernel": "local-moving decision, level-0 sub-round (all degree tiers)",
                "launches": stp["decide_launches"], "bytes_per_launch": stp["decide_bytes"] / max(1, stp["decide_launches"]),
                "ms_per_launch": stp["ms_decide"] / max(1, stp["decide_launches"])}

    # end to end through the C ABI: pinned host inputs, host labels out
    e2e = None
    if not args.no_e2e:
        hsnaps = [DevSnap(s, pin=True) for s in snaps]
        hlabels = torch.empty(N, dtype=torch.int32).pin_memory()
        h2d = sum(8 * s.indptr.size + 4 * s.indices.size + 4 * s.weights.size for s in snaps)
        d2h = 4 * N + 8

        def step_e2e():
            h = pkg.mslice_build(hsnaps, host_tensors=True, stream=stream.cuda_stream, **gen_kwargs(args)[0])
            _, Q, st = h.mslice_leiden(out=hlabels, **gen_kwargs(args)[1])
            h.close()
            return st

        step_e2e()
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        e_edges = 0
        k_e2e = max(2, args.steps // 4)
        for _ in range(k_e2e):
            e_edges += step_e2e()["lm_edges"]
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t)
        e2e = {"value": sum_over_ranks(e_edges) / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k_e2e, "ms_per_step": 1e3 * el / k_e2e}

    pvb = serving = None
    default_model = args.null == "multislice" and args.coupling == "ordinal" and not args.theta
    if args.workload == "plain" and rank == 0 and not args.no_batched and default_model:
        torch.cuda.empty_cache()
        pvb = plain_vs_batched(pkg, dsnaps, stream, {})
    if args.workload == "plain" and rank == 0 and not args.no_serving and default_model:
        # the serving workload with every live graph's n scaled by 1/20 (the
        # full-size run takes --workload serving)
        sargs = argparse.Namespace(**vars(args))
        sargs.scale, sargs.requests, sargs.slots, sargs.graphs = SERVING_SUB_SCALE, 4, 2, None
        sv = serving_measurement(sargs)
        serving = {"scale_n": SERVING_SUB_SCALE, "note": "serving workload with every live graph's n scaled by "
                   "1/20; full size: bench.py --workload serving", "achieved_per_s": sv["achieved_per_s"],
                   "offered_per_s": sv["offered_per_s"], "latency_s": sv["latency_s"], "service_s": sv["service_s"],
                   "capacity_per_s": sv["capacity"]["value"], "plain_per_s": sv["plain"]["value"],
                   "served_over_plain": sv["served_over_plain"], "overlap": sv["batching"]["overlap"],
                   "capped_levels": sv["capped_levels"],
                   "timed_requests": sv["config"]["timed_requests"], "identical_results": sv["identical_results"]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {**workload(args), "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": f"inputs larger than L2 (level-0 supra-CSR {csr_bytes / 1e9:.2f} GB vs 129 MB L2)"},
            "generate_s": t_gen,
            "Q": Qs[-1] if Qs else None, "gpu_launches": int(sum_over_ranks(launches)),
            "local_move_only": {"value": stp["lm_edges"] / (stp["ms_local_move"] / 1e3), "unit": UNIT,
                                "note": "same edges over local-moving device time only (profiled step)"},
            "phases_ms": {k: round(stp["ms_" + k], 2) for k in
                          ("total", "local_move", "refine", "aggregate", "modularity", "decide")},
            "capped_levels": {"levels": stp["capped_levels"], "rounds": stp["capped_rounds"],
                              "ms": round(stp["ms_capped"], 2),
                              "share_of_solve": stp["ms_capped"] / max(stp["ms_total"], 1e-9),
                              "note": "local-moving levels that stopped at max_rounds with nodes still moving"},
            "roofline": roofline, "clocks": clk, "e2e": e2e}
    if pvb is not None:
        line["plain_vs_batched"] = pvb
    if serving is not None:
        line["serving"] = serving
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
