#!/usr/bin/env python
"""Throughput benchmark of the multislice-Leiden hot path on GB300.

A step is one complete solve of the synthetic power-law temporal workload
(T=16 snapshots of n=100,000 nodes, degree-corrected SBM with power-law
degrees and community sizes, 5% edge churn per snapshot, weights 1..8,
ordinal coupling omega=1, gamma=1): supra-graph build from device-resident
snapshots, Leiden (two passes: local moving, refinement, aggregation) and
Q_MS.  The metric is local-moving supra-edges per second: the sum over all
local-moving rounds of the level's directed entries, divided by the whole
step's device time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mslice|reference]

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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {"workload": "multislice Leiden, power-law temporal DC-SBM", "T": 16, "n": 100000,
            "deg_exp": 2.5, "mean_deg": 20, "size_exp": 1.5, "sizes": "20-5000", "mixing": 0.3, "churn": 0.05,
            "weights": "1-8", "gamma": "1/1", "omega": "1/1", "n_iterations": 2, "K": 4, "seed": 0,
            "supra_nodes": 1600000}
METRIC = "supra-edges/s in Leiden local-move"
UNIT = "supra-edges/s"
ORACLE_SAMPLE_N = 20000  # same recipe, n scaled so one oracle solve takes ~10-30 s


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mslice", choices=["mslice", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-run", action="store_true",
                    help="one solve of the workload and exit (a short target for ncu captures)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def decide_traffic():
    """DRAM bytes per launch of the decision kernel from the committed ncu
    summary (None when absent)."""
    p = os.path.join(ROOT, "profiles", "local_move_decide_config2.md")
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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

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


def cpu_baseline():
    import oracle
    from paper_2608_03695_gb300 import synth
    snaps = synth.config_graph(2, scale_n=ORACLE_SAMPLE_N)
    t = time.perf_counter()
    _, _, st = oracle.leiden(snaps)
    el = time.perf_counter() - t
    return {"value": st["lm_edges"] / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one oracle solve of the same recipe at n={ORACLE_SAMPLE_N}, T=16 "
                      f"({st['lm_edges']} local-move supra-edges in {el:.1f} s, single thread)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2608_03695_gb300 import synth
    oracle.build()
    snaps = synth.config_graph(2, scale_n=ORACLE_SAMPLE_N)
    for _ in range(args.warmup):
        oracle.leiden(snaps, n_iterations=1, max_rounds=2)  # short warm-up (page-in, caches)
    edges, secs = 0, 0.0
    for _ in range(args.steps):
        t = time.perf_counter()
        _, _, st = oracle.leiden(snaps)
        secs += time.perf_counter() - t
        edges += st["lm_edges"]
    v = edges / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {**WORKLOAD, "n": ORACLE_SAMPLE_N, "supra_nodes": ORACLE_SAMPLE_N * 16,
                       "note": "bounded sample of the same recipe (n scaled) for the single-thread CPU oracle"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} oracle solves at n={ORACLE_SAMPLE_N}, T=16"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_2608_03695_gb300 as pkg
    from paper_2608_03695_gb300 import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    snaps = synth.config_graph(2)
    stream = torch.cuda.Stream()
    if args.profile_run:
        with pkg.mslice_build(snaps) as h:
            _, Q, st = h.mslice_leiden()
        print(json.dumps({"profile_run": True, "Q": Q, "kernel_launches": st["kernel_launches"],
                          "ms_total": st["ms_total"]}), flush=True)
        return

    class DevSnap:
        def __init__(self, s, pin=False, device=None):
            conv = (lambda a: torch.from_numpy(a).pin_memory()) if pin else (lambda a: torch.from_numpy(a).to(device))
            self.indptr, self.indices, self.weights = conv(s.indptr), conv(s.indices), conv(s.weights)

    dsnaps = [DevSnap(s, device="cuda") for s in snaps]
    N = snaps[0].n * len(snaps)
    dlabels = torch.empty(N, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def step_device(profile=False):
        h = pkg.mslice_build(dsnaps, device_ptrs=True, stream=stream.cuda_stream)
        _, Q, st = h.mslice_leiden(out=dlabels, profile=profile)
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
    ms_max = max_over_ranks(ms)
    total_edges = sum_over_ranks(edges)
    value = total_edges / (ms_max / 1e3)

    # decision-kernel roofline from one profiled step (not part of the timed region)
    stp, _, _ = step_device(profile=True)
    peak, peak_kind = measured_peak()
    achieved = stp["decide_bytes"] / (stp["ms_decide"] / 1e3) / 1e9 if stp["ms_decide"] > 0 else 0.0
    traffic = decide_traffic()
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
            h = pkg.mslice_build(hsnaps, host_tensors=True, stream=stream.cuda_stream)
            _, Q, st = h.mslice_leiden(out=hlabels)
            h.close()
            return st

        step_e2e()
        barrier()
        torch.cuda.synchronize()
        t = time.perf_counter()
        e_edges = 0
        k_e2e = max(1, args.steps // 2)
        for _ in range(k_e2e):
            e_edges += step_e2e()["lm_edges"]
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t)
        e2e = {"value": sum_over_ranks(e_edges) / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k_e2e, "ms_per_step": 1e3 * el / k_e2e}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {**WORKLOAD, "parallelism": f"replicas{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (level-0 supra-CSR 280 MB vs 129 MB L2)"},
            "Q": Qs[-1] if Qs else None, "gpu_launches": int(sum_over_ranks(launches)),
            "local_move_only": {"value": stp["lm_edges"] / (stp["ms_local_move"] / 1e3), "unit": UNIT,
                                "note": "same edges over local-moving device time only (profiled step)"},
            "roofline": roofline, "clocks": clk, "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
