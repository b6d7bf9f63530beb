"""Full-size parity cases and the oracle's results on them.

Run as a script, it solves every case with the oracle (nothing else) and
writes ``full_size_expected.json`` beside this file: per case the digest of
the generated input, the digest of the oracle's labels, Q (as a repr string)
and the oracle's counters.  The GPU tests regenerate each input; when its
digest matches the stored one they compare with the stored result, otherwise
(a platform whose floating-point library changes the generated graph) they
run the oracle live.

    python tests/golden/full_size_cases.py            # all cases (hours, one core)
    python tests/golden/full_size_cases.py powerlaw   # cases whose name starts so
    python tests/golden/full_size_cases.py --jobs 4 batched_full   # cases in parallel processes
    python tests/golden/full_size_cases.py 'powerlaw_t64_n200k_w1_1$'   # exactly one case

Each case is written to the JSON file as soon as it finishes (under a file
lock, so parallel runs may share it).
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from paper_2608_03695_gb300 import synth  # noqa: E402

EXPECTED = os.path.join(HERE, "full_size_expected.json")

# Graphs of the batched workload solved over the whole (gamma, omega) grid:
# the largest by n whose single-thread oracle solves take minutes (n = 151k,
# 139k and 124k with T = 3-4); the two largest (n = 166k and 159k, T = 28
# and 26) take the oracle 48 and 38 minutes per solve, too long for 17 more.
BATCHED_SWEEP_GRAPHS = [48, 13, 44]

# n of the largest stored T=64 case (the recipe's n = 1,000,000 needs ~120 GB
# in the single-thread oracle; 200,000 needs ~25 GB)
T64_ORACLE_N = 200_000


def digest_arrays(arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode())
        h.update(np.int64(a.size).tobytes())
        h.update(a.tobytes())
    return h.hexdigest()


def digest_snaps(snaps) -> str:
    return digest_arrays([x for s in snaps for x in (s.indptr, s.indices, s.weights)])


def digest_labels(labels) -> str:
    return digest_arrays([np.asarray(labels, dtype=np.int32)])


def cases():
    """name -> (builder returning a list of solves).  A solve is a dict with
    snaps, gamma, omega and optional init."""
    out = {}

    def powerlaw_t16():
        return [dict(snaps=synth.recipe_graph("powerlaw_t16_n100k"), gamma=(1, 1), omega=(1, 1))]

    out["powerlaw_t16_n100k"] = powerlaw_t16

    def powerlaw_t16_global():
        # the same graph under the global null model (plain modularity of the supra-graph)
        return [dict(snaps=synth.recipe_graph("powerlaw_t16_n100k"), gamma=(1, 1), omega=(1, 1), null="global")]

    out["powerlaw_t16_n100k_global"] = powerlaw_t16_global

    def powerlaw_t64_n20k():
        snaps = synth.recipe_graph("powerlaw_t64_n1m", scale_n=20000)
        return [dict(snaps=snaps, gamma=(1, 1), omega=om) for om in [(1, 10), (1, 1), (10, 1)]]

    out["powerlaw_t64_n20k"] = powerlaw_t64_n20k

    # the T=64 recipe at the largest n whose oracle solve fits this
    # container's memory next to the other cases (~12 GB per 100k nodes)
    for om in [(1, 1), (1, 10), (10, 1)]:
        def powerlaw_t64_large(om=om):
            snaps = synth.recipe_graph("powerlaw_t64_n1m", scale_n=T64_ORACLE_N)
            return [dict(snaps=snaps, gamma=(1, 1), omega=om)]

        out[f"powerlaw_t64_n{T64_ORACLE_N // 1000}k_w{om[0]}_{om[1]}"] = powerlaw_t64_large

    def batched_sample():
        specs = synth.batched_specs()
        picks = [0, 1, 2, 5]  # full-size graphs of the batched workload (n 1.6k-22k, T 7-21)
        solves = []
        for k in picks:
            snaps = synth.batched_graph(specs[k])
            for gm, om in [(synth.BATCHED_GAMMAS[k % 6], synth.BATCHED_OMEGAS[k % 3]),
                           (synth.BATCHED_GAMMAS[(k + 3) % 6], synth.BATCHED_OMEGAS[(k + 1) % 3])]:
                solves.append(dict(snaps=snaps, gamma=gm, omega=om, graph=k))
        return solves

    out["batched_sample"] = batched_sample

    # every graph of the batched workload at full size, at gamma = omega = 1
    for k in range(synth.BATCHED["n_graphs"]):
        def batched_full(k=k):
            return [dict(snaps=synth.batched_graph(synth.batched_specs()[k]), gamma=(1, 1), omega=(1, 1), graph=k)]

        out[f"batched_full_g{k:02d}"] = batched_full

    # the whole gamma x omega grid on the batched workload's largest graphs
    for k in BATCHED_SWEEP_GRAPHS:
        for gm in synth.BATCHED_GAMMAS:
            for om in synth.BATCHED_OMEGAS:
                def batched_sweep(k=k, gm=gm, om=om):
                    return [dict(snaps=synth.batched_graph(synth.batched_specs()[k]), gamma=gm, omega=om, graph=k)]

                out[f"batched_sweep_g{k:02d}_{gm[0]}_{gm[1]}_{om[0]}_{om[1]}"] = batched_sweep

    def serving_chain():
        W = synth.SERVING["window"]
        spec = sorted(synth.serving_specs(), key=lambda s: s[0])[0]  # the smallest live graph (n ~ 10k)
        stream = synth.serving_stream(spec, W + 3)
        return [dict(stream=stream, W=W)]

    out["serving_chain"] = serving_chain

    def serving_chain_largest():
        # the largest live graph of the serving workload (n ~ 2M): 11 requests,
        # the window growing to W = 8 snapshots and then sliding three times
        W = synth.SERVING["window"]
        spec = max(synth.serving_specs(), key=lambda s: s[0])
        return [dict(stream=synth.serving_stream(spec, W + 3), W=W)]

    out["serving_chain_largest"] = serving_chain_largest

    def serving_chain_largest_fifth():
        # the same live graph with the serving workload's n scaled by 1/5
        # (n ~ 400k, windows up to 3.2M supra-nodes), 11 requests
        W = synth.SERVING["window"]
        spec = max(synth.serving_specs(0.2), key=lambda s: s[0])
        return [dict(stream=synth.serving_stream(spec, W + 3), W=W)]

    out["serving_chain_largest_fifth"] = serving_chain_largest_fifth

    def school_full():
        # the school-shaped contact sequence (n = 327, T = 7,375) solved whole
        return [dict(snaps=synth.recipe_graph("school_t7375_n327"), gamma=(1, 1), omega=(1, 1))]

    out["school_t7375_full"] = school_full

    def school_windowed():
        # the same sequence in windows of 64 snapshots at stride 32
        return [dict(snaps=synth.recipe_graph("school_t7375_n327"), W=64, stride=32)]

    out["school_t7375_windowed"] = school_windowed
    return out


def run_solve(oracle, s):
    if "stream" in s:  # a serving chain: one result per request
        stream, W = s["stream"], s["W"]
        res = [{"labels": digest_labels(lab), "Q": repr(Q)} for lab, Q in oracle.serve_chain(stream, W)]
        return {"input": digest_snaps(stream), "chain": res}
    if "W" in s:  # windowed optimisation: stitched labels and every window's Q
        lab, Qs, nw = oracle.leiden_windowed(s["snaps"], s["W"], s["stride"])
        return {"input": digest_snaps(s["snaps"]), "W": s["W"], "stride": s["stride"], "labels": digest_labels(lab),
                "windows": nw, "Q_windows": [repr(q) for q in Qs], "Q": repr(oracle.modularity(s["snaps"], lab))}
    null = s.get("null", "multislice")
    lab, Q, st = oracle.leiden(s["snaps"], s["gamma"], s["omega"], null=null)
    return {"input": digest_snaps(s["snaps"]), "gamma": list(s["gamma"]), "omega": list(s["omega"]), "null": null,
            "labels": digest_labels(lab), "Q": repr(Q),
            "stats": {k: int(st[k]) for k in ("iterations", "levels", "lm_rounds", "lm_edges", "lm_moves")}}


def _store(name, result):
    """Writes one case's result into the JSON file (read-modify-write under
    an exclusive lock, replaced atomically)."""
    import fcntl
    with open(EXPECTED + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        data = json.load(open(EXPECTED)) if os.path.exists(EXPECTED) else {}
        data[name] = result
        tmp = EXPECTED + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, EXPECTED)


def _run_case(name):
    import oracle
    oracle.build()
    t = time.time()
    result = [run_solve(oracle, s) for s in cases()[name]()]
    _store(name, result)
    return name, time.time() - t


def main(argv):
    jobs = 1
    if argv[:1] == ["--jobs"]:
        jobs, argv = int(argv[1]), argv[2:]
    import oracle
    oracle.build()
    # a name ending in "$" selects that case only; others select by prefix
    names = list(cases()) if not argv else list(dict.fromkeys(
        n for p in argv for n in cases() if (n == p[:-1] if p.endswith("$") else n.startswith(p))))
    if jobs <= 1:
        for name in names:
            print("%s: %.1f s" % _run_case(name), flush=True)
        return
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(jobs, maxtasksperchild=1) as pool:
        for name, el in pool.imap_unordered(_run_case, names):
            print(f"{name}: {el:.1f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
