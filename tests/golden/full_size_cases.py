"""Full-size parity cases and the oracle's results on them.

Run as a script, it solves every case with the oracle (nothing else) and
writes ``full_size_expected.json`` beside this file: per case the digest of
the generated input, the digest of the oracle's labels, Q (as a repr string)
and the oracle's counters.  The GPU tests regenerate each input; when its
digest matches the stored one they compare with the stored result, otherwise
(a platform whose floating-point library changes the generated graph) they
run the oracle live.

    python tests/golden/full_size_cases.py            # all cases (~20 min, one core)
    python tests/golden/full_size_cases.py powerlaw   # cases whose name starts so
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

    def serving_chain():
        W = synth.SERVING["window"]
        spec = sorted(synth.serving_specs(), key=lambda s: s[0])[0]  # the smallest live graph (n ~ 10k)
        stream = synth.serving_stream(spec, W + 3)
        return [dict(stream=stream, W=W)]

    out["serving_chain"] = serving_chain

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


def main(prefixes):
    import oracle
    oracle.build()
    data = {}
    if os.path.exists(EXPECTED):
        data = json.load(open(EXPECTED))
    for name, make in cases().items():
        if prefixes and not any(name.startswith(p) for p in prefixes):
            continue
        t = time.time()
        data[name] = [run_solve(oracle, s) for s in make()]
        print(f"{name}: {time.time() - t:.1f} s", flush=True)
        with open(EXPECTED, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
