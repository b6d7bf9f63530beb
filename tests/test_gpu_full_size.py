"""Parity at the workloads' full sizes.

The expected labels (as digests) and Q come from the oracle alone, written by
``tests/golden/full_size_cases.py``.  Each test regenerates its inputs; if
their digest differs from the stored one (a platform whose floating-point
library changes the generated graph) the oracle is run live instead.

* power-law workload at full size (T=16, n=100,000), the benchmark's solve,
  under Q_MS and under the global null model;
* the T=64 power-law recipe at n=20,000 for omega in {1/10, 1, 10}, solved
  one by one and as one batch;
* four full-size graphs of the batched workload at two (gamma, omega) each,
  as one batch;
* a serving chain: the smallest live graph of the serving workload through
  11 snapshots with windows of 8;
* the school-shaped contact sequence (n = 327, T = 7,375) solved whole, and
  in windows of 64 snapshots at stride 32.
"""
import json
import os
import sys

import numpy as np
import pytest

import oracle
import paper_2608_03695_gb300 as pkg

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import full_size_cases as fsc  # noqa: E402
from qtol import q_close

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module", autouse=True)
def built():
    _cuda()
    pkg.build()
    oracle.build()


def expected(name, solves):
    """Stored oracle results, or live oracle results when the inputs differ."""
    stored = json.load(open(fsc.EXPECTED)).get(name)
    out = []
    for k, s in enumerate(solves):
        if stored and k < len(stored) and stored[k]["input"] == fsc.digest_snaps(s.get("snaps", s.get("stream"))):
            out.append(stored[k])
        else:
            out.append(fsc.run_solve(oracle, s))
    return out


def q_ok(q, ref):
    ref = float(ref)
    return q_close(q, ref)


def test_power_law_full_size():
    solves = fsc.cases()["powerlaw_t16_n100k"]()
    exp = expected("powerlaw_t16_n100k", solves)
    s = solves[0]
    with pkg.mslice_build(s["snaps"]) as h:
        lab, Q, st = h.mslice_leiden(gamma=s["gamma"], omega=s["omega"])
    assert fsc.digest_labels(lab) == exp[0]["labels"]
    assert q_ok(Q, exp[0]["Q"])
    for k in ("iterations", "levels", "lm_rounds", "lm_edges", "lm_moves"):
        assert st[k] == exp[0]["stats"][k], k


def test_power_law_full_size_global_null():
    solves = fsc.cases()["powerlaw_t16_n100k_global"]()
    exp = expected("powerlaw_t16_n100k_global", solves)
    s = solves[0]
    with pkg.mslice_build(s["snaps"]) as h:
        lab, Q, st = h.mslice_leiden(gamma=s["gamma"], omega=s["omega"], null="global")
    assert fsc.digest_labels(lab) == exp[0]["labels"]
    assert q_ok(Q, exp[0]["Q"])
    for k in ("iterations", "levels", "lm_rounds", "lm_edges", "lm_moves"):
        assert st[k] == exp[0]["stats"][k], k


def test_T64_recipe_plain_and_batched():
    solves = fsc.cases()["powerlaw_t64_n20k"]()
    exp = expected("powerlaw_t64_n20k", solves)
    with pkg.mslice_build(solves[0]["snaps"]) as h:
        for s, e in zip(solves, exp):
            lab, Q, _ = h.mslice_leiden(gamma=s["gamma"], omega=s["omega"])
            assert fsc.digest_labels(lab) == e["labels"], s["omega"]
            assert q_ok(Q, e["Q"])
        with pkg.Batch() as b:
            for s in solves:
                b.add(h, s["gamma"], s["omega"])
            b.run()
            for i, e in enumerate(exp):
                lab, Q = b.results(i)
                assert fsc.digest_labels(lab) == e["labels"], i
                assert q_ok(Q, e["Q"])


def test_batched_workload_graphs_in_one_batch():
    solves = fsc.cases()["batched_sample"]()
    exp = expected("batched_sample", solves)
    handles = {}
    with pkg.Batch() as b:
        for s in solves:
            if s["graph"] not in handles:
                handles[s["graph"]] = pkg.mslice_build(s["snaps"])
            b.add(handles[s["graph"]], s["gamma"], s["omega"])
        b.run()
        for i, e in enumerate(exp):
            lab, Q = b.results(i)
            assert fsc.digest_labels(lab) == e["labels"], i
            assert q_ok(Q, e["Q"])
    for h in handles.values():
        h.close()


def test_serving_chain_full_size():
    s = fsc.cases()["serving_chain"]()[0]
    exp = expected("serving_chain", [s])[0]["chain"]
    stream, W = s["stream"], s["W"]
    with pkg.Server(window=W, n_slots=2) as srv:
        g = srv.add_graph(stream[0].n)
        rids = [srv.submit(g, sn) for sn in stream]
        for t, rid in enumerate(rids):
            lab, info = srv.wait(rid)
            assert fsc.digest_labels(lab) == exp[t]["labels"], t
            assert q_ok(info["Q"], exp[t]["Q"])


def test_school_sequence_whole_and_windowed():
    s = fsc.cases()["school_t7375_full"]()[0]
    exp = expected("school_t7375_full", [s])[0]
    with pkg.mslice_build(s["snaps"]) as h:
        lab, Q, st = h.mslice_leiden()
    assert fsc.digest_labels(lab) == exp["labels"]
    assert q_ok(Q, exp["Q"])
    for k in ("iterations", "levels", "lm_rounds", "lm_edges", "lm_moves"):
        assert st[k] == exp["stats"][k], k
    w = fsc.cases()["school_t7375_windowed"]()[0]
    expw = expected("school_t7375_windowed", [w])[0]
    lab, Qs, _ = pkg.leiden_windowed(w["snaps"], w["W"], w["stride"])
    assert fsc.digest_labels(lab) == expw["labels"]
    assert len(Qs) == expw["windows"]
    assert all(q_ok(a, b) for a, b in zip(Qs, expw["Q_windows"]))
    with pkg.mslice_build(w["snaps"]) as h:
        assert q_ok(h.mslice_modularity(lab), expw["Q"])
