"""The bounds-checked build (-DMSLICE_CHECKED=1: indices and table
capacities tested on the hot paths, a violation reported as an error instead
of accessed) on randomised small cases against the oracle, on the hashed
tables, batched and served, under the other null models and general coupling,
on a long sequence and windowed, with randomised refinement, and twice over for
identical bits.  It runs in a
subprocess so that the checked library is the one loaded."""
import os
import subprocess
import sys

import pytest

import paper_2608_03695_gb300 as pkg

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import os, sys
import numpy as np
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))
import oracle
import paper_2608_03695_gb300 as pkg
from paper_2608_03695_gb300 import synth
from qtol import q_close
assert pkg.LIB_PATH.endswith("libmslice_checked.so")
oracle.build()
for seed in range(16):
    rng = np.random.default_rng(500 + seed)
    T, n = int(rng.integers(1, 6)), int(rng.integers(1, 70))
    if seed % 2:
        snaps = synth.random_temporal(n, T, p=float(rng.uniform(0.02, 0.4)), w_max=5, seed=seed, p_empty=0.1)
    else:
        snaps, _ = synth.planted_partition_temporal(max(n, 8), T, 3, 0.3, 0.03, 0.1, None, 4, seed)
    gamma = [(1, 1), (3, 2), (1, 2), (2, 1)][seed % 4]
    omega = [(1, 1), (0, 1), (1, 10), (10, 1)][(seed // 4) % 4]
    if seed % 3 == 0:
        os.environ["MSLICE_DENSE_LIMIT"] = "0"
    with pkg.mslice_build(snaps) as h:
        lab, Q, _ = h.mslice_leiden(gamma=gamma, omega=omega, K=1 + seed % 4, seed=seed)
        lab2, Q2, _ = h.mslice_leiden(gamma=gamma, omega=omega, K=1 + seed % 4, seed=seed)
    os.environ.pop("MSLICE_DENSE_LIMIT", None)
    ref, Qref, _ = oracle.leiden(snaps, gamma, omega, K=1 + seed % 4, seed=seed)
    assert np.array_equal(lab, ref) and np.array_equal(lab2, lab) and Q2 == Q, seed
    assert q_close(Q, Qref), seed
snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 3000, "T": 4})
with pkg.mslice_build(snaps) as h, pkg.Batch() as b:
    for gm in [(1, 1), (3, 2), (1, 2)]:
        b.add(h, gm, (1, 1))
    b.run()
    for i, gm in enumerate([(1, 1), (3, 2), (1, 2)]):
        assert np.array_equal(b.results(i)[0], oracle.leiden(snaps, gm)[0]), i
stream, _ = synth.planted_partition_temporal(100, 4, 3, 0.15, 0.015, 0.1, 0.05, 8, 9)
with pkg.Server(window=2, n_slots=2) as srv:
    g = srv.add_graph(100)
    prev = None
    for t, sn in enumerate(stream):
        lab, _ = srv.wait(srv.submit(g, sn))
        init = None
        if prev is not None:
            w_prev = len(prev) // 100
            e = 1 if w_prev == 2 else 0
            src = np.minimum(np.arange(min(w_prev + 1, 2)) + e, w_prev - 1)
            init = np.concatenate([prev[j * 100:(j + 1) * 100] for j in src]).astype(np.int32)
        assert np.array_equal(lab, oracle.leiden(stream[max(0, t - 1):t + 1], init=init)[0]), t
        prev = lab
# the other null models, general coupling (coupling-table lookups are bound-checked), long slice lists
# (block tiers' slice-parallel scoring) and windowed optimisation
for seed in range(8):
    rng = np.random.default_rng(900 + seed)
    T, n = int(rng.integers(2, 6)), int(rng.integers(8, 60))
    snaps, _ = synth.planted_partition_temporal(n, T, 3, 0.3, 0.03, 0.1, None, 4, seed)
    coupling = ["ordinal", "categorical"][seed % 2]
    if coupling == "ordinal":
        omegas = [int(x) for x in rng.integers(0, 4, size=T - 1)]
    else:
        M = np.zeros((T, T), np.int64)
        for a in range(T):
            for b in range(a + 1, T):
                M[a, b] = M[b, a] = int(rng.integers(0, 4))
        omegas = [int(x) for x in M.ravel()]
    null = ["multislice", "global", "cpm", "multislice"][seed % 4]
    gamma = (1, 4) if null == "cpm" else (1, 1)
    gammas = [(int(rng.integers(1, 4)), 2) for _ in range(T)] if null != "global" and seed % 3 == 0 else None
    with pkg.mslice_build(snaps, coupling=coupling) as h:
        lab, Q, _ = h.mslice_leiden(gamma=gamma, omega=(1, 2), omegas=omegas, gammas=gammas, null=null, seed=seed)
    ref, Qref, _ = oracle.leiden(snaps, gamma, (1, 2), coupling=coupling, omegas=omegas, gammas=gammas, null=null,
                                 seed=seed)
    assert np.array_equal(lab, ref), ("general", seed)
    assert q_close(Q, Qref), ("general", seed)
long = synth.recipe_graph("school_t7375_n327", T=600)
with pkg.mslice_build(long) as h:
    lab, Q, _ = h.mslice_leiden()
ref, Qref, _ = oracle.leiden(long)
assert np.array_equal(lab, ref) and q_close(Q, Qref), "long"
wl, wq, _ = pkg.leiden_windowed(long[:200], 24, 10)
owl, owq, _ = oracle.leiden_windowed(long[:200], 24, 10)
assert np.array_equal(wl, owl), "windowed"
# randomised refinement (theta > 0): its group and block kernels, on random cases, hashed tables and a
# graph with hubs of the block and global-table tiers
for seed in range(6):
    rng = np.random.default_rng(1300 + seed)
    T, n = int(rng.integers(1, 5)), int(rng.integers(4, 60))
    snaps, _ = synth.planted_partition_temporal(max(n, 8), T, 3, 0.3, 0.03, 0.1, None, 4, seed)
    theta = [(1, 10), (1, 1000), (2, 1)][seed % 3]
    if seed % 2:
        os.environ["MSLICE_DENSE_LIMIT"] = "0"
    with pkg.mslice_build(snaps) as h:
        lab, Q, _ = h.mslice_leiden(theta=theta, seed=seed)
    os.environ.pop("MSLICE_DENSE_LIMIT", None)
    ref, Qref, _ = oracle.leiden(snaps, theta=theta, seed=seed)
    assert np.array_equal(lab, ref) and q_close(Q, Qref), ("theta", seed)
rng = np.random.default_rng(31)
nh = 2500
u = np.concatenate([np.zeros(1200, np.int64), np.ones(300, np.int64), rng.integers(2, nh, 6000)])
v = np.concatenate([rng.choice(np.arange(2, nh), 1200, replace=False), rng.choice(np.arange(2, nh), 300, replace=False),
                    rng.integers(2, nh, 6000)])
key = np.unique(np.minimum(u, v) * nh + np.maximum(u, v))
u, v = key // nh, key % nh
u, v = u[u != v], v[u != v]
hubs = [synth.csr_from_edges(nh, u, v, rng.integers(1, 5, size=len(u))) for _ in range(2)]
with pkg.mslice_build(hubs) as h:
    lab, Q, _ = h.mslice_leiden(theta=(1, 100), omega=(1, 2))
ref, Qref, _ = oracle.leiden(hubs, (1, 1), (1, 2), theta=(1, 100))
assert np.array_equal(lab, ref), "theta hubs"
print("checked ok")
'''


def test_checked_build_against_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build(checked=True)
    env = {**os.environ, "MSLICE_LIBRARY": "checked"}
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CASES], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "checked ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
