"""Randomised refinement (mslice_opts.theta_num/theta_den) on the GPU against
the oracle's: the weights come from one integer recipe and the draws from the
schedule's hash, so labels must be bit-exact at every stage (counters equal,
Q within 1e-12 relative) -- on random cases, hubs of every degree tier
(including the global-table tier), hashed tables, batches, the other null
models, a long sequence (block tiers with long slice lists) and windowed runs.
"""
import numpy as np
import pytest

import oracle
import paper_2608_03695_gb300 as pkg
from paper_2608_03695_gb300 import synth
from qtol import q_close

pytestmark = pytest.mark.gpu

THETAS = [(1, 10), (1, 100), (1, 1000), (2, 1), (1, 10000)]


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


def solve_both(snaps, gamma=(1, 1), omega=(1, 1), **kw):
    with pkg.mslice_build(snaps, omega=omega) as h:
        g = h.mslice_leiden(gamma=gamma, omega=omega, **kw)
    o = oracle.leiden(snaps, gamma, omega, **kw)
    return g, o


def assert_same(g, o):
    gl, gq, gs = g
    ol, oq, os_ = o
    assert len(gl) == len(ol)
    bad = np.flatnonzero(gl != ol)
    assert bad.size == 0, f"{bad.size} labels differ, first at {bad[:5]}"
    assert q_close(gq, oq), (gq, oq)
    for k in ("iterations", "levels", "lm_rounds", "lm_edges", "lm_moves", "stop_reason", "last_level0_moves"):
        assert gs[k] == os_[k], (k, gs[k], os_[k])


@pytest.mark.parametrize("seed", range(20))
def test_random_small(seed):
    rng = np.random.default_rng(1100 + seed)
    T = int(rng.integers(1, 6))
    n = int(rng.integers(2, 70))
    if seed % 3 == 0:
        snaps = synth.random_temporal(n, T, p=float(rng.uniform(0.03, 0.4)), w_max=int(rng.integers(1, 9)),
                                      seed=seed, p_empty=0.1)
    else:
        snaps, _ = synth.planted_partition_temporal(max(n, 8), T, n_blocks=int(rng.integers(2, 5)), p_in=0.3,
                                                    p_out=0.03, switch_frac=0.1, w_max=4, seed=seed)
    gamma = [(1, 1), (1, 2), (3, 2)][seed % 3]
    omega = [(1, 1), (0, 1), (1, 10), (5, 1)][seed % 4]
    assert_same(*solve_both(snaps, gamma, omega, theta=THETAS[seed % 5], K=[4, 2, 3][seed % 3], seed=seed,
                            n_iterations=1 + seed % 3))


@pytest.mark.parametrize("level", [0, 1])
def test_refined_labels_at_a_stage(level):
    snaps = synth.recipe_graph("planted_t4_n1000")
    for theta in [(1, 10), (1, 1000)]:
        g, o = solve_both(snaps, theta=theta, stop_level=level, stop_stage=2)
        assert np.array_equal(g[0], o[0]), theta


# A star (leaves 3, 1, 4, 1, 5), a graph where node 0's target 1 has a key of
# exactly 0 (2m = 32, gamma 1/2) and two disjoint stars: node 0's (and node
# 6's) draw for every seed.
CHOICE_GRAPHS = [
    (6, [0, 0, 0, 0, 0], [1, 2, 3, 4, 5], [3, 1, 4, 1, 5], (1, 4)),
    (6, [0, 0, 0, 1, 4], [1, 2, 3, 4, 5], [1, 3, 4, 7, 1], (1, 2)),
    (12, [0] * 5 + [6] * 5, [1, 2, 3, 4, 5, 7, 8, 9, 10, 11], [3, 1, 4, 1, 5, 2, 6, 1, 3, 2], (1, 4)),
]


@pytest.mark.parametrize("graph", range(len(CHOICE_GRAPHS)))
def test_small_choices_match_for_every_seed(graph):
    n, u, v, w, gamma = CHOICE_GRAPHS[graph]
    snaps = [synth.csr_from_edges(n, np.array(u, np.int64), np.array(v, np.int64), np.array(w, np.int32))]
    with pkg.mslice_build(snaps) as h:
        for seed in range(200):
            kw = dict(K=2, seed=seed, init=np.zeros(n, np.int32), stop_level=0, stop_stage=2, stop_rounds=-1,
                      theta=(1, 10))
            lab, _, _ = h.mslice_leiden(gamma=gamma, **kw)
            ref, _, _ = oracle.leiden(snaps, gamma, **kw)
            assert np.array_equal(lab, ref), seed


def test_hubs_of_every_tier():
    rng = np.random.default_rng(3)
    n = 3000
    us, vs = [], []
    for hub, deg in [(0, 1500), (1, 200), (2, 40), (3, 1100)]:
        nb = rng.choice(np.arange(10, n), size=deg, replace=False)
        us.append(np.full(deg, hub))
        vs.append(nb)
    er = synth.random_temporal(n, 1, p=4.0 / n, seed=9)[0]
    r = np.repeat(np.arange(n), np.diff(er.indptr))
    keep = r < er.indices
    us.append(r[keep])
    vs.append(er.indices[keep])
    u = np.concatenate(us)
    v = np.concatenate(vs)
    key = np.unique(np.minimum(u, v) * n + np.maximum(u, v))
    u, v = key // n, key % n
    ok = u != v
    u, v = u[ok], v[ok]
    snaps = [synth.csr_from_edges(n, u, v, rng.integers(1, 5, size=len(u))) for _ in range(3)]
    for theta in [(1, 10), (1, 1000)]:
        assert_same(*solve_both(snaps, (1, 1), (1, 2), theta=theta))


def test_hashed_tables_and_medium_graph(monkeypatch):
    medium = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 5000, "T": 4})
    assert_same(*solve_both(medium, theta=(1, 100)))
    monkeypatch.setenv("MSLICE_DENSE_LIMIT", "0")
    assert_same(*solve_both(medium, theta=(1, 100), seed=7))


def test_other_models_and_long_sequence():
    snaps = synth.recipe_graph("planted_t4_n1000")
    assert_same(*solve_both(snaps, theta=(1, 50), null="global"))
    assert_same(*solve_both(snaps, (1, 8), theta=(1, 50), null="cpm"))
    long = synth.recipe_graph("school_t7375_n327", T=300)
    assert_same(*solve_both(long, theta=(1, 200)))


def test_batch_and_windowed():
    graphs = [synth.planted_partition_temporal(int(n), T, 3, 0.25, 0.03, 0.1, None, 4, k)[0]
              for k, (n, T) in enumerate([(40, 3), (120, 2), (80, 5), (30, 1)])]
    handles = [pkg.mslice_build(s) for s in graphs]
    with pkg.Batch() as b:
        for h in handles:
            b.add(h)
        b.run(theta=(1, 30), seed=5)
        for i, s in enumerate(graphs):
            lab, Q = b.results(i)
            ol, oq, _ = oracle.leiden(s, theta=(1, 30), seed=5)
            assert np.array_equal(lab, ol), i
            assert q_close(Q, oq)
    for h in handles:
        h.close()
    seq = synth.recipe_graph("school_t7375_n327", T=80)
    gl, gq, _ = pkg.leiden_windowed(seq, 20, 8, theta=(1, 100))
    ol, oq, _ = oracle.leiden_windowed(seq, 20, 8, theta=(1, 100))
    assert np.array_equal(gl, ol) and all(q_close(a, b) for a, b in zip(gq, oq))


def test_theta_is_validated_and_zero_is_greedy():
    snaps = synth.recipe_graph("planted_t4_n1000")
    with pkg.mslice_build(snaps) as h:
        with pytest.raises(pkg.MsliceError) as e:
            h.mslice_leiden(theta=(-1, 1))
        assert e.value.code == pkg.MSLICE_EINVAL
        a = h.mslice_leiden(theta=(0, 1))
        b = h.mslice_leiden()
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
