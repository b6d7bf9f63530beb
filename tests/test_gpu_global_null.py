"""The global null model (MSLICE_NULL_GLOBAL) on the GPU against the oracle.

Under this model the library optimises the plain modularity (Eq. modularity)
of the supra-graph of Eq. supra-adjacency: the objective cuGraph's Leiden
optimises when it is handed the supra-graph (Sec. 3.2).  The oracle's
``null="global"`` mode is pinned on the CPU (networkx on the supra-graph,
exact rationals, brute force); here every GPU result must equal it: labels
bit-exact at every stage, Q within 1e-12 relative (bit-equal in practice),
through single solves, batches, the hashed tables and the server.
"""
import numpy as np
import pytest

import oracle
import paper_2608_03695_gb300 as pkg
from paper_2608_03695_gb300 import synth
from qtol import q_close

pytestmark = pytest.mark.gpu

G = "global"


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
        g = h.mslice_leiden(gamma=gamma, omega=omega, null=G, **kw)
    o = oracle.leiden(snaps, gamma, omega, null=G, **kw)
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


def test_planted_t4_n1000():
    snaps = synth.recipe_graph("planted_t4_n1000")
    g, o = solve_both(snaps)
    assert_same(g, o)
    assert g[1] == o[1]
    # and it is a different optimisation from Q_MS
    with pkg.mslice_build(snaps) as h:
        ms = h.mslice_leiden()
    assert ms[1] != g[1]


@pytest.mark.parametrize("seed", range(16))
def test_random_small(seed):
    rng = np.random.default_rng(300 + seed)
    T = int(rng.integers(1, 6))
    n = int(rng.integers(1, 60))
    if seed % 3 == 0:
        snaps = synth.random_temporal(n, T, p=float(rng.uniform(0.02, 0.4)), w_max=int(rng.integers(1, 9)),
                                      seed=seed, p_empty=0.15)
    else:
        snaps, _ = synth.planted_partition_temporal(max(n, 8), T, n_blocks=int(rng.integers(2, 5)), p_in=0.3,
                                                    p_out=0.03, switch_frac=0.1, w_max=4, seed=seed)
    gamma = [(1, 1), (1, 2), (3, 2), (2, 1), (5, 4)][seed % 5]
    omega = [(1, 1), (0, 1), (1, 10), (10, 1), (3, 7)][(seed // 3) % 5]
    K = [4, 1, 2, 3, 5][seed % 5]
    g, o = solve_both(snaps, gamma, omega, K=K, seed=seed * 5 + 2, n_iterations=1 + seed % 3)
    assert_same(g, o)


@pytest.mark.parametrize("stage", [1, 2, 3])
@pytest.mark.parametrize("level", [0, 1])
def test_stages(stage, level):
    snaps = synth.recipe_graph("planted_t4_n1000")
    g, o = solve_both(snaps, (1, 1), (1, 2), stop_level=level, stop_stage=stage)
    assert np.array_equal(g[0], o[0])
    if stage == 3:
        for k in ("next_n", "next_nnz", "next_checksum"):
            assert g[2][k] == o[2][k], k


def test_degree_tiers_and_medium_graph():
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
    assert_same(*solve_both(snaps, (1, 1), (1, 2)))
    medium = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 6000, "T": 5})
    assert_same(*solve_both(medium))


def test_modularity_of_given_labels():
    snaps = synth.recipe_graph("planted_t4_n1000")
    rng = np.random.default_rng(1)
    with pkg.mslice_build(snaps) as h:
        for trial in range(6):
            labels = rng.integers(0, [4, 40, 4000][trial % 3], size=4000).astype(np.int32)
            for gamma, omega in [((1, 1), (1, 1)), ((3, 2), (1, 10)), ((1, 3), (0, 1)), ((1, 1), (7, 2))]:
                qg = h.mslice_modularity(labels, gamma, omega, null=G)
                qo = oracle.modularity(snaps, labels, gamma, omega, null=G)
                assert qg == qo or q_close(qg, qo)


def test_edge_cases():
    for snaps in ([synth.random_temporal(5, 1, p=0.0, seed=0)[0]],
                  synth.random_temporal(1, 3, p=0.0, seed=0),
                  synth.random_temporal(4, 3, p=0.0, seed=0),  # coupling edges only
                  [synth.Snapshot(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))]):
        for omega in [(1, 1), (0, 1)]:
            assert_same(*solve_both(snaps, (1, 1), omega))


@pytest.mark.parametrize("seed", range(4))
def test_hashed_tables(seed, monkeypatch):
    monkeypatch.setenv("MSLICE_DENSE_LIMIT", "0")
    rng = np.random.default_rng(70 + seed)
    T = int(rng.integers(1, 6))
    snaps, _ = synth.planted_partition_temporal(int(rng.integers(30, 200)), T, n_blocks=3, p_in=0.2, p_out=0.02,
                                                switch_frac=0.1, w_max=5, seed=seed)
    gamma = [(1, 1), (3, 2), (2, 1), (1, 2)][seed]
    omega = [(1, 1), (1, 10), (0, 1), (5, 1)][seed]
    assert_same(*solve_both(snaps, gamma, omega, K=[4, 2, 3, 4][seed], seed=seed))
    if seed == 0:
        medium = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 4000, "T": 4})
        assert_same(*solve_both(medium))


def test_rejections_and_bound():
    sn = synth.random_temporal(6, 1, p=0.5, seed=1)[0]
    sn = synth.Snapshot(sn.indptr, sn.indices, np.full(sn.nnz, 2 ** 30, np.int32))
    snaps = [sn] * 4
    on = 2 ** 31
    sum2m = 4 * sn.nnz * 2 ** 30
    g = -(-(2 ** 61) // (sum2m + 2 * on * 6 * 3))  # gamma * 2M' just reaches 2^61
    with pkg.mslice_build(snaps, omega=(on, 1)) as h:
        h.mslice_leiden(gamma=(g, 1), omega=(on, 1), n_iterations=1, max_rounds=1, max_levels=1)
        with pytest.raises(pkg.MsliceError) as e:
            h.mslice_leiden(gamma=(g, 1), omega=(on, 1), null=G)
        assert e.value.code == pkg.MSLICE_EOVERFLOW
        with pytest.raises(pkg.MsliceError) as e:
            h.mslice_modularity(np.zeros(24, np.int32), (g, 1), (on, 1), null=G)
        assert e.value.code == pkg.MSLICE_EOVERFLOW
        with pkg.Batch() as b:
            b.add(h, (g, 1), (on, 1))
            with pytest.raises(pkg.MsliceError) as e:
                b.run(null=G)
            assert e.value.code == pkg.MSLICE_EOVERFLOW
        lab, Q, _ = h.mslice_leiden(gamma=(g - 1, 1), omega=(on, 1), null=G, n_iterations=1, max_rounds=1,
                                    max_levels=1)
        ol, oq, _ = oracle.leiden(snaps, (g - 1, 1), (on, 1), null=G, n_iterations=1, max_rounds=1, max_levels=1)
        assert np.array_equal(lab, ol) and q_close(Q, oq)


# ----------------------------------------------------------------- batches
def test_batch_mixed_instances():
    rng = np.random.default_rng(5)
    graphs = []
    for k in range(6):
        T = int(rng.integers(1, 6))
        snaps, _ = synth.planted_partition_temporal(int(rng.integers(10, 150)), T, n_blocks=3, p_in=0.25,
                                                    p_out=0.03, switch_frac=0.1, w_max=4, seed=k)
        graphs.append(snaps)
    params = [((1, 1), (1, 1)), ((3, 2), (1, 10)), ((1, 2), (0, 1)), ((2, 1), (10, 1)), ((5, 4), (3, 7)),
              ((1, 1), (1, 2))]
    handles = [pkg.mslice_build(s) for s in graphs]
    with pkg.Batch() as b:
        for h, (gm, om) in zip(handles, params):
            b.add(h, gm, om)
        st = b.run(null=G)
        for i, (snaps, (gm, om)) in enumerate(zip(graphs, params)):
            lab, Q = b.results(i)
            ol, oq, _ = oracle.leiden(snaps, gm, om, null=G)
            assert np.array_equal(lab, ol), i
            assert Q == oq or q_close(Q, oq), (i, Q, oq)
        # the same batch again under Q_MS gives the multislice results
        b.run()
        for i, (snaps, (gm, om)) in enumerate(zip(graphs, params)):
            lab, Q = b.results(i)
            ol, oq, _ = oracle.leiden(snaps, gm, om)
            assert np.array_equal(lab, ol), i
    for h in handles:
        h.close()
    assert st["iterations"] >= 1


def test_batch_sweep_hashed(monkeypatch):
    monkeypatch.setenv("MSLICE_DENSE_LIMIT", "0")
    snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 2000, "T": 4})
    params = [((gn, gd), om) for gn, gd in [(1, 1), (3, 2)] for om in [(1, 1), (0, 1), (4, 1)]]
    with pkg.mslice_build(snaps) as h, pkg.Batch() as b:
        for gm, om in params:
            b.add(h, gm, om)
        b.run(null=G)
        for i, (gm, om) in enumerate(params):
            lab, Q = b.results(i)
            ol, oq, _ = oracle.leiden(snaps, gm, om, null=G)
            assert np.array_equal(lab, ol), i
            assert q_close(Q, oq)


# ----------------------------------------------------------------- serving
def test_served_chain():
    W, n = 3, 150
    stream, _ = synth.planted_partition_temporal(n, 6, n_blocks=3, p_in=12.0 / n, p_out=1.2 / n, switch_frac=0.1,
                                                 churn=0.05, w_max=8, seed=17)
    prev = None
    with pkg.Server(window=W, n_slots=2, null=G) as srv:
        g = srv.add_graph(n)
        for t, sn in enumerate(stream):
            lab, info = srv.wait(srv.submit(g, sn))
            init = None
            if prev is not None:
                w_prev = len(prev) // n
                e = 1 if w_prev == W else 0
                src = np.minimum(np.arange(min(w_prev + 1, W)) + e, w_prev - 1)
                init = np.concatenate([prev[j * n:(j + 1) * n] for j in src]).astype(np.int32)
            ol, oq, _ = oracle.leiden(stream[max(0, t + 1 - W):t + 1], init=init, null=G)
            assert np.array_equal(lab, ol), t
            assert q_close(info["Q"], oq)
            prev = lab
