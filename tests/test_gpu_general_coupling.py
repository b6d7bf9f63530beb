"""General coupling on the GPU against the oracle.

The general form of Eq. multislice-modularity: omega^(sr) per pair of
snapshots (ordinal pairs with their own weights, or categorical coupling of
every pair) and a resolution gamma^(s) per snapshot.  The oracle's general
mode is pinned on the CPU (exact-rational dense form, networkx, exact key
differences, brute force); here every GPU result must equal it: labels
bit-exact (at every stage), counters equal, Q within 1e-12 relative --
through single solves, Q of given labels, the global null model, hashed
tables and batches that mix patterns and tables.
"""
import numpy as np
import pytest

import oracle
import paper_2608_03695_gb300 as pkg
from paper_2608_03695_gb300 import synth
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


def rand_table(rng, T, coupling, hi=5):
    if coupling == "ordinal":
        return [int(x) for x in rng.integers(0, hi, size=max(T - 1, 0))]
    M = np.zeros((T, T), dtype=np.int64)
    for s in range(T):
        for r in range(s + 1, T):
            M[s, r] = M[r, s] = int(rng.integers(0, hi))
    return [int(x) for x in M.ravel()]


def solve_both(snaps, coupling="ordinal", gamma=(1, 1), omega=(1, 1), omegas=None, gammas=None, **kw):
    with pkg.mslice_build(snaps, omega=omega, coupling=coupling) as h:
        g = h.mslice_leiden(gamma=gamma, omega=omega, omegas=omegas, gammas=gammas, **kw)
    o = oracle.leiden(snaps, gamma, omega, coupling=coupling, omegas=omegas, gammas=gammas, **kw)
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


def case(seed):
    rng = np.random.default_rng(500 + seed)
    T = int(rng.integers(1, 7))
    n = int(rng.integers(2, 60))
    if seed % 3 == 0:
        snaps = synth.random_temporal(n, T, p=float(rng.uniform(0.03, 0.4)), w_max=int(rng.integers(1, 9)),
                                      seed=seed, p_empty=0.15)
    else:
        snaps, _ = synth.planted_partition_temporal(max(n, 8), T, n_blocks=int(rng.integers(2, 5)), p_in=0.3,
                                                    p_out=0.03, switch_frac=0.1, w_max=4, seed=seed)
    coupling = ["ordinal", "categorical"][seed % 2]
    omega = [(1, 1), (1, 3), (2, 1), (0, 1)][seed % 4]
    omegas = rand_table(rng, T, coupling) if seed % 3 != 1 else None
    gammas = [(int(rng.integers(1, 5)), int(rng.integers(1, 4))) for _ in range(T)] if seed % 4 < 2 else None
    return rng, snaps, coupling, omega, omegas, gammas


@pytest.mark.parametrize("seed", range(24))
def test_random_small(seed):
    rng, snaps, coupling, omega, omegas, gammas = case(seed)
    K = [4, 1, 2, 3, 5][seed % 5]
    g, o = solve_both(snaps, coupling, (1, 1), omega, omegas, gammas, K=K, seed=seed * 3 + 1,
                      n_iterations=1 + seed % 3)
    assert_same(g, o)


@pytest.mark.parametrize("stage", [1, 2, 3])
@pytest.mark.parametrize("level", [0, 1])
def test_stages_categorical(stage, level):
    snaps = synth.recipe_graph("planted_t4_n1000")
    rng = np.random.default_rng(2)
    omegas = rand_table(rng, 4, "categorical")
    gammas = [(1, 1), (3, 2), (4, 5), (1, 1)]
    g, o = solve_both(snaps, "categorical", (1, 1), (1, 2), omegas, gammas, stop_level=level, stop_stage=stage)
    assert np.array_equal(g[0], o[0])
    if stage == 3:
        for k in ("next_n", "next_nnz", "next_checksum"):
            assert g[2][k] == o[2][k], k


def test_medium_power_law():
    snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 4000, "T": 6})
    rng = np.random.default_rng(4)
    assert_same(*solve_both(snaps, "categorical", (1, 1), (1, 4), rand_table(rng, 6, "categorical")))
    assert_same(*solve_both(snaps, "ordinal", (1, 1), (1, 1), [1, 0, 3, 1, 2], [(1, 1), (2, 1), (1, 2), (1, 1),
                                                                             (3, 2), (1, 1)]))


def test_modularity_of_given_labels():
    snaps = synth.recipe_graph("planted_t4_n1000")
    rng = np.random.default_rng(6)
    for coupling in ("ordinal", "categorical"):
        with pkg.mslice_build(snaps, coupling=coupling) as h:
            for trial in range(4):
                labels = rng.integers(0, [4, 40, 4000][trial % 3], size=4000).astype(np.int32)
                omegas = rand_table(rng, 4, coupling)
                gammas = [(int(rng.integers(1, 5)), int(rng.integers(1, 4))) for _ in range(4)]
                for kw in (dict(omegas=omegas), dict(gammas=gammas), dict(omegas=omegas, gammas=gammas), {}):
                    qg = h.mslice_modularity(labels, (1, 1), (1, 3), **kw)
                    qo = oracle.modularity(snaps, labels, (1, 1), (1, 3), coupling=coupling, **kw)
                    assert qg == qo or q_close(qg, qo), (coupling, kw)
                qg = h.mslice_modularity(labels, (3, 2), (1, 3), null="global", omegas=omegas)
                qo = oracle.modularity(snaps, labels, (3, 2), (1, 3), null="global", coupling=coupling, omegas=omegas)
                assert qg == qo or q_close(qg, qo)


@pytest.mark.parametrize("seed", range(6))
def test_global_null_with_general_coupling(seed):
    rng, snaps, coupling, omega, omegas, _ = case(100 + seed)
    g, o = solve_both(snaps, coupling, (3, 2), omega, omegas, None, null="global", seed=seed)
    assert_same(g, o)


@pytest.mark.parametrize("seed", range(4))
def test_hashed_tables(seed, monkeypatch):
    monkeypatch.setenv("MSLICE_DENSE_LIMIT", "0")
    rng, snaps, coupling, omega, omegas, gammas = case(200 + seed)
    assert_same(*solve_both(snaps, coupling, (1, 1), omega, omegas, gammas, K=[4, 2, 3, 4][seed]))


def test_uniform_tables_give_the_uniform_bits():
    snaps = synth.recipe_graph("planted_t4_n1000")
    with pkg.mslice_build(snaps) as h:
        a = h.mslice_leiden(gamma=(3, 2), omega=(1, 2))
        b = h.mslice_leiden(gamma=(3, 2), omega=(1, 2), omegas=[1, 1, 1], gammas=[(3, 2)] * 4)
    assert np.array_equal(a[0], b[0]) and abs(a[1] - b[1]) <= 1e-14
    with pkg.mslice_build(snaps[:2], coupling="categorical") as hc, pkg.mslice_build(snaps[:2]) as ho:
        c = hc.mslice_leiden(omega=(2, 1))
        d = ho.mslice_leiden(omega=(2, 1))
    assert np.array_equal(c[0], d[0]) and c[1] == d[1]


def test_batch_mixing_patterns_and_tables():
    items = []
    for k in range(8):
        rng, snaps, coupling, omega, omegas, gammas = case(300 + k)
        items.append((snaps, coupling, omega, omegas, gammas))
    handles = [pkg.mslice_build(s, coupling=c) for s, c, _, _, _ in items]
    with pkg.Batch() as b:
        for h, (snaps, coupling, omega, omegas, gammas) in zip(handles, items):
            b.add(h, (1, 1), omega, omegas=omegas, gammas=gammas)
        b.run()
        for i, (snaps, coupling, omega, omegas, gammas) in enumerate(items):
            lab, Q = b.results(i)
            ol, oq, _ = oracle.leiden(snaps, (1, 1), omega, coupling=coupling, omegas=omegas, gammas=gammas)
            assert np.array_equal(lab, ol), i
            assert q_close(Q, oq), (i, Q, oq)
    # the same graphs under the global null model (tables of omega only)
    with pkg.Batch() as b:
        for h, (snaps, coupling, omega, omegas, gammas) in zip(handles, items):
            b.add(h, (3, 2), omega, omegas=omegas)
        b.run(null="global")
        for i, (snaps, coupling, omega, omegas, gammas) in enumerate(items):
            lab, Q = b.results(i)
            ol, oq, _ = oracle.leiden(snaps, (3, 2), omega, null="global", coupling=coupling, omegas=omegas)
            assert np.array_equal(lab, ol), i
            assert q_close(Q, oq), (i, Q, oq)
    for h in handles:
        h.close()


def test_rejections():
    snaps = synth.random_temporal(6, 3, p=0.5, seed=1)
    with pkg.mslice_build(snaps, coupling="categorical") as h:
        for kw in (dict(omegas=[0, 1, 2, 1, 0, 1, 3, 1, 0]),          # asymmetric
                   dict(omegas=[1, 1, 1, 1, 0, 1, 1, 1, 0]),          # diagonal
                   dict(omegas=[0, 1, -1, 1, 0, 1, -1, 1, 0]),        # negative
                   dict(gammas=[(1, 1), (0, 1), (1, 1)])):            # gamma 0
            with pytest.raises(pkg.MsliceError) as e:
                h.mslice_leiden(**kw)
            assert e.value.code == pkg.MSLICE_EINVAL, kw
        with pytest.raises(pkg.MsliceError) as e:
            h.mslice_leiden(gammas=[(1, 1)] * 3, null="global")
        assert e.value.code == pkg.MSLICE_EINVAL
        with pkg.Batch() as b:
            b.add(h, gammas=[(1, 1), (2, 1), (1, 1)])
            with pytest.raises(pkg.MsliceError) as e:
                b.run(null="global")
            assert e.value.code == pkg.MSLICE_EINVAL
        lab, Q, _ = h.mslice_leiden(omegas=[0, 1, 2, 1, 0, 1, 2, 1, 0])  # the handle still works
        ol, oq, _ = oracle.leiden(snaps, coupling="categorical", omegas=[0, 1, 2, 1, 0, 1, 2, 1, 0])
        assert np.array_equal(lab, ol) and q_close(Q, oq)
    # the bound takes the largest gamma^(s)
    sn = synth.Snapshot(snaps[0].indptr, snaps[0].indices, np.full(snaps[0].nnz, 2 ** 30, np.int32))
    big = [sn] * 3
    g = -(-(2 ** 61) // (3 * sn.nnz * 2 ** 30))
    with pkg.mslice_build(big) as h:
        with pytest.raises(pkg.MsliceError) as e:
            h.mslice_leiden(gammas=[(1, 1), (g, 1), (1, 1)])
        assert e.value.code == pkg.MSLICE_EOVERFLOW
        h.mslice_leiden(gammas=[(1, 1), (g - 1, 1), (1, 1)], n_iterations=1, max_rounds=1, max_levels=1)
