"""The temporal Constant Potts Model (MSLICE_NULL_CPM) on the GPU against the
oracle's CPM mode (pinned on the CPU to the dense exact-rational form, closed
forms, exact key differences, brute force and CPM's density threshold).

Labels bit-exact at every stage, counters equal, Q within 1e-12 relative:
single solves (with and without general coupling and per-snapshot gamma),
Q of given labels, hashed tables, batches, a served chain, rejections and
CPM's own overflow bound.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2608_03695_gb300 as pkg
from paper_2608_03695_gb300 import synth
from qtol import q_close

pytestmark = pytest.mark.gpu

CPM = "cpm"


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


def solve_both(snaps, gamma=(1, 1), omega=(1, 1), coupling="ordinal", omegas=None, gammas=None, **kw):
    with pkg.mslice_build(snaps, omega=omega, coupling=coupling) as h:
        g = h.mslice_leiden(gamma=gamma, omega=omega, omegas=omegas, gammas=gammas, null=CPM, **kw)
    o = oracle.leiden(snaps, gamma, omega, coupling=coupling, omegas=omegas, gammas=gammas, null=CPM, **kw)
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
    rng = np.random.default_rng(700 + seed)
    T = int(rng.integers(1, 6))
    n = int(rng.integers(2, 60))
    if seed % 3 == 0:
        snaps = synth.random_temporal(n, T, p=float(rng.uniform(0.05, 0.4)), w_max=int(rng.integers(1, 9)),
                                      seed=seed, p_empty=0.15)
    else:
        snaps, _ = synth.planted_partition_temporal(max(n, 8), T, n_blocks=int(rng.integers(2, 5)), p_in=0.3,
                                                    p_out=0.03, switch_frac=0.1, w_max=4, seed=seed)
    gamma = [(1, 2), (1, 1), (3, 2), (1, 4), (2, 1)][seed % 5]
    omega = [(1, 1), (0, 1), (1, 3), (2, 1)][seed % 4]
    coupling = ["ordinal", "categorical"][(seed // 2) % 2]
    omegas = None
    if seed % 5 == 4:
        omegas = ([int(x) for x in rng.integers(0, 4, size=max(T - 1, 0))] if coupling == "ordinal" else None)
    gammas = [(int(rng.integers(1, 4)), int(rng.integers(1, 5))) for _ in range(T)] if seed % 4 == 3 else None
    return snaps, gamma, omega, coupling, omegas, gammas


@pytest.mark.parametrize("seed", range(20))
def test_random_small(seed):
    snaps, gamma, omega, coupling, omegas, gammas = case(seed)
    assert_same(*solve_both(snaps, gamma, omega, coupling, omegas, gammas, K=[4, 1, 2, 3, 5][seed % 5],
                            seed=seed, n_iterations=1 + seed % 3))


@pytest.mark.parametrize("stage", [1, 2, 3])
@pytest.mark.parametrize("level", [0, 1])
def test_stages(stage, level):
    snaps = synth.recipe_graph("planted_t4_n1000")
    g, o = solve_both(snaps, (1, 4), (1, 2), stop_level=level, stop_stage=stage)
    assert np.array_equal(g[0], o[0])
    if stage == 3:
        for k in ("next_n", "next_nnz", "next_checksum"):
            assert g[2][k] == o[2][k], k


def test_planted_and_medium():
    snaps = synth.recipe_graph("planted_t4_n1000")
    g, o = solve_both(snaps, (1, 8), (1, 1))
    assert_same(g, o)
    assert g[1] == o[1]
    medium = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 5000, "T": 5})
    assert_same(*solve_both(medium, (1, 20), (1, 1)))


def test_modularity_of_given_labels():
    snaps = synth.recipe_graph("planted_t4_n1000")
    rng = np.random.default_rng(8)
    with pkg.mslice_build(snaps) as h:
        for trial in range(6):
            labels = rng.integers(0, [4, 40, 4000][trial % 3], size=4000).astype(np.int32)
            for gamma, omega in [((1, 1), (1, 1)), ((1, 8), (1, 10)), ((3, 2), (0, 1))]:
                qg = h.mslice_modularity(labels, gamma, omega, null=CPM)
                qo = oracle.modularity(snaps, labels, gamma, omega, null=CPM)
                assert qg == qo or q_close(qg, qo)
            gammas = [(1, 2), (1, 3), (1, 4), (1, 5)]
            qg = h.mslice_modularity(labels, (1, 1), (1, 1), null=CPM, gammas=gammas)
            qo = oracle.modularity(snaps, labels, (1, 1), (1, 1), null=CPM, gammas=gammas)
            assert qg == qo or q_close(qg, qo)


@pytest.mark.parametrize("seed", range(3))
def test_hashed_tables(seed, monkeypatch):
    monkeypatch.setenv("MSLICE_DENSE_LIMIT", "0")
    snaps, gamma, omega, coupling, omegas, gammas = case(50 + seed)
    assert_same(*solve_both(snaps, gamma, omega, coupling, omegas, gammas))


def test_batch():
    items = [case(80 + k) for k in range(6)]
    handles = [pkg.mslice_build(s, coupling=c) for s, _, _, c, _, _ in items]
    with pkg.Batch() as b:
        for h, (snaps, gamma, omega, coupling, omegas, gammas) in zip(handles, items):
            b.add(h, gamma, omega, omegas=omegas, gammas=gammas)
        b.run(null=CPM)
        for i, (snaps, gamma, omega, coupling, omegas, gammas) in enumerate(items):
            lab, Q = b.results(i)
            ol, oq, _ = oracle.leiden(snaps, gamma, omega, null=CPM, coupling=coupling, omegas=omegas, gammas=gammas)
            assert np.array_equal(lab, ol), i
            assert q_close(Q, oq), (i, Q, oq)
    for h in handles:
        h.close()


def test_served_chain():
    W, n = 3, 120
    stream, _ = synth.planted_partition_temporal(n, 5, n_blocks=3, p_in=12.0 / n, p_out=1.2 / n, switch_frac=0.1,
                                                 churn=0.05, w_max=8, seed=23)
    prev = None
    with pkg.Server(window=W, n_slots=2, gamma=(1, 10), null=CPM) as srv:
        g = srv.add_graph(n)
        for t, sn in enumerate(stream):
            lab, info = srv.wait(srv.submit(g, sn))
            init = None
            if prev is not None:
                w_prev = len(prev) // n
                e = 1 if w_prev == W else 0
                src = np.minimum(np.arange(min(w_prev + 1, W)) + e, w_prev - 1)
                init = np.concatenate([prev[j * n:(j + 1) * n] for j in src]).astype(np.int32)
            ol, oq, _ = oracle.leiden(stream[max(0, t + 1 - W):t + 1], (1, 10), init=init, null=CPM)
            assert np.array_equal(lab, ol), t
            assert q_close(info["Q"], oq)
            prev = lab


def test_rejections_and_bound():
    both = pkg.MSLICE_NULL_GLOBAL | pkg.MSLICE_NULL_CPM
    snaps = synth.random_temporal(6, 3, p=0.5, seed=1)
    with pkg.mslice_build(snaps) as h:
        o = pkg.default_opts()
        o.flags = both
        lab = np.zeros(18, np.int32)
        Q = C.c_double(0)
        rc = pkg.lib().mslice_leiden_ex(h._h, C.byref(o), None, lab.ctypes.data_as(C.c_void_p), C.byref(Q), None)
        assert rc == pkg.MSLICE_EINVAL
    so = pkg.ServerOpts()
    pkg.lib().mslice_server_default_opts(C.byref(so))
    so.solve.flags = both
    s = C.c_void_p()
    assert pkg.lib().mslice_server_create(C.byref(so), C.byref(s)) == pkg.MSLICE_EINVAL
    # CPM's bound: gamma*od*n*N < 2^61 (a sparse graph passes Q_MS's bound)
    sn = synth.csr_from_edges(64, np.array([0], np.int64), np.array([1], np.int64), np.ones(1, np.int32))
    with pkg.mslice_build([sn] * 4) as h:
        h.mslice_leiden(gamma=(2 ** 24, 1), omega=(1, 2 ** 24), n_iterations=1, max_rounds=1, max_levels=1)
        with pytest.raises(pkg.MsliceError) as e:
            h.mslice_leiden(gamma=(2 ** 24, 1), omega=(1, 2 ** 24), null=CPM)
        assert e.value.code == pkg.MSLICE_EOVERFLOW
        lab, Q, _ = h.mslice_leiden(gamma=(2 ** 22, 1), omega=(1, 2 ** 24), null=CPM)
        ol, oq, _ = oracle.leiden([sn] * 4, (2 ** 22, 1), (1, 2 ** 24), null=CPM)
        assert np.array_equal(lab, ol) and q_close(Q, oq)
