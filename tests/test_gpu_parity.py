"""GPU path against the oracle, through the C ABI.

Integer work (labels at every stage, the aggregated level's checksum) must be
bit-exact; Q is FP64 from exact integer sums in one fixed order and must be
within 1e-12 relative (it is in practice bit-equal).
"""
import numpy as np
import pytest

import oracle
import paper_2608_03695_gb300 as pkg
from paper_2608_03695_gb300 import synth
from qtol import QTOL, q_close

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


def test_planted_t4_n1000():
    snaps = synth.recipe_graph("planted_t4_n1000")
    g, o = solve_both(snaps)
    assert_same(g, o)
    assert g[1] == o[1]  # same FP64 operation order: bit-equal Q


@pytest.mark.parametrize("seed", range(24))
def test_random_small(seed):
    rng = np.random.default_rng(seed)
    T = int(rng.integers(1, 6))
    n = int(rng.integers(1, 60))
    kind = seed % 3
    if kind == 0:
        snaps = synth.random_temporal(n, T, p=float(rng.uniform(0.02, 0.4)), w_max=int(rng.integers(1, 9)),
                                      seed=seed, p_empty=0.15)
    else:
        snaps, _ = synth.planted_partition_temporal(max(n, 8), T, n_blocks=int(rng.integers(2, 5)), p_in=0.3,
                                                    p_out=0.03, switch_frac=0.1, w_max=4, seed=seed)
    gamma = [(1, 1), (1, 2), (3, 2), (2, 1), (5, 4)][seed % 5]
    omega = [(1, 1), (0, 1), (1, 10), (10, 1), (3, 7)][(seed // 5) % 5]
    K = [4, 1, 2, 3, 5][seed % 5]
    g, o = solve_both(snaps, gamma, omega, K=K, seed=seed * 7 + 1, n_iterations=1 + seed % 3)
    assert_same(g, o)


@pytest.mark.parametrize("stage", [1, 2, 3])
@pytest.mark.parametrize("level", [0, 1])
def test_stages_planted_t4_n1000(stage, level):
    snaps = synth.recipe_graph("planted_t4_n1000")
    g, o = solve_both(snaps, stop_level=level, stop_stage=stage)
    assert np.array_equal(g[0], o[0])
    if stage == 3:
        for k in ("next_n", "next_nnz", "next_checksum"):
            assert g[2][k] == o[2][k], k


@pytest.mark.parametrize("rounds", [1, 2, -1])
def test_stage_rounds(rounds):
    snaps = synth.recipe_graph("planted_t4_n1000")
    for stage in (1, 2):
        g, o = solve_both(snaps, stop_level=0, stop_stage=stage, stop_rounds=rounds, K=3, seed=5)
        assert np.array_equal(g[0], o[0])


def test_degree_tiers():
    """Hubs of degree > 32 (block tier) and > 1024 (global tier)."""
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
    snaps = []
    for t in range(3):
        w = rng.integers(1, 5, size=len(u))
        snaps.append(synth.csr_from_edges(n, u, v, w))
    g, o = solve_both(snaps, (1, 1), (1, 2))
    assert_same(g, o)
    g, o = solve_both(snaps, (1, 1), (1, 2), stop_level=1, stop_stage=3)
    assert np.array_equal(g[0], o[0]) and g[2]["next_checksum"] == o[2]["next_checksum"]


@pytest.mark.parametrize("shared", ["1", "0"])
def test_hubs_past_the_shared_table(shared, monkeypatch):
    """Hubs of degree 5,000 and 9,000, past the 8,192-slot shared tables of
    the top tier (their tables live in global scratch), beside one that fits
    (1,500); shared = 0 puts every top-tier node in global scratch."""
    monkeypatch.setenv("MSLICE_TIER4_SHARED", shared)
    rng = np.random.default_rng(11)
    n = 12000
    us, vs = [], []
    for hub, deg in [(0, 9000), (1, 5000), (2, 1500)]:
        us.append(np.full(deg, hub))
        vs.append(rng.choice(np.arange(10, n), size=deg, replace=False))
    us.append(rng.integers(10, n, 30000))
    vs.append(rng.integers(10, n, 30000))
    u = np.concatenate(us)
    v = np.concatenate(vs)
    key = np.unique(np.minimum(u, v) * n + np.maximum(u, v))
    u, v = key // n, key % n
    ok = u != v
    u, v = u[ok], v[ok]
    snaps = [synth.csr_from_edges(n, u, v, rng.integers(1, 5, size=len(u))) for _ in range(2)]
    for gamma, omega in [((1, 1), (1, 2)), ((1, 4), (1, 1))]:
        g, o = solve_both(snaps, gamma, omega)
        assert_same(g, o)


def test_modularity_parity():
    snaps = synth.recipe_graph("planted_t4_n1000")
    rng = np.random.default_rng(0)
    with pkg.mslice_build(snaps) as h:
        for trial in range(6):
            labels = rng.integers(0, [4, 40, 4000][trial % 3], size=4000).astype(np.int32)
            for gamma, omega in [((1, 1), (1, 1)), ((3, 2), (1, 10)), ((1, 3), (0, 1))]:
                qg = h.mslice_modularity(labels, gamma, omega)
                qo = oracle.modularity(snaps, labels, gamma, omega)
                assert qg == qo or q_close(qg, qo)


def test_hand_worked_cases_on_gpu():
    from test_oracle_pins import load_golden_case
    for name in ["local_move_path_ties.txt", "local_move_empty_target.txt", "refine_wellconnected.txt"]:
        d, snaps = load_golden_case(name)
        lvl, stage, rounds = d["stop"]
        with pkg.mslice_build(snaps, omega=tuple(d["omega"])) as h:
            labels, _, _ = h.mslice_leiden(tuple(d["gamma"]), tuple(d["omega"]), K=d["K"][0], seed=d["seed"][0],
                                           init=np.array(d["init"], np.int32) if "init" in d else None,
                                           stop_level=lvl, stop_stage=stage, stop_rounds=rounds)
        assert labels.tolist() == d["expect"], name


def test_warm_start_and_device_pointers():
    torch = _cuda()
    snaps = synth.recipe_graph("planted_t4_n1000")
    ref, Qref, _ = oracle.leiden(snaps)
    init = np.roll(ref, 7).astype(np.int32)
    o = oracle.leiden(snaps, init=init, n_iterations=1)
    with pkg.mslice_build(snaps) as h:
        g = h.mslice_leiden(init=init, n_iterations=1)
        assert np.array_equal(g[0], o[0])
        out = torch.empty(h.N, dtype=torch.int32, device="cuda")
        lab, Q, _ = h.mslice_leiden(out=out)
        assert np.array_equal(lab.cpu().numpy(), ref)
        assert h.mslice_modularity(lab) == pytest.approx(Qref, rel=QTOL)


def test_device_pointer_build():
    torch = _cuda()
    snaps = synth.recipe_graph("planted_t4_n1000")

    class DSnap:
        def __init__(self, s):
            self.indptr = torch.from_numpy(s.indptr).cuda()
            self.indices = torch.from_numpy(s.indices).cuda()
            self.weights = torch.from_numpy(s.weights).cuda()

    d = [DSnap(s) for s in snaps]
    with pkg.mslice_build(d, device_ptrs=True) as h:
        lab, Q, _ = h.mslice_leiden()
    ref, Qref, _ = oracle.leiden(snaps)
    assert np.array_equal(lab, ref) and Q == Qref


def test_repeatable_bits():
    snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 20000, "T": 4})
    with pkg.mslice_build(snaps) as h:
        a = h.mslice_leiden()
        b = h.mslice_leiden()
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]


def test_medium_dcsbm_parity():
    snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 6000, "T": 5})
    g, o = solve_both(snaps)
    assert_same(g, o)


def test_edge_cases():
    # a single snapshot with no edges; n = 1; empty graph
    for snaps in ([synth.random_temporal(5, 1, p=0.0, seed=0)[0]],
                  synth.random_temporal(1, 3, p=0.0, seed=0),
                  [synth.Snapshot(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))]):
        g, o = solve_both(snaps)
        assert_same(g, o)


def test_invalid_inputs_rejected():
    good = synth.random_temporal(6, 2, p=0.5, seed=1)
    sn = good[0]
    w = sn.weights.copy()
    w[0] += 1
    with pytest.raises(pkg.MsliceError) as e:
        pkg.mslice_build([synth.Snapshot(sn.indptr, sn.indices, w), good[1]])
    assert e.value.code == pkg.MSLICE_EINVAL
    ip = np.array([0, 2, 3, 4], np.int64)
    ix = np.array([2, 1, 0, 0], np.int32)
    with pytest.raises(pkg.MsliceError):
        pkg.mslice_build([synth.Snapshot(ip, ix, np.ones(4, np.int32))])
    with pkg.mslice_build(good) as h:
        with pytest.raises(pkg.MsliceError):
            h.mslice_leiden(gamma=(0, 1))
        with pytest.raises(pkg.MsliceError):
            h.mslice_leiden(init=np.full(12, 12, np.int32))
        with pytest.raises(pkg.MsliceError):
            h.mslice_modularity(np.full(12, -1, np.int32))
        # the handle stays usable after rejected calls
        lab, Q, _ = h.mslice_leiden()
        assert np.array_equal(lab, oracle.leiden(good)[0])
    big = synth.Snapshot(sn.indptr, sn.indices, np.full(sn.nnz, 2 ** 30, np.int32))
    with pkg.mslice_build([big, big]) as h:
        with pytest.raises(pkg.MsliceError) as e:
            h.mslice_leiden(omega=(1, 2 ** 31))
        assert e.value.code == pkg.MSLICE_EOVERFLOW


@pytest.mark.parametrize("wide", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_hashed_tables_path(seed, wide, monkeypatch):
    """The hashed (label, snapshot) tables used when labels x T exceeds the
    dense budget give the same bits as the dense rows, with 8-byte slots (the
    default while every snapshot's mass is below 2^32) and 16-byte ones."""
    monkeypatch.setenv("MSLICE_DENSE_LIMIT", "0")
    monkeypatch.setenv("MSLICE_WIDE_SLOTS", str(wide))
    rng = np.random.default_rng(40 + seed)
    T = int(rng.integers(1, 6))
    snaps, _ = synth.planted_partition_temporal(int(rng.integers(30, 200)), T, n_blocks=3, p_in=0.2, p_out=0.02,
                                                switch_frac=0.1, w_max=5, seed=seed)
    gamma = [(1, 1), (3, 2), (2, 1)][seed % 3]
    omega = [(1, 1), (1, 10), (0, 1)][seed % 3]
    g, o = solve_both(snaps, gamma, omega, K=[4, 2, 3][seed % 3], seed=seed)
    assert_same(g, o)
    if seed == 0:
        g, o = solve_both(snaps, gamma, omega, stop_level=1, stop_stage=3)
        assert np.array_equal(g[0], o[0]) and g[2]["next_checksum"] == o[2]["next_checksum"]


def test_hashed_tables_medium(monkeypatch):
    monkeypatch.setenv("MSLICE_DENSE_LIMIT", "0")
    snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 6000, "T": 5})
    g, o = solve_both(snaps)
    assert_same(g, o)


def test_hashed_tables_masses_past_32_bits(monkeypatch):
    """Snapshots whose mass 2m_s passes 2^32 (sums that 8-byte slots cannot
    hold) run on 16-byte slots and still match the oracle; a light snapshot
    beside them does not change that."""
    monkeypatch.setenv("MSLICE_DENSE_LIMIT", "0")
    snaps, _ = synth.planted_partition_temporal(150, 3, n_blocks=4, p_in=0.3, p_out=0.03, switch_frac=0.1,
                                                w_max=5, seed=3)
    rng = np.random.default_rng(3)
    heavy = []
    for s, sn in enumerate(snaps):
        w = sn.weights.astype(np.int64)
        if s < 2:  # symmetric scaling keeps the snapshot symmetric
            w = w * (1 << 25) + 7
        heavy.append(synth.Snapshot(sn.indptr, sn.indices, w.astype(np.int32)))
    assert int(heavy[0].weights.astype(np.int64).sum()) >= 1 << 32
    assert int(heavy[2].weights.astype(np.int64).sum()) < 1 << 32
    for gamma, omega in [((1, 1), (1, 1)), ((2, 1), (1 << 20, 1))]:
        g, o = solve_both(heavy, gamma, omega)
        assert_same(g, o)


def test_tier_cuts_and_autotune_do_not_change_results():
    """The degree cuts decide only which kernel decides a node: any valid
    cuts, and the autotuner's choice, give the same bits."""
    snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 6000, "T": 5})
    ref, Qref, _ = oracle.leiden(snaps)
    with pkg.mslice_build(snaps) as h:
        for cuts in [(16, 32, 256, 1024), (0, 0, 0, 0), (4, 8, 16, 32), (16, 16, 64, 64), (0, 32, 256, 1024)]:
            lab, Q, st = h.mslice_leiden(tier_cuts=cuts)
            assert np.array_equal(lab, ref) and Q == Qref, cuts
        lab, Q, st = h.mslice_leiden(autotune=True)
        assert np.array_equal(lab, ref) and Q == Qref
        c = st["tier_cuts"]
        assert 0 <= c[0] <= 16 and c[0] <= c[1] <= 32 and c[1] <= c[2] <= 256 and c[2] <= c[3] <= 1024
        for bad in [(17, 32, 256, 1024), (16, 8, 256, 1024), (16, 32, 256, 2048), (-1, 32, 256, 1024)]:
            with pytest.raises(pkg.MsliceError):
                h.mslice_leiden(tier_cuts=bad)


def test_round_graphs_give_the_same_bits(monkeypatch):
    """Rounds replayed from a captured CUDA graph (forced on for a single
    solve) give the oracle's bits, on dense and hashed tables."""
    monkeypatch.setenv("MSLICE_GRAPHS", "1")
    for limit in (None, "0"):
        if limit is not None:
            monkeypatch.setenv("MSLICE_DENSE_LIMIT", limit)
        snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 4000, "T": 4})
        g, o = solve_both(snaps, (1, 1), (1, 2), K=3, seed=4)
        assert_same(g, o)
