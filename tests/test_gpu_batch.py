"""Batched solves (many independent (graph, gamma, omega) instances in one
pass) through the C ABI: every instance must give the labels of the oracle
run on that instance alone, bit for bit, and its Q within 1e-12 relative."""
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


def small_instance(seed):
    rng = np.random.default_rng(1000 + seed)
    T = int(rng.integers(1, 6))
    n = int(rng.integers(1, 80))
    if seed % 3 == 0:
        snaps = synth.random_temporal(n, T, p=float(rng.uniform(0.02, 0.4)), w_max=int(rng.integers(1, 9)),
                                      seed=seed, p_empty=0.15)
    else:
        snaps, _ = synth.planted_partition_temporal(max(n, 8), T, n_blocks=int(rng.integers(2, 5)), p_in=0.3,
                                                    p_out=0.03, switch_frac=0.1, w_max=4, seed=seed)
    gamma = [(1, 1), (1, 2), (3, 2), (2, 1), (5, 4)][seed % 5]
    omega = [(1, 1), (0, 1), (1, 10), (10, 1), (3, 7)][(seed // 5) % 5]
    return snaps, gamma, omega


def run_batch(instances, **opts):
    """instances: list of (handle, snaps, gamma, omega, init)."""
    with pkg.Batch() as b:
        for h, _, gamma, omega, init in instances:
            b.add(h, gamma, omega, init)
        st = b.run(**opts)
        out = [b.results(i) for i in range(len(instances))]
        all_lab, all_Q = b.results()
        B, N, off = b.info()
    assert B == len(instances)
    for i, (lab, Q) in enumerate(out):
        assert np.array_equal(all_lab[off[i]:off[i + 1]], lab)
        assert all_Q[i] == Q
    return out, st


def check_against_oracle(instances, out, **opts):
    for i, ((h, snaps, gamma, omega, init), (lab, Q)) in enumerate(zip(instances, out)):
        ol, oq, _ = oracle.leiden(snaps, gamma, omega, init=init, **opts)
        bad = np.flatnonzero(lab != ol)
        assert bad.size == 0, f"instance {i}: {bad.size} labels differ, first at {bad[:5]}"
        assert q_close(Q, oq), (i, Q, oq)


@pytest.mark.parametrize("opts", [{}, {"K": 3, "seed": 11, "n_iterations": 3}, {"K": 1, "max_levels": 2}])
def test_mixed_small_instances(opts):
    handles, instances = [], []
    for seed in range(20):
        snaps, gamma, omega = small_instance(seed)
        h = pkg.mslice_build(snaps)
        handles.append(h)
        instances.append((h, snaps, gamma, omega, None))
    out, st = run_batch(instances, **opts)
    check_against_oracle(instances, out, **opts)
    assert st["kernel_launches"] > 0
    for h in handles:
        h.close()


def test_gamma_omega_sweep_one_graph():
    snaps = synth.recipe_graph("planted_t4_n1000")
    with pkg.mslice_build(snaps) as h:
        grid = [((g, 4), (w, 4)) for g in (2, 4, 6) for w in (0, 1, 4)]
        instances = [(h, snaps, gamma, omega, None) for gamma, omega in grid]
        out, _ = run_batch(instances)
        check_against_oracle(instances, out)
        # the same instance solved alone on the GPU
        lab, Q, _ = h.mslice_leiden(gamma=grid[4][0], omega=grid[4][1])
        assert np.array_equal(lab, out[4][0]) and Q == out[4][1]


def test_warm_starts_and_repeat_runs():
    snaps = synth.recipe_graph("planted_t4_n1000")
    ref, _, _ = oracle.leiden(snaps)
    rng = np.random.default_rng(5)
    small = [small_instance(s) for s in (3, 7)]
    with pkg.mslice_build(snaps) as h, pkg.mslice_build(small[0][0]) as h1, pkg.mslice_build(small[1][0]) as h2:
        init_a = np.roll(ref, 7).astype(np.int32)
        n1 = h1.N
        init_b = rng.integers(0, max(n1, 1), size=n1).astype(np.int32)
        instances = [(h, snaps, (1, 1), (1, 1), init_a), (h1, small[0][0], small[0][1], small[0][2], init_b),
                     (h2, small[1][0], small[1][1], small[1][2], None), (h, snaps, (3, 2), (1, 2), None)]
        with pkg.Batch() as b:
            for hh, _, gamma, omega, init in instances:
                b.add(hh, gamma, omega, init)
            with pytest.raises(pkg.MsliceError):
                b.results(0)  # not run yet
            b.run(n_iterations=1)
            first = [b.results(i) for i in range(4)]
            b.run(n_iterations=1)  # the cached concatenation is reused
            again = [b.results(i) for i in range(4)]
            for x, y in zip(first, again):
                assert np.array_equal(x[0], y[0]) and x[1] == y[1]
            b.clear()
            b.add(h2, small[1][1], small[1][2])
            b.run()
            lab, Q = b.results(0)
        check_against_oracle(instances, first, n_iterations=1)
        ol, oq, _ = oracle.leiden(small[1][0], small[1][1], small[1][2])
        assert np.array_equal(lab, ol) and q_close(Q, oq)


def test_degenerate_instances():
    empty = [synth.Snapshot(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))]
    single = synth.random_temporal(1, 3, p=0.0, seed=0)
    edgeless = [synth.random_temporal(5, 1, p=0.0, seed=0)[0]]
    planted = synth.recipe_graph("planted_t4_n1000")
    graphs = [empty, single, planted, edgeless, planted]
    handles = [pkg.mslice_build(s) for s in graphs]
    instances = [(h, s, (1, 1), (1, 1), None) for h, s in zip(handles, graphs)]
    out, _ = run_batch(instances)
    check_against_oracle(instances, out)
    for h in handles:
        h.close()


def test_batch_hashed_tables(monkeypatch):
    monkeypatch.setenv("MSLICE_DENSE_LIMIT", "0")
    handles, instances = [], []
    for seed in range(8):
        snaps, gamma, omega = small_instance(40 + seed)
        h = pkg.mslice_build(snaps)
        handles.append(h)
        instances.append((h, snaps, gamma, omega, None))
    out, _ = run_batch(instances)
    check_against_oracle(instances, out)
    for h in handles:
        h.close()


def test_batch_medium_graphs_match_single_solves():
    """Larger instances (several degree tiers, several levels): each equals
    the standalone GPU solve, which the parity suite ties to the oracle; one
    of them is checked against the oracle directly."""
    graphs = [synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 6000, "T": 5}),
              synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 3000, "T": 3, "seed": 7}),
              synth.recipe_graph("planted_t4_n1000")]
    handles = [pkg.mslice_build(s) for s in graphs]
    params = [((1, 1), (1, 1)), ((3, 2), (1, 4)), ((1, 2), (2, 1)), ((1, 1), (0, 1))]
    instances = [(handles[i % 3], graphs[i % 3], g, w, None) for i, (g, w) in enumerate(params)]
    out, _ = run_batch(instances)
    for (h, snaps, gamma, omega, _), (lab, Q) in zip(instances, out):
        sl, sq, _ = h.mslice_leiden(gamma=gamma, omega=omega)
        assert np.array_equal(lab, sl) and Q == sq
    check_against_oracle(instances[:1], out[:1])
    for h in handles:
        h.close()


def test_batch_rejects_bad_input():
    snaps = synth.random_temporal(6, 2, p=0.5, seed=1)
    with pkg.mslice_build(snaps) as h, pkg.Batch() as b:
        with pytest.raises(pkg.MsliceError):
            b.run()  # empty
        with pytest.raises(pkg.MsliceError):
            b.add(h, (0, 1), (1, 1))
        with pytest.raises(pkg.MsliceError):
            b.add(h, (1, 1), (1, 1), init=np.full(12, 12, np.int32))
        b.add(h)
        with pytest.raises(pkg.MsliceError):
            b.results(1)
        b.run()
        lab, Q = b.results(0)
        assert np.array_equal(lab, oracle.leiden(snaps)[0])


def test_many_tiny_instances():
    """More instances than fit any fixed host staging area (600 Q values),
    each against the oracle."""
    handles, instances = [], []
    rng = np.random.default_rng(77)
    for k in range(600):
        n, T = int(rng.integers(1, 25)), int(rng.integers(1, 4))
        snaps = synth.random_temporal(n, T, p=float(rng.uniform(0.05, 0.5)), w_max=3, seed=k)
        h = pkg.mslice_build(snaps)
        handles.append(h)
        instances.append((h, snaps, [(1, 1), (3, 2), (1, 2)][k % 3], [(1, 1), (0, 1), (2, 1)][(k // 3) % 3], None))
    out, _ = run_batch(instances)
    check_against_oracle(instances, out)
    for h in handles:
        h.close()
