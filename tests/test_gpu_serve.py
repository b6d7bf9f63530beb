"""Serving (mslice_server_*): sliding windows solved warm-started, admitted by
memory footprint and batched continuously.  Every result must equal the
oracle run on that window's slices from the warm-start labels (bit-exact
labels, Q within 1e-12 relative), and be the same whether the request was
served alone or mixed with other graphs' requests."""
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


def stream(n, steps, seed, churn=0.05):
    snaps, _ = synth.planted_partition_temporal(n, steps, n_blocks=3, p_in=min(1.0, 12.0 / n), p_out=1.2 / n,
                                                switch_frac=0.1, churn=churn, w_max=8, seed=seed)
    return snaps


def oracle_chain(snaps, W, gamma=(1, 1), omega=(1, 1)):
    """Expected (labels, Q) of every request of one graph's stream: the
    oracle's serving chain (window of the last W snapshots, warm-started from
    the previous request's labels)."""
    return oracle.serve_chain(snaps, W, gamma, omega)


def test_window_chain_matches_oracle():
    W = 4
    snaps = stream(120, 9, seed=3)
    expect = oracle_chain(snaps, W)
    with pkg.Server(window=W, n_slots=1) as srv:
        g = srv.add_graph(120)
        for t, sn in enumerate(snaps):
            lab, info = srv.wait(srv.submit(g, sn))
            assert info["slices"] == min(t + 1, W) and info["N"] == 120 * min(t + 1, W)
            assert np.array_equal(lab, expect[t][0]), t
            assert q_close(info["Q"], expect[t][1])


def test_alone_and_in_the_mix_agree():
    """Six graphs submitted all at once to three workers (batches of up to 4)
    give, request by request, what each graph gets served alone, and what the
    oracle chain gives."""
    W = 3
    graphs = [stream(int(n), 6, seed=10 + k) for k, n in enumerate([40, 90, 150, 60, 200, 75])]
    alone = []
    for snaps in graphs:
        with pkg.Server(window=W, n_slots=1, max_batch=1) as srv:
            g = srv.add_graph(snaps[0].n)
            alone.append([srv.wait(srv.submit(g, sn)) for sn in snaps])
    with pkg.Server(window=W, n_slots=3, max_batch=4) as srv:
        ids = [srv.add_graph(s[0].n) for s in graphs]
        reqs = []
        for t in range(6):
            for k, snaps in enumerate(graphs):
                reqs.append((k, t, srv.submit(ids[k], snaps[t])))
        mixed = {}
        batch_sizes = []
        for k, t, rid in reqs:
            mixed[(k, t)] = srv.wait(rid)
            batch_sizes.append(mixed[(k, t)][1]["batch_size"])
    for k in range(len(graphs)):
        for t in range(6):
            a, b = alone[k][t], mixed[(k, t)]
            assert np.array_equal(a[0], b[0]) and a[1]["Q"] == b[1]["Q"], (k, t)
    assert max(batch_sizes) > 1  # some requests were solved together
    for k in (0, 3):
        expect = oracle_chain(graphs[k], W)
        for t in range(6):
            assert np.array_equal(mixed[(k, t)][0], expect[t][0]), (k, t)


def test_tiny_budget_serialises_but_agrees():
    W = 3
    graphs = [stream(int(n), 4, seed=30 + k) for k, n in enumerate([50, 80, 30])]
    with pkg.Server(window=W, n_slots=2, max_batch=8, hbm_budget=1) as srv:
        ids = [srv.add_graph(s[0].n) for s in graphs]
        reqs = [(k, t, srv.submit(ids[k], graphs[k][t])) for t in range(4) for k in range(3)]
        res = {(k, t): srv.wait(rid) for k, t, rid in reqs}
    for k in range(3):
        expect = oracle_chain(graphs[k], W)
        for t in range(4):
            lab, info = res[(k, t)]
            assert info["batch_size"] == 1  # nothing fits beside another request
            assert np.array_equal(lab, expect[t][0])


def test_bad_snapshot_leaves_window_unchanged():
    W = 3
    snaps = stream(60, 5, seed=7)
    bad_w = snaps[2].weights.copy()
    bad_w[0] += 1  # asymmetric weight
    bad = synth.Snapshot(snaps[2].indptr, snaps[2].indices, bad_w)
    kept = [snaps[0], snaps[1], snaps[3], snaps[4]]
    expect = oracle_chain(kept, W)
    with pkg.Server(window=W, n_slots=2) as srv:
        g = srv.add_graph(60)
        r = [srv.submit(g, snaps[0]), srv.submit(g, snaps[1]), srv.submit(g, bad), srv.submit(g, snaps[3]),
             srv.submit(g, snaps[4])]
        out = [srv.wait(r[0]), srv.wait(r[1])]
        with pytest.raises(pkg.MsliceError) as e:
            srv.wait(r[2])
        assert e.value.code == pkg.MSLICE_EINVAL
        out += [srv.wait(r[3]), srv.wait(r[4])]
    for t in range(4):
        assert np.array_equal(out[t][0], expect[t][0]), t


def test_server_rejects_bad_arguments():
    with pytest.raises(pkg.MsliceError):
        pkg.Server(window=0)
    with pkg.Server(window=2) as srv:
        g = srv.add_graph(10)
        with pytest.raises(pkg.MsliceError):
            srv.submit(g + 1, stream(10, 1, 0)[0])
        with pytest.raises(pkg.MsliceError):
            srv.submit(g, stream(12, 1, 0)[0])  # n differs
        with pytest.raises(pkg.MsliceError):
            srv.wait(12345)


def test_checkpoint_and_resume_give_identical_bits():
    """A window checkpointed after some requests and restored into a new
    server continues exactly as the uninterrupted server does."""
    W, n = 3, 120
    snaps = stream(n, 8, seed=41)
    with pkg.Server(window=W, n_slots=2) as srv:
        g = srv.add_graph(n)
        whole = [srv.wait(srv.submit(g, sn)) for sn in snaps]
    with pkg.Server(window=W, n_slots=1) as srv:
        g = srv.add_graph(n)
        for t in range(5):
            srv.wait(srv.submit(g, snaps[t]))
        saved, labels = srv.checkpoint(g)
    assert len(saved) == W and len(labels) == W * n
    for k, sn in enumerate(saved):  # the window holds the last W snapshots
        ref = snaps[5 - W + k]
        assert np.array_equal(sn.indptr, ref.indptr) and np.array_equal(sn.indices, ref.indices)
    assert np.array_equal(labels, whole[4][0])
    with pkg.Server(window=W, n_slots=2) as srv:
        g = srv.add_graph(n)
        srv.restore(g, saved, labels)
        for t in range(5, 8):
            lab, info = srv.wait(srv.submit(g, snaps[t]))
            assert np.array_equal(lab, whole[t][0]) and info["Q"] == whole[t][1]["Q"], t


def test_restore_rejects_bad_state_and_keeps_the_window():
    W, n = 3, 60
    snaps = stream(n, 5, seed=43)
    expect = oracle_chain(snaps, W)
    with pkg.Server(window=W, n_slots=1) as srv:
        g = srv.add_graph(n)
        for t in range(3):
            srv.wait(srv.submit(g, snaps[t]))
        saved, labels = srv.checkpoint(g)
        bad_w = saved[1].weights.copy()
        bad_w[0] += 1
        bad = synth.Snapshot(saved[1].indptr, saved[1].indices, bad_w)
        with pytest.raises(pkg.MsliceError):
            srv.restore(g, [saved[0], bad, saved[2]], labels)  # asymmetric snapshot
        with pytest.raises(pkg.MsliceError):
            srv.restore(g, saved, np.full(len(labels), len(labels), np.int32))  # labels out of range
        with pytest.raises(pkg.MsliceError):
            srv.restore(g, saved + saved, np.zeros(6 * n, np.int32))  # more than W snapshots
        for t in (3, 4):  # the window is the one before the failed restores
            lab, _ = srv.wait(srv.submit(g, snaps[t]))
            assert np.array_equal(lab, expect[t][0]), t
