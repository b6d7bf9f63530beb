"""Failure handling, with failures made on the host (nothing faults the GPU).

MSLICE_FAIL_ALLOC_AFTER=k makes every device allocation after the k-th fail
as if the device were out of memory.  Whatever step it hits, the call must
return MSLICE_ENOMEM, and once injection stops the same handle, batch or
server must give the oracle's bits again.
"""
import numpy as np
import pytest

import oracle
import paper_2608_03695_gb300 as pkg
from paper_2608_03695_gb300 import synth

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


@pytest.fixture
def inject(monkeypatch):
    def on(k):
        monkeypatch.setenv("MSLICE_FAIL_ALLOC_AFTER", str(k))

    def off():
        monkeypatch.delenv("MSLICE_FAIL_ALLOC_AFTER", raising=False)

    yield on, off
    off()


def test_allocation_failures_in_build_and_solve(inject):
    on, off = inject
    snaps = synth.recipe_graph("planted_t4_n1000")
    ref, Qref, _ = oracle.leiden(snaps)
    failures = 0
    for k in [0, 1, 3, 8, 16, 32, 64, 128]:
        on(k)
        try:
            with pkg.mslice_build(snaps) as h:
                lab, Q, _ = h.mslice_leiden()
            # enough allocations were allowed: the result must be right
            assert np.array_equal(lab, ref) and Q == Qref
        except pkg.MsliceError as e:
            assert e.code == pkg.MSLICE_ENOMEM, (k, e)
            failures += 1
        off()
    assert failures > 0
    with pkg.mslice_build(snaps) as h:
        lab, Q, _ = h.mslice_leiden()
    assert np.array_equal(lab, ref) and Q == Qref


def test_handle_survives_a_failed_solve(inject):
    on, off = inject
    snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 3000, "T": 4})
    ref, Qref, _ = oracle.leiden(snaps)
    other, Qo, _ = oracle.leiden(snaps, gamma=(3, 2))
    with pkg.mslice_build(snaps) as h:
        on(0)  # the handle's first solve needs fresh buffers: it fails
        with pytest.raises(pkg.MsliceError) as e:
            h.mslice_leiden()
        assert e.value.code == pkg.MSLICE_ENOMEM
        off()
        lab, Q, _ = h.mslice_leiden()
        assert np.array_equal(lab, ref) and Q == Qref
        on(2)  # a later solve that fails part way
        try:
            h.mslice_leiden(gamma=(3, 2), K=7)
        except pkg.MsliceError as e2:
            assert e2.code == pkg.MSLICE_ENOMEM
        off()
        lab, Q, _ = h.mslice_leiden(gamma=(3, 2))
        assert np.array_equal(lab, other) and Q == Qo


def test_batch_survives_a_failed_run(inject):
    on, off = inject
    snaps = synth.recipe_graph("planted_t4_n1000")
    params = [((1, 1), (1, 1)), ((3, 2), (1, 4)), ((1, 2), (2, 1))]
    with pkg.mslice_build(snaps) as h, pkg.Batch() as b:
        for gm, om in params:
            b.add(h, gm, om)
        on(0)
        with pytest.raises(pkg.MsliceError) as e:
            b.run()
        assert e.value.code == pkg.MSLICE_ENOMEM
        with pytest.raises(pkg.MsliceError):
            b.results(0)  # a failed run leaves no results
        off()
        b.run()
        for i, (gm, om) in enumerate(params):
            lab, Q = b.results(i)
            ol, oq, _ = oracle.leiden(snaps, gm, om)
            assert np.array_equal(lab, ol) and Q == oq


def test_served_request_failure_leaves_the_window(inject):
    on, off = inject
    W, n = 3, 80
    stream, _ = synth.planted_partition_temporal(n, 5, 3, 0.15, 0.015, 0.1, 0.05, 8, 21)
    with pkg.Server(window=W, n_slots=1) as srv:
        g = srv.add_graph(n)
        first = [srv.wait(srv.submit(g, stream[t]))[0] for t in range(2)]
        on(0)
        with pytest.raises(pkg.MsliceError) as e:
            srv.wait(srv.submit(g, stream[2]))
        assert e.value.code == pkg.MSLICE_ENOMEM
        off()
        rest = [srv.wait(srv.submit(g, stream[t]))[0] for t in (3, 4)]
    # expected: the chain without the failed snapshot
    kept = [stream[0], stream[1], stream[3], stream[4]]
    prev, expect = None, []
    for t in range(len(kept)):
        init = None
        if prev is not None:
            w_prev = len(prev) // n
            e_ = 1 if w_prev == W else 0
            src = np.minimum(np.arange(min(w_prev + 1, W)) + e_, w_prev - 1)
            init = np.concatenate([prev[j * n:(j + 1) * n] for j in src]).astype(np.int32)
        lab, _, _ = oracle.leiden(kept[max(0, t + 1 - W):t + 1], init=init)
        expect.append(lab)
        prev = lab
    for got, exp in zip(first + rest, expect):
        assert np.array_equal(got, exp)


def test_windowed_run_fails_cleanly_and_recovers(inject):
    on, off = inject
    snaps = synth.recipe_graph("school_t7375_n327", T=60)
    ref, _, _ = oracle.leiden_windowed(snaps, 16, 8)
    failures = 0
    for k in [0, 2, 8, 40]:
        on(k)
        try:
            lab, _, _ = pkg.leiden_windowed(snaps, 16, 8)
            assert np.array_equal(lab, ref)
        except pkg.MsliceError as e:
            assert e.code == pkg.MSLICE_ENOMEM, (k, e)
            failures += 1
        off()
    assert failures > 0
    lab, _, _ = pkg.leiden_windowed(snaps, 16, 8)
    assert np.array_equal(lab, ref)
