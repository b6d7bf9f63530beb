"""Windowed optimisation (mslice_leiden_windowed) on the GPU against the
oracle's leiden_windowed: the stitched labels bit-exact, every window's Q
within 1e-12 relative and the same number of windows -- on random sequences
of every overlap, a school-shaped contact sequence, the other null models,
device-pointer input, and a sequence that fits one window (the plain solve).
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


def both(snaps, W, S, gamma=(1, 1), omega=(1, 1), null="multislice", **kw):
    g = pkg.leiden_windowed(snaps, W, S, gamma, omega, null=null, **kw)
    o = oracle.leiden_windowed(snaps, W, S, gamma, omega, null=null, **kw)
    return g, o


def assert_same(g, o):
    gl, gq, _ = g
    ol, oq, nw = o
    assert len(gq) == nw == len(oq)
    bad = np.flatnonzero(gl != ol)
    assert bad.size == 0, f"{bad.size} labels differ, first at {bad[:5]}"
    for k, (a, b) in enumerate(zip(gq, oq)):
        assert q_close(a, b), (k, a, b)


@pytest.mark.parametrize("seed", range(16))
def test_random_sequences(seed):
    rng = np.random.default_rng(900 + seed)
    T = int(rng.integers(4, 40))
    n = int(rng.integers(3, 40))
    snaps, _ = synth.planted_partition_temporal(n, T, n_blocks=int(rng.integers(2, 4)), p_in=0.3, p_out=0.03,
                                                switch_frac=0.1, churn=0.1, w_max=4, seed=seed)
    W = int(rng.integers(2, 10))
    S = int(rng.integers(1, W))
    gamma = [(1, 1), (3, 2), (1, 2)][seed % 3]
    omega = [(1, 1), (1, 4), (3, 1), (0, 1)][seed % 4]
    assert_same(*both(snaps, W, S, gamma, omega, K=[4, 2, 3][seed % 3], seed=seed))


def test_school_shaped_sequence():
    snaps = synth.recipe_graph("school_t7375_n327", T=400)
    for W, S in [(32, 16), (50, 49), (16, 1)]:
        assert_same(*both(snaps, W, S))


@pytest.mark.parametrize("null", ["global", "cpm"])
def test_other_null_models(null):
    snaps = synth.recipe_graph("school_t7375_n327", T=120)
    gamma = (1, 1) if null == "global" else (1, 20)
    assert_same(*both(snaps, 24, 10, gamma, (1, 2), null=null))


def test_one_window_is_the_plain_solve():
    snaps = synth.recipe_graph("planted_t4_n1000")
    lab, Qs, st = pkg.leiden_windowed(snaps, 8, 3)
    with pkg.mslice_build(snaps) as h:
        ref, Q, _ = h.mslice_leiden()
    assert np.array_equal(lab, ref) and Qs == [Q]


def test_device_pointer_input():
    torch = _cuda()
    snaps = synth.recipe_graph("school_t7375_n327", T=90)

    class D:
        def __init__(self, s):
            self.indptr = torch.from_numpy(s.indptr).cuda()
            self.indices = torch.from_numpy(s.indices).cuda()
            self.weights = torch.from_numpy(s.weights).cuda()

    dev = [D(s) for s in snaps]
    g = pkg.leiden_windowed(dev, 20, 8, device_ptrs=True)
    o = oracle.leiden_windowed(snaps, 20, 8)
    assert_same(g, o)


def test_rejections():
    snaps = synth.random_temporal(10, 12, p=0.3, seed=2)
    for W, S in [(0, 1), (4, 0), (4, 4), (4, 5)]:
        with pytest.raises(pkg.MsliceError) as e:
            pkg.leiden_windowed(snaps, W, S)
        assert e.value.code == pkg.MSLICE_EINVAL, (W, S)
    bad = synth.Snapshot(snaps[5].indptr, snaps[5].indices, snaps[5].weights.copy())
    if bad.nnz:
        bad.weights[0] += 1  # asymmetric
        with pytest.raises(pkg.MsliceError) as e:
            pkg.leiden_windowed(snaps[:5] + [bad] + snaps[6:], 4, 2)
        assert e.value.code == pkg.MSLICE_EINVAL
    lab, Qs, _ = pkg.leiden_windowed(snaps, 12, 5)  # T == W: one window, any stride
    assert len(Qs) == 1
