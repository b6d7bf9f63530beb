"""The allocation-free Q entry point (mslice_modularity_noalloc) through the C
ABI, against the oracle's Q and the handle-based mslice_modularity.

That entry point serves callers that cannot allocate device memory (plug-ins
held to a memory budget by their host application, services that reserve all
device memory up front): its scratch is one fixed array inside the library,
shared by every call.  The checks run two calls in a row, so a second call
that saw the first call's leftovers would fail, and they check that the
device's free memory does not change across calls.  This file is collected
last so a run that stops at the first failure has already run everything
else; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2608_03695_gb300 as pkg
from paper_2608_03695_gb300 import synth
from qtol import q_close

pytestmark = pytest.mark.gpu

# scratch capacity of the entry point, in 8-byte words (4 + 6*T + N*T must fit)
SCRATCH_WORDS = 4 * 1024 * 1024


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


class DeviceCase:
    """Snapshots and labels copied to the device once (torch allocations made
    before any measured call)."""

    def __init__(self, torch, snaps, labels, n=None):
        self.keep, self.arr = [], (pkg.Csr * len(snaps))()
        for s, sn in enumerate(snaps):
            ip = torch.from_numpy(np.ascontiguousarray(sn.indptr)).cuda()
            ix = torch.from_numpy(np.ascontiguousarray(sn.indices)).cuda() if len(sn.indices) else None
            w = torch.from_numpy(np.ascontiguousarray(sn.weights)).cuda() if len(sn.weights) else None
            self.keep += [ip, ix, w]
            self.arr[s] = pkg.Csr(sn.n if n is None else n, ip.data_ptr(), ix.data_ptr() if ix is not None else None,
                                  w.data_ptr() if w is not None else None)
        self.T = len(snaps)
        self.dlab = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.int32)).cuda()

    def q(self, gamma=(1, 1), omega=(1, 1)):
        out = C.c_double(0.0)
        rc = pkg.lib().mslice_modularity_noalloc(C.cast(self.arr, C.c_void_p), self.T,
                                                C.c_void_p(self.dlab.data_ptr()), gamma[0], gamma[1], omega[0],
                                                omega[1], None, C.byref(out))
        return rc, out.value


@pytest.fixture(scope="module", autouse=True)
def built():
    _torch()
    pkg.build()
    oracle.build()


@pytest.mark.parametrize("case", range(3))
def test_noalloc_matches_oracle_and_handle_path_twice(case):
    torch = _torch()
    rng = np.random.default_rng(case)
    if case == 0:
        snaps = synth.recipe_graph("planted_t4_n1000")
    elif case == 1:
        snaps = synth.recipe_graph({**synth.RECIPES["powerlaw_t16_n100k"], "n": 5000, "T": 6})
    else:
        snaps = synth.random_temporal(40, 3, p=0.2, w_max=5, seed=7, p_empty=0.3)
    N = snaps[0].n * len(snaps)
    with pkg.mslice_build(snaps) as h:
        labels, _, _ = h.mslice_leiden()
        other = rng.integers(0, max(1, N // 10), size=N).astype(np.int32)
        for lab, gamma, omega in [(labels, (1, 1), (1, 1)), (other, (3, 2), (1, 10)), (labels, (1, 2), (0, 1))]:
            want = oracle.modularity(snaps, lab, gamma, omega)
            assert q_close(h.mslice_modularity(lab, gamma, omega), want)
            dc = DeviceCase(torch, snaps, lab)
            for _ in range(2):  # the second call must not see the first call's scratch
                rc, got = dc.q(gamma, omega)
                assert rc == pkg.MSLICE_OK, pkg.lib().mslice_last_error()
                assert q_close(got, want), (got, want)


def test_noalloc_allocates_no_device_memory():
    torch = _torch()
    snaps = synth.recipe_graph("planted_t4_n1000")
    lab = (np.arange(4000) % 9).astype(np.int32)
    dc = DeviceCase(torch, snaps, lab)
    assert dc.q()[0] == pkg.MSLICE_OK  # first call: the scratch address is looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        rc, _ = dc.q((3, 2), (1, 4))
        assert rc == pkg.MSLICE_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_at_the_scratch_limit():
    """T = 2 and n = 1,048,572 use exactly 4 + 6T + nT*T = 4,194,304 words; one
    more node is rejected."""
    torch = _torch()
    T = 2
    n = (SCRATCH_WORDS - 4 - 6 * T) // (T * T)
    assert 4 + 6 * T + n * T * T == SCRATCH_WORDS
    rng = np.random.default_rng(5)
    snaps = []
    for s in range(T):
        u = rng.integers(0, n, 300_000)
        v = rng.integers(0, n, 300_000)
        key = np.unique(np.minimum(u, v) * n + np.maximum(u, v))
        a, b = key // n, key % n
        a, b = a[a != b], b[a != b]
        snaps.append(synth.csr_from_edges(n, a, b, rng.integers(1, 6, len(a)).astype(np.int32)))
    lab = rng.integers(0, 500, n * T).astype(np.int32)
    want = oracle.modularity(snaps, lab, (1, 1), (1, 3))
    dc = DeviceCase(torch, snaps, lab)
    for _ in range(2):
        rc, got = dc.q((1, 1), (1, 3))
        assert rc == pkg.MSLICE_OK, pkg.lib().mslice_last_error()
        assert q_close(got, want), (got, want)
    over = [synth.Snapshot(np.zeros(n + 2, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))] * T
    rc, _ = DeviceCase(torch, over, np.zeros((n + 1) * T, np.int32)).q()
    assert rc == pkg.MSLICE_EINVAL
    assert b"scratch" in pkg.lib().mslice_last_error()


def test_noalloc_rejections_leave_the_next_call_working():
    torch = _torch()
    snaps = synth.recipe_graph("planted_t4_n1000")
    labels = np.arange(4000, dtype=np.int32) % 7
    want = oracle.modularity(snaps, labels)
    good = DeviceCase(torch, snaps, labels)

    def ok_again():
        rc, q = good.q()
        assert rc == pkg.MSLICE_OK and q_close(q, want)

    # a label out of [0, N)
    assert DeviceCase(torch, snaps, np.full(4000, 4000, np.int32)).q()[0] == pkg.MSLICE_EINVAL
    ok_again()
    # bounds of the 2^61 conventions: gamma * omega_den * sum 2m_s
    assert good.q((1 << 31, 1), (1, 1 << 31))[0] == pkg.MSLICE_EOVERFLOW
    ok_again()
    # malformed snapshots: a self-loop, a repeated column, descending columns
    base = synth.csr_from_edges(4, np.array([0, 1, 2]), np.array([1, 2, 3]), np.ones(3, np.int32))
    lab4 = np.zeros(4, np.int32)
    assert DeviceCase(torch, [base], lab4).q()[0] == pkg.MSLICE_OK
    for bad_ix in ([0, 0, 2, 1, 3, 2], [1, 0, 0, 1, 3, 2], [1, 0, 2, 3, 1, 2]):
        # rows 0:{1} 1:{0,2} 2:{1,3} 3:{2}; the variants give row 0 a self-loop,
        # row 1 a repeated column and row 2 descending columns
        ip = base.indptr.copy()
        sn = synth.Snapshot(ip, np.array(bad_ix, np.int32), base.weights.copy())
        assert DeviceCase(torch, [sn], lab4).q()[0] == pkg.MSLICE_EINVAL, bad_ix
        ok_again()
    # entries present but no index or weight array
    sn = synth.Snapshot(base.indptr.copy(), np.zeros(0, np.int32), base.weights.copy())
    assert DeviceCase(torch, [sn], lab4).q()[0] == pkg.MSLICE_EINVAL
    sn = synth.Snapshot(base.indptr.copy(), base.indices.copy(), np.zeros(0, np.int32))
    assert DeviceCase(torch, [sn], lab4).q()[0] == pkg.MSLICE_EINVAL
    ok_again()
