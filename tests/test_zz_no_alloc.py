"""The allocation-free Q entry point (mslice_modularity_noalloc) against the
handle-based one (mslice_modularity), through the C ABI.

That entry point serves callers that cannot allocate device memory (graph
capture, fixed memory budgets): its scratch is one fixed array inside the
library, shared by every call.  The checks run two calls in a row, so a
second call that saw the first call's leftovers would fail.  This file is
collected last so a run that stops at the first failure has already run
everything else; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import paper_2608_03695_gb300 as pkg
from paper_2608_03695_gb300 import synth
from qtol import q_close

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _device_slices(torch, snaps):
    keep, arr = [], (pkg.Csr * len(snaps))()
    for s, sn in enumerate(snaps):
        ip = torch.from_numpy(sn.indptr).cuda()
        ix = torch.from_numpy(sn.indices).cuda()
        w = torch.from_numpy(sn.weights).cuda()
        keep += [ip, ix, w]
        arr[s] = pkg.Csr(sn.n, ip.data_ptr(), ix.data_ptr(), w.data_ptr())
    return arr, keep


def _noalloc_q(torch, snaps, labels, gamma, omega):
    arr, keep = _device_slices(torch, snaps)
    dlab = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.int32)).cuda()
    q = C.c_double(0.0)
    rc = pkg.lib().mslice_modularity_noalloc(C.cast(arr, C.c_void_p), len(snaps), C.c_void_p(dlab.data_ptr()),
                                            gamma[0], gamma[1], omega[0], omega[1], None, C.byref(q))
    return rc, q.value


def _close(a, b):
    return q_close(a, b)


@pytest.mark.parametrize("case", range(3))
def test_noalloc_matches_handle_path_twice(case):
    torch = _torch()
    pkg.build()
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
            want = h.mslice_modularity(lab, gamma, omega)
            for _ in range(2):  # the second call must not see the first call's scratch
                rc, got = _noalloc_q(torch, snaps, lab, gamma, omega)
                assert rc == pkg.MSLICE_OK, pkg.lib().mslice_last_error()
                assert _close(got, want), (got, want)


def test_noalloc_rejects_oversize_and_bad_labels():
    torch = _torch()
    pkg.build()
    snaps = synth.recipe_graph("planted_t4_n1000")
    bad = np.full(4000, 4000, np.int32)
    rc, _ = _noalloc_q(torch, snaps, bad, (1, 1), (1, 1))
    assert rc == pkg.MSLICE_EINVAL
    # a valid call right after a rejected one still works
    labels = np.arange(4000, dtype=np.int32) % 7
    rc, q = _noalloc_q(torch, snaps, labels, (1, 1), (1, 1))
    assert rc == pkg.MSLICE_OK
    with pkg.mslice_build(snaps) as h:
        assert _close(q, h.mslice_modularity(labels))
    # n*T*T beyond the fixed scratch: 3000 nodes x 40 snapshots x 40
    big = [synth.Snapshot(np.zeros(3001, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))] * 40
    rc, _ = _noalloc_q(torch, big, np.zeros(3000 * 40, np.int32), (1, 1), (1, 1))
    assert rc == pkg.MSLICE_EINVAL
    assert b"scratch" in pkg.lib().mslice_last_error()
