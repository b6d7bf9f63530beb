"""ctypes wrapper of the multislice-Leiden ORACLE (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU baseline import this
package.  The shared object ``liboracle.so`` is compiled from ``oracle.cpp``
by :func:`build` (plain g++, single-threaded code, ``-ffp-contract=off`` so
that the fixed FP64 evaluation order of Q is kept on every host).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")

OK, EINVAL, EOVERFLOW = 0, -1, -3
NULL_MULTISLICE, NULL_GLOBAL, NULL_CPM = 0, 1, 2
_NULLS = {"multislice": NULL_MULTISLICE, "global": NULL_GLOBAL, "cpm": NULL_CPM}
ORDINAL, CATEGORICAL = 0, 1
_COUPLINGS = {"ordinal": ORDINAL, "categorical": CATEGORICAL}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("indptr", C.c_void_p), ("indices", C.c_void_p), ("weights", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("n_iterations", C.c_int32), ("K", C.c_int32), ("max_rounds", C.c_int32),
                ("max_levels", C.c_int32), ("seed", C.c_uint64), ("stop_level", C.c_int32),
                ("stop_stage", C.c_int32), ("stop_rounds", C.c_int32), ("null_model", C.c_int32),
                ("pad_", C.c_int32), ("theta_num", C.c_int64), ("theta_den", C.c_int64)]


class _General(C.Structure):
    _fields_ = [("coupling", C.c_int32), ("pad_", C.c_int32), ("omega_num", C.c_void_p), ("gamma_num", C.c_void_p),
                ("gamma_den", C.c_void_p)]


class _Gen:
    """The general form (coupling pattern, per-pair omega numerators over the
    call's omega denominator, per-slice gamma as (num, den) pairs); None when
    every part takes its default, so the plain path is exercised."""

    def __init__(self, coupling="ordinal", omegas=None, gammas=None):
        self.arrays = []
        self.struct = None
        if coupling == "ordinal" and omegas is None and gammas is None:
            return
        g = _General(_COUPLINGS[coupling] if isinstance(coupling, str) else int(coupling), 0, None, None, None)
        if omegas is not None:
            om = np.ascontiguousarray(np.asarray(omegas, dtype=np.int64).ravel())
            self.arrays.append(om)
            g.omega_num = _ptr(om)
        if gammas is not None:
            gn = np.ascontiguousarray([int(x[0]) for x in gammas], dtype=np.int64)
            gd = np.ascontiguousarray([int(x[1]) for x in gammas], dtype=np.int64)
            self.arrays += [gn, gd]
            g.gamma_num, g.gamma_den = _ptr(gn), _ptr(gd)
        self.struct = g

    @property
    def ptr(self):
        return C.byref(self.struct) if self.struct is not None else None


class _LevelOut(C.Structure):
    _fields_ = [("N", C.c_int64), ("nnz", C.c_int64), ("ns", C.c_int64), ("cap_N", C.c_int64),
                ("cap_nnz", C.c_int64), ("cap_ns", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("W", C.c_void_p), ("sptr", C.c_void_p), ("sidx", C.c_void_p), ("sval", C.c_void_p),
                ("init_labels", C.c_void_p), ("node_map", C.c_void_p)]


class _Stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("levels", C.c_int32), ("lm_rounds", C.c_int64),
                ("lm_edges", C.c_int64), ("lm_moves", C.c_int64), ("last_level0_moves", C.c_int64),
                ("out_n", C.c_int64), ("next_n", C.c_int64), ("next_nnz", C.c_int64),
                ("next_checksum", C.c_uint64), ("stop_reason", C.c_int32), ("pad_", C.c_int32)]


def build(force: bool = False) -> str:
    src = os.path.join(HERE, "oracle.cpp")
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC",
                               src, "-o", tmp])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.orc_leiden.argtypes = [P, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int64, P, P, P, P,
                                 C.c_int64, P, P]
        L.orc_modularity.argtypes = [P, C.c_int32, P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int32, P,
                                     P]
        L.orc_move_key.argtypes = [P, C.c_int32, P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int32, P,
                                   C.c_int64, C.c_int64, P]
        L.orc_lambda.argtypes = [P, C.c_int32, C.c_int64, C.c_int64, P, P]
        L.orc_count_improving.argtypes = [P, C.c_int32, P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int32,
                                          P, P]
        L.orc_aggregate.argtypes = [P, C.c_int32, C.c_int64, C.c_int64, C.c_int32, P, P, P, P]
        L.orc_level_key.argtypes = [P, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int32, P, P, P,
                                    P, C.c_int64, C.c_int64, P]
        L.orc_exp_weight.argtypes = [C.c_uint64] * 5
        L.orc_exp_weight.restype = C.c_uint64
        L.orc_mix64.argtypes = [C.c_uint64]
        L.orc_mix64.restype = C.c_uint64
        L.orc_default_opts.argtypes = [P]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _Slices:
    """Keeps the numpy arrays alive while the struct array is in use."""

    def __init__(self, snaps):
        self.arrays = []
        self.arr = (_Csr * max(len(snaps), 1))()
        for s, sn in enumerate(snaps):
            ip = np.ascontiguousarray(sn.indptr, dtype=np.int64)
            ix = np.ascontiguousarray(sn.indices, dtype=np.int32)
            w = np.ascontiguousarray(sn.weights, dtype=np.int32)
            self.arrays += [ip, ix, w]
            self.arr[s] = _Csr(len(ip) - 1, _ptr(ip), _ptr(ix), _ptr(w))
        self.T = len(snaps)
        self.N = (len(snaps[0].indptr) - 1) * len(snaps) if snaps else 0

    @property
    def ptr(self):
        return C.cast(self.arr, C.c_void_p)


def _check(rc, what):
    if rc != OK:
        raise OracleError(rc, what)


def _null(null) -> int:
    """'multislice' (Q_MS's per-slice null term) or 'global' (plain modularity
    of the supra-graph); an int passes through unchanged."""
    return _NULLS[null] if isinstance(null, str) else int(null)


def leiden(snaps, gamma=(1, 1), omega=(1, 1), n_iterations=2, K=4, max_rounds=100, max_levels=32, seed=0,
           init=None, stop_level=-1, stop_stage=0, stop_rounds=0, null="multislice", coupling="ordinal",
           omegas=None, gammas=None, theta=None):
    """Returns (labels int32[...], Q, stats dict).  coupling / omegas /
    gammas: the general form (omega^(sr) numerators over omega[1], per-slice
    gamma pairs).  theta: (num, den) of the randomised refinement (None:
    the greedy limit)."""
    S = _Slices(snaps)
    tn, td = theta if theta is not None else (0, 1)
    o = _Opts(n_iterations, K, max_rounds, max_levels, seed, stop_level, stop_stage, stop_rounds, _null(null), 0,
              tn, td)
    cap = max(S.N, 1)
    out = np.zeros(cap, dtype=np.int32)
    Q = C.c_double(0.0)
    st = _Stats()
    init_a = None if init is None else np.ascontiguousarray(init, dtype=np.int32)
    gen = _Gen(coupling, omegas, gammas)
    rc = lib().orc_leiden(S.ptr, S.T, gamma[0], gamma[1], omega[0], omega[1], C.byref(o), gen.ptr, _ptr(init_a),
                          _ptr(out), cap, C.byref(Q), C.byref(st))
    _check(rc, "orc_leiden")
    stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
    return out[: st.out_n].copy(), Q.value, stats


def modularity(snaps, labels, gamma=(1, 1), omega=(1, 1), null="multislice", coupling="ordinal", omegas=None,
               gammas=None):
    S = _Slices(snaps)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    Q = C.c_double(0.0)
    gen = _Gen(coupling, omegas, gammas)
    _check(lib().orc_modularity(S.ptr, S.T, _ptr(lab), gamma[0], gamma[1], omega[0], omega[1], _null(null),
                                gen.ptr, C.byref(Q)), "orc_modularity")
    return Q.value


def move_key(snaps, labels, v, c, gamma=(1, 1), omega=(1, 1), null="multislice", coupling="ordinal",
             omegas=None, gammas=None) -> int:
    S = _Slices(snaps)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    out = (C.c_uint64 * 2)()
    gen = _Gen(coupling, omegas, gammas)
    _check(lib().orc_move_key(S.ptr, S.T, _ptr(lab), gamma[0], gamma[1], omega[0], omega[1], _null(null), gen.ptr,
                              v, c, out), "orc_move_key")
    x = out[0] | (out[1] << 64)
    return x - (1 << 128) if x >> 127 else x


def lambdas(snaps, gamma=(1, 1)):
    S = _Slices(snaps)
    lam = np.zeros(2 * S.T, dtype=np.uint64)
    tm = np.zeros(S.T, dtype=np.int64)
    _check(lib().orc_lambda(S.ptr, S.T, gamma[0], gamma[1], _ptr(lam), _ptr(tm)), "orc_lambda")
    return [int(lam[2 * s]) | (int(lam[2 * s + 1]) << 64) for s in range(S.T)], [int(x) for x in tm]


def count_improving(snaps, labels, gamma=(1, 1), omega=(1, 1), null="multislice", coupling="ordinal",
                    omegas=None, gammas=None) -> int:
    S = _Slices(snaps)
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    cnt = C.c_int64(0)
    gen = _Gen(coupling, omegas, gammas)
    _check(lib().orc_count_improving(S.ptr, S.T, _ptr(lab), gamma[0], gamma[1], omega[0], omega[1], _null(null),
                                     gen.ptr, C.byref(cnt)), "orc_count_improving")
    return cnt.value


def aggregate(snaps, P, R, omega=(1, 1), null="multislice", coupling="ordinal", omegas=None):
    """One aggregation step of the level-0 supra-graph for the local-moving
    partition P and its refinement R.  Returns a dict: N, rows (per new node a
    list of (column, W) pairs, W in units of 1/omega[1]), slices (per new node
    a list of (snapshot, strength) pairs), init (initial labels of the new
    level) and map (new id of every level-0 node)."""
    S = _Slices(snaps)
    Pa = np.ascontiguousarray(P, dtype=np.int32)
    Ra = np.ascontiguousarray(R, dtype=np.int32)
    gen = _Gen(coupling, omegas, None)
    out = _LevelOut()
    _check(lib().orc_aggregate(S.ptr, S.T, omega[0], omega[1], _null(null), gen.ptr, _ptr(Pa), _ptr(Ra),
                               C.byref(out)), "orc_aggregate")
    N, nnz, ns = out.N, out.nnz, out.ns
    rowptr = np.zeros(N + 1, np.int64)
    col = np.zeros(max(nnz, 1), np.int32)
    W = np.zeros(max(nnz, 1), np.int64)
    sptr = np.zeros(N + 1, np.int64)
    sidx = np.zeros(max(ns, 1), np.int32)
    sval = np.zeros(max(ns, 1), np.int64)
    init = np.zeros(max(N, 1), np.int32)
    mp = np.zeros(max(S.N, 1), np.int32)
    out.cap_N, out.cap_nnz, out.cap_ns = N, nnz, ns
    for f, a in [("rowptr", rowptr), ("col", col), ("W", W), ("sptr", sptr), ("sidx", sidx), ("sval", sval),
                 ("init_labels", init), ("node_map", mp)]:
        setattr(out, f, _ptr(a))
    _check(lib().orc_aggregate(S.ptr, S.T, omega[0], omega[1], _null(null), gen.ptr, _ptr(Pa), _ptr(Ra),
                               C.byref(out)), "orc_aggregate")
    rows = [[(int(col[e]), int(W[e])) for e in range(rowptr[x], rowptr[x + 1])] for x in range(N)]
    slices = [[(int(sidx[j]), int(sval[j])) for j in range(sptr[x], sptr[x + 1])] for x in range(N)]
    return {"N": N, "rows": rows, "slices": slices, "init": init[:N].tolist(), "map": mp[:S.N].tolist()}


def level_key(snaps, P, R, labels1, x, c, gamma=(1, 1), omega=(1, 1), null="multislice", coupling="ordinal",
              omegas=None, gammas=None) -> int:
    """Key G(x, c) at the level aggregated from (P, R), under that level's
    labels labels1 (c = -1: an empty community)."""
    S = _Slices(snaps)
    Pa = np.ascontiguousarray(P, dtype=np.int32)
    Ra = np.ascontiguousarray(R, dtype=np.int32)
    La = np.ascontiguousarray(labels1, dtype=np.int32)
    out = (C.c_uint64 * 2)()
    gen = _Gen(coupling, omegas, gammas)
    _check(lib().orc_level_key(S.ptr, S.T, gamma[0], gamma[1], omega[0], omega[1], _null(null), gen.ptr, _ptr(Pa),
                               _ptr(Ra), _ptr(La), x, c, out), "orc_level_key")
    v = out[0] | (out[1] << 64)
    return v - (1 << 128) if v >> 127 else v


def serve_warm_start(prev, n, W):
    """Initial labels of the next served window (the serving rule; the paper
    names windowed optimisation, Sec. 4, without a procedure): with w_prev
    slices in the previous result and e = 1 when the window already held W
    slices (the oldest is evicted), supra-node (j, i) of the new window of
    min(w_prev + 1, W) slices starts with the previous label of
    (min(j + e, w_prev - 1), i): surviving slices keep their labels and the
    new slice copies the previous newest one.  None (the first snapshot):
    singletons."""
    if prev is None:
        return None
    prev = np.asarray(prev)
    w_prev = len(prev) // n
    e = 1 if w_prev == W else 0
    w_new = min(w_prev + 1, W)
    src = np.minimum(np.arange(w_new) + e, w_prev - 1)
    return np.concatenate([prev[s * n:(s + 1) * n] for s in src]).astype(np.int32)


def serve_chain(stream, W, gamma=(1, 1), omega=(1, 1), **kw):
    """What a server computes for one live graph: request t solves the window
    of the last min(t + 1, W) snapshots, warm-started by serve_warm_start from
    the previous request's labels.  Returns [(labels, Q), ...] per request."""
    n = stream[0].n
    prev, out = None, []
    for t in range(len(stream)):
        window = stream[max(0, t + 1 - W):t + 1]
        lab, Q, _ = leiden(window, gamma, omega, init=serve_warm_start(prev, n, W), **kw)
        out.append((lab, Q))
        prev = lab
    return out


def exp_weight(d: int, div: int, theta_den: int) -> int:
    """The randomised refinement's fixed-point weight for key difference d and
    divisor div = 2M * theta_num (Python ints, each below 2^128)."""
    m = (1 << 64) - 1
    return int(lib().orc_exp_weight(d & m, d >> 64, div & m, div >> 64, theta_den))


def mix64(x: int) -> int:
    return int(lib().orc_mix64(x & ((1 << 64) - 1)))


def window_starts(T: int, W: int, stride: int):
    """First snapshot of every window: 0, stride, 2*stride, ... with the last
    start clamped to T - W, so every window holds W snapshots and the last
    ends at T (a single window [0, T) when T <= W)."""
    if T <= W:
        return [0]
    starts = [0]
    while starts[-1] + W < T:
        starts.append(min(starts[-1] + stride, T - W))
    return starts


def leiden_windowed(snaps, W, stride, gamma=(1, 1), omega=(1, 1), null="multislice", **kw):
    """Windowed optimisation of a long snapshot sequence (the paper names
    windowed optimisation for its 7,375-snapshot case, Sec. 4, and gives no
    procedure; this is the reading both implementations follow):

    * windows of W snapshots start at window_starts(T, W, stride);
    * window 0 starts from singletons; window k is warm-started by the
      serving rule with the shift e = start_k - start_{k-1}: its local
      snapshot j takes the previous window's labels of local snapshot
      min(j + e, W - 1), so the overlap keeps its labels and the new
      snapshots copy the previous window's last one;
    * stitching: the communities of window k are taken in order of first
      occurrence (supra-node order); one whose first supra-node lies in the
      overlap (the window's first W - e snapshots) continues the stitched
      label of that supra-node unless an earlier community of the window
      already continued it; every other community gets the next fresh label.
      Window k's labels then overwrite its snapshots' stitched labels, so
      within a window the stitched labels are a renaming of its partition;
    * the stitched labels are renumbered by first occurrence at the end.

    Returns (labels int32[n*T], Q of every window's solve, number of windows)."""
    T, n = len(snaps), snaps[0].n
    starts = window_starts(T, W, stride)
    out = np.full(n * T, -1, dtype=np.int64)
    fresh = 0
    prev, prev_start, Qs = None, None, []
    for a in starts:
        b = min(a + W, T)
        e = 0 if prev is None else a - prev_start
        init = None
        if prev is not None:
            src = np.minimum(np.arange(b - a) + e, len(prev) // n - 1)
            init = np.concatenate([prev[s * n:(s + 1) * n] for s in src]).astype(np.int32)
        lab, Q, _ = leiden(snaps[a:b], gamma, omega, init=init, null=null, **kw)
        Qs.append(Q)
        n_comm = int(lab.max()) + 1 if len(lab) else 0
        first = np.full(n_comm, len(lab), dtype=np.int64)
        np.minimum.at(first, lab, np.arange(len(lab)))
        overlap = 0 if prev is None else (b - a - e) * n
        stitched = np.empty(n_comm, dtype=np.int64)
        taken = set()
        for c in range(n_comm):  # canonical labels: c ascending is first-occurrence order
            if first[c] < overlap and int(out[a * n + first[c]]) not in taken:
                stitched[c] = out[a * n + first[c]]
                taken.add(int(stitched[c]))
            else:
                stitched[c] = fresh
                fresh += 1
        out[a * n:b * n] = stitched[lab]
        prev, prev_start = lab, a
    # renumber by first occurrence
    seen = {}
    final = np.empty(n * T, dtype=np.int32)
    for v, x in enumerate(out.tolist()):
        final[v] = seen.setdefault(x, len(seen))
    return final, Qs, len(starts)
