"""Python binding of the mslice CUDA library (multislice-modularity Leiden).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libmslice.so`` (built from ``csrc/`` for sm_103a).  Importing the
package does not need a GPU; calling into the library does, and there is no
CPU fallback: a missing library raises :class:`LibraryMissing`.

The entry points mirror ``include/mslice.h``:

* :func:`mslice_build` -- supra-graph of T snapshots (Eq. supra-adjacency)
* :meth:`Handle.mslice_leiden` -- Leiden on multislice modularity (Sec. 3.2)
* :meth:`Handle.mslice_modularity` -- Q_MS of a labelling
  (Eq. multislice-modularity)
* :class:`Batch` -- many (graph, gamma, omega) solves in one pass
  (``mslice_batch_create/add/run/results``)
* :class:`Server` -- sliding windows of live temporal graphs, warm-started,
  admitted by device-memory footprint and batched continuously
  (``mslice_server_*``)
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MSLICE_LIBRARY=checked loads the bounds-checked build (build(checked=True))
LIB_PATH = os.path.join(HERE, "libmslice_checked.so" if os.environ.get("MSLICE_LIBRARY") == "checked"
                        else "libmslice.so")

MSLICE_OK, MSLICE_EINVAL, MSLICE_ENOMEM, MSLICE_EOVERFLOW, MSLICE_ECUDA, MSLICE_ETIMEOUT = 0, -1, -2, -3, -4, -5
MSLICE_DEVICE_PTRS = 1
MSLICE_PROFILE = 2
MSLICE_AUTOTUNE = 4
MSLICE_NULL_GLOBAL = 8
MSLICE_NULL_CPM = 16
_NULLS = {"multislice": 0, "global": MSLICE_NULL_GLOBAL, "cpm": MSLICE_NULL_CPM}
MSLICE_ORDINAL = 0
MSLICE_CATEGORICAL = 1
_COUPLINGS = {"ordinal": MSLICE_ORDINAL, "categorical": MSLICE_CATEGORICAL}

# every symbol include/mslice.h declares
EXPORTS = ["mslice_default_opts", "mslice_build", "mslice_build_ex", "mslice_leiden", "mslice_leiden_ex",
           "mslice_leiden_general", "mslice_modularity", "mslice_modularity_ex", "mslice_modularity_general",
           "mslice_modularity_noalloc", "mslice_info", "mslice_batch_add_general", "mslice_leiden_windowed",
           "mslice_kernel_launches", "mslice_free", "mslice_last_error", "mslice_batch_create",
           "mslice_batch_add", "mslice_batch_run", "mslice_batch_results", "mslice_batch_info",
           "mslice_batch_clear", "mslice_batch_kernel_launches", "mslice_batch_free",
           "mslice_server_default_opts", "mslice_server_create", "mslice_server_add_graph",
           "mslice_server_submit", "mslice_server_wait", "mslice_server_free", "mslice_server_window_info",
           "mslice_server_window_read", "mslice_server_window_restore"]


class LibraryMissing(RuntimeError):
    pass


class MsliceError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mslice error {code}: {msg}")
        self.code = code


class Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("indptr", C.c_void_p), ("indices", C.c_void_p), ("weights", C.c_void_p)]


class Opts(C.Structure):
    _fields_ = [("n_iterations", C.c_int32), ("K", C.c_int32), ("max_rounds", C.c_int32),
                ("max_levels", C.c_int32), ("seed", C.c_uint64), ("gamma_num", C.c_int64),
                ("gamma_den", C.c_int64), ("omega_num", C.c_int64), ("omega_den", C.c_int64),
                ("flags", C.c_int32), ("stop_level", C.c_int32), ("stop_stage", C.c_int32),
                ("stop_rounds", C.c_int32), ("tier_cuts", C.c_int32 * 4), ("theta_num", C.c_int64),
                ("theta_den", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("levels", C.c_int32), ("lm_rounds", C.c_int64),
                ("lm_edges", C.c_int64), ("lm_moves", C.c_int64), ("last_level0_moves", C.c_int64),
                ("out_n", C.c_int64), ("next_n", C.c_int64), ("next_nnz", C.c_int64),
                ("next_checksum", C.c_uint64), ("stop_reason", C.c_int32), ("pad_", C.c_int32),
                ("kernel_launches", C.c_int64), ("ms_total", C.c_double), ("ms_local_move", C.c_double),
                ("ms_refine", C.c_double), ("ms_aggregate", C.c_double), ("ms_modularity", C.c_double),
                ("ms_decide", C.c_double), ("decide_launches", C.c_int64), ("decide_bytes", C.c_int64),
                ("tier_cuts", C.c_int32 * 4), ("ms_capped", C.c_double), ("capped_levels", C.c_int64),
                ("capped_rounds", C.c_int64), ("host_launches", C.c_int64)]


class ServerOpts(C.Structure):
    _fields_ = [("window", C.c_int32), ("n_slots", C.c_int32), ("max_batch", C.c_int32), ("pad_", C.c_int32),
                ("max_batch_nodes", C.c_int64), ("hbm_budget", C.c_int64), ("gamma_num", C.c_int64), ("gamma_den", C.c_int64),
                ("omega_num", C.c_int64), ("omega_den", C.c_int64), ("solve", Opts)]


class RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("slices", C.c_int32), ("N", C.c_int64), ("Q", C.c_double),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("batch_size", C.c_int32), ("slot", C.c_int32), ("footprint", C.c_int64),
                ("t_batch_start", C.c_double), ("t_batch_end", C.c_double)]


_lib = None


def build(force: bool = False, checked: bool = False) -> str:
    """Compiles libmslice.so (or, checked=True, libmslice_checked.so) in-tree
    (nvcc, sm_103a)."""
    from . import build_lib
    return build_lib.build(force=force, checked=checked)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LibraryMissing(f"{LIB_PATH} is not built; run paper_2608_03695_gb300.build()")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.mslice_default_opts.argtypes = [P]
        L.mslice_build.argtypes = [P, C.c_int32, C.c_int, C.c_int64, C.c_int64, P]
        L.mslice_build_ex.argtypes = [P, C.c_int32, C.c_int, C.c_int64, C.c_int64, C.c_int32, P, P]
        L.mslice_leiden.argtypes = [P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int32, C.c_uint64, P, P]
        L.mslice_leiden_ex.argtypes = [P, P, P, P, P, P]
        L.mslice_leiden_general.argtypes = [P, P, P, P, P, P, P]
        L.mslice_modularity_general.argtypes = [P, P, P, P, P]
        L.mslice_batch_add_general.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, P, P, P]
        L.mslice_leiden_windowed.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, C.c_int32, P, P]
        L.mslice_modularity.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, P]
        L.mslice_modularity_ex.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int32, P]
        L.mslice_modularity_noalloc.argtypes = [P, C.c_int32, P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, P, P]
        L.mslice_info.argtypes = [P, P, P, P, P]
        L.mslice_kernel_launches.argtypes = [P]
        L.mslice_kernel_launches.restype = C.c_int64
        L.mslice_free.argtypes = [P]
        L.mslice_free.restype = None
        L.mslice_last_error.restype = C.c_char_p
        L.mslice_batch_create.argtypes = [C.c_int32, P, P]
        L.mslice_batch_add.argtypes = [P, P, C.c_int64, C.c_int64, C.c_int64, C.c_int64, P, P]
        L.mslice_batch_run.argtypes = [P, P, P]
        L.mslice_batch_results.argtypes = [P, C.c_int32, P, P]
        L.mslice_batch_info.argtypes = [P, P, P, P]
        L.mslice_batch_clear.argtypes = [P]
        L.mslice_batch_kernel_launches.argtypes = [P]
        L.mslice_batch_kernel_launches.restype = C.c_int64
        L.mslice_batch_free.argtypes = [P]
        L.mslice_batch_free.restype = None
        L.mslice_server_default_opts.argtypes = [P]
        L.mslice_server_default_opts.restype = None
        L.mslice_server_create.argtypes = [P, P]
        L.mslice_server_add_graph.argtypes = [P, C.c_int64, P]
        L.mslice_server_submit.argtypes = [P, C.c_int32, P, P]
        L.mslice_server_wait.argtypes = [P, C.c_int64, P, P]
        L.mslice_server_free.argtypes = [P]
        L.mslice_server_free.restype = None
        L.mslice_server_window_info.argtypes = [P, C.c_int32, P, P]
        L.mslice_server_window_read.argtypes = [P, C.c_int32, C.c_int32, P, P, P, P]
        L.mslice_server_window_restore.argtypes = [P, C.c_int32, P, C.c_int32, P]
        _lib = L
    return _lib


class General(C.Structure):
    """``mslice_general``: per-pair omega numerators and per-snapshot gamma."""
    _fields_ = [("omega_num", C.c_void_p), ("gamma_num", C.c_void_p), ("gamma_den", C.c_void_p)]


class _Gen:
    """Marshals ``omegas`` (omega^(sr) numerators over the call's omega
    denominator, in the handle's slot layout: T-1 for ordinal coupling, a
    T x T matrix for categorical) and ``gammas`` (T (num, den) pairs); None
    when neither is given."""

    def __init__(self, omegas=None, gammas=None):
        self.arrays = []
        self.struct = None
        if omegas is None and gammas is None:
            return
        g = General(None, None, None)
        if omegas is not None:
            om = np.ascontiguousarray(np.asarray(omegas, dtype=np.int64).ravel())
            self.arrays.append(om)
            g.omega_num = om.ctypes.data
        if gammas is not None:
            gn = np.ascontiguousarray([int(x[0]) for x in gammas], dtype=np.int64)
            gd = np.ascontiguousarray([int(x[1]) for x in gammas], dtype=np.int64)
            self.arrays += [gn, gd]
            g.gamma_num, g.gamma_den = gn.ctypes.data, gd.ctypes.data
        self.struct = g

    @property
    def ptr(self):
        return C.byref(self.struct) if self.struct is not None else None


def _check(rc, what):
    if rc != MSLICE_OK:
        raise MsliceError(rc, f"{what}: {lib().mslice_last_error().decode()}")


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor (device or host)
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _stats_dict(st) -> dict:
    d = {f: getattr(st, f) for f, _ in Stats._fields_}
    d["tier_cuts"] = tuple(st.tier_cuts)
    return d


def default_opts() -> Opts:
    o = Opts()
    lib().mslice_default_opts(C.byref(o))
    return o


class Handle:
    """An mslice handle: the level-0 supra-graph resident on the device."""

    def __init__(self, h, keep):
        self._h = h
        self._keep = keep
        N, T, n, nnz = C.c_int64(), C.c_int32(), C.c_int64(), C.c_int64()
        _check(lib().mslice_info(h, C.byref(N), C.byref(T), C.byref(n), C.byref(nnz)), "mslice_info")
        self.N, self.T, self.n, self.nnz = N.value, T.value, n.value, nnz.value

    def close(self):
        if self._h:
            lib().mslice_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def kernel_launches(self) -> int:
        return int(lib().mslice_kernel_launches(self._h))

    def mslice_leiden(self, gamma=(1, 1), omega=(1, 1), max_levels=32, seed=0, n_iterations=2, K=4,
                      max_rounds=100, init=None, stop_level=-1, stop_stage=0, stop_rounds=0, out=None,
                      profile=False, tier_cuts=None, autotune=False, null="multislice", omegas=None, gammas=None,
                      theta=None):
        """Returns (labels, Q, stats).  With ``out`` a device tensor (int32[N])
        the labels stay on the device (MSLICE_DEVICE_PTRS); ``init`` may then
        be a device tensor as well.  ``null="global"`` optimises the plain
        modularity of the supra-graph instead of Q_MS (MSLICE_NULL_GLOBAL).
        ``omegas`` / ``gammas``: the general form (mslice_leiden_general).
        ``theta``: (num, den) of the randomised refinement (None: greedy)."""
        o = default_opts()
        o.gamma_num, o.gamma_den = gamma
        o.omega_num, o.omega_den = omega
        o.max_levels, o.seed, o.n_iterations, o.K, o.max_rounds = max_levels, seed, n_iterations, K, max_rounds
        o.stop_level, o.stop_stage, o.stop_rounds = stop_level, stop_stage, stop_rounds
        if theta is not None:
            o.theta_num, o.theta_den = theta
        dev = out is not None and hasattr(out, "is_cuda") and out.is_cuda
        if profile:
            o.flags |= MSLICE_PROFILE
        if autotune:
            o.flags |= MSLICE_AUTOTUNE
        o.flags |= _NULLS[null]
        if tier_cuts is not None:
            o.tier_cuts[:] = list(tier_cuts)
        if dev:
            o.flags |= MSLICE_DEVICE_PTRS
        labels = out if out is not None else np.zeros(max(self.N, 1), dtype=np.int32)
        init_a = init
        if init is not None and not hasattr(init, "data_ptr"):
            init_a = np.ascontiguousarray(init, dtype=np.int32)
        Q = C.c_double(0.0)
        st = Stats()
        gen = _Gen(omegas, gammas)
        _check(lib().mslice_leiden_general(self._h, C.byref(o), gen.ptr, _ptr(init_a), _ptr(labels), C.byref(Q),
                                           C.byref(st)), "mslice_leiden_general")
        stats = _stats_dict(st)
        if out is not None:
            return labels, Q.value, stats
        return labels[: st.out_n].copy(), Q.value, stats

    def mslice_modularity(self, labels, gamma=(1, 1), omega=(1, 1), null="multislice", omegas=None, gammas=None):
        dev = hasattr(labels, "is_cuda") and labels.is_cuda
        lab = labels if dev else np.ascontiguousarray(labels, dtype=np.int32)
        Q = C.c_double(0.0)
        flags = (MSLICE_DEVICE_PTRS if dev else 0) | _NULLS[null]
        if omegas is None and gammas is None:
            _check(lib().mslice_modularity_ex(self._h, _ptr(lab), gamma[0], gamma[1], omega[0], omega[1], flags,
                                              C.byref(Q)), "mslice_modularity_ex")
            return Q.value
        o = default_opts()
        o.gamma_num, o.gamma_den = gamma
        o.omega_num, o.omega_den = omega
        o.flags = flags
        gen = _Gen(omegas, gammas)
        _check(lib().mslice_modularity_general(self._h, _ptr(lab), C.byref(o), gen.ptr, C.byref(Q)),
               "mslice_modularity_general")
        return Q.value

    # short aliases
    leiden = mslice_leiden
    modularity = mslice_modularity


class Batch:
    """A batch of independent (graph, gamma, omega) instances solved together
    (``mslice_batch_*``).  Each instance's labels and Q equal those of
    :meth:`Handle.mslice_leiden` on its graph alone."""

    def __init__(self, stream=None, device_ptrs=False):
        b = C.c_void_p()
        _check(lib().mslice_batch_create(MSLICE_DEVICE_PTRS if device_ptrs else 0,
                                         C.c_void_p(stream) if stream is not None else None, C.byref(b)),
               "mslice_batch_create")
        self._b = b
        self._dev = device_ptrs
        self._graphs = []

    def close(self):
        if self._b:
            lib().mslice_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def mslice_batch_add(self, graph: "Handle", gamma=(1, 1), omega=(1, 1), init=None, omegas=None,
                         gammas=None) -> int:
        init_a = init
        if init is not None and not hasattr(init, "data_ptr"):
            init_a = np.ascontiguousarray(init, dtype=np.int32)
        idx = C.c_int32(-1)
        if omegas is None and gammas is None:
            _check(lib().mslice_batch_add(self._b, graph._h, gamma[0], gamma[1], omega[0], omega[1], _ptr(init_a),
                                          C.byref(idx)), "mslice_batch_add")
        else:
            gen = _Gen(omegas, gammas)
            _check(lib().mslice_batch_add_general(self._b, graph._h, gamma[0], gamma[1], omega[0], omega[1],
                                                  gen.ptr, _ptr(init_a), C.byref(idx)), "mslice_batch_add_general")
        self._graphs.append(graph)
        return idx.value

    def mslice_batch_run(self, n_iterations=2, K=4, max_rounds=100, max_levels=32, seed=0, profile=False,
                         tier_cuts=None, autotune=False, null="multislice", theta=None) -> dict:
        o = default_opts()
        o.n_iterations, o.K, o.max_rounds, o.max_levels, o.seed = n_iterations, K, max_rounds, max_levels, seed
        if theta is not None:
            o.theta_num, o.theta_den = theta
        if profile:
            o.flags |= MSLICE_PROFILE
        if autotune:
            o.flags |= MSLICE_AUTOTUNE
        o.flags |= _NULLS[null]
        if tier_cuts is not None:
            o.tier_cuts[:] = list(tier_cuts)
        st = Stats()
        _check(lib().mslice_batch_run(self._b, C.byref(o), C.byref(st)), "mslice_batch_run")
        return _stats_dict(st)

    def mslice_batch_info(self):
        B, N = C.c_int32(), C.c_int64()
        _check(lib().mslice_batch_info(self._b, C.byref(B), C.byref(N), None), "mslice_batch_info")
        off = np.zeros(B.value + 1, dtype=np.int64)
        _check(lib().mslice_batch_info(self._b, None, None, _ptr(off)), "mslice_batch_info")
        return B.value, N.value, off

    def mslice_batch_results(self, i=-1, out=None):
        """(labels, Q) of instance i; i = -1: all labels one after another and
        the B values of Q."""
        B, N, off = self.mslice_batch_info()
        n = int(N if i < 0 else (off[i + 1] - off[i] if i < B else 0))  # a bad index is the library's to reject
        labels = out if out is not None else np.zeros(max(n, 1), dtype=np.int32)
        if i < 0:
            Q = np.zeros(max(B, 1), dtype=np.float64)
            _check(lib().mslice_batch_results(self._b, -1, _ptr(labels), _ptr(Q)), "mslice_batch_results")
            return (labels if out is not None else labels[:n]), Q[:B]
        Q = C.c_double(0.0)
        _check(lib().mslice_batch_results(self._b, i, _ptr(labels), C.byref(Q)), "mslice_batch_results")
        return (labels if out is not None else labels[:n]), Q.value

    def mslice_batch_clear(self):
        _check(lib().mslice_batch_clear(self._b), "mslice_batch_clear")
        self._graphs = []

    @property
    def kernel_launches(self) -> int:
        return int(lib().mslice_batch_kernel_launches(self._b))

    add = mslice_batch_add
    run = mslice_batch_run
    results = mslice_batch_results
    info = mslice_batch_info
    clear = mslice_batch_clear


class Server:
    """Serving loop over live temporal graphs (``mslice_server_*``): every
    submitted snapshot advances its graph's window of ``window`` slices and is
    solved warm-started from the previous window's labels; the result equals
    :meth:`Handle.mslice_leiden` on the window with those initial labels."""

    def __init__(self, window=8, n_slots=2, max_batch=64, hbm_budget=0, gamma=(1, 1), omega=(1, 1),
                 n_iterations=2, K=4, max_rounds=100, max_levels=32, seed=0, max_batch_nodes=None,
                 null="multislice", theta=None):
        o = ServerOpts()
        lib().mslice_server_default_opts(C.byref(o))
        o.window, o.n_slots, o.max_batch, o.hbm_budget = window, n_slots, max_batch, hbm_budget
        if max_batch_nodes is not None:
            o.max_batch_nodes = max_batch_nodes
        o.gamma_num, o.gamma_den = gamma
        o.omega_num, o.omega_den = omega
        o.solve.n_iterations, o.solve.K, o.solve.max_rounds = n_iterations, K, max_rounds
        o.solve.max_levels, o.solve.seed = max_levels, seed
        o.solve.flags = _NULLS[null]
        if theta is not None:
            o.solve.theta_num, o.solve.theta_den = theta
        s = C.c_void_p()
        _check(lib().mslice_server_create(C.byref(o), C.byref(s)), "mslice_server_create")
        self._s = s
        self.window = window
        self._n = {}
        self._pending = {}

    def close(self):
        if self._s:
            lib().mslice_server_free(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def mslice_server_add_graph(self, n: int) -> int:
        gid = C.c_int32(-1)
        _check(lib().mslice_server_add_graph(self._s, n, C.byref(gid)), "mslice_server_add_graph")
        self._n[gid.value] = n
        return gid.value

    def mslice_server_submit(self, graph_id: int, snap) -> int:
        ip = np.ascontiguousarray(snap.indptr, dtype=np.int64)
        ix = np.ascontiguousarray(snap.indices, dtype=np.int32)
        w = np.ascontiguousarray(snap.weights, dtype=np.int32)
        csr = Csr(len(ip) - 1, _ptr(ip).value, _ptr(ix).value, _ptr(w).value)
        rid = C.c_int64(-1)
        _check(lib().mslice_server_submit(self._s, graph_id, C.byref(csr), C.byref(rid)), "mslice_server_submit")
        self._pending[rid.value] = graph_id
        return rid.value

    def mslice_server_wait(self, request_id: int):
        """(labels, info dict) of a finished request; raises MsliceError when
        the request failed."""
        gid = self._pending.pop(request_id, None)
        n = self._n.get(gid, 0) * self.window
        labels = np.zeros(max(n, 1), dtype=np.int32)
        info = RequestInfo()
        rc = lib().mslice_server_wait(self._s, request_id, _ptr(labels), C.byref(info))
        d = {f: getattr(info, f) for f, _ in RequestInfo._fields_}
        _check(rc, "mslice_server_wait")
        return labels[: info.N].copy(), d

    def mslice_server_checkpoint(self, graph_id: int):
        """(snapshots, labels) of an idle graph's window: the state its next
        request reads (snapshots oldest first, as Snapshot-like objects)."""
        from .synth import Snapshot
        w = C.c_int32(0)
        _check(lib().mslice_server_window_info(self._s, graph_id, C.byref(w), None), "mslice_server_window_info")
        nnz = np.zeros(max(w.value, 1), dtype=np.int64)
        _check(lib().mslice_server_window_info(self._s, graph_id, C.byref(w), _ptr(nnz)), "mslice_server_window_info")
        n = self._n[graph_id]
        snaps = []
        for k in range(w.value):
            ip = np.zeros(n + 1, dtype=np.int64)
            ix = np.zeros(max(int(nnz[k]), 1), dtype=np.int32)
            wt = np.zeros(max(int(nnz[k]), 1), dtype=np.int32)
            _check(lib().mslice_server_window_read(self._s, graph_id, k, _ptr(ip), _ptr(ix), _ptr(wt), None),
                   "mslice_server_window_read")
            snaps.append(Snapshot(ip, ix[: nnz[k]], wt[: nnz[k]]))
        labels = np.zeros(max(n * w.value, 1), dtype=np.int32)
        _check(lib().mslice_server_window_read(self._s, graph_id, -1, None, None, None, _ptr(labels)),
               "mslice_server_window_read")
        return snaps, labels[: n * w.value]

    def mslice_server_restore(self, graph_id: int, snaps, labels):
        arr = (Csr * len(snaps))()
        keep = []
        for k, sn in enumerate(snaps):
            ip = np.ascontiguousarray(sn.indptr, dtype=np.int64)
            ix = np.ascontiguousarray(sn.indices, dtype=np.int32)
            wt = np.ascontiguousarray(sn.weights, dtype=np.int32)
            keep += [ip, ix, wt]
            arr[k] = Csr(len(ip) - 1, _ptr(ip).value, _ptr(ix).value, _ptr(wt).value)
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        _check(lib().mslice_server_window_restore(self._s, graph_id, C.cast(arr, C.c_void_p), len(snaps), _ptr(lab)),
               "mslice_server_window_restore")

    add_graph = mslice_server_add_graph
    submit = mslice_server_submit
    wait = mslice_server_wait
    checkpoint = mslice_server_checkpoint
    restore = mslice_server_restore


def mslice_build(snaps, omega=(1, 1), stream=None, device_ptrs=False, host_tensors=False,
                 coupling="ordinal") -> Handle:
    """Builds a handle from T snapshots.  ``snaps`` holds objects with
    ``indptr``/``indices``/``weights`` arrays: numpy host arrays, torch host
    tensors (``host_tensors=True``, e.g. pinned memory) or torch device
    tensors (``device_ptrs=True``).  ``coupling``: "ordinal" (adjacent
    snapshots) or "categorical" (every pair of snapshots)."""
    T = len(snaps)
    arr = (Csr * max(T, 1))()
    keep = []
    for s, sn in enumerate(snaps):
        if device_ptrs or host_tensors:
            ip, ix, w = sn.indptr, sn.indices, sn.weights
            n = ip.numel() - 1
        else:
            ip = np.ascontiguousarray(sn.indptr, dtype=np.int64)
            ix = np.ascontiguousarray(sn.indices, dtype=np.int32)
            w = np.ascontiguousarray(sn.weights, dtype=np.int32)
            n = len(ip) - 1
        keep += [ip, ix, w]
        arr[s] = Csr(n, _ptr(ip).value, _ptr(ix).value if _ptr(ix) is not None else None,
                     _ptr(w).value if _ptr(w) is not None else None)
    h = C.c_void_p()
    st = C.c_void_p(stream) if stream is not None else None
    _check(lib().mslice_build_ex(C.cast(arr, C.c_void_p), T, _COUPLINGS[coupling], omega[0], omega[1],
                                 MSLICE_DEVICE_PTRS if device_ptrs else 0, st, C.byref(h)), "mslice_build_ex")
    return Handle(h, keep)


build_graph = mslice_build


def _csr_array(snaps, device_ptrs=False, host_tensors=False):
    T = len(snaps)
    arr = (Csr * max(T, 1))()
    keep = []
    for s, sn in enumerate(snaps):
        if device_ptrs or host_tensors:
            ip, ix, w = sn.indptr, sn.indices, sn.weights
            n = ip.numel() - 1
        else:
            ip = np.ascontiguousarray(sn.indptr, dtype=np.int64)
            ix = np.ascontiguousarray(sn.indices, dtype=np.int32)
            w = np.ascontiguousarray(sn.weights, dtype=np.int32)
            n = len(ip) - 1
        keep += [ip, ix, w]
        arr[s] = Csr(n, _ptr(ip).value, _ptr(ix).value if _ptr(ix) is not None else None,
                     _ptr(w).value if _ptr(w) is not None else None)
    return arr, keep


def mslice_leiden_windowed(snaps, W, stride, gamma=(1, 1), omega=(1, 1), null="multislice", n_iterations=2, K=4,
                           max_rounds=100, max_levels=32, seed=0, stream=None, device_ptrs=False, theta=None):
    """Windowed optimisation of a long snapshot sequence
    (``mslice_leiden_windowed``): windows of W snapshots at the given stride,
    warm-started and stitched through their overlaps.  Returns (labels
    int32[n*T], Q of every window, stats)."""
    arr, keep = _csr_array(snaps, device_ptrs=device_ptrs)
    T = len(snaps)
    n = (snaps[0].indptr.numel() if device_ptrs else len(snaps[0].indptr)) - 1 if T else 0
    o = default_opts()
    o.gamma_num, o.gamma_den = gamma
    o.omega_num, o.omega_den = omega
    o.n_iterations, o.K, o.max_rounds, o.max_levels, o.seed = n_iterations, K, max_rounds, max_levels, seed
    o.flags = _NULLS[null] | (MSLICE_DEVICE_PTRS if device_ptrs else 0)
    if theta is not None:
        o.theta_num, o.theta_den = theta
    labels = np.zeros(max(n * T, 1), dtype=np.int32)
    cap = T + 1
    Qw = np.zeros(cap, dtype=np.float64)
    nw = C.c_int32(0)
    st = Stats()
    s = C.c_void_p(stream) if stream is not None else None
    _check(lib().mslice_leiden_windowed(C.cast(arr, C.c_void_p), T, W, stride, C.byref(o), s, _ptr(labels),
                                        _ptr(Qw), cap, C.byref(nw), C.byref(st)), "mslice_leiden_windowed")
    del keep
    return labels[: n * T].copy(), [float(x) for x in Qw[: nw.value]], _stats_dict(st)


leiden_windowed = mslice_leiden_windowed
