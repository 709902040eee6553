"""Python binding of libfpp, the GB300 Falconn++ search library.

Argument marshalling only: every step of build and search runs in the CUDA
kernels of ``libfpp.so`` behind the C ABI declared in ``include/fpp.h``.  The
functions keep the C names.  Arrays may be numpy arrays (host memory) or
torch tensors (host or CUDA); outputs are allocated like the query array when
not given.

The library is built in-tree by ``paper_2206_01382_gb300._build.build()``.
Loading fails loudly when it is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import _build

FPP_OK, FPP_EINVAL, FPP_ENOMEM, FPP_ECUDA, FPP_ETIMEOUT, FPP_EBUSY, FPP_EINTERNAL = range(7)
FPP_FP32, FPP_BF16, FPP_FP8E4M3 = 0, 1, 2
FPP_SEARCH_GRAPH = 1
FPP_SEARCH_PIPELINE = 2
STATUS_NAMES = {0: "FPP_OK", 1: "FPP_EINVAL", 2: "FPP_ENOMEM", 3: "FPP_ECUDA",
                4: "FPP_ETIMEOUT", 5: "FPP_EBUSY", 6: "FPP_EINTERNAL"}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "fpp.h")


class FppError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fpp_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("D", ctypes.c_int32), ("iprobes", ctypes.c_int32),
                ("kappa", ctypes.c_int32), ("alpha", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("R", ctypes.c_void_p), ("precision", ctypes.c_int32),
                ("rerank_k", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("center", ctypes.c_int32), ("simhash_bits", ctypes.c_int32),
                ("center_vec", ctypes.c_void_p), ("hash_precision", ctypes.c_int32)]


class fpp_search_opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("probes", ctypes.c_int32),
                ("k_per_query", ctypes.c_void_p), ("probes_per_query", ctypes.c_void_p),
                ("k_max", ctypes.c_int32), ("table_begin", ctypes.c_int32),
                ("table_end", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("stream", ctypes.c_void_p), ("global_probes", ctypes.c_int32),
                ("simhash_keep", ctypes.c_int32), ("score_range_rows", ctypes.c_int32),
                ("reserved0", ctypes.c_int32)]


class fpp_search_stats(ctypes.Structure):
    _fields_ = [("queries", ctypes.c_uint64), ("probes", ctypes.c_uint64),
                ("entries", ctypes.c_uint64), ("unique", ctypes.c_uint64),
                ("probe_rechecks", ctypes.c_uint64), ("topk_rechecks", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("probe_full_rechecks", ctypes.c_uint64),
                ("ms_project", ctypes.c_float), ("ms_probe", ctypes.c_float),
                ("ms_probe_exact", ctypes.c_float), ("ms_gather_score", ctypes.c_float),
                ("ms_dedup", ctypes.c_float), ("ms_score", ctypes.c_float),
                ("ms_topk", ctypes.c_float), ("ms_total", ctypes.c_float)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class fpp_server_cfg(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("k_max", ctypes.c_int32), ("probes_max", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("candidate_budget_bytes", ctypes.c_uint64)]


class fpp_server_stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "completed", "failed", "queued",
                                               "batches", "queries", "entries", "probes",
                                               "splits", "serving_allocs")]


class fpp_tune_report(ctypes.Structure):
    _fields_ = [("score_lanes", ctypes.c_int32), ("score_waves", ctypes.c_int32),
                ("ms_default", ctypes.c_float), ("ms_best", ctypes.c_float),
                ("shapes_tried", ctypes.c_int32), ("reserved0", ctypes.c_int32)]


class fpp_index_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("L", ctypes.c_int32),
                ("D", ctypes.c_int32), ("iprobes", ctypes.c_int32), ("kappa", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("kept_total", ctypes.c_uint64), ("max_bucket_kept", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64), ("build_ms", ctypes.c_float),
                ("rerank_k", ctypes.c_int32), ("center", ctypes.c_int32),
                ("simhash_bits", ctypes.c_int32), ("r_pieces", ctypes.c_int32),
                ("score_error_factor", ctypes.c_double), ("q_pieces", ctypes.c_int32),
                ("graph_fallbacks", ctypes.c_uint32)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Loads libfpp.so (raises if it has not been built).  The environment
    variable FPP_LIBRARY may name another build of it, such as the
    FPP_DEBUG_BOUNDS one (``_build.LIB_DEBUG``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or os.environ.get("FPP_LIBRARY") or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libfpp.so not found at {p}; build it with "
                           "paper_2206_01382_gb300._build.build()")
    L = ctypes.CDLL(p)
    vp, i32, i64, u64, f32p = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                               ctypes.c_uint64, ctypes.c_void_p)
    sig = {
        "fpp_default_params": (None, [ctypes.POINTER(fpp_params)]),
        "fpp_default_search_opts": (None, [ctypes.POINTER(fpp_search_opts)]),
        "fpp_build": (ctypes.c_int, [f32p, i64, i32, ctypes.POINTER(fpp_params),
                                     ctypes.POINTER(ctypes.c_void_p)]),
        "fpp_search": (ctypes.c_int, [vp, f32p, i64, i32, i32, vp, vp]),
        "fpp_search_ex": (ctypes.c_int, [vp, f32p, i64, ctypes.POINTER(fpp_search_opts), vp, vp,
                                         ctypes.POINTER(fpp_search_stats)]),
        "fpp_free": (None, [vp]),
        "fpp_last_error": (ctypes.c_char_p, []),
        "fpp_rotations": (ctypes.c_int, [u64, i32, i32, i32, vp]),
        "fpp_keep_count": (u64, [u64, ctypes.c_double, i32, i32]),
        "fpp_index_get_info": (ctypes.c_int, [vp, ctypes.POINTER(fpp_index_info)]),
        "fpp_debug_point_buckets": (ctypes.c_int, [vp, i32, vp]),
        "fpp_debug_table": (ctypes.c_int, [vp, i32, vp, vp]),
        "fpp_debug_probes": (ctypes.c_int, [vp, f32p, i64, i32, i32, i32, vp]),
        "fpp_debug_candidates": (ctypes.c_int, [vp, f32p, i64, i32, vp, vp]),
        "fpp_bruteforce": (ctypes.c_int, [f32p, i64, i32, f32p, i64, i32, vp, vp, vp]),
        "fpp_debug_projections": (ctypes.c_int, [vp, f32p, i64, i32, i32, vp]),
        "fpp_projection_error_bound": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_double)]),
        "fpp_bruteforce_static": (ctypes.c_int, [f32p, i64, i32, f32p, i64, i32, vp, vp, vp]),
        "fpp_debug_wait_test": (ctypes.c_int, [i32, i64]),
        "fpp_search_flush": (ctypes.c_int, [vp, vp]),
        "fpp_launch_count": (u64, []),
        "fpp_alloc_count": (u64, []),
        "fpp_set_candidate_budget": (ctypes.c_int, [vp, u64]),
        "fpp_merge_topk": (ctypes.c_int, [vp, vp, i32, i64, i32, vp, vp]),
        "fpp_autotune": (ctypes.c_int, [vp, f32p, i64, i32, i32, ctypes.POINTER(fpp_tune_report)]),
        "fpp_default_server_cfg": (None, [ctypes.POINTER(fpp_server_cfg)]),
        "fpp_server_create": (ctypes.c_int, [vp, ctypes.POINTER(fpp_server_cfg),
                                             ctypes.POINTER(ctypes.c_void_p)]),
        "fpp_server_submit": (ctypes.c_int, [vp, f32p, i32, i32, i32,
                                             ctypes.POINTER(ctypes.c_uint64)]),
        "fpp_server_poll": (ctypes.c_int, [vp, u64, vp, vp, i32, ctypes.POINTER(ctypes.c_float)]),
        "fpp_server_submit_many": (ctypes.c_int, [vp, f32p, i32, vp, vp, vp, vp]),
        "fpp_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(fpp_server_stats)]),
        "fpp_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def header_functions() -> list:
    """Names of the functions declared in include/fpp.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fpp_[a-z0-9_]+)\s*\(", txt)))


# ----------------------------------------------------------------- marshalling

def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def _f32(a):
    if _is_torch(a):
        import torch
        return a.to(torch.float32).contiguous()
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    if a is None:
        return None
    if _is_torch(a):
        import torch
        return a.to(torch.int32).contiguous()
    return np.ascontiguousarray(a, dtype=np.int32)


def _alloc_like(ref, shape, kind):
    if _is_torch(ref):
        import torch
        dt = torch.int64 if kind == "i64" else torch.float32
        return torch.empty(shape, dtype=dt, device=ref.device)
    return np.empty(shape, dtype=np.int64 if kind == "i64" else np.float32)


def _check(status):
    if status != FPP_OK:
        raise FppError(status, load().fpp_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ----------------------------------------------------------------- API

def fpp_default_params() -> fpp_params:
    p = fpp_params()
    load().fpp_default_params(ctypes.byref(p))
    return p


def fpp_build(X, L: int, D: int, alpha: float, seed: int = 0, R=None, iprobes: int = 1,
              kappa: int = 0, precision: int = FPP_FP32, rerank_k: int = 100,
              center: bool = False, center_vec=None, simhash_bits: int = 0,
              stream=None, hash_precision: int = FPP_FP32) -> ctypes.c_void_p:
    """Builds an index over X [n][d]; returns the opaque handle."""
    lib = load()
    X = _f32(X)
    p = fpp_default_params()
    p.L, p.D, p.alpha, p.seed = L, D, float(alpha), int(seed)
    p.iprobes, p.kappa, p.precision, p.rerank_k = iprobes, kappa, precision, rerank_k
    p.center = 1 if center else 0
    p.simhash_bits = simhash_bits
    p.hash_precision = hash_precision
    cv = _f32(center_vec) if center_vec is not None else None
    p.center_vec = _ptr(cv)
    Rc = _f32(R) if R is not None else None
    p.R = _ptr(Rc)
    p.stream = _stream_ptr(stream)
    out = ctypes.c_void_p()
    n, d = X.shape
    _check(lib.fpp_build(_ptr(X), n, d, ctypes.byref(p), ctypes.byref(out)))
    return out


def fpp_free(ix) -> None:
    if ix is not None:
        load().fpp_free(ix)


def fpp_search(ix, Q, k: int, probes: int, ids=None, scores=None):
    """Top-k ids [m][k] (int64) and scores [m][k] (float32)."""
    Q = _f32(Q)
    m = Q.shape[0]
    ids = _alloc_like(Q, (m, k), "i64") if ids is None else ids
    scores = _alloc_like(Q, (m, k), "f32") if scores is None else scores
    _check(load().fpp_search(ix, _ptr(Q), m, k, probes, _ptr(ids), _ptr(scores)))
    return ids, scores


def fpp_search_ex(ix, Q, k: int = 10, probes: int = 1, k_per_query=None, probes_per_query=None,
                  k_max: int | None = None, table_begin: int = 0, table_end: int = 0,
                  stream=None, ids=None, scores=None, want_stats: bool = True,
                  graph: bool = False, global_probes: int = 0, simhash_keep: int = 0,
                  score_range_rows: int = 0, pipeline: bool = False):
    """fpp_search with per-query k / probes, a table range, a stream and stats."""
    Q = _f32(Q)
    m = Q.shape[0]
    kpq = _i32(k_per_query)
    ppq = _i32(probes_per_query)
    if k_max is None:
        k_max = int(kpq.max()) if kpq is not None and m else k
    o = fpp_search_opts()
    load().fpp_default_search_opts(ctypes.byref(o))
    o.k, o.probes = k, probes
    o.k_per_query, o.probes_per_query = _ptr(kpq), _ptr(ppq)
    o.k_max, o.table_begin, o.table_end = k_max, table_begin, table_end
    o.stream = _stream_ptr(stream)
    o.flags = (FPP_SEARCH_GRAPH if graph else 0) | (FPP_SEARCH_PIPELINE if pipeline else 0)
    o.global_probes = global_probes
    o.simhash_keep = simhash_keep
    o.score_range_rows = score_range_rows
    ids = _alloc_like(Q, (m, k_max), "i64") if ids is None else ids
    scores = _alloc_like(Q, (m, k_max), "f32") if scores is None else scores
    st = fpp_search_stats()
    _check(load().fpp_search_ex(ix, _ptr(Q), m, ctypes.byref(o), _ptr(ids), _ptr(scores),
                                ctypes.byref(st) if want_stats else None))
    return ids, scores, (st.as_dict() if want_stats else None)


def fpp_search_flush(ix, stream=None) -> None:
    """Makes the stream wait for every pipelined call of the index."""
    _check(load().fpp_search_flush(ix, _stream_ptr(stream)))


def fpp_rotations(seed: int, L: int, D: int, d: int) -> np.ndarray:
    R = np.empty((L, 2, D, d), dtype=np.float32)
    _check(load().fpp_rotations(seed, L, D, d, R.ctypes.data))
    return R


def fpp_keep_count(B: int, alpha: float, iprobes: int = 1, kappa: int = 0) -> int:
    return int(load().fpp_keep_count(B, alpha, iprobes, kappa))


def fpp_index_get_info(ix) -> dict:
    info = fpp_index_info()
    _check(load().fpp_index_get_info(ix, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in info._fields_}


def fpp_debug_point_buckets(ix, t: int) -> np.ndarray:
    """[n] bucket ids (iprobes = 1) or [n][iprobes] ranked bucket ids."""
    info = fpp_index_get_info(ix)
    n, ip = info["n"], info["iprobes"]
    out = np.empty((n, ip) if ip > 1 else n, dtype=np.uint32)
    _check(load().fpp_debug_point_buckets(ix, t, out.ctypes.data))
    return out


def fpp_debug_table(ix, t: int):
    info = fpp_index_get_info(ix)
    off = np.empty(4 * info["D"] ** 2 + 1, dtype=np.uint32)
    _check(load().fpp_debug_table(ix, t, off.ctypes.data, None))
    ids = np.empty(int(off[-1]), dtype=np.uint32)
    _check(load().fpp_debug_table(ix, t, off.ctypes.data, ids.ctypes.data))
    return off, ids


def fpp_debug_probes(ix, Q, probes: int, table_begin: int = 0, table_end: int = 0) -> np.ndarray:
    info = fpp_index_get_info(ix)
    te = table_end or info["L"]
    Q = _f32(Q)
    m = Q.shape[0]
    out = np.empty((m, te - table_begin, probes), dtype=np.uint32)
    _check(load().fpp_debug_probes(ix, _ptr(Q), m, probes, table_begin, table_end, out.ctypes.data))
    return out


def fpp_debug_candidates(ix, Q, probes: int):
    """De-duplicated candidate ids of every query, ascending: a list of arrays."""
    Q = _f32(Q)
    m = Q.shape[0]
    off = np.zeros(m + 1, dtype=np.int64)
    lib = load()
    _check(lib.fpp_debug_candidates(ix, _ptr(Q), m, probes, off.ctypes.data, None))
    cand = np.empty(max(int(off[-1]), 1), dtype=np.uint32)
    _check(lib.fpp_debug_candidates(ix, _ptr(Q), m, probes, off.ctypes.data, cand.ctypes.data))
    return [cand[off[i]:off[i + 1]] for i in range(m)]


def fpp_debug_projections(ix, Q, table_begin: int = 0, table_end: int = 0) -> np.ndarray:
    info = fpp_index_get_info(ix)
    te = table_end or info["L"]
    Q = _f32(Q)
    m = Q.shape[0]
    out = np.empty((m, 2 * (te - table_begin) * info["D"]), dtype=np.float32)
    _check(load().fpp_debug_projections(ix, _ptr(Q), m, table_begin, table_end, out.ctypes.data))
    return out


def fpp_debug_wait_test(withhold: int, wait_cycles: int) -> None:
    """Test hook of the projection kernel's bounded waits (see include/fpp.h)."""
    _check(load().fpp_debug_wait_test(int(withhold), int(wait_cycles)))


def fpp_projection_error_bound(ix) -> float:
    f = ctypes.c_double()
    _check(load().fpp_projection_error_bound(ix, ctypes.byref(f)))
    return f.value


def fpp_bruteforce(X, Q, k: int, stream=None):
    X = _f32(X)
    Q = _f32(Q)
    m = Q.shape[0]
    ids = _alloc_like(Q, (m, k), "i64")
    scores = _alloc_like(Q, (m, k), "f32")
    _check(load().fpp_bruteforce(_ptr(X), X.shape[0], X.shape[1], _ptr(Q), m, k, _ptr(ids),
                                 _ptr(scores), _stream_ptr(stream)))
    return ids, scores


def fpp_bruteforce_static(X, Q, k: int, ids=None, scores=None, stream=None):
    """Exact search that allocates no device memory inside the library; X, Q
    and the outputs must be CUDA tensors (d a multiple of 4)."""
    m = Q.shape[0]
    ids = _alloc_like(Q, (m, k), "i64") if ids is None else ids
    scores = _alloc_like(Q, (m, k), "f32") if scores is None else scores
    _check(load().fpp_bruteforce_static(_ptr(X), X.shape[0], X.shape[1], _ptr(Q), m, k,
                                        _ptr(ids), _ptr(scores), _stream_ptr(stream)))
    return ids, scores


def fpp_launch_count() -> int:
    return int(load().fpp_launch_count())


def fpp_alloc_count() -> int:
    """Device allocations libfpp has made in this process."""
    return int(load().fpp_alloc_count())


def fpp_set_candidate_budget(ix, nbytes: int) -> None:
    """Candidate buffer bytes a call may provision without a read-back."""
    _check(load().fpp_set_candidate_budget(ix, int(nbytes)))


class Index:
    """Owning wrapper of an fpp_index handle."""

    def __init__(self, X, L, D, alpha, seed=0, **kw):
        self.handle = fpp_build(X, L, D, alpha, seed=seed, **kw)

    def search(self, Q, k, probes, **kw):
        if kw:
            return fpp_search_ex(self.handle, Q, k=k, probes=probes, **kw)
        return fpp_search(self.handle, Q, k, probes)

    def info(self):
        return fpp_index_get_info(self.handle)

    def close(self):
        if self.handle is not None:
            fpp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fpp_autotune(ix, Q, k: int, probes: int) -> dict:
    """Tunes the scoring kernel's launch shape on one batch of Q; returns the report."""
    Q = _f32(Q)
    r = fpp_tune_report()
    _check(load().fpp_autotune(ix, _ptr(Q), Q.shape[0], k, probes, ctypes.byref(r)))
    return {f: getattr(r, f) for f, _ in r._fields_}


def fpp_merge_topk(ids, scores):
    """Merges per-part top-k lists ids/scores [parts][m][k] (host arrays) into
    the global top-k [m][k] (score desc, id asc, each id once)."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    scores = np.ascontiguousarray(scores, dtype=np.float32)
    parts, m, k = ids.shape
    oi = np.empty((m, k), dtype=np.int64)
    osc = np.empty((m, k), dtype=np.float32)
    _check(load().fpp_merge_topk(ids.ctypes.data, scores.ctypes.data, parts, m, k,
                                 oi.ctypes.data, osc.ctypes.data))
    return oi, osc


class Server:
    """Continuous-batching search server over an Index (see fpp_server_* in
    include/fpp.h).  submit() returns a request id; poll() returns
    (ids [nq][k], scores [nq][k], latency_ms), or None when timeout_us ran
    out first."""

    def __init__(self, index, **cfg):
        lib = load()
        c = fpp_server_cfg()
        lib.fpp_default_server_cfg(ctypes.byref(c))
        for key, v in cfg.items():
            setattr(c, key, v)
        self.cfg = {f: getattr(c, f) for f, _ in c._fields_}
        self.index = index          # the index must outlive the server
        self.d = index.info()["d"]
        h = ctypes.c_void_p()
        _check(lib.fpp_server_create(index.handle, ctypes.byref(c), ctypes.byref(h)))
        self.handle = h
        self._shape = {}

    def submit(self, q, k: int, probes: int) -> int:
        if not _is_torch(q):
            q = np.atleast_2d(np.asarray(q, dtype=np.float32))
        q = _f32(q)
        nq = int(q.shape[0])
        rid = ctypes.c_uint64()
        _check(load().fpp_server_submit(self.handle, _ptr(q), nq, k, probes, ctypes.byref(rid)))
        self._shape[rid.value] = (nq, k)
        return rid.value

    def submit_many(self, q, sizes, ks, probes) -> list:
        """Queues len(sizes) requests whose query rows follow each other in q."""
        q = _f32(np.atleast_2d(np.asarray(q, dtype=np.float32)) if not _is_torch(q) else q)
        sz = np.ascontiguousarray(sizes, dtype=np.int32)
        kk = np.ascontiguousarray(ks, dtype=np.int32)
        pp = np.ascontiguousarray(np.broadcast_to(np.asarray(probes, dtype=np.int32), sz.shape))
        ids = np.zeros(sz.size, dtype=np.uint64)
        _check(load().fpp_server_submit_many(self.handle, _ptr(q), int(sz.size), sz.ctypes.data,
                                             kk.ctypes.data, pp.ctypes.data, ids.ctypes.data))
        for rid, n, k in zip(ids.tolist(), sz.tolist(), kk.tolist()):
            self._shape[rid] = (n, k)
        return ids.tolist()

    def poll(self, rid: int, timeout_us: int = -1):
        nq, k = self._shape[rid]
        ids = np.empty((nq, k), dtype=np.int64)
        sc = np.empty((nq, k), dtype=np.float32)
        lat = ctypes.c_float()
        st = load().fpp_server_poll(self.handle, rid, ids.ctypes.data, sc.ctypes.data,
                                    timeout_us, ctypes.byref(lat))
        if st == 4:   # FPP_ETIMEOUT: not complete yet
            return None
        del self._shape[rid]
        _check(st)
        return ids, sc, lat.value

    def stats(self) -> dict:
        st = fpp_server_stats()
        _check(load().fpp_server_get_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if self.handle is not None:
            load().fpp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
