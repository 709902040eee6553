"""The oracle's index build spread over host processes, one table at a time.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The tables of a Falconn++ index are independent (Section 2.1: L tables, each
with its own random vectors), so ``build_index_parallel`` runs the same
``falconn.build_table`` for each table in a pool of single-threaded worker
processes and assembles the same ``OracleIndex`` that ``build_index`` returns.
Nothing of the arithmetic changes: each table is computed by the one plain
function, in FP64, in the order it states.  The pool uses the ``spawn`` start
method (safe in a process that already holds a CUDA context), and the points
reach the workers through one shared-memory block.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from .falconn import OracleIndex, build_table, center_points
from .rotations import gaussian_rotations

_W = {}


def _init(shm_name, shape, dtype, R64, alpha, iprobes, kappa):
    shm = shared_memory.SharedMemory(name=shm_name)
    X = np.ndarray(shape, dtype=dtype, buffer=shm.buf)
    _W.update(shm=shm, X64=np.asarray(X, dtype=np.float64), R=R64, alpha=alpha,
              iprobes=iprobes, kappa=kappa)


def _one_table(t):
    o, ids, cnt, pb, hf, ff = build_table(_W["X64"], _W["R"][t], _W["alpha"], _W["iprobes"],
                                          _W["kappa"])
    return (t, o, ids, cnt.astype(np.int32), None if pb is None else pb.astype(np.int32),
            np.packbits(hf), np.packbits(ff))


def build_index_parallel(X, L: int, D: int, alpha: float, seed: int | None = None,
                         R: np.ndarray | None = None, iprobes: int = 1, kappa: int = 0,
                         tables=None, center: bool = False, c=None,
                         workers: int | None = None) -> OracleIndex:
    """``build_index`` with its tables built in ``workers`` processes (default:
    the host's cores).  Same arguments and result, except that point buckets
    and bucket counts are held as int32."""
    X32 = np.ascontiguousarray(X)
    n, d = X32.shape
    Xh = X32
    if center:
        _, Xh = center_points(X32, c)
    if R is None:
        R = gaussian_rotations(seed, L, D, d)
    R64 = np.asarray(R, dtype=np.float64).reshape(L, 2, D, d)
    NB = 4 * D * D
    todo = list(range(L)) if tables is None else [int(t) for t in tables]
    workers = max(1, min(workers or os.cpu_count() or 1, len(todo)))
    offsets = np.zeros((L, NB + 1), dtype=np.int64)
    counts = np.zeros((L, NB), dtype=np.int32)
    ids = [np.zeros(0, dtype=np.int64) for _ in range(L)]
    pb = np.full((L, n), -1, dtype=np.int32) if iprobes == 1 else None
    hflag = np.zeros((L, n), dtype=bool)
    fflag = np.zeros((L, NB), dtype=bool)
    Xh = np.ascontiguousarray(Xh)
    shm = shared_memory.SharedMemory(create=True, size=max(Xh.nbytes, 1))
    try:
        np.ndarray(Xh.shape, dtype=Xh.dtype, buffer=shm.buf)[...] = Xh
        # one BLAS thread per worker: the pool is the parallelism
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                 "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            # a worker that dies raises BrokenProcessPool here instead of
            # leaving the build waiting
            with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"),
                                        initializer=_init,
                                        initargs=(shm.name, Xh.shape, Xh.dtype, R64, float(alpha),
                                                  iprobes, kappa)) as pool:
                for t, o, i, cnt, b, hf, ff in pool.map(_one_table, todo):
                    offsets[t], ids[t], counts[t] = o, i, cnt
                    hflag[t] = np.unpackbits(hf, count=n).astype(bool)
                    fflag[t] = np.unpackbits(ff, count=NB).astype(bool)
                    if pb is not None:
                        pb[t] = b
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    finally:
        shm.close()
        shm.unlink()
    return OracleIndex(n, d, L, D, float(alpha), iprobes, kappa, R64,
                       np.asarray(X32, dtype=np.float64), offsets, ids, counts, pb, hflag, fflag,
                       np.asarray(Xh, dtype=np.float64) if center else None)
