"""Parity run on the FPP_DEBUG_BOUNDS build of libfpp (run as a child process
by tests/test_gpu_debug_bounds.py, with FPP_LIBRARY naming that build).

In that build every gather and scatter index of the candidate path (probed
bucket ids, bucket offsets, kept-id and candidate-slot indices, candidate
ids, score work items, top-k regions) is checked on the device; the first
violation makes the call return FPP_EINTERNAL.  Each case below must run
without one and still match the FP64 oracle.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402
from tests import parity as PT  # noqa: E402
import paper_2206_01382_gb300 as F  # noqa: E402


def check(ix_o, ix_g, Q, k, P, L, **kw):
    gi, gs, _ = F.fpp_search_ex(ix_g.handle, Q, k=k, probes=P, want_stats=False, **kw)
    _, _, res = O.search_batch(ix_o, Q, k, P)
    excl = {t: PT.excluded_buckets(ix_o, t, F.fpp_debug_point_buckets(ix_g.handle, t))
            for t in range(L)}
    c, s, fails = PT.compare_search(res, gi, gs, k, list(range(L)), excl)
    assert not fails, fails[:3]
    return c


def main():
    lib = F.load()
    assert os.path.basename(lib._name) == "libfpp_debug.so", lib._name
    n_searches, compared = 0, 0
    # the tiny workload: the small dedup tier, row-range grouping forced
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    ix_o = O.build_index(X, w.L, w.D, w.alpha, seed=w.rot_seed)
    ix_g = F.Index(X, w.L, w.D, w.alpha, seed=w.rot_seed)
    for P in (1, 4, 16):
        for rr in (0, 512):
            compared += check(ix_o, ix_g, Q, w.k, P, w.L, score_range_rows=rr)
            n_searches += 1
    # queries above 3,072 and above 16,384 entries: the larger tiers, no de-duplication
    for n, L, D, P in ((30000, 24, 4, 8), (12000, 6, 8, 12)):
        X2, Q2 = W.small_mixture(n, 30, 16, 8, 0.3, 92 + D)
        io = O.build_index(X2, L, D, 1.0, seed=44)
        ig = F.Index(X2, L, D, 1.0, seed=44)
        compared += check(io, ig, Q2, 20, P, L)
        n_searches += 1
    # BF16 rows and per-query budgets through the server
    X3, Q3 = W.small_mixture(20000, 200, 64, 128, 0.25, 401)
    ib = F.Index(X3, 8, 32, 0.2, seed=17, precision=F.FPP_BF16)
    ref = [F.fpp_search_ex(ib.handle, Q3[i:i + 20], k=10, probes=4, want_stats=False)
           for i in range(0, 200, 20)]
    srv = F.Server(ib, k_max=10, probes_max=4, slots=2, max_batch=64)
    rids = [srv.submit(Q3[i:i + 20], 10, 4) for i in range(0, 200, 20)]
    for rid, (gi, gs, _) in zip(rids, ref):
        ids, sc, _ = srv.poll(rid)
        assert np.array_equal(ids, gi) and np.array_equal(sc, gs)
    srv.close()
    n_searches += len(rids)
    print(f"debug bounds build: {n_searches} searches, {compared} queries compared with the "
          f"oracle, no bounds violation")


if __name__ == "__main__":
    main()
