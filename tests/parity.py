"""Comparison helpers for GPU-vs-oracle parity: exact equality of every
discrete decision except where the oracle flags an FP64 near-tie."""
import numpy as np

import oracle as O

SCORE_RTOL = 1e-5


def excluded_buckets(ix: O.OracleIndex, t: int, gpu_point_buckets=None) -> set:
    """Buckets of table t whose content may legitimately differ: those that
    hold a point whose assignment is a near-tie (under either assignment),
    and those whose filter boundary is a near-tie."""
    ex = set(np.nonzero(ix.filter_flag[t])[0].tolist())
    flagged = np.nonzero(ix.hash_flag[t])[0]
    if ix.point_buckets is not None:
        ex.update(ix.point_buckets[t, flagged].tolist())
    if gpu_point_buckets is not None:
        ex.update(np.asarray(gpu_point_buckets)[flagged].tolist())
    return ex


def compare_point_buckets(ix, t, gpu_pb):
    ora = ix.point_buckets[t]
    bad = np.nonzero(ora != gpu_pb.astype(np.int64))[0]
    unexplained = [int(p) for p in bad if not ix.hash_flag[t, p]]
    return len(bad), unexplained


def compare_table(ix, t, gpu_off, gpu_ids, exclude):
    """Returns the list of buckets whose kept ids differ and are not excluded."""
    off = ix.offsets[t]
    bad = []
    g_off = gpu_off.astype(np.int64)
    for b in np.nonzero((np.diff(off) != np.diff(g_off)) | (off[:-1] != g_off[:-1]))[0]:
        if int(b) not in exclude:
            bad.append(int(b))
    # same kept counts: compare ids bucket by bucket.  The order inside a
    # bucket is part of the CSR contract (filter score desc, id asc); two ids
    # may change places only inside a run of FP64 filter scores whose
    # neighbours are closer than the near-tie threshold.
    if not bad:
        diff = np.nonzero(ix.ids[t] != gpu_ids.astype(np.int64))[0]
        if diff.size:
            bk = np.searchsorted(off, diff, side="right") - 1
            for b in np.unique(bk):
                if int(b) in exclude:
                    continue
                a = ix.bucket_ids(t, int(b))
                g = gpu_ids[off[b]: off[b + 1]].astype(np.int64)
                if not same_up_to_near_ties(a, g, bucket_filter_scores(ix, t, int(b), a)):
                    bad.append(int(b))
    return bad


def bucket_filter_scores(ix, t, b, ids):
    """FP64 filter scores of points ``ids`` in bucket b of table t: the
    bucket's pair score v1(h1) + v2(h2) of each point (Section 3.4 filter,
    with the signed-wedge values of the probe ranking)."""
    D = ix.D
    h1, h2 = b // (2 * D), b % (2 * D)
    x = (ix.X if ix.Xh is None else ix.Xh)[np.asarray(ids, dtype=np.int64)]

    def v(j, h):
        p = x @ ix.R[t, j, h % D]
        return p if h < D else -p
    return v(0, h1) + v(1, h2)


def same_up_to_near_ties(want, got, scores):
    """True if ``got`` lists the ids of ``want`` in the same order, except
    that ids inside one run of consecutive ``scores`` (the FP64 keys of
    ``want`` in its order) closer than NEAR_TIE may appear in any order."""
    want = np.asarray(want)
    got = np.asarray(got)
    if want.shape != got.shape:
        return False
    lo = 0
    for i in range(1, len(want) + 1):
        if i == len(want) or scores[i - 1] - scores[i] >= O.NEAR_TIE:
            if set(want[lo:i].tolist()) != set(got[lo:i].tolist()):
                return False
            lo = i
    return True


def ambiguous_ids(ix, t, b, gpu_point_buckets=None):
    """Points whose presence among the kept ids of bucket b of table t an
    FP64 near-tie leaves open: the points whose hash is a near-tie and that
    either side places in b, and the points around the filter cut, over the
    range of kept counts those points can cause (plus any filter-score
    near-tie at the cut)."""
    pb = ix.point_buckets[t]
    members = np.nonzero(pb == b)[0]
    flagged = np.nonzero(ix.hash_flag[t])[0]
    fl = flagged[pb[flagged] == b]
    if gpu_point_buckets is not None:
        fl = np.union1d(fl, flagged[np.asarray(gpu_point_buckets)[flagged] == b])
    pool = np.union1d(members, fl)
    if pool.size == 0:
        return pool
    sc = bucket_filter_scores(ix, t, b, pool)
    order = np.lexsort((pool, -sc))
    pool, sc = pool[order], sc[order]
    fixed = np.setdiff1d(members, fl).size
    kmin = int(O.keep_count(fixed, ix.alpha, ix.iprobes, ix.kappa))
    kmax = int(O.keep_count(pool.size, ix.alpha, ix.iprobes, ix.kappa))
    lo, hi = max(kmin - 1, 0), min(kmax + 1, pool.size)
    # widen over filter-score near-ties at either end of the window
    while lo > 0 and sc[lo - 1] - sc[lo] < O.NEAR_TIE:
        lo -= 1
    while hi < pool.size and sc[hi - 1] - sc[hi] < O.NEAR_TIE:
        hi += 1
    return np.union1d(fl, pool[lo:hi])


def topk_determined(ix, q, cand, amb, k):
    """True if every candidate set between cand minus amb and cand plus amb
    has the same top-k (then it is the oracle's top-k of cand)."""
    q64 = np.asarray(q, dtype=np.float64)
    lo = np.setdiff1d(cand, amb)
    hi = np.union1d(cand, amb)
    a, _, fa = O.falconn.topk_exact(lo, ix.X[lo] @ q64, k)
    b, _, fb = O.falconn.topk_exact(hi, ix.X[hi] @ q64, k)
    return not fa and not fb and np.array_equal(a, b)


def compare_search(res, gpu_ids, gpu_scores, k, tables, excl_by_table, ambiguous=None, Q=None,
                   ix=None):
    """Per query: exact ids and scores within SCORE_RTOL unless a flag
    (probe boundary, top-k boundary, or a probed bucket that is excluded)
    allows another answer.  With ``ambiguous`` ((t, b) -> ids, e.g.
    ambiguous_ids), a query that probes excluded buckets is still compared
    when its top-k is the same for every resolution of their ambiguous ids.
    Returns (n_compared, n_skipped, failures)."""
    compared, skipped, fails = 0, 0, []
    for i, r in enumerate(res):
        flagged = bool(r.topk_flag) or bool(np.any(r.probe_flag))
        if not flagged:
            hit = [(t, int(b)) for ti, t in enumerate(tables) if excl_by_table[t]
                   for b in r.buckets[ti] if int(b) in excl_by_table[t]]
            if hit:
                flagged = True
                if ambiguous is not None:
                    amb = np.unique(np.concatenate([ambiguous(t, b) for t, b in hit]
                                                   + [np.zeros(0, dtype=np.int64)]))
                    kk = len(r.ids)
                    flagged = not topk_determined(ix, Q[i], r.cand, amb.astype(np.int64), kk)
        if flagged:
            skipped += 1
            continue
        compared += 1
        kk = len(r.ids)
        gi = np.asarray(gpu_ids[i][:kk]).astype(np.int64)
        gs = np.asarray(gpu_scores[i][:kk]).astype(np.float64)
        if not np.array_equal(gi, r.ids):
            fails.append((i, "ids", r.ids.tolist(), gi.tolist()))
            continue
        fin = np.isfinite(r.scores)
        if not np.array_equal(np.isfinite(gs), fin):
            fails.append((i, "padding", r.scores.tolist(), gs.tolist()))
            continue
        err = np.abs(gs[fin] - r.scores[fin])
        tol = SCORE_RTOL * np.maximum(np.abs(r.scores[fin]), 1e-3)
        if np.any(err > tol):
            fails.append((i, "scores", r.scores.tolist(), gs.tolist()))
    return compared, skipped, fails


def compare_probes(ix, Q, P, gpu_probes, tables):
    """Probe sets per (query, table) must agree unless the oracle flags the
    P-th / (P+1)-th boundary.  Returns (compared, skipped, failures)."""
    compared, skipped, fails = 0, 0, []
    for i, q in enumerate(Q):
        b, _, flag = O.probe_buckets(ix, q, P, tables)
        for ti in range(len(tables)):
            if flag[ti]:
                skipped += 1
                continue
            compared += 1
            if set(b[ti].tolist()) != set(gpu_probes[i, ti].astype(np.int64).tolist()):
                fails.append((i, tables[ti]))
    return compared, skipped, fails


def compare_candidates(res, gpu_cands, tables, excl_by_table, ambiguous=None):
    """Per query: the de-duplicated candidate set must equal the oracle's
    unless a probe boundary is flagged; where probed buckets are excluded,
    the skip, or with ``ambiguous`` ((t, b) -> ids) the two sets must agree
    outside the ids those buckets leave open.  Returns (n_compared,
    n_skipped, failures)."""
    compared, skipped, fails = 0, 0, []
    for i, r in enumerate(res):
        if bool(np.any(r.probe_flag)):
            skipped += 1
            continue
        hit = [(t, int(b)) for ti, t in enumerate(tables) if excl_by_table[t]
               for b in r.buckets[ti] if int(b) in excl_by_table[t]]
        if hit and ambiguous is None:
            skipped += 1
            continue
        compared += 1
        g = np.asarray(gpu_cands[i]).astype(np.int64)
        want = r.cand
        if hit:
            amb = np.unique(np.concatenate([ambiguous(t, b) for t, b in hit])).astype(np.int64)
            g, want = np.setdiff1d(g, amb), np.setdiff1d(want, amb)
        if not np.array_equal(g, want):
            fails.append((i, len(r.cand), len(g)))
    return compared, skipped, fails
