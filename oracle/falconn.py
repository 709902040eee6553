"""Falconn++ in plain FP64 numpy: index build, probing, search, brute force.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Notation follows the paper: n points X on the unit sphere, query q, L hash
tables, each the concatenation of l = 2 cross-polytope hashes over D Gaussian
random vectors r_i (Section 2.2), filter fraction alpha (Section 3.4),
indexing probes iProbes and limit kappa (Algorithm 1 and Section 3.4),
query probes P per table, k results.

Readings of passages the paper leaves open:

* Hash value encoding (Eq. 1).  A hash returns one of the 2D signed vectors
  +r_i or -r_i.  We number them h = i for +r_i and h = i + D for -r_i.  The
  argmax over |q^T r_i| takes the lowest i on exact ties; the sign is +
  iff q^T r_i >= 0 (Eq. 1 says sgn >= 0).  The table key of the pair
  (h1, h2) is the bucket id h1 * 2D + h2, giving the 4D^2 buckets the paper
  counts for l = 2 (Section 4, parameter settings).
* Filter score of a point in a bucket (Section 3.4 keeps the top alpha*B
  points by |x^T r_i|; with l = 2 a bucket corresponds to two vectors).  We
  rank by the sum |x^T r_{i1}| + |x^T r_{i2}| = v1(h1) + v2(h2), the same
  quantity the probe ranking uses.  Ties: lower point id first.
* Kept count.  A bucket of size B keeps ceil(alpha * B) points, evaluated as
  one IEEE FP64 multiply and a ceil.  (floor would empty every bucket with
  B < 1/alpha.)  With multi-probe indexing and limit scaling it keeps
  min(B, max(kappa, ceil(alpha * B / iProbes))) (Algorithm 1, Section 3.4).
* Probe ranking (Section 3.4, "a new criteria").  Each hash j gives the
  signed list v_j(h) over the 2D wedges: v_j(i) = q^T r_i and
  v_j(i + D) = -q^T r_i, so its top D entries are the |q^T r_i| in the wedge
  on q's side, ranked by |q^T r_i| as the paper asks.  A bucket (h1, h2) is
  scored v1(h1) + v2(h2); a query probes the P highest-scoring buckets of
  every table (ties: lower bucket id).  P = 1 probes exactly the query's
  own bucket.
* Multi-probe indexing (Algorithm 1).  With iProbes > 1 a point is added to
  its iProbes highest-scoring buckets under the same pair score, and its
  filter score in each is that bucket's pair score.
* Short results.  With fewer than k candidates the tail is id -1, score -inf.

Near-ties.  Wherever an FP64 decision has a margin below NEAR_TIE the oracle
raises a flag; a different but equally valid answer is then allowed there.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .rotations import gaussian_rotations

NEAR_TIE = 1e-6


# ---------------------------------------------------------------------------
# Hashing (Section 2.2, Eq. 1) and the per-bucket filter (Section 3.4)
# ---------------------------------------------------------------------------

def cross_polytope_hash(p: np.ndarray):
    """Cross-polytope hash of projection rows ``p`` [..., D] (Eq. 1).

    Returns (h, value, flag): the wedge h in [0, 2D) (i for +r_i, i + D for
    -r_i), the winning |q^T r_i|, and a near-tie flag (the two largest |p|
    closer than NEAR_TIE, or the winner within NEAR_TIE of zero so that its
    sign is uncertain)."""
    D = p.shape[-1]
    a = np.abs(p)
    i_star = np.argmax(a, axis=-1)                  # first index on ties
    win = np.take_along_axis(p, i_star[..., None], axis=-1)[..., 0]
    h = i_star + D * (win < 0)                      # sign + iff q^T r >= 0
    top = np.abs(win)
    if D > 1:
        second = -np.partition(-a, 1, axis=-1)[..., 1]
    else:
        second = np.full_like(top, -np.inf)
    flag = ((top - second) < NEAR_TIE) | (top < NEAR_TIE)
    return h.astype(np.int64), top, flag


def keep_count(B, alpha: float, iprobes: int = 1, kappa: int = 0):
    """Points kept in a bucket holding ``B`` entries (Section 3.4,
    Algorithm 1 and the limit-scaling add-on): ceil(alpha * B / iProbes),
    raised to kappa when kappa > 0, never above B."""
    B = np.asarray(B, dtype=np.int64)
    c = np.ceil((float(alpha) * B.astype(np.float64)) / float(iprobes)).astype(np.int64)
    if kappa > 0:
        c = np.maximum(c, int(kappa))
    return np.minimum(c, B)


def _signed_lists(p: np.ndarray) -> np.ndarray:
    """v(h) over the 2D wedges of one hash: [p, -p] along the last axis."""
    return np.concatenate([p, -p], axis=-1)


def _top_pairs(v1: np.ndarray, v2: np.ndarray, P: int):
    """The P highest-scoring wedge pairs of each row (rows are leading axes).

    v1, v2: [..., 2D] signed lists.  Score v1[h1] + v2[h2]; ties by lower
    bucket id h1 * 2D + h2.  Only the top-T entries of each list can take
    part in the top-T pairs, T = min(P + 1, 2D), because a pair whose
    first wedge is ranked a-th in its list is preceded by the pairs made
    with the a - 1 wedges ranked above it (and likewise for the second).
    One extra pair is kept for the boundary near-tie flag.

    Returns (buckets [..., P], scores [..., P], margin [...]) where margin is
    the gap between the P-th and (P+1)-th pair scores (inf if none)."""
    W = v1.shape[-1]                           # 2D
    T = min(P + 1, W)
    o1 = np.argsort(-v1, axis=-1, kind="stable")[..., :T]
    o2 = np.argsort(-v2, axis=-1, kind="stable")[..., :T]
    a = np.take_along_axis(v1, o1, axis=-1)
    b = np.take_along_axis(v2, o2, axis=-1)
    s = a[..., :, None] + b[..., None, :]                        # [..., T, T]
    bid = o1[..., :, None] * W + o2[..., None, :]
    lead = s.shape[:-2]
    s = s.reshape(lead + (T * T,))
    bid = bid.reshape(lead + (T * T,))
    # order each row by (score desc, bucket asc)
    flat_s = s.reshape(-1, T * T)
    flat_b = bid.reshape(-1, T * T)
    order = np.empty_like(flat_b)
    for r in range(flat_s.shape[0]):
        order[r] = np.lexsort((flat_b[r], -flat_s[r]))
    s_sorted = np.take_along_axis(flat_s, order, axis=-1).reshape(lead + (T * T,))
    b_sorted = np.take_along_axis(flat_b, order, axis=-1).reshape(lead + (T * T,))
    Pe = min(P, T * T)
    if T * T > P:
        margin = s_sorted[..., P - 1] - s_sorted[..., P]
    else:
        margin = np.full(lead, np.inf)
    return b_sorted[..., :Pe], s_sorted[..., :Pe], margin


@dataclasses.dataclass
class OracleIndex:
    """The Falconn++ index as the oracle holds it."""

    n: int
    d: int
    L: int
    D: int
    alpha: float
    iprobes: int
    kappa: int
    R: np.ndarray                 # FP64 [L][2][D][d]
    X: np.ndarray                 # FP64 [n][d]
    offsets: np.ndarray           # int64 [L][4D^2 + 1]  kept CSR offsets
    ids: list                     # per table: int64 kept ids, bucket-major,
                                  # (filter score desc, id asc) inside a bucket
    counts: np.ndarray            # int64 [L][4D^2] bucket sizes before filtering
    point_buckets: np.ndarray     # int64 [L][n] (iProbes = 1 only, else None)
    hash_flag: np.ndarray         # bool [L][n]: near-tie bucket assignment
    filter_flag: np.ndarray       # bool [L][4D^2]: near-tie filter boundary
    Xh: np.ndarray | None = None  # FP64 points the tables hash (centered), if not X

    @property
    def nbuckets(self) -> int:
        return 4 * self.D * self.D

    def bucket_ids(self, t: int, b: int) -> np.ndarray:
        return self.ids[t][self.offsets[t, b]: self.offsets[t, b + 1]]


def _table_entries(X64, Rt, iprobes, chunk=1 << 16):
    """Bucket entries of one table: (point id, bucket, filter score, flag).

    iProbes = 1: one entry per point, its hash pair (Eq. 1) and score
    |x^T r_{i1}| + |x^T r_{i2}|.  iProbes > 1: the point's iProbes
    highest-scoring buckets (Algorithm 1) under the pair score."""
    n = X64.shape[0]
    D = Rt.shape[1]
    pid, bkt, fsc, flg = [], [], [], []
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        p1 = X64[s:e] @ Rt[0].T
        p2 = X64[s:e] @ Rt[1].T
        if iprobes == 1:
            h1, a1, f1 = cross_polytope_hash(p1)
            h2, a2, f2 = cross_polytope_hash(p2)
            pid.append(np.arange(s, e, dtype=np.int64))
            bkt.append(h1 * (2 * D) + h2)
            fsc.append(a1 + a2)
            flg.append(f1 | f2)
        else:
            b, sc, margin = _top_pairs(_signed_lists(p1), _signed_lists(p2), iprobes)
            _, _, f1 = cross_polytope_hash(p1)
            _, _, f2 = cross_polytope_hash(p2)
            flag = (margin < NEAR_TIE) | f1 | f2
            pid.append(np.repeat(np.arange(s, e, dtype=np.int64), b.shape[1]))
            bkt.append(b.reshape(-1))
            fsc.append(sc.reshape(-1))
            flg.append(np.repeat(flag, b.shape[1]))
    return (np.concatenate(pid), np.concatenate(bkt), np.concatenate(fsc),
            np.concatenate(flg))


def build_table(X64, Rt, alpha, iprobes=1, kappa=0):
    """One Falconn++ table: hash every point, then keep in every bucket the
    top keep_count(B) entries by filter score (Section 3.4, Algorithm 1).

    Returns (offsets, ids, counts, point_bucket or None, hash_flag [n],
    filter_flag [4D^2])."""
    n = X64.shape[0]
    D = Rt.shape[1]
    NB = 4 * D * D
    pid, bkt, fsc, flg = _table_entries(X64, Rt, iprobes)
    counts = np.bincount(bkt, minlength=NB).astype(np.int64)
    # group by bucket; inside a bucket, filter score desc then point id asc
    order = np.lexsort((pid, -fsc, bkt))
    b_sorted, f_sorted, p_sorted = bkt[order], fsc[order], pid[order]
    start = np.concatenate([[0], np.cumsum(counts)])[:-1]
    rank = np.arange(b_sorted.size) - start[b_sorted]
    keep = keep_count(counts, alpha, iprobes, kappa)
    kept = rank < keep[b_sorted]
    ids = p_sorted[kept]
    offsets = np.concatenate([[0], np.cumsum(keep)]).astype(np.int64)
    # filter boundary near-tie: last kept vs first dropped score
    filter_flag = np.zeros(NB, dtype=bool)
    cut = np.nonzero((keep < counts) & (keep > 0))[0]
    if cut.size:
        gap = f_sorted[start[cut] + keep[cut] - 1] - f_sorted[start[cut] + keep[cut]]
        filter_flag[cut] = gap < NEAR_TIE
    hash_flag = np.zeros(n, dtype=bool)
    np.logical_or.at(hash_flag, pid, flg)
    point_bucket = bkt if iprobes == 1 else None
    return offsets, ids, counts, point_bucket, hash_flag, filter_flag


def center_points(X, c=None):
    """Centering (Section 3.4, heuristic (1)): c = the mean of the points,
    x -> x - c.  c is the FP64 mean rounded to FP32 (or the given vector);
    each centered coordinate is the FP32 rounding of the exact difference.
    Returns (c as FP32, centered points as FP32)."""
    X32 = np.asarray(X, dtype=np.float32)
    if c is None:
        c = X32.astype(np.float64).mean(axis=0)
    c32 = np.asarray(c, dtype=np.float32)
    Xc = (X32.astype(np.float64) - c32.astype(np.float64)).astype(np.float32)
    return c32, Xc


def build_index(X, L: int, D: int, alpha: float, seed: int | None = None,
                R: np.ndarray | None = None, iprobes: int = 1, kappa: int = 0,
                tables=None, center: bool = False, c=None) -> OracleIndex:
    """Build the index over ``X`` [n][d] (FP32 or FP64 input, promoted).

    R comes from ``seed`` through the rotation generator, or is given.
    ``tables`` restricts the build to a subset of table numbers (the other
    tables are left empty) so that full-size cases can be checked table by
    table.  ``center``: the tables are built over the centered points
    x - c (Section 3.4, heuristic (1); queries are not centered, and search
    scores stay the inner products with the original points, whose order
    the centering does not change)."""
    X64 = np.asarray(X, dtype=np.float64)
    n, d = X64.shape
    Xh = X64
    if center:
        _, Xc = center_points(X, c)
        Xh = Xc.astype(np.float64)
    if R is None:
        R = gaussian_rotations(seed, L, D, d)
    R64 = np.asarray(R, dtype=np.float64).reshape(L, 2, D, d)
    NB = 4 * D * D
    offsets = np.zeros((L, NB + 1), dtype=np.int64)
    counts = np.zeros((L, NB), dtype=np.int64)
    ids = [np.zeros(0, dtype=np.int64) for _ in range(L)]
    pb = np.full((L, n), -1, dtype=np.int64) if iprobes == 1 else None
    hflag = np.zeros((L, n), dtype=bool)
    fflag = np.zeros((L, NB), dtype=bool)
    for t in (range(L) if tables is None else tables):
        o, i, cnt, b, hf, ff = build_table(Xh, R64[t], alpha, iprobes, kappa)
        offsets[t], ids[t], counts[t], hflag[t], fflag[t] = o, i, cnt, hf, ff
        if pb is not None:
            pb[t] = b
    return OracleIndex(n, d, L, D, float(alpha), iprobes, kappa, R64, X64,
                       offsets, ids, counts, pb, hflag, fflag, Xh if center else None)


# ---------------------------------------------------------------------------
# Query side: probing (Section 3.4), candidates, exact top-k
# ---------------------------------------------------------------------------

def probe_buckets(index: OracleIndex, q, P: int, tables=None):
    """The P buckets probed in each table for query ``q``.

    Returns (buckets [L', P], scores [L', P], flags [L']) where the flag
    marks a near-tie between the P-th and (P+1)-th pair score."""
    q64 = np.asarray(q, dtype=np.float64)
    tsel = np.arange(index.L) if tables is None else np.asarray(tables)
    p = index.R[tsel] @ q64                              # [L', 2, D]
    b, s, margin = _top_pairs(_signed_lists(p[:, 0]), _signed_lists(p[:, 1]), P)
    return b, s, margin < NEAR_TIE


def probe_global(index: OracleIndex, q, Qp: int, tables=None):
    """Global probe budget (qProbes, Sections 2.2 and 4): the Qp best
    (table, bucket) pairs over all 4D^2 buckets of every table, ranked by the
    pair score v1(h1) + v2(h2); ties go to the lower table, then the lower
    bucket.  A table can give at most Qp of them, so its best min(Qp, 4D^2)
    pairs are the only ones that can be selected; one more per table is
    ranked for the boundary flag.

    Returns (buckets: one array per table of its selected buckets in rank
    order, flag: near-tie between the Qp-th and (Qp+1)-th pair scores)."""
    q64 = np.asarray(q, dtype=np.float64)
    tsel = np.arange(index.L) if tables is None else np.asarray(tables)
    p = index.R[tsel] @ q64                              # [L', 2, D]
    T = min(Qp + 1, index.nbuckets)
    b, s, _ = _top_pairs(_signed_lists(p[:, 0]), _signed_lists(p[:, 1]), T)
    tt = np.repeat(np.arange(len(tsel)), b.shape[1])
    bb, ss = b.reshape(-1), s.reshape(-1)
    order = np.lexsort((bb, tt, -ss))
    take = order[:Qp]
    flag = bool(order.size > Qp and ss[order[Qp - 1]] - ss[order[Qp]] < NEAR_TIE)
    per = [bb[take][tt[take] == ti] for ti in range(len(tsel))]
    return per, flag


def simhash_signatures(index: OracleIndex, V, bits: int) -> np.ndarray:
    """SimHash signatures (Charikar, STOC 2002) from the index's own random
    vectors, as the paper suggests (Section 4: the projections are reused):
    bit i of a vector v is [v^T r_i >= 0] for the i-th of the 2 L D vectors
    in table-major order (r of table t, hash j, index i at (2t + j) D + i),
    packed little-endian into uint32 words.  V: [m][d]; returns [m][bits/32]."""
    if bits % 32 or not 0 < bits <= 2 * index.L * index.D:
        raise ValueError("bits must be a multiple of 32 in (0, 2 L D]")
    R = index.R.reshape(-1, index.d)[:bits]
    P = np.atleast_2d(np.asarray(V, dtype=np.float64)) @ R.T          # [m][bits]
    b = (P >= 0).astype(np.uint64)
    w = np.zeros((b.shape[0], bits // 32), dtype=np.uint64)
    for i in range(bits):
        w[:, i // 32] |= b[:, i] << np.uint64(i % 32)
    return w.astype(np.uint32)


def hamming(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Bit differences between signature rows a [..., W] and b [W]."""
    x = np.bitwise_xor(a, b)
    return np.array([sum(bin(int(v)).count("1") for v in row) for row in np.atleast_2d(x)],
                    dtype=np.int64)


def simhash_select(sig_x: np.ndarray, sig_q: np.ndarray, cand: np.ndarray, keep: int):
    """The ``keep`` candidates whose signatures differ from the query's in
    the fewest bits (ties: lower id), sorted by id: SimHash pre-ranking of
    the candidates before exact scoring (Section 4)."""
    if cand.size <= keep:
        return cand
    h = hamming(sig_x[cand], sig_q)
    order = np.lexsort((cand, h))
    return np.sort(cand[order[:keep]])


def topk_exact(cand: np.ndarray, scores: np.ndarray, k: int):
    """Top-k of (cand, scores) by score desc then id asc, padded with
    (-1, -inf); also the near-tie flag at the k-th / (k+1)-th boundary."""
    order = np.lexsort((cand, -scores))
    ids = np.full(k, -1, dtype=np.int64)
    sc = np.full(k, -np.inf)
    kk = min(k, order.size)
    ids[:kk] = cand[order[:kk]]
    sc[:kk] = scores[order[:kk]]
    flag = bool(order.size > k and scores[order[k - 1]] - scores[order[k]] < NEAR_TIE)
    return ids, sc, flag


def candidates(index: OracleIndex, buckets: np.ndarray, tables=None) -> np.ndarray:
    """Union of the kept ids of the probed buckets over the tables, as a
    sorted array of distinct point ids (the bitset de-duplication)."""
    tsel = np.arange(index.L) if tables is None else np.asarray(tables)
    parts = [index.bucket_ids(int(t), int(b))
             for ti, t in enumerate(tsel) for b in buckets[ti]]
    if not parts:
        return np.zeros(0, dtype=np.int64)
    return np.unique(np.concatenate(parts))


@dataclasses.dataclass
class QueryResult:
    ids: np.ndarray          # int64 [k]
    scores: np.ndarray       # FP64 [k]
    cand: np.ndarray         # sorted distinct candidate ids
    buckets: np.ndarray      # [L', P] probed buckets
    probe_flag: np.ndarray   # [L'] near-tie at the probe boundary
    topk_flag: bool          # near-tie at the top-k boundary
    entries: int             # bucket entries scanned (with duplicates)


def search(index: OracleIndex, q, k: int, P: int, tables=None,
           global_probes: int = 0, simhash=None) -> QueryResult:
    """One Falconn++ query: project, probe P buckets per table (or, with a
    global budget, the global_probes best buckets over all tables), union
    their kept points, score them exactly and return the top-k."""
    q64 = np.asarray(q, dtype=np.float64)
    if global_probes:
        b, gflag = probe_global(index, q64, global_probes, tables)
        pflag = np.full(len(b), gflag)
    else:
        b, _, pflag = probe_buckets(index, q64, P, tables)
    tsel = np.arange(index.L) if tables is None else np.asarray(tables)
    entries = int(sum(index.offsets[t, bb + 1] - index.offsets[t, bb]
                      for ti, t in enumerate(tsel) for bb in b[ti]))
    cand = candidates(index, b, tables)
    if simhash is not None:
        # simhash = (signatures of X [n][W], bits, keep): only the keep
        # candidates closest in Hamming distance are scored
        sig_x, bits, keep = simhash
        sig_q = simhash_signatures(index, q64[None, :], bits)[0]
        cand = simhash_select(sig_x, sig_q, cand, keep)
    s = index.X[cand] @ q64
    ids, sc, tflag = topk_exact(cand, s, k)
    return QueryResult(ids, sc, cand, b, pflag, tflag, entries)


def search_batch(index: OracleIndex, Q, k, P, tables=None, global_probes: int = 0,
                 simhash=None):
    """``search`` over the rows of Q; k and P may be scalars or per-query
    arrays.  Returns ids [m][kmax], scores, and the per-query results."""
    Q = np.asarray(Q)
    m = Q.shape[0]
    ks = np.broadcast_to(np.asarray(k), (m,))
    ps = np.broadcast_to(np.asarray(P), (m,))
    kmax = int(ks.max()) if m else 0
    ids = np.full((m, kmax), -1, dtype=np.int64)
    sc = np.full((m, kmax), -np.inf)
    res = []
    for i in range(m):
        r = search(index, Q[i], int(ks[i]), int(ps[i]), tables, global_probes, simhash)
        ids[i, : ks[i]] = r.ids
        sc[i, : ks[i]] = r.scores
        res.append(r)
    return ids, sc, res


def brute_force(X, Q, k: int, chunk: int = 1 << 18):
    """Exact top-k by FP64 inner product over all of X (ties: lower id).
    Returns ids [m][k], scores [m][k], and per-query near-tie flags."""
    X64 = np.asarray(X, dtype=np.float64)
    Q64 = np.atleast_2d(np.asarray(Q, dtype=np.float64))
    m, n = Q64.shape[0], X64.shape[0]
    ids = np.full((m, k), -1, dtype=np.int64)
    sc = np.full((m, k), -np.inf)
    flags = np.zeros(m, dtype=bool)
    S = np.empty((m, n))
    for s in range(0, n, chunk):
        S[:, s: s + chunk] = Q64 @ X64[s: s + chunk].T
    kk = min(k + 1, n)
    for i in range(m):
        row = S[i]
        if n > kk:
            thr = np.partition(row, n - kk)[n - kk]
            cand = np.nonzero(row >= thr)[0]
        else:
            cand = np.arange(n)
        ids[i], sc[i], flags[i] = topk_exact(cand.astype(np.int64), row[cand], k)
    return ids, sc, flags


def recall_at(found: np.ndarray, truth: np.ndarray, k: int) -> float:
    """Mean |found[:k] intersect truth[:k]| / k over queries."""
    hits = 0
    for f, t in zip(found, truth):
        tt = set(int(x) for x in t[:k] if x >= 0)
        hits += len(tt.intersection(int(x) for x in f[:k] if x >= 0))
    return hits / (k * len(found)) if len(found) else math.nan
