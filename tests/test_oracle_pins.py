"""Pins of the CPU oracle against facts fixed outside it.

Each test checks the oracle against something other than itself: published
test vectors, closed forms, brute-force enumeration written independently in
plain Python loops, invariants the paper fixes, and exact special cases.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import falconn as F
from oracle import rotations as RG
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- rotations

def test_splitmix64_published_vectors():
    want = [int(x) for x in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    got = [int(v) for v in RG.splitmix64(1234567, 5)]
    assert got == want


def test_splitmix64_counter_offset_matches_sequence():
    full = RG.splitmix64(99, 40)
    assert np.array_equal(RG.splitmix64(99, 10, start=30), full[30:])


def test_box_muller_closed_forms():
    # sqrt(-2 ln u1) cos(2 pi u2) at points where it is exact by hand
    u1 = np.array([math.exp(-0.5), math.exp(-2.0), 1.0, math.exp(-4.5)])
    u2 = np.array([0.0, 0.5, 0.3, 0.25])
    z = RG.box_muller(u1, u2)
    assert z[0] == pytest.approx(1.0, abs=1e-15)
    assert z[1] == pytest.approx(-2.0, abs=1e-15)
    assert z[2] == 0.0
    assert abs(z[3]) < 1e-15


def test_rotations_are_standard_normal():
    from scipy import stats
    R = O.gaussian_rotations(7, 4, 64, 128).reshape(-1).astype(np.float64)
    assert abs(R.mean()) < 0.01
    assert abs(R.var() - 1.0) < 0.01
    assert stats.kstest(R[:50000], "norm").pvalue > 1e-3
    # streams of different (table, hash) are uncorrelated
    a = RG.gaussian_stream(7, 0, 20000).astype(np.float64)
    b = RG.gaussian_stream(7, 1, 20000).astype(np.float64)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.03


def _nearest_bf16(x: float) -> float:
    # the two BF16 neighbours of an FP32 value and the closer one, ties to
    # the one with an even last kept bit
    u = int(np.float32(x).view(np.uint32))
    lo = u & 0xFFFF0000
    hi = lo + 0x10000
    flo = float(np.uint32(lo).view(np.float32))
    fhi = float(np.uint32(hi).view(np.float32))
    dlo, dhi = abs(x - flo), abs(fhi - x)
    if dlo != dhi:
        return flo if dlo < dhi else fhi
    return flo if (lo >> 16) % 2 == 0 else fhi


def test_rotations_on_bf16_grid():
    # hand cases of the rounding: 1 + 2^-8 is a tie (to 1, even), 1 + 3 2^-9
    # rounds up, -1.00390625 (tie) goes to -1
    for x, want in ((1.0 + 2.0 ** -8, 1.0), (1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7),
                    (-(1.0 + 2.0 ** -8), -1.0), (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6)):
        assert float(RG.round_bf16(np.array([x], np.float32))[0]) == want
    # every coordinate is the BF16 value nearest to the FP32 Box-Muller value
    raw = RG.splitmix64(RG.stream_state(5, 3), 2 * 300)
    u1, u2 = RG.uniform_pair(raw)
    z32 = RG.box_muller(u1, u2).astype(np.float32)
    got = RG.gaussian_stream(5, 3, 300)
    assert np.all(got.view(np.uint32) & 0xFFFF == 0)
    for a, b in zip(z32, got):
        assert _nearest_bf16(float(a)) == float(b)
    R = O.gaussian_rotations(9, 2, 16, 24)
    assert np.all(R.view(np.uint32) & 0xFFFF == 0)


def test_uniforms_in_range():
    raw = RG.splitmix64(RG.stream_state(5, 3), 20000)
    u1, u2 = RG.uniform_pair(raw)
    assert (u1 > 0).all() and (u1 <= 1).all()
    assert (u2 >= 0).all() and (u2 < 1).all()


# ---------------------------------------------------------------- hashing

def _hash_by_enumeration(p):
    """Eq. 1 restated as a search over the 2D signed vectors +-r_i: the wedge
    whose signed projection s * p_i is largest, first wedge on ties."""
    D = len(p)
    best_h, best_v = None, -math.inf
    for i in range(D):           # +r_i wedges first, then ties keep lower i
        for s, h in ((1.0, i), (-1.0, i + D)):
            v = s * p[i]
            if v > best_v:
                best_h, best_v = h, v
    return best_h


def test_hash_golden_2d():
    g = json.load(open(os.path.join(GOLDEN, "cross_polytope_2d.json")))
    X = np.array(g["points"])
    R1, R2 = np.array(g["R_hash1"]), np.array(g["R_hash2"])
    h1, _, _ = O.cross_polytope_hash(X @ R1.T)
    assert h1.tolist() == g["hash1"]
    h2, _, _ = O.cross_polytope_hash(X @ R2.T)
    assert int(h2[0]) == g["hash2_point0"]
    assert int(h1[0]) * 6 + int(h2[0]) == g["bucket_point0"]


def test_probe_golden_2d():
    g = json.load(open(os.path.join(GOLDEN, "cross_polytope_2d.json")))
    R = np.array([g["R_hash1"], g["R_hash2"]], dtype=np.float64)[None]
    X = np.array(g["points"])
    ix = O.build_index(X, L=1, D=3, alpha=1.0, R=R)
    b, s, flag = O.probe_buckets(ix, np.array(g["query"]), 3)
    assert b[0].tolist() == g["probes_P3"]
    assert not flag[0]


def test_hash_matches_enumeration():
    rng = np.random.default_rng(1)
    for D in (1, 2, 3, 8, 17):
        p = rng.standard_normal((200, D))
        h, top, _ = O.cross_polytope_hash(p)
        for r in range(p.shape[0]):
            assert h[r] == _hash_by_enumeration(list(p[r]))
            assert top[r] == max(abs(x) for x in p[r])


def test_hash_standard_basis_is_nearest_cross_polytope_vertex():
    # r_i = e_i: the hash is the nearest vertex +-e_i of the cross-polytope,
    # i.e. the coordinate of largest magnitude with its sign.
    rng = np.random.default_rng(2)
    x = rng.standard_normal((500, 6))
    h, _, _ = O.cross_polytope_hash(x @ np.eye(6).T)
    verts = np.concatenate([np.eye(6), -np.eye(6)])
    dist = ((x[:, None, :] / np.linalg.norm(x, axis=1)[:, None, None] - verts[None]) ** 2).sum(-1)
    assert np.array_equal(h, np.argmin(dist, axis=1))


def test_hash_invariances():
    rng = np.random.default_rng(3)
    D = 16
    R = rng.standard_normal((D, 10))
    x = rng.standard_normal((300, 10))
    h, _, _ = O.cross_polytope_hash(x @ R.T)
    h_scaled, _, _ = O.cross_polytope_hash((3.5 * x) @ R.T)
    h_neg, _, _ = O.cross_polytope_hash((-x) @ R.T)
    assert np.array_equal(h, h_scaled)
    assert np.array_equal(h_neg, (h + D) % (2 * D))     # antipodal wedge


# ---------------------------------------------------------------- index build

def test_every_point_in_exactly_one_bucket(tiny_data, tiny_index):
    w, X, _ = tiny_data
    ix = tiny_index
    assert (ix.counts.sum(axis=1) == w.n).all()
    for t in range(ix.L):
        assert np.array_equal(np.bincount(ix.point_buckets[t], minlength=ix.nbuckets),
                              ix.counts[t])


def test_point_buckets_match_per_point_hash(tiny_data, tiny_index):
    w, X, _ = tiny_data
    ix = tiny_index
    R = O.gaussian_rotations(w.rot_seed, w.L, w.D, w.d).astype(np.float64)
    rng = np.random.default_rng(4)
    for pid in rng.choice(w.n, 40, replace=False):
        for t in (0, w.L - 1):
            x = X[pid].astype(np.float64)
            h1 = _hash_by_enumeration(list(R[t, 0] @ x))
            h2 = _hash_by_enumeration(list(R[t, 1] @ x))
            assert ix.point_buckets[t, pid] == h1 * 2 * w.D + h2


def test_kept_count_is_ceil_alpha_B(tiny_index):
    ix = tiny_index
    kept = np.diff(ix.offsets, axis=1)
    for B, c in zip(ix.counts.reshape(-1), kept.reshape(-1)):
        assert c == -((-2 * int(B)) // 10)      # ceil(0.2 B) in integers


def test_keep_count_matches_rational_ceil():
    B = np.arange(0, 200001)
    for a, b in ((1, 10), (1, 5), (1, 20), (1, 100), (3, 10)):
        want = -((-a * B) // b)
        assert np.array_equal(O.keep_count(B, a / b), want), (a, b)


def test_limit_scaling_keep_count():
    B = np.arange(0, 500)
    got = O.keep_count(B, 0.01, iprobes=3, kappa=20)
    want = np.minimum(B, np.maximum(20, -((-B) // 300)))
    assert np.array_equal(got, want)


def test_alpha_one_keeps_everything(tiny_data):
    w, X, _ = tiny_data
    ix = O.build_index(X[:2000], 3, 16, 1.0, seed=11)
    for t in range(3):
        assert np.array_equal(np.sort(ix.ids[t]), np.arange(2000))


def test_filter_keeps_top_by_projection_magnitude():
    # brute force per bucket: recompute |x^T r_i1| + |x^T r_i2| in Python
    X, _ = W.small_mixture(600, 1, 8, 4, 0.2, 5)
    R = O.gaussian_rotations(12, 2, 4, 8).astype(np.float64)
    ix = O.build_index(X, 2, 4, 0.3, R=R)
    for t in range(2):
        buckets = {}
        for pid in range(600):
            x = [float(v) for v in X[pid]]
            p1 = [sum(a * b for a, b in zip(x, r)) for r in R[t, 0]]
            p2 = [sum(a * b for a, b in zip(x, r)) for r in R[t, 1]]
            h1, h2 = _hash_by_enumeration(p1), _hash_by_enumeration(p2)
            f = max(abs(v) for v in p1) + max(abs(v) for v in p2)
            buckets.setdefault(h1 * 8 + h2, []).append((-f, pid))
        for b in range(ix.nbuckets):
            members = sorted(buckets.get(b, []))
            c = math.ceil(0.3 * len(members) - 1e-12)
            assert ix.bucket_ids(t, b).tolist() == [pid for _, pid in members[:c]]


def test_multiprobe_indexing_counts():
    X, _ = W.small_mixture(500, 1, 8, 4, 0.2, 6)
    ix = O.build_index(X, 2, 4, 0.5, seed=3, iprobes=3, kappa=2)
    assert (ix.counts.sum(axis=1) == 3 * 500).all()     # Algorithm 1: n*iProbes entries
    kept = np.diff(ix.offsets, axis=1)
    assert np.array_equal(kept, O.keep_count(ix.counts, 0.5, 3, 2))
    for t in range(2):   # a point appears at most once per bucket
        for b in range(ix.nbuckets):
            ids = ix.bucket_ids(t, b)
            assert len(set(ids.tolist())) == len(ids)


def _algorithm1_by_enumeration(X, R, alpha_num, alpha_den, iprobes, kappa):
    """Multi-probe indexing (Algorithm 1) in plain Python loops for one table:
    each point goes to its iProbes best buckets under the pair score
    v1(h1) + v2(h2) over all (2D)^2 wedge pairs (ties: lower bucket), with
    that score as its filter score there; a bucket of B entries keeps its
    best min(B, max(kappa, ceil(alpha B / iProbes))) by (score desc, id asc).
    alpha = alpha_num / alpha_den so that the ceil is taken in integers."""
    D = len(R[0])
    buckets = {}
    for pid, x in enumerate(X):
        x = [float(v) for v in x]
        p1 = [sum(a * b for a, b in zip(x, r)) for r in R[0]]
        p2 = [sum(a * b for a, b in zip(x, r)) for r in R[1]]
        v1 = p1 + [-v for v in p1]
        v2 = p2 + [-v for v in p2]
        pairs = sorted((-(v1[a] + v2[b]), a * 2 * D + b)
                       for a in range(2 * D) for b in range(2 * D))
        for negs, b in pairs[:iprobes]:
            buckets.setdefault(b, []).append((negs, pid))
    kept = {}
    for b, members in buckets.items():
        members.sort()
        B = len(members)
        c = -((-alpha_num * B) // (alpha_den * iprobes))
        c = min(B, max(kappa, c))
        kept[b] = [pid for _, pid in members[:c]]
    return kept


@pytest.mark.parametrize("iprobes,kappa", [(3, 2), (2, 0), (4, 5)])
def test_multiprobe_kept_set_matches_algorithm1_enumeration(iprobes, kappa):
    X, _ = W.small_mixture(400, 1, 6, 4, 0.25, 7)
    L, D = 2, 3
    R = O.gaussian_rotations(21, L, D, 6).astype(np.float64)
    ix = O.build_index(X, L, D, 0.5, R=R, iprobes=iprobes, kappa=kappa)
    checked = 0
    for t in range(L):
        want = _algorithm1_by_enumeration(X, R[t], 1, 2, iprobes, kappa)
        for b in range(ix.nbuckets):
            got = ix.bucket_ids(t, b).tolist()
            if ix.filter_flag[t, b] or any(ix.hash_flag[t, i] for i in got):
                continue
            assert got == want.get(b, []), (t, b)
            checked += len(got)
    assert checked > 0.9 * ix.offsets[:, -1].sum()


# ---------------------------------------------------------------- probing

def _pairs_by_enumeration(p1, p2, P):
    D = len(p1)
    v1 = list(p1) + [-x for x in p1]
    v2 = list(p2) + [-x for x in p2]
    allp = [(-(v1[a] + v2[b]), a * 2 * D + b) for a in range(2 * D) for b in range(2 * D)]
    allp.sort()
    return [b for _, b in allp[:P]]


@pytest.mark.parametrize("D", [1, 2, 3, 5])
def test_probe_ranking_matches_full_enumeration(D):
    rng = np.random.default_rng(D)
    R = rng.standard_normal((1, 2, D, 4))
    ix = O.build_index(rng.standard_normal((5, 4)), 1, D, 1.0, R=R)
    for _ in range(20):
        q = rng.standard_normal(4)
        p = R[0] @ q
        for P in sorted({1, 2, 3, D, 2 * D, 4 * D * D - 1, 4 * D * D} - {0}):
            b, _, _ = O.probe_buckets(ix, q, P)
            assert b[0].tolist() == _pairs_by_enumeration(p[0], p[1], P)


def test_single_probe_is_query_bucket(tiny_data, tiny_index):
    w, X, Q = tiny_data
    ix = tiny_index
    for q in Q[:20]:
        b, _, _ = O.probe_buckets(ix, q, 1)
        p = ix.R @ q.astype(np.float64)
        h1, _, _ = O.cross_polytope_hash(p[:, 0])
        h2, _, _ = O.cross_polytope_hash(p[:, 1])
        assert np.array_equal(b[:, 0], h1 * 2 * w.D + h2)


def test_probe_sets_nested_and_scores_sorted(tiny_data, tiny_index):
    w, X, Q = tiny_data
    for q in Q[:10]:
        b4, s4, _ = O.probe_buckets(tiny_index, q, 4)
        b16, s16, _ = O.probe_buckets(tiny_index, q, 16)
        assert (np.diff(s16, axis=1) <= 0).all()
        assert np.array_equal(b16[:, :4], b4)


# ---------------------------------------------------------------- search

def test_bruteforce_matches_full_sort():
    rng = np.random.default_rng(8)
    X = rng.standard_normal((300, 5))
    Q = rng.standard_normal((7, 5))
    ids, sc, _ = O.brute_force(X, Q, 12)
    for i in range(7):
        s = [(-sum(float(a) * float(b) for a, b in zip(X[j], Q[i])), j) for j in range(300)]
        s.sort()
        assert ids[i].tolist() == [j for _, j in s[:12]]


def test_short_results_are_padded():
    X = np.eye(4)
    ids, sc, _ = O.brute_force(X, np.ones((1, 4)), 6)
    assert ids[0, 4:].tolist() == [-1, -1]
    assert np.isneginf(sc[0, 4:]).all()


def test_unfiltered_full_probe_equals_bruteforce():
    # alpha = 1 and all 4D^2 buckets probed: every point is a candidate, so
    # Falconn++ returns the exact top-k.
    X, Q = W.small_mixture(3000, 20, 16, 32, 0.1, 9)
    ix = O.build_index(X, 2, 4, 1.0, seed=21)
    ids, sc, res = O.search_batch(ix, Q, 10, 4 * 4 * 4)
    bi, bs, _ = O.brute_force(X, Q, 10)
    assert all(r.cand.size == 3000 for r in res)
    assert np.array_equal(ids, bi)
    assert np.allclose(sc, bs)


def test_search_topk_is_exact_over_candidates(tiny_data, tiny_index):
    w, X, Q = tiny_data
    for q in Q[:10]:
        r = O.search(tiny_index, q, 10, 4)
        s = sorted((-float(np.dot(X[c].astype(np.float64), q.astype(np.float64))), int(c))
                   for c in r.cand)
        assert r.ids.tolist() == [c for _, c in s[:10]]


def test_candidates_are_union_of_probed_buckets(tiny_data, tiny_index):
    w, X, Q = tiny_data
    ix = tiny_index
    r = O.search(ix, Q[0], 10, 4)
    u = set()
    for t in range(ix.L):
        for b in r.buckets[t]:
            u.update(ix.ids[t][ix.offsets[t, b]: ix.offsets[t, b + 1]].tolist())
    assert sorted(u) == r.cand.tolist()


def test_recall_monotone_in_probes(tiny_data, tiny_index):
    # probe sets are nested, so candidate sets are nested, so the exact top-k
    # over them can only gain true neighbours
    w, X, Q = tiny_data
    bi, _, _ = O.brute_force(X, Q[:30], 10)
    prev = -1.0
    prev_c = None
    for P in (1, 2, 4, 8, 32):
        ids, _, res = O.search_batch(tiny_index, Q[:30], 10, P)
        r = O.recall_at(ids, bi, 10)
        assert r >= prev
        prev = r
        if prev_c is not None:
            for a, b in zip(prev_c, res):
                assert set(a.cand.tolist()) <= set(b.cand.tolist())
        prev_c = res
    assert prev > 0.9


def test_lemma1_collision_probability_band():
    # Lemma 1 (Section 2.2, quoted from the Falconn analysis): two unit
    # vectors at distance r collide under one cross-polytope hash with
    # probability about D^(-1 / (4 / r^2 - 1)).  The form is asymptotic in D
    # (lower-order factors), so it pins a loose band; orthogonal vectors
    # (r = sqrt 2) hash independently over the 2D signed vectors, which pins
    # 1 / (2D) tightly (a hash that dropped the sign would give 1 / D).
    rng = np.random.default_rng(11)
    d, T = 32, 20000
    p = {}
    for D in (8, 32):
        for r in (0.5, 1.0, np.sqrt(2.0)):
            q = rng.standard_normal((T, d))
            q /= np.linalg.norm(q, axis=1)[:, None]
            u = rng.standard_normal((T, d))
            u -= (u * q).sum(1)[:, None] * q
            u /= np.linalg.norm(u, axis=1)[:, None]
            th = 2.0 * np.arcsin(r / 2.0)
            x = np.cos(th) * q + np.sin(th) * u
            R = rng.standard_normal((T, D, d))
            hx = O.cross_polytope_hash(np.einsum("td,tkd->tk", x, R))[0]
            hq = O.cross_polytope_hash(np.einsum("td,tkd->tk", q, R))[0]
            p[D, r] = float((hx == hq).mean())
        assert 0.8 < 2 * D * p[D, np.sqrt(2.0)] < 1.2, (D, p[D, np.sqrt(2.0)])
        for r in (0.5, 1.0):
            pred = D ** (-1.0 / (4.0 / r ** 2 - 1.0))
            assert 0.25 < p[D, r] / pred <= 1.0, (D, r, p[D, r], pred)
        assert p[D, 0.5] > p[D, 1.0] > p[D, np.sqrt(2.0)]
    for r in (0.5, 1.0, np.sqrt(2.0)):
        assert p[8, r] > p[32, r]


def test_ceos_projection_preserves_inner_product_order():
    # Lemma 2 (CEOs): on the vector r_1 = argmax |q^T r_i|, x^T r_1 is
    # centred at sgn(q^T r_1) x^T q sqrt(2 ln D).  Loose statistical check
    # of the mean over many independent draws.
    rng = np.random.default_rng(10)
    d, D, trials = 64, 512, 300
    q = rng.standard_normal(d); q /= np.linalg.norm(q)
    z = rng.standard_normal(d); z -= z.dot(q) * q; z /= np.linalg.norm(z)
    c = 0.6
    x = c * q + math.sqrt(1 - c * c) * z
    vals = []
    for _ in range(trials):
        R = rng.standard_normal((D, d))
        p = R @ q
        i = int(np.argmax(np.abs(p)))
        vals.append(np.sign(p[i]) * (R[i] @ x))
    mean = float(np.mean(vals))
    # asymptotic value c * sqrt(2 ln D) = 2.13; the finite-D mean of the top
    # order statistic is a little smaller, so a band of +-20%
    assert 0.8 * c * math.sqrt(2 * math.log(D)) < mean < 1.2 * c * math.sqrt(2 * math.log(D))


def test_theorem1_keep_rates():
    # Theorem 1 (Section 3.3): with r_1 the signed random vector the query
    # hashes to, the threshold t = (1 - r^2 / 2) sqrt(2 ln D) keeps a point
    # at distance r with probability about 1/2 and one at distance >= c r
    # with probability at most q2 = exp(-g^2 / 2) / (g sqrt(2 pi)),
    # g = c r (1 - 1/c^2) / sqrt(4 - c^2 r^2) sqrt(2 ln D).  The statement is
    # asymptotic in D: at D = 256 the near rate sits a little below 1/2.
    # The oracle's hash picks r_1 and its signed lists give x^T r_1, so a
    # wrong sign or a wrong argmax in either sends the near rate to ~0.
    rng = np.random.default_rng(5)
    d, D, T = 64, 256, 4000
    for r, c in ((1.0, 1.3), (0.8, 1.5)):
        q = rng.standard_normal((T, d))
        q /= np.linalg.norm(q, axis=1)[:, None]

        def at(dist):
            u = rng.standard_normal((T, d))
            u -= (u * q).sum(1)[:, None] * q
            u /= np.linalg.norm(u, axis=1)[:, None]
            th = 2.0 * np.arcsin(dist / 2.0)
            return np.cos(th) * q + np.sin(th) * u

        x, y = at(r), at(c * r)
        R = rng.standard_normal((T, D, d))
        h, _, _ = O.cross_polytope_hash(np.einsum("td,tkd->tk", q, R))
        vx = np.take_along_axis(F._signed_lists(np.einsum("td,tkd->tk", x, R)), h[:, None], 1)[:, 0]
        vy = np.take_along_axis(F._signed_lists(np.einsum("td,tkd->tk", y, R)), h[:, None], 1)[:, 0]
        t = (1.0 - r * r / 2.0) * math.sqrt(2.0 * math.log(D))
        g = c * r * (1.0 - 1.0 / c ** 2) / math.sqrt(4.0 - (c * r) ** 2) * math.sqrt(2.0 * math.log(D))
        q2 = math.exp(-g * g / 2.0) / (g * math.sqrt(2.0 * math.pi))
        near, far = float((vx >= t).mean()), float((vy >= t).mean())
        assert 0.33 < near < 0.6, (r, near)
        assert far < q2, (r, c, far, q2)
        assert far < 0.5 * near


def test_recall_at_by_hand():
    found = np.array([[1, 2, 3, -1], [5, 6, 7, 8]])
    truth = np.array([[3, 2, 9, 10], [8, 7, 6, 5]])
    # k = 4: query 0 finds {2, 3} of 4, query 1 all 4: 6 / 8
    assert O.recall_at(found, truth, 4) == 0.75
    # k = 2: {1, 2} vs {3, 2} is 1 hit, {5, 6} vs {8, 7} none: 1 / 4
    assert O.recall_at(found, truth, 2) == 0.25
    # padding ids (-1) never count, even against padded truth
    assert O.recall_at(np.array([[-1, -1]]), np.array([[-1, -1]]), 2) == 0.0


def test_centering_transform_pinned():
    # Section 3.4, heuristic (1): c is the mean of the points and x -> x - c,
    # here on values where every step is exact
    X = np.array([[1.0, 2.0, -3.0], [3.0, 4.0, 5.0]], dtype=np.float32)
    c, Xc = O.center_points(X)
    assert c.tolist() == [2.0, 3.0, 1.0]
    assert Xc.tolist() == [[-1.0, -1.0, -4.0], [1.0, 1.0, 4.0]]
    # an explicit centre is used as given
    c2, Xc2 = O.center_points(X, np.array([1.0, 1.0, 1.0]))
    assert Xc2.tolist() == [[0.0, 1.0, -4.0], [2.0, 3.0, 4.0]]


def test_centered_index_is_the_index_of_centered_points():
    # the centered build hashes and filters the centered points, so its
    # tables equal those of a plain build over x - c; the search still
    # scores the original points
    import workloads as W
    X, Q = W.small_mixture(3000, 20, 24, 16, 0.3, 81)
    X = X + np.float32(0.2)   # a common offset, then centering
    ixc = O.build_index(X, 4, 8, 0.5, seed=5, center=True)
    _, Xc = O.center_points(X)
    ixp = O.build_index(Xc, 4, 8, 0.5, seed=5)
    for t in range(4):
        assert np.array_equal(ixc.offsets[t], ixp.offsets[t])
        assert np.array_equal(ixc.ids[t], ixp.ids[t])
    ids, sc, _ = O.search_batch(ixc, Q, 5, 2)
    X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
    for i in range(len(Q)):
        ok = ids[i] >= 0
        assert np.allclose(sc[i][ok], X64[ids[i][ok]] @ Q64[i], rtol=0, atol=1e-12)


def test_centering_spreads_skewed_data_over_buckets():
    # the point of centering (Section 3.4): data crowded on one area of the
    # sphere falls into few buckets; after centering it spreads out
    rng = np.random.default_rng(12)
    d = 32
    base = np.zeros(d); base[0] = 1.0
    X = base + 0.15 * rng.standard_normal((4000, d))
    X = (X / np.linalg.norm(X, axis=1, keepdims=True)).astype(np.float32)
    plain = O.build_index(X, 2, 8, 1.0, seed=3)
    cent = O.build_index(X, 2, 8, 1.0, seed=3, center=True)
    for t in range(2):
        assert cent.counts[t].max() < 0.5 * plain.counts[t].max()
        assert np.count_nonzero(cent.counts[t]) > np.count_nonzero(plain.counts[t])


def test_global_probes_equal_brute_force_enumeration():
    # qProbes (Sections 2.2 and 4): the Qp best (table, bucket) pairs over
    # all tables, checked against a plain enumeration of every pair
    import workloads as W
    X, Q = W.small_mixture(500, 6, 12, 8, 0.3, 83)
    L, D = 3, 2
    ix = O.build_index(X, L, D, 1.0, seed=7)
    for q in Q:
        q64 = q.astype(np.float64)
        allp = []
        for t in range(L):
            p1 = ix.R[t, 0] @ q64
            p2 = ix.R[t, 1] @ q64
            v1 = np.concatenate([p1, -p1])
            v2 = np.concatenate([p2, -p2])
            for h1 in range(2 * D):
                for h2 in range(2 * D):
                    allp.append((-(v1[h1] + v2[h2]), t, h1 * 2 * D + h2))
        allp.sort()
        for Qp in (1, 5, 12, 4 * D * D * L):
            per, flag = O.probe_global(ix, q, Qp)
            want = allp[:Qp]
            got = sorted((t, int(b)) for t in range(L) for b in per[t])
            if not flag:
                assert got == sorted((t, b) for _, t, b in want)
            assert sum(len(x) for x in per) == Qp


def test_global_probes_uncapped_past_128_per_table():
    # qProbes ranks the buckets of all tables together with no per-table
    # limit: with D = 8 a table has 256 buckets, and budgets above 128 must
    # take more than 128 from one table when its pairs score highest
    X, Q = W.small_mixture(300, 5, 10, 8, 0.3, 85)
    L, D = 3, 8
    ix = O.build_index(X, L, D, 1.0, seed=9)
    over_128 = 0
    for q in Q:
        q64 = q.astype(np.float64)
        allp = []
        for t in range(L):
            p1 = [float(v) for v in ix.R[t, 0] @ q64]
            p2 = [float(v) for v in ix.R[t, 1] @ q64]
            v1 = p1 + [-v for v in p1]
            v2 = p2 + [-v for v in p2]
            for h1 in range(2 * D):
                for h2 in range(2 * D):
                    allp.append((-(v1[h1] + v2[h2]), t, h1 * 2 * D + h2))
        allp.sort()
        for Qp in (129, 300, 700):
            per, flag = O.probe_global(ix, q, Qp)
            assert sum(len(x) for x in per) == Qp
            if flag:
                continue
            got = sorted((t, int(b)) for t in range(L) for b in per[t])
            assert got == sorted((t, b) for _, t, b in allp[:Qp])
            # each table's buckets come in rank order
            for t in range(L):
                mine = [b for _, tt, b in allp[:Qp] if tt == t]
                assert [int(b) for b in per[t]] == mine
            over_128 += max(len(x) for x in per) > 128
    assert over_128 > 0


def test_global_probes_all_buckets_is_bruteforce_and_monotone():
    import workloads as W
    X, Q = W.small_mixture(1500, 8, 16, 8, 0.3, 84)
    ix = O.build_index(X, 3, 3, 1.0, seed=8)
    bi, _, bflag = O.brute_force(X, Q, 5)
    _, _, res = O.search_batch(ix, Q, 5, 1, global_probes=3 * 36)
    for i, r in enumerate(res):
        if not bflag[i]:
            assert np.array_equal(r.ids, bi[i])
    prev = None
    for Qp in (1, 3, 9, 27):
        _, _, res = O.search_batch(ix, Q, 5, 1, global_probes=Qp)
        if prev is not None:
            for a, b in zip(prev, res):
                if not (np.any(a.probe_flag) or np.any(b.probe_flag)):
                    assert set(a.cand.tolist()) <= set(b.cand.tolist())
        prev = res


def test_simhash_signature_bits_by_hand():
    # bit i = [v^T r_i >= 0] over the index's vectors in table-major order
    R = np.zeros((1, 2, 16, 3))   # 32 vectors; all but the first four are zero
    R[0, 0, 0] = [1, 0, 0]
    R[0, 0, 1] = [0, 1, 0]
    R[0, 0, 2] = [0, 0, 1]
    R[0, 0, 3] = [1, 1, 1]
    X = np.array([[0.6, -0.8, 0.0]], dtype=np.float32)
    ix = O.build_index(X, 1, 16, 1.0, R=R)
    sig = O.simhash_signatures(ix, np.array([[0.6, -0.8, 0.0], [-1.0, 2.0, -3.0]]), 32)
    # v1: +, -, 0 (>= 0 -> 1), -0.2 -> bits 1,0,1,0 ; v2: -, +, -, - -> 0,1,0,0;
    # the zero vectors give 0 >= 0 -> 1 in bits 4..31
    assert sig[0, 0] == 0xFFFFFFF5 and sig[1, 0] == 0xFFFFFFF2
    assert O.hamming(sig, sig[0]).tolist() == [0, 3]


def test_simhash_estimates_angle():
    # Charikar: a random hyperplane separates two vectors with probability
    # theta / pi
    rng = np.random.default_rng(13)
    d = 64
    X = rng.standard_normal((2, d)).astype(np.float32)
    ix = O.build_index(X, 8, 64, 1.0, seed=9)   # 1,024 vectors
    q = rng.standard_normal(d)
    for c in (0.9, 0.5, 0.0, -0.7):
        z = rng.standard_normal(d); z -= z.dot(q) * q / q.dot(q)
        v = c * q / np.linalg.norm(q) + math.sqrt(1 - c * c) * z / np.linalg.norm(z)
        s = O.simhash_signatures(ix, np.stack([q, v]), 1024)
        frac = O.hamming(s[1:], s[0])[0] / 1024.0
        assert abs(frac - math.acos(c) / math.pi) < 0.05


def test_simhash_keep_all_equals_plain_search(tiny_data, tiny_index):
    w, X, Q = tiny_data
    sig = O.simhash_signatures(tiny_index, X, 256)
    a, sa, _ = O.search_batch(tiny_index, Q[:20], w.k, 4)
    b, sb, _ = O.search_batch(tiny_index, Q[:20], w.k, 4, simhash=(sig, 256, 10 ** 6))
    assert np.array_equal(a, b) and np.array_equal(sa, sb)
    # a small keep scores fewer candidates; the result is within the kept ones
    _, _, res = O.search_batch(tiny_index, Q[:20], w.k, 4, simhash=(sig, 256, 50))
    for r in res:
        assert r.cand.size <= 50
        assert set(r.ids[r.ids >= 0].tolist()) <= set(r.cand.tolist())


def test_parallel_build_equals_serial_build():
    # the process-pool build runs the same per-table function: identical index
    from oracle.parallel import build_index_parallel
    X, _ = W.small_mixture(3000, 1, 16, 8, 0.3, 86)
    for kw in ({}, {"iprobes": 2, "kappa": 1}, {"center": True}):
        a = O.build_index(X, 3, 4, 0.3, seed=5, **kw)
        b = build_index_parallel(X, 3, 4, 0.3, seed=5, workers=2, **kw)
        assert np.array_equal(a.offsets, b.offsets)
        assert all(np.array_equal(x, y) for x, y in zip(a.ids, b.ids))
        assert np.array_equal(a.counts, b.counts)
        assert np.array_equal(a.hash_flag, b.hash_flag)
        assert np.array_equal(a.filter_flag, b.filter_flag)
        if a.point_buckets is not None:
            assert np.array_equal(a.point_buckets, b.point_buckets)


def test_in_bucket_order_comparison_allows_only_near_tie_swaps():
    from tests import parity as PT
    want = np.array([5, 3, 9, 1])
    s = np.array([0.9, 0.5, 0.5 - 1e-8, 0.1])
    assert PT.same_up_to_near_ties(want, want, s)
    assert PT.same_up_to_near_ties(want, np.array([5, 9, 3, 1]), s)    # near-tied pair
    assert not PT.same_up_to_near_ties(want, np.array([3, 5, 9, 1]), s)
    assert not PT.same_up_to_near_ties(want, np.array([5, 3, 1, 9]), s)
