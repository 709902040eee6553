"""BF16 precision path (FPP_BF16) against the FP64 oracle and the exact path.

The BF16 path hashes and probes exactly as the FP32 path does and scores
candidates from BF16 rows; a shortlist is re-scored exactly and a top-k
boundary inside the statistical BF16 window is re-decided.  It is graded by
recall and score error: bucket ids and probe sets equal the exact path's,
top-k ids agree with the oracle except on a small fraction of queries,
returned scores are exact inner products of the returned ids, and recall
matches the exact path's.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2206_01382_gb300 as F
    from paper_2206_01382_gb300 import _build
    _build.build()
    F.load()
    return F


def _exact_scores(X, Q, ids):
    X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
    out = np.full(ids.shape, -np.inf)
    for i in range(ids.shape[0]):
        ok = ids[i] >= 0
        out[i, ok] = X64[ids[i, ok]] @ Q64[i]
    return out


def _round_bf16(x):
    """Round-to-nearest-even of FP32 values to BF16, returned as FP32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32)


def test_bf16_hashing_equals_exact_path_and_window_covers_bf16_scores(F):
    for d, D, L in ((128, 256, 2), (960, 64, 1), (37, 5, 3)):
        X, Q = W.small_mixture(800, 400, d, 32, 0.25, 300 + d)
        ix16 = F.Index(X, L, D, 0.5, seed=50 + d, precision=F.FPP_BF16)
        ix32 = F.Index(X, L, D, 0.5, seed=50 + d)
        # hashing and probing run on the same exact-split projections
        assert np.array_equal(F.fpp_debug_projections(ix16.handle, Q),
                              F.fpp_debug_projections(ix32.handle, Q))
        # first-pass scores from BF16 rows stay inside the statistical window
        c = ix16.info()["score_error_factor"]
        Xb = _round_bf16(X).astype(np.float64)
        X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
        err = np.abs(Q64 @ Xb.T - Q64 @ X64.T)
        win = c * np.linalg.norm(Q64, axis=1)[:, None] * np.linalg.norm(X64, axis=1)[None, :]
        assert float((err / win).max()) < 1.0, d
        assert ix32.info()["score_error_factor"] < 0.1 * c   # FP32 bound gamma_d


def test_bf16_tiny_decisions_match_oracle(F):
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    ix_o = O.build_index(X, w.L, w.D, w.alpha, seed=w.rot_seed)
    ix_b = F.Index(X, w.L, w.D, w.alpha, seed=w.rot_seed, precision=F.FPP_BF16)
    excl = {}
    for t in range(w.L):
        gpb = F.fpp_debug_point_buckets(ix_b.handle, t)
        nbad, unexplained = PT.compare_point_buckets(ix_o, t, gpb)
        assert not unexplained, (t, unexplained[:10])
        excl[t] = PT.excluded_buckets(ix_o, t, gpb)
        # buckets holding a point hashed differently may differ too
        ora = ix_o.point_buckets[t]
        diff = np.nonzero(ora != gpb.astype(np.int64))[0]
        excl[t].update(ora[diff].tolist())
        excl[t].update(gpb[diff].astype(np.int64).tolist())
        off, ids = F.fpp_debug_table(ix_b.handle, t)
        assert not PT.compare_table(ix_o, t, off, ids, excl[t]), t
    for P in (1, 4, 16):
        gp = F.fpp_debug_probes(ix_b.handle, Q, P)
        c, s, fails = PT.compare_probes(ix_o, Q, P, gp, list(range(w.L)))
        assert not fails, (P, fails[:5])
        gi, gs = ix_b.search(Q, w.k, P)
        _, _, res = O.search_batch(ix_o, Q, w.k, P)
        c, s, fails = PT.compare_search(res, gi, gs, w.k, list(range(w.L)), excl)
        assert len(fails) <= 0.01 * max(c, 1), (P, len(fails), c, fails[:3])
        assert c >= 0.8 * len(res)
        # scores are exact inner products of the returned ids
        ex = _exact_scores(X, Q, gi)
        fin = gi >= 0
        assert np.all(np.isfinite(gs) == fin)
        err = np.abs(gs[fin].astype(np.float64) - ex[fin])
        assert float(err.max(initial=0.0)) <= 1e-5 * max(1.0, float(np.abs(ex[fin]).max()))


def test_bf16_recall_matches_exact_path(F):
    X, Q = W.small_mixture(60000, 300, 96, 256, 0.3 / np.sqrt(96), 311)
    k = 10
    bi, _, _ = O.brute_force(X, Q, k)
    ix32 = F.Index(X, 20, 64, 0.1, seed=12)
    ix16 = F.Index(X, 20, 64, 0.1, seed=12, precision=F.FPP_BF16)
    for P in (1, 4, 16):
        i32, _ = ix32.search(Q, k, P)
        i16, s16 = ix16.search(Q, k, P)
        r32 = O.recall_at(i32, bi, k)
        r16 = O.recall_at(i16, bi, k)
        assert r16 >= r32 - 0.005, (P, r32, r16)
        same = np.mean([np.array_equal(a, b) for a, b in zip(i32, i16)])
        assert same >= 0.99, (P, same)


@pytest.mark.parametrize("rerank_k", [0, 5, 100, 256])
def test_bf16_rerank_lengths(F, rerank_k):
    # shortlists shorter or longer than k + 16 give the same answer here
    X, Q = W.small_mixture(20000, 100, 64, 64, 0.25, 312)
    ix = F.Index(X, 8, 32, 0.2, seed=3, precision=F.FPP_BF16, rerank_k=rerank_k)
    ref = F.Index(X, 8, 32, 0.2, seed=3)
    gi, gs = ix.search(Q, 20, 4)
    ri, rs = ref.search(Q, 20, 4)
    same = np.mean([np.array_equal(a, b) for a, b in zip(gi, ri)])
    assert same >= 0.99, same


def test_bf16_ragged_dimension(F):
    # d not a multiple of 8: the BF16 rows are zero padded
    X, Q = W.small_mixture(3000, 50, 37, 30, 0.2, 313)
    ix = F.Index(X, 3, 5, 0.37, seed=5, precision=F.FPP_BF16)
    gi, gs = ix.search(Q, 7, 11)
    ex = _exact_scores(X, Q, gi)
    fin = gi >= 0
    assert fin.any()
    assert float(np.abs(gs[fin] - ex[fin]).max()) <= 1e-5
    info = ix.info()
    assert info["precision"] == F.FPP_BF16


@pytest.mark.parametrize("rerank_k", [0, 100])
def test_fp8_rows_match_exact_path(F, rerank_k):
    # FP8 e4m3 candidate rows with per-row scales: the same candidates as the
    # exact path, results equal except where the statistical window misses
    X, Q = W.small_mixture(40000, 300, 96, 128, 0.3 / np.sqrt(96), 314)
    ix8 = F.Index(X, 16, 64, 0.1, seed=16, precision=F.FPP_FP8E4M3, rerank_k=rerank_k)
    ix32 = F.Index(X, 16, 64, 0.1, seed=16)
    assert ix8.info()["precision"] == F.FPP_FP8E4M3
    for P in (1, 4):
        i8, s8 = ix8.search(Q, 10, P)
        i32, s32 = ix32.search(Q, 10, P)
        same = np.mean([np.array_equal(a, b) for a, b in zip(i8, i32)])
        assert same >= 0.98, (P, same)
        ex = _exact_scores(X, Q, i8)
        fin = i8 >= 0
        assert float(np.abs(s8[fin] - ex[fin]).max()) <= 1e-5


@pytest.mark.parametrize("d,D,L,P,K", [(256, 256, 6, 2, 512),     # lists of 4, thread per item
                                       (128, 256, 4, 4, 256),     # lists of 8
                                       (960, 1024, 2, 4, 256)])   # stored projections
def test_one_piece_bf16_hashing_keeps_every_winner_exact(F, d, D, L, P, K):
    # hash_precision FPP_BF16: the queries are projected with one BF16
    # product; every hash's winner (the query's own bucket, the first probe)
    # is re-decided exactly when its BF16 lead is inside the window, so the
    # single-probe buckets equal the oracle's; the other probes are ranked by
    # the BF16 values (graded by recall); scores stay exact
    X, Q = W.small_mixture(20000, 300, d, K, 0.3 / np.sqrt(d), 600 + D + d)
    ix = F.Index(X, L, D, 0.3, seed=60 + d, precision=F.FPP_BF16, hash_precision=F.FPP_BF16)
    assert ix.info()["q_pieces"] == 1
    ix_o = O.build_index(X, L, D, 0.3, seed=60 + d)
    gp = F.fpp_debug_probes(ix.handle, Q, 1)
    c, s, fails = PT.compare_probes(ix_o, Q, 1, gp, list(range(L)))
    assert not fails, fails[:5]
    assert c >= 0.95 * len(Q) * L
    # every probe set contains the query's own bucket and P distinct buckets
    gpP = F.fpp_debug_probes(ix.handle, Q, P)
    for i in range(len(Q)):
        for t in range(L):
            row = gpP[i, t].astype(np.int64)
            assert len(set(row.tolist())) == P and gp[i, t] in row
    # recall against exact search stays with the exact-split BF16 path's
    ix3 = F.Index(X, L, D, 0.3, seed=60 + d, precision=F.FPP_BF16)
    ti, _ = F.fpp_bruteforce(X, Q, 10)
    got, _ = ix.search(Q, 10, P)
    ref, _ = ix3.search(Q, 10, P)
    rec = O.recall_at(got, ti, 10)
    rec3 = O.recall_at(ref, ti, 10)
    print(f"\none-piece BF16 hashing d={d} D={D} P={P}: recall@10 {rec:.4f} (exact split {rec3:.4f}), "
          f"{c} single-probe sets equal to the oracle's, {s} near-tie skipped")
    assert rec >= rec3 - 0.01
    gi, gs = ix.search(Q, 10, P)
    ex = _exact_scores(X, Q, gi)
    ok = gi >= 0
    assert np.allclose(gs[ok], ex[ok], rtol=1e-5, atol=1e-6)


def test_one_piece_bf16_hashing_is_refused_where_it_does_not_apply(F):
    X, _ = W.small_mixture(1000, 1, 32, 8, 0.3, 610)
    for kw in (dict(precision=F.FPP_FP32), dict(precision=F.FPP_BF16, simhash_bits=256)):
        with pytest.raises(F.FppError) as e:
            F.Index(X, 4, 32, 0.5, seed=1, hash_precision=F.FPP_BF16, **kw)
        assert e.value.status == F.FPP_EINVAL


def test_one_piece_bf16_hashing_with_centering_multiprobe_and_global_probes(F):
    # the one-product query projections compose with the other options: the
    # index's own hashing stays exact (centered, or iProbes = 2), every
    # single-probe set equals the oracle's, and a global budget returns
    # results with exact scores
    X, Q = W.small_mixture(12000, 120, 64, 96, 0.3 / 8, 620)
    X = (X + np.float32(0.1)).astype(np.float32)
    for kw in ({"center": True}, {"iprobes": 2, "kappa": 2}):
        ix = F.Index(X, 4, 32, 0.3, seed=61, precision=F.FPP_BF16, hash_precision=F.FPP_BF16, **kw)
        ix_o = O.build_index(X, 4, 32, 0.3, seed=61, **kw)
        gp = F.fpp_debug_probes(ix.handle, Q, 1)
        c, s, fails = PT.compare_probes(ix_o, Q, 1, gp, list(range(4)))
        assert not fails, (kw, fails[:5])
        assert c >= 0.95 * len(Q) * 4
        gi, gs, _ = F.fpp_search_ex(ix.handle, Q, k=10, global_probes=40)
        assert (gi[:, 0] >= 0).all()
        ex = _exact_scores(X, Q, gi)
        ok = gi >= 0
        assert np.allclose(gs[ok], ex[ok], rtol=1e-5, atol=1e-6)
