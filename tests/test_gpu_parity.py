"""GPU path vs the FP64 oracle, through the C ABI.

Bucket ids, kept CSR, probe sets, candidate sets and top-k ids must be equal
except where the oracle flags an FP64 near-tie (margin < 1e-6); scores agree
within 1e-5 relative.
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


def _full_parity(F, X, Q, L, D, alpha, seed, k, probes_list, min_compared=0.9, R=None,
                 ix_o=None, tag=""):
    """Every intermediate of the GPU path against the oracle: each point's
    bucket, each table's kept CSR (ids and their order), probe sets,
    candidate sets and the top-k; prints what was compared and skipped."""
    if ix_o is None:
        ix_o = O.build_index(X, L, D, alpha, seed=seed, R=R)
    ix_g = F.Index(X, L, D, alpha, seed=seed, R=R)
    excl = {}
    moved = 0
    for t in range(L):
        gpb = F.fpp_debug_point_buckets(ix_g.handle, t)
        nbad, unexplained = PT.compare_point_buckets(ix_o, t, gpb)
        assert not unexplained, f"table {t}: points {unexplained[:10]}"
        moved += nbad
        excl[t] = PT.excluded_buckets(ix_o, t, gpb)
        off, ids = F.fpp_debug_table(ix_g.handle, t)
        bad = PT.compare_table(ix_o, t, off, ids, excl[t])
        assert not bad, f"table {t}: buckets {bad[:10]}"
    print(f"\n{tag} build: {L} tables, {moved} near-tie points placed differently, "
          f"{sum(len(e) for e in excl.values())} buckets excluded")
    for P in probes_list:
        gp = F.fpp_debug_probes(ix_g.handle, Q, P)
        c, s, fails = PT.compare_probes(ix_o, Q, P, gp, list(range(L)))
        assert not fails, fails[:5]
        print(f"{tag} P={P} probes: {c} (query, table) sets compared, {s} near-tie skipped")
        gi, gs = ix_g.search(Q, k, P)
        _, _, res = O.search_batch(ix_o, Q, k, P)
        c, s, fails = PT.compare_search(res, gi, gs, k, list(range(L)), excl)
        assert not fails, fails[:3]
        print(f"{tag} P={P} top-{k}: {c} queries compared, {s} near-tie skipped")
        assert c >= min_compared * len(res), (c, s)
        gc = F.fpp_debug_candidates(ix_g.handle, Q, P)
        c, s, fails = PT.compare_candidates(res, gc, list(range(L)), excl)
        assert not fails, fails[:3]
        print(f"{tag} P={P} candidates: {c} queries compared, {s} near-tie skipped")
        assert c >= min_compared * len(res), (c, s)
    return ix_o, ix_g


def test_tiny_workload_full_parity(F):
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    _full_parity(F, X, Q, w.L, w.D, w.alpha, w.rot_seed, w.k, (1, 4, 16))


@pytest.mark.parametrize("D", [128, 256])
def test_list_epilogue_full_parity(F, D):
    # D = 128 and 256 take the projection epilogue's wide path (sign masks,
    # keys without the sign until the end); P = 1, 3, 7 give lists of 2, 4, 8
    X, Q = W.small_mixture(30000, 60, 64, 64, 0.25, 90 + D)
    _full_parity(F, X, Q, L=3, D=D, alpha=0.5, seed=7 + D, k=10, probes_list=(1, 3, 7))


def test_fp32_random_vectors_full_parity(F):
    # random vectors off the BF16 grid: six-product projections, and the exact
    # passes read the FP32 rows of R (the seeded vectors use their BF16 copy)
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    R = np.random.default_rng(17).standard_normal((w.L, 2, w.D, w.d)).astype(np.float32)
    ix_o, ix_g = _full_parity(F, X, Q, w.L, w.D, w.alpha, 0, w.k, (1, 4, 16), R=R)
    assert ix_g.info()["r_pieces"] == 3


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_scoring_by_row_range_changes_nothing(F, prec):
    # the candidates grouped by row range (forced here: 512 rows per range,
    # 20 ranges) give the same ids and scores as one range
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    p = F.FPP_BF16 if prec == "bf16" else F.FPP_FP32
    ix = F.Index(X, w.L, w.D, w.alpha, seed=w.rot_seed, precision=p)
    rng = np.random.default_rng(5)
    kq = rng.choice([1, 10, 50], size=len(Q)).astype(np.int32)
    pq = rng.choice([1, 4, 16], size=len(Q)).astype(np.int32)
    for kw in ({"k": 10, "probes": 4}, {"k_per_query": kq, "probes_per_query": pq}):
        a_i, a_s, _ = F.fpp_search_ex(ix.handle, Q, **kw)
        b_i, b_s, _ = F.fpp_search_ex(ix.handle, Q, score_range_rows=512, **kw)
        assert np.array_equal(a_i, b_i) and np.array_equal(a_s, b_s)


def test_scoring_by_row_range_large_lists(F):
    # queries with more than 16,384 entries (not de-duplicated) and with
    # 2,049..16,384 entries, grouped by row range: the same results
    for n, L, D, P in ((30000, 24, 4, 8), (12000, 6, 8, 12)):
        X, Q = W.small_mixture(n, 30, 16, 8, 0.3, 92 + D)
        ix = F.Index(X, L, D, 1.0, seed=44)
        a_i, a_s, st = F.fpp_search_ex(ix.handle, Q, k=20, probes=P)
        b_i, b_s, _ = F.fpp_search_ex(ix.handle, Q, k=20, probes=P, score_range_rows=256)
        assert np.array_equal(a_i, b_i) and np.array_equal(a_s, b_s)
        assert st["entries"] > 2048 * len(Q)


def test_queries_without_candidates_after_a_full_search(F):
    # a query whose probed buckets are all empty returns only padding, also
    # when the workspace still holds an earlier search's candidate counts
    X, Q = W.small_mixture(50, 200, 16, 4, 0.3, 93)
    ix = F.Index(X, 2, 64, 1.0, seed=3)
    ix.search(X, 5, 1)
    gi, gs = ix.search(Q, 5, 1)
    _, _, res = O.search_batch(O.build_index(X, 2, 64, 1.0, seed=3), Q, 5, 1)
    empty = [i for i, r in enumerate(res) if r.entries == 0 and not np.any(r.probe_flag)]
    assert len(empty) > 20
    for i in empty:
        assert np.all(gi[i] == -1) and not np.any(np.isfinite(gs[i])), i


def test_ragged_shapes_full_parity(F):
    # n, d, D, k, probes off every tile size; d not a multiple of 4
    X, Q = W.small_mixture(2999, 37, 30, 40, 0.2, 77)
    _full_parity(F, X, Q, L=3, D=5, alpha=0.37, seed=5, k=7, probes_list=(1, 11, 100))


def test_large_k_and_probes_parity(F):
    X, Q = W.small_mixture(20000, 25, 48, 128, 0.15, 78)
    # 24 of the 25 queries are free of FP64 near-ties (one top-100 boundary)
    _full_parity(F, X, Q, L=4, D=16, alpha=0.5, seed=6, k=100, probes_list=(128,),
                 tag="k=100 P=128")


def test_unfiltered_all_buckets_equals_bruteforce(F):
    # alpha = 1 and every one of the 4D^2 buckets probed: exact search
    X, Q = W.small_mixture(5000, 40, 24, 16, 0.2, 79)
    ix = F.Index(X, 3, 3, 1.0, seed=9)
    gi, gs = ix.search(Q, 10, 36)
    bi, bs, bf = O.brute_force(X, Q, 10)
    for i in range(len(Q)):
        if not bf[i]:
            assert np.array_equal(gi[i], bi[i])
        assert np.allclose(gs[i], bs[i], rtol=1e-5, atol=1e-6)


def test_gpu_bruteforce_matches_oracle(F):
    X, Q = W.small_mixture(30000, 50, 64, 64, 0.25, 80)
    gi, gs = F.fpp_bruteforce(X, Q, 20)
    bi, bs, bf = O.brute_force(X, Q, 20)
    for i in range(len(Q)):
        if not bf[i]:
            assert np.array_equal(gi[i], bi[i])
        assert np.allclose(gs[i], bs[i], rtol=1e-5, atol=1e-6)


def test_short_results_are_padded(F):
    X, Q = W.small_mixture(40, 3, 16, 4, 0.2, 81)
    ix = F.Index(X, 1, 2, 0.2, seed=1)
    gi, gs = ix.search(Q, 50, 1)
    ix_o = O.build_index(X, 1, 2, 0.2, seed=1)
    _, _, res = O.search_batch(ix_o, Q, 50, 1)
    for i, r in enumerate(res):
        assert np.array_equal(gi[i], r.ids)
        assert np.array_equal(np.isneginf(gs[i]), np.isneginf(r.scores))


def test_per_query_k_and_probes(F):
    X, Q = W.small_mixture(20000, 60, 32, 128, 0.2, 82)
    rng = np.random.default_rng(3)
    kq = rng.choice([1, 10, 100], size=len(Q)).astype(np.int32)
    pq = rng.choice([2, 8, 32, 128], size=len(Q)).astype(np.int32)
    L, D = 5, 12
    ix_o = O.build_index(X, L, D, 0.3, seed=4)
    ix = F.Index(X, L, D, 0.3, seed=4)
    gi, gs, st = ix.search(Q, 10, 1, k_per_query=kq, probes_per_query=pq)
    assert gi.shape == (len(Q), 100)
    _, _, res = O.search_batch(ix_o, Q, kq, pq)
    excl = {t: PT.excluded_buckets(ix_o, t) for t in range(L)}
    c, s, fails = PT.compare_search(res, gi, gs, 100, list(range(L)), excl)
    assert not fails, fails[:3]
    for i in range(len(Q)):       # past a query's own k: padding
        assert (gi[i, kq[i]:] == -1).all()
    assert st["queries"] == len(Q)
    assert st["entries"] == sum(r.entries for r in res)
    assert st["unique"] == sum(r.cand.size for r in res)


def test_table_range(F):
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    ix_o = O.build_index(X, w.L, w.D, w.alpha, seed=w.rot_seed)
    ix = F.Index(X, w.L, w.D, w.alpha, seed=w.rot_seed)
    tabs = [3, 4, 5, 6]
    gi, gs, _ = ix.search(Q, 10, 4, table_begin=3, table_end=7)
    _, _, res = O.search_batch(ix_o, Q, 10, 4, tables=tabs)
    excl = {t: PT.excluded_buckets(ix_o, t) for t in range(w.L)}
    c, s, fails = PT.compare_search(res, gi, gs, 10, tabs, excl)
    assert not fails and c > 80


def test_device_pointers_and_stream(F):
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    ix = F.Index(torch.from_numpy(X).cuda(), w.L, w.D, w.alpha, seed=w.rot_seed)
    hi, hs = ix.search(Q, 10, 4)
    Qd = torch.from_numpy(Q).cuda()
    s = torch.cuda.Stream()
    gi, gs, _ = ix.search(Qd, 10, 4, stream=s, want_stats=False)
    s.synchronize()
    assert gi.is_cuda
    assert np.array_equal(gi.cpu().numpy(), hi)
    assert np.array_equal(gs.cpu().numpy(), hs)


@pytest.mark.parametrize("d", [64, 37])
def test_pinned_host_queries_upload_ahead(F, d):
    # page-locked host queries on a stream: each call's upload runs ahead on
    # the index's copy stream into one of two query tiles.  Back-to-back
    # calls with different queries, one device-query call among them, give
    # the synchronous results (d = 37: padded tiles, zeroed on first use)
    X, Q = W.small_mixture(4000, 300, d, 32, 0.25, 330 + d)
    ix = F.Index(X, 6, 16, 0.3, seed=22)
    rng = np.random.default_rng(23)
    batches = [Q[rng.permutation(len(Q))[: 200 + 20 * j]] for j in range(6)]
    ref = [ix.search(b, 10, 4) for b in batches]
    s = torch.cuda.Stream()
    keep, outs = [], []
    for j, b in enumerate(batches):
        if j == 3:
            Qd = torch.from_numpy(b).cuda()
            gi, gs, _ = F.fpp_search_ex(ix.handle, Qd, k=10, probes=4, stream=s,
                                        want_stats=False)
            keep.append(Qd)
            outs.append((gi, gs))
            continue
        qh = torch.from_numpy(b).pin_memory()
        ih = torch.empty((len(b), 10), dtype=torch.int64).pin_memory()
        sh = torch.empty((len(b), 10), dtype=torch.float32).pin_memory()
        F.fpp_search_ex(ix.handle, qh, k=10, probes=4, stream=s, ids=ih, scores=sh,
                        want_stats=False)
        keep.append(qh)
        outs.append((ih, sh))
    s.synchronize()
    for (gi, gs), (ri, rs) in zip(outs, ref):
        assert np.array_equal(gi.cpu().numpy(), ri)
        assert np.array_equal(gs.cpu().numpy(), rs)


def test_empty_query_batch(F):
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    ix = F.Index(X[:500], 2, 8, 0.5, seed=1)
    gi, gs = ix.search(Q[:0], 10, 4)
    assert gi.shape == (0, 10)


def test_repeat_search_is_deterministic(F):
    w = W.WORKLOADS["tiny"]
    X, Q = W.dataset(w)
    ix = F.Index(X, w.L, w.D, w.alpha, seed=w.rot_seed)
    a = ix.search(Q, 10, 16)
    b = ix.search(Q, 10, 16)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_plain1m_full_size_all_tables(F):
    """The 1M x 128 workload that the benchmark times, at full size, against
    the oracle built over all 100 tables (a process per host core): every
    point's bucket and every kept CSR in every table, probe sets, candidate
    sets and the top-10 of 300 queries at P = 1 and P = 16 over all tables."""
    from oracle.parallel import build_index_parallel
    w = W.WORKLOADS["plain1m"]
    X, Q = W.dataset(w, m=300)
    ix_o = build_index_parallel(X, w.L, w.D, w.alpha, seed=w.rot_seed)
    ix = F.Index(X, w.L, w.D, w.alpha, seed=w.rot_seed)
    excl, gpbs = {}, {}
    moved = 0
    for t in range(w.L):
        gpb = F.fpp_debug_point_buckets(ix.handle, t)
        nbad, unexplained = PT.compare_point_buckets(ix_o, t, gpb)
        assert not unexplained, (t, unexplained[:5])
        moved += nbad
        excl[t] = PT.excluded_buckets(ix_o, t, gpb)
        fl = np.nonzero(ix_o.hash_flag[t])[0]
        gpbs[t] = np.full(w.n, -1, dtype=np.int64)
        gpbs[t][fl] = gpb[fl]
        off, ids = F.fpp_debug_table(ix.handle, t)
        bad = PT.compare_table(ix_o, t, off, ids, excl[t])
        assert not bad, (t, bad[:5])
    print(f"\nplain1m build: 100 tables x 1M points, {moved} near-tie points placed "
          f"differently, {sum(len(e) for e in excl.values())} buckets excluded")
    tabs = list(range(w.L))
    for P in (1, 16):
        gp = F.fpp_debug_probes(ix.handle, Q, P)
        c, s, fails = PT.compare_probes(ix_o, Q, P, gp, tabs)
        assert not fails, fails[:5]
        print(f"plain1m P={P} probes: {c} (query, table) sets compared, {s} near-tie skipped")
        gi, gs = ix.search(Q, w.k, P)
        _, _, res = O.search_batch(ix_o, Q, w.k, P)
        # a query probing a bucket that holds a near-tie point is compared
        # when no resolution of that point can change its top-10
        c, s, fails = PT.compare_search(
            res, gi, gs, w.k, tabs, excl, Q=Q, ix=ix_o,
            ambiguous=lambda t, b: PT.ambiguous_ids(ix_o, t, b, gpbs[t]))
        assert not fails, fails[:3]
        print(f"plain1m P={P} top-10: {c} queries compared, {s} near-tie skipped")
        assert c >= 0.9 * len(Q), (c, s)
        gc = F.fpp_debug_candidates(ix.handle, Q, P)
        c, s, fails = PT.compare_candidates(
            res, gc, tabs, excl, ambiguous=lambda t, b: PT.ambiguous_ids(ix_o, t, b, gpbs[t]))
        assert not fails, fails[:3]
        print(f"plain1m P={P} candidates: {c} queries compared, {s} near-tie skipped")
        assert c >= 0.9 * len(Q), (c, s)


@pytest.mark.parametrize("d,D,K,sigma,L,probes", [
    (960, 1024, 256, 0.35 / np.sqrt(960), 2, (1, 4, 16)),   # the precision workload's shape
    (128, 512, 512, 0.25 / np.sqrt(128), 3, (1, 4, 16, 64)),
])
def test_stored_projection_shapes_full_parity(F, d, D, K, sigma, L, probes):
    # D > 256: the projections are stored and the pair-window, full and
    # global passes run over 2D-entry rows; every step against the oracle
    X, Q = W.small_mixture(30000, 60, d, K, sigma, 400 + D)
    _full_parity(F, X, Q, L=L, D=D, alpha=0.1, seed=31 + D, k=10, probes_list=probes,
                 tag=f"d={d} D={D}")


def test_table_slices_merged_equal_full_search(F):
    # the table-sharded plan on one GPU: every slice searched through
    # fpp_search_ex's table range, merged by fpp_merge_topk
    from paper_2206_01382_gb300 import sharded
    X, Q = W.small_mixture(20000, 200, 48, 64, 0.25, 90)
    ix = F.Index(X, 10, 16, 0.3, seed=21)
    for P in (1, 3):
        fi, fs = ix.search(Q, 10, P)
        parts_i, parts_s = [], []
        for r in range(3):
            tb, te = sharded.table_range(r, 3, 10)
            gi, gs, _ = F.fpp_search_ex(ix.handle, Q, k=10, probes=P, table_begin=tb,
                                        table_end=te, want_stats=False)
            parts_i.append(gi)
            parts_s.append(gs)
        mi, ms = F.fpp_merge_topk(np.stack(parts_i), np.stack(parts_s))
        assert np.array_equal(mi, fi)
        assert np.array_equal(ms, fs)


def _oracle_point_probes(ix_o, t, ip):
    """Each point's ip best buckets in table t (Algorithm 1) and a near-tie
    flag per point (hash ties or the ip-th / (ip+1)-th pair boundary)."""
    p1 = ix_o.X @ ix_o.R[t, 0].T
    p2 = ix_o.X @ ix_o.R[t, 1].T
    from oracle import falconn as OF
    b, _, margin = OF._top_pairs(OF._signed_lists(p1), OF._signed_lists(p2), ip)
    _, _, f1 = O.cross_polytope_hash(p1)
    _, _, f2 = O.cross_polytope_hash(p2)
    return b, (margin < O.NEAR_TIE) | f1 | f2


@pytest.mark.parametrize("ip,kappa,D", [(3, 0, 8), (2, 3, 16), (5, 2, 4)])
def test_multiprobe_indexing_and_limit_scaling_parity(F, ip, kappa, D):
    # Algorithm 1 with iProbes > 1 and the limit-scaling floor kappa
    X, Q = W.small_mixture(6000, 80, 32, 48, 0.25, 91 + ip)
    L, alpha = 4, 0.3
    ix_o = O.build_index(X, L, D, alpha, seed=33, iprobes=ip, kappa=kappa)
    ix_g = F.Index(X, L, D, alpha, seed=33, iprobes=ip, kappa=kappa)
    excl = {}
    for t in range(L):
        ob, flag = _oracle_point_probes(ix_o, t, ip)
        gb = F.fpp_debug_point_buckets(ix_g.handle, t).astype(np.int64)
        bad = np.nonzero(np.any(ob != gb, axis=1) & ~flag)[0]
        assert bad.size == 0, (t, bad[:5], ob[bad[:2]], gb[bad[:2]])
        ex = set(np.nonzero(ix_o.filter_flag[t])[0].tolist())
        fl = np.nonzero(flag)[0]
        ex.update(ob[fl].reshape(-1).tolist())
        ex.update(gb[fl].reshape(-1).tolist())
        excl[t] = ex
        off, ids = F.fpp_debug_table(ix_g.handle, t)
        assert not PT.compare_table(ix_o, t, off, ids, ex), t
    for P in (1, 4):
        gi, gs = ix_g.search(Q, 10, P)
        _, _, res = O.search_batch(ix_o, Q, 10, P)
        c, s, fails = PT.compare_search(res, gi, gs, 10, list(range(L)), excl)
        assert not fails, fails[:3]
        assert c >= 0.7 * len(res), (c, s)


@pytest.mark.parametrize("n,L,D,P", [(30000, 24, 4, 8), (12000, 6, 8, 12)])
def test_large_candidate_lists_parity(F, n, L, D, P):
    # queries with more than 16,384 bucket entries (first case: ~90,000 per
    # query, most of them repeats) skip de-duplication; the mid-size table
    # takes 2,049..16,384 entries (second case); results are unchanged
    X, Q = W.small_mixture(n, 30, 16, 8, 0.3, 92 + D)
    ix_o = O.build_index(X, L, D, 1.0, seed=44)
    ix_g = F.Index(X, L, D, 1.0, seed=44)
    excl = {t: PT.excluded_buckets(ix_o, t, F.fpp_debug_point_buckets(ix_g.handle, t))
            for t in range(L)}
    gi, gs = ix_g.search(Q, 20, P)
    _, _, res = O.search_batch(ix_o, Q, 20, P)
    c, s, fails = PT.compare_search(res, gi, gs, 20, list(range(L)), excl)
    assert not fails, fails[:3]
    assert c >= 0.5 * len(res), (c, s)   # D = 4 leaves many probe-boundary near-ties
    for i in range(len(Q)):   # no id twice in a result
        row = gi[i][gi[i] >= 0]
        assert len(set(row.tolist())) == len(row)
    _, _, st = F.fpp_search_ex(ix_g.handle, Q, k=20, probes=P)
    assert st["entries"] > 2048 * len(Q)


def test_graph_replay_equals_plain_calls(F):
    # FPP_SEARCH_GRAPH: captured once, replayed with new query data in the
    # same buffers, re-captured when an argument changes
    X, Q = W.small_mixture(30000, 700, 64, 64, 0.25, 93)
    ix = F.Index(X, 8, 32, 0.2, seed=4)
    st = torch.cuda.Stream()
    Qd = torch.empty((300, 64), dtype=torch.float32, device="cuda")
    ids = torch.empty((300, 10), dtype=torch.int64, device="cuda")
    sc = torch.empty((300, 10), dtype=torch.float32, device="cuda")
    n0 = F.fpp_launch_count()
    for r, (lo, P) in enumerate(((0, 2), (300, 2), (100, 4), (400, 4))):
        Qd.copy_(torch.from_numpy(Q[lo:lo + 300]))
        torch.cuda.synchronize()
        F.fpp_search_ex(ix.handle, Qd, k=10, probes=P, stream=st, ids=ids, scores=sc,
                        want_stats=False, graph=True)
        st.synchronize()
        gi, gs = ix.search(Q[lo:lo + 300], 10, P)
        assert np.array_equal(ids.cpu().numpy(), gi)
        assert np.array_equal(sc.cpu().numpy(), gs)
    assert F.fpp_launch_count() - n0 > 4 * 8   # graph kernels are counted at each replay


def test_optimistic_graph_checks_regions_and_falls_back(F):
    # a worst-case bound past the candidate budget makes the graph
    # optimistic: every candidate region is checked against the buffer on the
    # device; a call whose entries fit runs as the graph, one whose entries do
    # not is repeated without it (and its buffers grow), so a second such
    # call fits
    X, Q = W.small_mixture(30000, 700, 64, 64, 0.25, 95)
    ref = F.Index(X, 8, 32, 0.2, seed=5)
    m = 300
    _, _, s1 = F.fpp_search_ex(ref.handle, Q[:m], k=10, probes=1)
    _, _, s8 = F.fpp_search_ex(ref.handle, Q[:m], k=10, probes=8)
    e1, e8 = int(s1["entries"]), int(s8["entries"])
    assert e8 > 2 * e1
    budget = (e1 + e8) // 2   # candidate slots: P = 1 fits, P = 8 does not
    ix = F.Index(X, 8, 32, 0.2, seed=5)
    assert m * 8 * 1 * ix.info()["max_bucket_kept"] > budget   # optimistic even at P = 1
    F.fpp_set_candidate_budget(ix.handle, budget * 8)
    st = torch.cuda.Stream()
    Qd = torch.from_numpy(Q[:m]).cuda()
    ids = torch.empty((m, 10), dtype=torch.int64, device="cuda")
    sc = torch.empty((m, 10), dtype=torch.float32, device="cuda")
    for P, fallbacks in ((1, 0), (8, 1), (8, 1), (1, 1)):
        ids.fill_(-7)
        torch.cuda.synchronize()
        F.fpp_search_ex(ix.handle, Qd, k=10, probes=P, stream=st, ids=ids, scores=sc,
                        want_stats=False, graph=True)
        st.synchronize()
        gi, gs = ref.search(Q[:m], 10, P)
        assert np.array_equal(ids.cpu().numpy(), gi), P
        assert np.array_equal(sc.cpu().numpy(), gs), P
        assert ix.info()["graph_fallbacks"] == fallbacks, (P, fallbacks)
    with pytest.raises(F.FppError):
        F.fpp_set_candidate_budget(ix.handle, 1024)


def test_autotune_keeps_results(F):
    X, Q = W.small_mixture(40000, 500, 96, 64, 0.25, 94)
    for prec in (F.FPP_FP32, F.FPP_BF16):
        ix = F.Index(X, 8, 64, 0.2, seed=8, precision=prec)
        gi, gs = ix.search(Q, 10, 2)
        rep = F.fpp_autotune(ix.handle, Q, 10, 2)
        assert rep["shapes_tried"] >= 4
        assert 0 < rep["ms_best"] <= rep["ms_default"] * 1.0001
        ti, ts = ix.search(Q, 10, 2)
        assert np.array_equal(gi, ti) and np.array_equal(gs, ts)


@pytest.mark.parametrize("given_c", [False, True])
def test_centering_parity(F, given_c):
    # Section 3.4, heuristic (1): tables over x - c, queries and scores as usual
    X, Q = W.small_mixture(8000, 100, 32, 64, 0.25, 95)
    X = (X + np.float32(0.15)).astype(np.float32)
    c, _ = O.center_points(X)
    ix_o = O.build_index(X, 6, 16, 0.3, seed=12, center=True)
    ix_g = F.Index(X, 6, 16, 0.3, seed=12, center=True, center_vec=c if given_c else None)
    assert ix_g.info()["center"] == 1
    excl = {}
    for t in range(6):
        gpb = F.fpp_debug_point_buckets(ix_g.handle, t)
        nbad, unexplained = PT.compare_point_buckets(ix_o, t, gpb)
        assert not unexplained, (t, unexplained[:5])
        excl[t] = PT.excluded_buckets(ix_o, t, gpb)
        off, ids = F.fpp_debug_table(ix_g.handle, t)
        assert not PT.compare_table(ix_o, t, off, ids, excl[t]), t
    for P in (1, 4):
        gi, gs = ix_g.search(Q, 10, P)
        _, _, res = O.search_batch(ix_o, Q, 10, P)
        c_, s_, fails = PT.compare_search(res, gi, gs, 10, list(range(6)), excl)
        assert not fails, fails[:3]
        assert c_ >= 0.8 * len(res)


@pytest.mark.parametrize("Qp,L,D", [(1, 8, 16), (12, 6, 16), (40, 10, 8), (200, 10, 64),
                                    (600, 24, 32)])
def test_global_probes_parity(F, Qp, L, D):
    # qProbes over all tables together (Sections 2.2 and 4), list mode
    # (small per-table cap; Qp = 1 caps every table at one probe) and stored
    # projections (large)
    X, Q = W.small_mixture(6000, 60, 32, 64, 0.25, 96 + Qp)
    ix_o = O.build_index(X, L, D, 0.3, seed=14)
    ix_g = F.Index(X, L, D, 0.3, seed=14)
    excl = {t: PT.excluded_buckets(ix_o, t, F.fpp_debug_point_buckets(ix_g.handle, t))
            for t in range(L)}
    gi, gs, _ = F.fpp_search_ex(ix_g.handle, Q, k=10, global_probes=Qp, want_stats=False)
    _, _, res = O.search_batch(ix_o, Q, 10, 1, global_probes=Qp)
    c, s, fails = PT.compare_search(res, gi, gs, 10, list(range(L)), excl)
    assert not fails, fails[:3]
    assert c >= 0.7 * len(res), (c, s)


@pytest.mark.parametrize("bits,keep", [(256, 40), (512, 7)])
def test_simhash_preranking_parity(F, bits, keep):
    # Section 4: candidates pre-ranked by SimHash signatures of the index's
    # random vectors; the keep closest (Hamming) are scored exactly
    X, Q = W.small_mixture(8000, 60, 48, 64, 0.25, 97 + keep)
    L, D = 8, 32
    ix_o = O.build_index(X, L, D, 0.3, seed=15)
    ix_g = F.Index(X, L, D, 0.3, seed=15, simhash_bits=bits)
    assert ix_g.info()["simhash_bits"] == bits
    sig = O.simhash_signatures(ix_o, X, bits)
    excl = {t: PT.excluded_buckets(ix_o, t, F.fpp_debug_point_buckets(ix_g.handle, t))
            for t in range(L)}
    for P in (2, 6):
        gi, gs, _ = F.fpp_search_ex(ix_g.handle, Q, k=10, probes=P, simhash_keep=keep)
        _, _, res = O.search_batch(ix_o, Q, 10, P, simhash=(sig, bits, keep))
        c, s, fails = PT.compare_search(res, gi, gs, 10, list(range(L)), excl)
        assert not fails, fails[:3]
        assert c >= 0.7 * len(res), (c, s)


def test_global_probes_past_the_per_table_cap_are_refused(F):
    # D = 8: 256 buckets per table, so a budget of 300 over two tables takes
    # more than 128 from one of them; the library offers at most 128 per
    # table and must refuse rather than return a capped selection
    X, Q = W.small_mixture(3000, 20, 16, 16, 0.25, 98)
    ix_g = F.Index(X, 2, 8, 0.5, seed=16)
    with pytest.raises(F.FppError) as e:
        F.fpp_search_ex(ix_g.handle, Q, k=10, global_probes=300, want_stats=False)
    assert e.value.status == F.FPP_EINVAL and "128" in str(e.value)
    # the oracle's uncapped selection does take more than 128 from a table
    ix_o = O.build_index(X, 2, 8, 0.5, seed=16)
    per, _ = O.probe_global(ix_o, Q[0], 300)
    assert max(len(b) for b in per) > 128


def test_pipelined_calls_equal_plain_calls(F):
    # FPP_SEARCH_PIPELINE: consecutive calls alternate two workspaces on two
    # internal streams; after a flush every call's results equal the plain
    # call's, with device or page-locked host buffers, a change of budget
    # between calls and a plain call among them
    X, Q = W.small_mixture(30000, 2400, 64, 64, 0.25, 97)
    ix = F.Index(X, 8, 32, 0.2, seed=5)
    parts = [(i * 400, (i + 1) * 400, 1 + (i % 3)) for i in range(6)]
    ref = [ix.search(Q[lo:hi], 10, P) for lo, hi, P in parts]
    st = torch.cuda.Stream()
    Qd = torch.from_numpy(Q).cuda()
    Qh = torch.from_numpy(Q).pin_memory()
    outs = []
    for j, (lo, hi, P) in enumerate(parts):
        if j == 3:   # a plain call among the pipelined ones
            gi, gs = ix.search(Q[lo:hi], 10, P)
            outs.append((gi, gs))
            continue
        if j % 2:
            ids = torch.empty((hi - lo, 10), dtype=torch.int64).pin_memory()
            sc = torch.empty((hi - lo, 10), dtype=torch.float32).pin_memory()
            q = Qh[lo:hi]
        else:
            ids = torch.empty((hi - lo, 10), dtype=torch.int64, device="cuda")
            sc = torch.empty((hi - lo, 10), dtype=torch.float32, device="cuda")
            q = Qd[lo:hi]
        F.fpp_search_ex(ix.handle, q, k=10, probes=P, stream=st, ids=ids, scores=sc,
                        want_stats=False, pipeline=True)
        outs.append((ids, sc))
    F.fpp_search_flush(ix.handle, st)
    st.synchronize()
    for (gi, gs), (ri, rs) in zip(outs, ref):
        gi = gi.cpu().numpy() if hasattr(gi, "cpu") else gi
        gs = gs.cpu().numpy() if hasattr(gs, "cpu") else gs
        assert np.array_equal(gi, ri) and np.array_equal(gs, rs)
