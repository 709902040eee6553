"""Serving (fpp_server_*): continuous batching gives every request exactly
the result fpp_search_ex gives its queries alone, whatever the batch mix,
the number of slots or the candidate budget."""
import numpy as np
import pytest

import workloads as W

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


@pytest.fixture(scope="module")
def data(F):
    X, Q = W.small_mixture(30000, 600, 64, 128, 0.25, 401)
    ix = F.Index(X, 8, 32, 0.2, seed=17)
    return X, Q, ix


def _requests(nq_total, seed):
    rng = np.random.default_rng(seed)
    reqs, q0 = [], 0
    while q0 < nq_total:
        nq = int(min(rng.integers(1, 40), nq_total - q0))
        reqs.append((q0, nq, int(rng.choice([1, 5, 10, 20])), int(rng.choice([1, 2, 4, 8]))))
        q0 += nq
    return reqs


def _alone(F, ix, Q, reqs):
    out = []
    for q0, nq, k, p in reqs:
        gi, gs, _ = F.fpp_search_ex(ix.handle, Q[q0:q0 + nq], k=k, probes=p, want_stats=False)
        out.append((gi, gs))
    return out


@pytest.mark.parametrize("cfg", [dict(slots=1, max_batch=64), dict(slots=3, max_batch=128),
                                 dict(slots=2, max_batch=4096, candidate_budget_bytes=1 << 20)])
def test_server_results_equal_requests_alone(F, data, cfg):
    X, Q, ix = data
    reqs = _requests(len(Q), 402)
    ref = _alone(F, ix, Q, reqs)
    srv = F.Server(ix, k_max=20, probes_max=8, **cfg)
    rids = [srv.submit(Q[q0:q0 + nq], k, p) for q0, nq, k, p in reqs]
    for rid, (gi, gs) in zip(rids, ref):
        ids, sc, lat = srv.poll(rid)
        assert np.array_equal(ids, gi)
        assert np.array_equal(sc, gs)
        assert lat >= 0.0
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["queries"] == len(Q)
    assert 1 <= st["batches"] <= len(reqs)
    srv.close()


def test_server_same_query_alone_and_in_a_mix(F, data):
    X, Q, ix = data
    srv = F.Server(ix, k_max=20, probes_max=8, slots=2, max_batch=256)
    alone = srv.poll(srv.submit(Q[7:8], 10, 4))
    rng = np.random.default_rng(403)
    rids = []
    for i in range(30):
        lo = int(rng.integers(0, len(Q) - 50))
        rids.append(srv.submit(Q[lo:lo + 50], int(rng.choice([5, 20])), int(rng.choice([1, 8]))))
    mixed = srv.submit(Q[7:8], 10, 4)
    rids.append(srv.submit(Q[100:180], 20, 2))
    got = srv.poll(mixed)
    for r in rids:
        srv.poll(r)
    assert np.array_equal(got[0], alone[0]) and np.array_equal(got[1], alone[1])
    srv.close()


def test_server_rejects_bad_requests_and_times_out_polls(F, data):
    X, Q, ix = data
    srv = F.Server(ix, k_max=10, probes_max=4, max_batch=32)
    for args in ((Q[:33], 5, 1), (Q[:4], 11, 1), (Q[:4], 5, 5), (Q[:4], 0, 1)):
        with pytest.raises(F.FppError) as e:
            srv.submit(*args)
        assert e.value.status == F.FPP_EINVAL
    with pytest.raises(F.FppError):
        srv._shape[12345] = (1, 1)
        srv.poll(12345)
    rid = srv.submit(Q[:32], 10, 4)
    res = srv.poll(rid, timeout_us=0)      # may or may not be complete yet
    while res is None:
        res = srv.poll(rid, timeout_us=1000)
    assert res[0].shape == (32, 10)
    srv.close()
    srv.close()   # idempotent


def test_server_device_queries_and_destroy_with_pending(F, data):
    X, Q, ix = data
    srv = F.Server(ix, k_max=10, probes_max=4, slots=1, max_batch=16)
    Qd = torch.from_numpy(Q[:16]).cuda()
    r = srv.poll(srv.submit(Qd, 10, 2))
    gi, gs, _ = F.fpp_search_ex(ix.handle, Q[:16], k=10, probes=2, want_stats=False)
    assert np.array_equal(r[0], gi)
    for i in range(20):
        srv.submit(Q[i * 16:(i + 1) * 16], 10, 4)
    srv.close()   # drops what is still queued, joins the worker


def test_server_splits_batches_that_do_not_fit_and_allocates_nothing(F, data):
    # a 1 MiB candidate buffer per slot holds 131,072 entries; one request of
    # 600 queries at 8 probes per table scans more, so the slot must halve the
    # batch (the first request is always admitted whole) instead of growing
    # its buffers: no device allocation while serving, the same results
    X, Q, _ = data
    ix = F.Index(X, 16, 16, 0.5, seed=19)   # about 1,000 entries per query at 8 probes
    gi, gs, st = F.fpp_search_ex(ix.handle, Q, k=10, probes=8)
    assert st["entries"] > 2 * ((1 << 20) // 8), st["entries"]
    srv = F.Server(ix, k_max=10, probes_max=8, slots=1, max_batch=4096,
                   candidate_budget_bytes=1 << 20)
    a0 = F.fpp_alloc_count()
    ids, sc, _ = srv.poll(srv.submit(Q, 10, 8))
    reqs = _requests(len(Q), 404)
    rids = [srv.submit(Q[q0:q0 + nq], 10, 8) for q0, nq, _, _ in reqs]
    outs = [srv.poll(r) for r in rids]
    assert F.fpp_alloc_count() == a0
    s = srv.stats()
    srv.close()
    assert s["serving_allocs"] == 0 and s["failed"] == 0
    assert s["splits"] >= 1, s
    assert np.array_equal(ids, gi) and np.array_equal(sc, gs)
    for (q0, nq, _, _), o in zip(reqs, outs):
        assert np.array_equal(o[0], gi[q0:q0 + nq]) and np.array_equal(o[1], gs[q0:q0 + nq])
    print(f"\nserver: {s['batches']} batches, {s['splits']} halvings, 0 allocations")


def test_server_refuses_a_buffer_below_one_querys_worst_case(F, data):
    X, Q, _ = data
    ix = F.Index(X, 16, 2, 1.0, seed=3)     # 16 buckets per table: very large buckets
    worst = 16 * 8 * ix.info()["max_bucket_kept"] * 8
    assert worst > 1 << 20
    with pytest.raises(F.FppError) as e:
        F.Server(ix, k_max=10, probes_max=8, candidate_budget_bytes=1 << 20)
    assert e.value.status == F.FPP_EINVAL and "worst case" in str(e.value)
    srv = F.Server(ix, k_max=10, probes_max=8, candidate_budget_bytes=worst)
    gi, gs, _ = F.fpp_search_ex(ix.handle, Q[:50], k=10, probes=8, want_stats=False)
    ids, sc, _ = srv.poll(srv.submit(Q[:50], 10, 8))
    srv.close()
    assert np.array_equal(ids, gi) and np.array_equal(sc, gs)


def test_server_bulk_submit_equals_single_submits(F, data):
    X, Q, ix = data
    reqs = _requests(300, 405)
    ref = _alone(F, ix, Q, reqs)
    srv = F.Server(ix, k_max=20, probes_max=8, slots=2, max_batch=512)
    rows = np.concatenate([Q[q0:q0 + nq] for q0, nq, _, _ in reqs])
    rids = []
    for p in sorted({r[3] for r in reqs}):   # one probe budget per call
        sel = [i for i, r in enumerate(reqs) if r[3] == p]
        part = np.concatenate([Q[reqs[i][0]:reqs[i][0] + reqs[i][1]] for i in sel])
        got = srv.submit_many(part, [reqs[i][1] for i in sel], [reqs[i][2] for i in sel], p)
        rids += list(zip(sel, got))
    for i, rid in rids:
        ids, sc, _ = srv.poll(rid)
        assert np.array_equal(ids, ref[i][0]) and np.array_equal(sc, ref[i][1])
    with pytest.raises(F.FppError):   # a bad request stops the call there
        srv.submit_many(rows[:10], [5, 0, 5], [5, 5, 5], 2)
    srv.close()


def test_server_refuses_requests_past_its_queue_limit(F, data):
    # admission: with max_queue = 3, a group of 8 requests queued in one call
    # (the queue lock is held while it is filled, so no slot drains it in
    # between) keeps the first 3 and refuses the rest with FPP_EBUSY; the
    # admitted ones complete normally
    X, Q, ix = data
    srv = F.Server(ix, k_max=10, probes_max=4, slots=1, max_batch=64, max_queue=3)
    with pytest.raises(F.FppError) as e:
        srv.submit_many(Q[:40], [5] * 8, [10] * 8, 2)
    assert e.value.status == F.FPP_EBUSY and "queue full" in str(e.value)
    st = srv.stats()
    assert st["submitted"] == 3
    gi, gs, _ = F.fpp_search_ex(ix.handle, Q[:15], k=10, probes=2, want_stats=False)
    srv.close()
    assert gi.shape == (15, 10)
