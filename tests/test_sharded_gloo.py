"""Table-sharded search across two processes (gloo, CPU): each rank takes
its slice of the tables, the ranks' top-k lists are all-gathered and merged
by the library's fpp_merge_topk, and the result equals the search over all
tables.  The per-slice results come from the oracle (the same search the GPU
ranks run with fpp_search_ex's table range), so this needs no GPU."""
import os
import socket

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, P):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2206_01382_gb300 import sharded

        w = W.WORKLOADS["tiny"]
        X, Q = W.dataset(w, m=40)
        ix = O.build_index(X, w.L, w.D, w.alpha, seed=w.rot_seed)
        tb, te = sharded.table_range(rank, world, w.L)
        ids, sc, _ = O.search_batch(ix, Q, w.k, P, tables=list(range(tb, te)))
        mi, ms = sharded.gather_merge(ids, sc.astype(np.float32))
        fi, fs, res = O.search_batch(ix, Q, w.k, P)
        compared = 0
        for i, r in enumerate(res):
            if r.topk_flag:
                continue
            compared += 1
            assert np.array_equal(mi[i], fi[i]), (rank, i, mi[i], fi[i])
            fin = np.isfinite(fs[i])
            assert np.allclose(ms[i][fin], fs[i][fin], rtol=1e-6)
        assert compared >= 35
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("P", [1, 4])
def test_table_sharded_merge_equals_full_search(P):
    import torch.multiprocessing as mp
    from paper_2206_01382_gb300 import _build

    _build.build()
    mp.spawn(_worker, args=(2, _free_port(), P), nprocs=2, join=True)


def test_table_range_partitions_the_tables():
    from paper_2206_01382_gb300 import sharded

    for L in (2, 3, 10, 100, 101):
        for world in (1, 2, 3, 8):
            if world > L:
                continue
            spans = [sharded.table_range(r, world, L) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == L
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1


def test_merge_topk_dedups_orders_and_pads():
    import paper_2206_01382_gb300 as F
    from paper_2206_01382_gb300 import _build

    _build.build()
    ids = np.array([[[5, 3, -1]], [[3, 9, 2]]], dtype=np.int64)
    sc = np.array([[[0.9, 0.5, -np.inf]], [[0.5, 0.5, 0.1]]], dtype=np.float32)
    oi, osc = F.fpp_merge_topk(ids, sc)
    assert oi.tolist() == [[5, 3, 9]]
    assert osc[0].tolist() == pytest.approx([0.9, 0.5, 0.5])
    oi, osc = F.fpp_merge_topk(np.full((2, 1, 3), -1, np.int64), np.full((2, 1, 3), -np.inf, np.float32))
    assert oi.tolist() == [[-1, -1, -1]] and np.all(np.isneginf(osc))
