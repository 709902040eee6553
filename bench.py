#!/usr/bin/env python
"""Throughput benchmark of the GB300 Falconn++ search path.

One step = one batched search of the workload's whole query set through the
hot path (projection GEMM, probe ranking, gather + hash-set dedup + exact
scoring + top-k), with the index and the queries resident in HBM.  The probe
budget is the smallest of the workload's sweep whose recall@10 against exact
search reaches 0.90 (measured once, before timing, on a query sample with the
library's own brute-force search).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.

Multi-GPU (torchrun, N > 1): every rank is an independent replica with its
own index and query set (query sharding, no collective on the data path), so
the aggregate QPS is N x queries / max-over-ranks time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = ("QPS at recall@10>=0.90 on 1 GB300 (BF16 serving vs plain FP32 GPU); "
          "p50/p99 ms; HBM GB/s")
RECALL_TARGET = 0.90
CALIB_QUERIES = 1000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="plain1m", choices=sorted(W.WORKLOADS))
    ap.add_argument("--probes", type=int, default=0, help="force a probe budget")
    ap.add_argument("--precision", choices=["fp32", "bf16", "fp8"], default=None,
                    help="fp32: exact decisions; bf16 / fp8: candidate rows in BF16 / FP8 e4m3 "
                         "with an exactly re-scored shortlist (default: the workload's stored "
                         "precision, bf16 for precision1m and serve2m)")
    ap.add_argument("--rerank-k", type=int, default=None,
                    help="bf16 / fp8 rows: FP32 re-ranked shortlist (default: 100 for the precision "
                         "workload, which states it; 0 = the minimum k + 16 for serving)")
    ap.add_argument("--hash", choices=["auto", "exact", "bf16"], default="auto",
                    help="query projections of bf16 / fp8 rows: bf16 = one BF16 product (each "
                         "hash's winner re-decided exactly, the other probes ranked by the BF16 "
                         "values); exact = the three-piece split; auto = bf16 for the precision "
                         "workload (whose projections are BF16), exact otherwise (measured faster "
                         "for serving)")
    ap.add_argument("--serve-seconds", type=float, default=3.0,
                    help="serving workload: seconds of arrivals per offered rate")
    ap.add_argument("--slots", type=int, default=5,
                    help="serving: batches in flight (host copies of one slot overlap the others' "
                         "device work; 5 measured faster than 3)")
    ap.add_argument("--serve-seconds-default", type=float, default=1.0,
                    help="default run: seconds of arrivals per offered rate in its serving block")
    ap.add_argument("--no-serve", action="store_true",
                    help="default run: skip the serving comparison block")
    ap.add_argument("--max-batch", type=int, default=4096, help="serving: queries per batch")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--graph", action="store_true",
                    help="time the steps as replays of the library's captured search graph")
    ap.add_argument("--no-graph", action="store_true",
                    help="batch10m: steps as plain (pipelined) calls instead of graph replays")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--score-range-rows", type=int, default=0,
                    help="rows per candidate row range of the scoring (0: the library's choice)")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="run the steps one after another (no FPP_SEARCH_PIPELINE)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def peaks():
    """HBM GB/s and dense BF16 TFLOP/s: the measured copy bandwidth and the
    cuBLAS burst figure (each kernel runs well under a second per step)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# headers whose device code the kernels of a source file compile in
KERNEL_HEADERS = {"search_kernels.cu": ("topk.cuh", "common.cuh"),
                  "gemm_tc.cu": ("common.cuh",)}


def kernel_source_hash(name: str) -> str:
    d = os.path.join(ROOT, "paper_2206_01382_gb300", "csrc")
    h = hashlib.sha256()
    for f in (name,) + KERNEL_HEADERS.get(name, ()):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload: str, src: str):
    """DRAM bytes per launch from a committed ncu summary, if the kernel's
    source has not changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(f"{kernel}@{workload}")
    except (OSError, ValueError):
        return None
    if not d or d.get("source_sha") != kernel_source_hash(src):
        return None
    return d.get("bytes_per_launch")


class OracleSearchPool:
    """The FP64 oracle's query path in spawned single-threaded processes over
    one shared copy of a full-size oracle index (points, kept CSR and random
    vectors in shared memory; each worker promotes the points to FP64 once).
    The paper parallelises its search over queries (Section 4)."""

    def __init__(self, ix, workers):
        from multiprocessing import shared_memory
        self.workers = workers
        ids = np.concatenate([np.asarray(t, dtype=np.int64) for t in ix.ids])
        starts = np.concatenate([[0], np.cumsum([len(t) for t in ix.ids])]).astype(np.int64)
        X32 = ix.X.astype(np.float32)   # the points are FP32 inputs: exact round trip
        self.blocks, meta = [], {}
        for name, a in (("X", X32), ("offsets", ix.offsets), ("ids", ids), ("R", ix.R)):
            shm = shared_memory.SharedMemory(create=True, size=max(a.nbytes, 1))
            np.ndarray(a.shape, dtype=a.dtype, buffer=shm.buf)[...] = a
            self.blocks.append(shm)
            meta[name] = (shm.name, a.shape, a.dtype.str)
        meta["starts"] = starts
        meta["shape"] = (ix.n, ix.d, ix.L, ix.D, ix.alpha)
        self.meta = meta
        self.pool = None

    def __enter__(self):
        import concurrent.futures as cf
        import multiprocessing as mp
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                 "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"   # inherited by the spawned workers
        try:
            self.pool = cf.ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"),
                                               initializer=_oracle_worker_init,
                                               initargs=(self.meta,))
            # start every worker and load its index before any timing
            list(self.pool.map(_oracle_worker_ready, range(self.workers)))
        finally:
            for v, old in saved.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old
        return self

    def run(self, Q, ks, ps):
        """Searches the rows of Q (query i with k = ks[i], P = ps[i]) spread
        over the workers; returns the wall time in seconds."""
        c = self.workers
        jobs = [(Q[i::c], ks[i::c], ps[i::c]) for i in range(c) if len(Q[i::c])]
        t0 = time.perf_counter()
        list(self.pool.map(_oracle_worker_search, jobs))
        return time.perf_counter() - t0

    def __exit__(self, *exc):
        if self.pool is not None:
            self.pool.shutdown()
        for shm in self.blocks:
            shm.close()
            shm.unlink()


_ORACLE_IX = {}


def _oracle_worker_init(meta):
    from multiprocessing import shared_memory
    import oracle as O
    arrs = {}
    for name in ("X", "offsets", "ids", "R"):
        shm_name, shape, dt = meta[name]
        shm = shared_memory.SharedMemory(name=shm_name)
        _ORACLE_IX.setdefault("shm", []).append(shm)
        arrs[name] = np.ndarray(shape, dtype=np.dtype(dt), buffer=shm.buf)
    n, d, L, D, alpha = meta["shape"]
    st = meta["starts"]
    ids = [arrs["ids"][st[t]:st[t + 1]] for t in range(L)]
    _ORACLE_IX["ix"] = O.OracleIndex(n, d, L, D, alpha, 1, 0, arrs["R"],
                                     arrs["X"].astype(np.float64), arrs["offsets"], ids,
                                     None, None, None, None)


def _oracle_worker_ready(_):
    return os.getpid()


def _oracle_worker_search(job):
    import oracle as O
    Qs, ks, ps = job
    for q, k, p in zip(Qs, ks, ps):
        O.search(_ORACLE_IX["ix"], q, int(k), int(p))
    return len(Qs)


def oracle_index_full(w, X):
    """The oracle's index over every point of the workload (its tables built
    in one spawned process per host core); returns (index, build seconds)."""
    from oracle.parallel import build_index_parallel
    t0 = time.perf_counter()
    ix = build_index_parallel(X, w.L, w.D, w.alpha, seed=w.rot_seed)
    ix.point_buckets = ix.hash_flag = ix.filter_flag = ix.counts = None   # not used by search
    return ix, time.perf_counter() - t0


def cpu_baseline(w, X, Q, P, k, n1=500, budget_s=20.0):
    """The FP64 oracle, as it stands, on the same full-size index: the query
    path on one core (one single-threaded process, n1 queries) and on every
    host core (one single-threaded process per core; about budget_s of work
    in all).  value = the all-core figure."""
    cores = os.cpu_count() or 1
    ix, build_s = oracle_index_full(w, X)
    m = len(Q)
    kk = np.broadcast_to(np.asarray(k), (m,))
    pp = np.broadcast_to(np.asarray(P), (m,))
    with OracleSearchPool(ix, 1) as one:
        one.run(Q[:4], kk[:4], pp[:4])   # warm
        t1 = one.run(Q[:n1], kk[:n1], pp[:n1])
    qps1 = n1 / t1
    nall = int(min(m, max(n1, qps1 * cores * budget_s / 2)))
    with OracleSearchPool(ix, cores) as pool:
        pool.run(Q[:cores], kk[:cores], pp[:cores])
        tall = pool.run(Q[:nall], kk[:nall], pp[:nall])
    return {"value": nall / tall, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "value_1core": qps1, "oracle_build_s": build_s,
            "sample": f"FP64 numpy oracle over the full index (n={w.n}, L={w.L}, D={w.D}, "
                      f"alpha={w.alpha}): the first {nall} queries over {cores} single-threaded "
                      f"processes ({n1} on one process for value_1core) at "
                      f"{'per-query' if np.ndim(P) else P} probes/table, "
                      f"k={'per-query' if np.ndim(k) else k}"}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    X, Q = W.dataset(w)
    # the budget our arm's calibration picks: the smallest of the sweep that
    # reaches recall@10 >= 0.90 (plain1m: 1 probe per table, recall 0.964)
    P = args.probes or w.probes[0]
    cores = os.cpu_count() or 1
    per_step = 4 * cores   # queries per step, spread over one process per core
    ix, build_s = oracle_index_full(w, X)
    qi = 0
    ks = np.full(per_step, w.k)
    ps = np.full(per_step, P)
    with OracleSearchPool(ix, cores) as pool:
        def step():
            nonlocal qi
            idx = [(qi + i) % len(Q) for i in range(per_step)]
            qi += per_step
            return pool.run(Q[idx], ks, ps)
        for _ in range(args.warmup):
            step()
        times = [step() for _ in range(args.steps)]
    tot = sum(times)
    qps = per_step * args.steps / tot
    sample = (f"FP64 numpy oracle over the full index (n={w.n}, L={w.L}, D={w.D}, "
              f"alpha={w.alpha}, built in {build_s:.0f} s): {per_step} queries per step over "
              f"{cores} single-threaded processes")
    line = {
        "impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "note": w.note, "probes": P, "k": w.k, "sample": sample},
        "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def calibrate_probes(F, ix, Xd, Qd, k, sweep):
    """Smallest probe budget of the sweep whose recall@k against the
    library's brute-force search reaches RECALL_TARGET on a query sample."""
    mcal = min(CALIB_QUERIES, Qd.shape[0])
    ti, _ = F.fpp_bruteforce(Xd, Qd[:mcal], k)
    truth = ti.cpu().numpy()
    recalls, chosen = {}, None
    for P in sweep:
        gi, _ = ix.search(Qd[:mcal], k, P)
        g = gi.cpu().numpy()
        hit = sum(len(set(a.tolist()) & set(b.tolist())) for a, b in zip(g, truth))
        recalls[P] = hit / (k * mcal)
        if chosen is None and recalls[P] >= RECALL_TARGET:
            chosen = P
    if chosen is None:
        chosen = max(recalls, key=lambda p: recalls[p])
    return chosen, recalls, mcal


def serve_drive(srv, Q, P, t, sizes, ks, paced):
    """Submits the requests (arrival times t, sizes, k) to the server, paced
    or not, and times each from submit to completion (host queries in, host
    results out)."""
    import threading
    m = Q.shape[0]
    rids = [None] * len(t)
    lat = np.zeros(len(t))
    start = time.perf_counter()

    def submitter():
        qi = 0
        if not paced:
            # unpaced: the requests go in 16 at a time (one library call), so
            # that the client's per-call overhead does not set the pace
            # (16 x 4,096 rows fit the query pool)
            for i0 in range(0, len(t), 16):
                sz = np.asarray(sizes[i0:i0 + 16], dtype=np.int64)
                tot = int(sz.sum())
                if qi + tot > m:
                    qi = 0
                ids = srv.submit_many(Q[qi:qi + tot], sz, ks[i0:i0 + 16], P)
                for j, rid in enumerate(ids):
                    rids[i0 + j] = rid
                qi += tot
            return
        for i in range(len(t)):
            wait = t[i] - (time.perf_counter() - start)
            if wait > 0:
                time.sleep(wait)
            nq = int(sizes[i])
            if qi + nq > m:
                qi = 0
            rids[i] = srv.submit(Q[qi:qi + nq], int(ks[i]), P)
            qi += nq

    th = threading.Thread(target=submitter)
    th.start()
    for i in range(len(t)):
        while rids[i] is None:
            time.sleep(5e-5)
        lat[i] = srv.poll(rids[i])[2]
    th.join()
    wall = time.perf_counter() - start
    return {"requests": int(len(t)), "queries": int(sizes.sum()),
            "qps": float(sizes.sum() / wall),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_request": float(sizes.mean())}


def serve_session(F, ix, Q, P, slots, seconds, max_batch=4096):
    """Poisson arrivals at each offered query rate (sizes log-uniform in
    1..4096, k in {10, 100}) through the continuous-batching server, then the
    same kind of mix unpaced (saturation)."""
    srv = F.Server(ix, k_max=100, probes_max=P, slots=slots, max_batch=max_batch)
    try:
        t, sizes, ks = W.serve_arrivals(99, 100_000, 0.2)
        serve_drive(srv, Q, P, t, sizes, ks, paced=False)   # warm-up
        s0 = srv.stats()
        rates = {}
        for ri, rate in enumerate(W.SERVE_RATES):
            t, sizes, ks = W.serve_arrivals(ri, rate, seconds)
            r = serve_drive(srv, Q, P, t, sizes, ks, paced=True)
            r["offered_qps"] = rate
            rates[str(rate)] = r
        # saturation: three windows' worth of the highest rate's mix, unpaced
        t, sizes, ks = W.serve_arrivals(len(W.SERVE_RATES), W.SERVE_RATES[-1], 3 * seconds)
        s_sat = srv.stats()
        sat = serve_drive(srv, Q, P, t, sizes, ks, paced=False)
        s1 = srv.stats()
        sat["mean_batch_queries"] = (s1["queries"] - s_sat["queries"]) / max(
            s1["batches"] - s_sat["batches"], 1)
    finally:
        srv.close()
    batches = s1["batches"] - s0["batches"]
    return {"probes": P, "offered": rates, "saturation": sat,
            "mean_batch_queries": (s1["queries"] - s0["queries"]) / max(batches, 1),
            "h2d_bytes": int(sizes.sum() * Q.shape[1] * 4),
            "d2h_bytes": int((np.asarray(sizes) * np.asarray(ks)).sum() * 12)}


def serving_compare(F, w, precision, rerank_k, slots, seconds, probes=0, hash_bf16=False,
                    max_batch=4096):
    """The serving workload with candidate rows in ``precision`` against the
    plain FP32 path under the same request mix, each at its own calibrated
    probe budget (the smallest of the sweep with recall@10 >= 0.90), with
    the GPU clocks sampled over both serving windows."""
    import torch
    X, Q = W.dataset(w)
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q[:CALIB_QUERIES]).cuda()
    sweep = [probes] if probes else list(w.probes)
    prec = {"fp32": F.FPP_FP32, "bf16": F.FPP_BF16, "fp8": F.FPP_FP8E4M3}[precision]
    out = {"workload": w.name, "note": w.note, "seconds_per_rate": seconds, "slots": slots,
           "rerank_k": rerank_k}
    sampler = ClockSampler(torch.cuda.current_device())
    arms = [(precision, prec)] + ([("fp32", F.FPP_FP32)] if prec != F.FPP_FP32 else [])
    res = {}
    for name, pc in arms:
        tb = time.perf_counter()
        hp = F.FPP_BF16 if (hash_bf16 and pc != F.FPP_FP32) else F.FPP_FP32
        ix = F.Index(Xd, w.L, w.D, w.alpha, seed=w.rot_seed, precision=pc, rerank_k=rerank_k,
                     hash_precision=hp)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - tb
        P, rec, mcal = calibrate_probes(F, ix, Xd, Qd, w.k, sweep)
        # the device time of each phase on one 10,000-query batch (k = 10)
        Qb = torch.from_numpy(Q[:10_000]).cuda()
        ph = {}
        for rep in range(3):
            _, _, st = F.fpp_search_ex(ix.handle, Qb, k=10, probes=P)
            if rep:
                for key in ("ms_project", "ms_probe", "ms_probe_exact", "ms_dedup", "ms_score",
                            "ms_topk", "probe_rechecks", "topk_rechecks"):
                    ph[key] = ph.get(key, 0.0) + st[key] / 2
        del Qb
        if not res:
            sampler.start()
        r = serve_session(F, ix, Q, P, slots, seconds, max_batch)
        r.update(precision=name, recall_at_10=rec[P], recall_sweep=rec, recall_sample=mcal,
                 build_s=build_s, batch_phases_10k=ph,
                 query_projection="bf16 one product" if hp == F.FPP_BF16 else "exact split")
        res[name] = r
        ix.close()
    out["clocks"] = sampler.stop()
    out[precision] = res[precision]
    if "fp32" in res and precision != "fp32":
        out["fp32_same_mix"] = dict(res["fp32"])
        out["fp32_same_mix"]["bf16_over_fp32_qps"] = (res[precision]["saturation"]["qps"]
                                                     / res["fp32"]["saturation"]["qps"])
    del Xd, Qd
    torch.cuda.empty_cache()
    return out


def run_serve(args, w):
    """Serving workload alone (``--workload serve2m``): the serving
    comparison above, its saturation throughput as ``value``, and the gather
    + score roofline of the served index on one 10,000-query batch."""
    import torch
    import paper_2206_01382_gb300 as F
    from paper_2206_01382_gb300 import _build

    torch.cuda.set_device(0)
    _build.build()
    F.load()
    srv = serving_compare(F, w, args.precision, args.rerank_k, args.slots, args.serve_seconds,
                          args.probes, args.hash_bf16, args.max_batch)
    main_arm = srv[args.precision]
    sat = main_arm["saturation"]
    line = {
        "metric": METRIC, "value": sat["qps"], "unit": "queries/s", "n_gpus": 1,
        "steps": len(W.SERVE_RATES) + 1, "warmup": 1, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "fp8e4m3"}[args.precision],
        "data": "synthetic",
        "config": {"workload": w.name, "note": w.note, "precision": args.precision,
                   "rerank_k": args.rerank_k if args.precision != "fp32" else None,
                   "n": w.n, "d": w.d, "L": w.L, "D": w.D, "alpha": w.alpha,
                   "probes": main_arm["probes"], "recall_at_10": main_arm["recall_at_10"],
                   "slots": args.slots, "max_batch": args.max_batch,
                   "l2": "inputs larger than L2 (X is "
                         f"{w.n * w.d * 4 / 2**20:.0f} MiB FP32), no flush"},
        "serving": srv,
        "latency_ms": {"p50": sat["p50_ms"], "p99": sat["p99_ms"]},
        "clocks": srv["clocks"],
        "e2e": {"value": sat["qps"], "unit": "queries/s",
                "h2d_bytes_per_step": main_arm["h2d_bytes"],
                "d2h_bytes_per_step": main_arm["d2h_bytes"]},
        "roofline": None,
        "cpu_baseline": None,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    w = W.WORKLOADS[args.workload]
    if args.precision is None:   # the workload's stored precision
        args.precision = "bf16" if w.storage == "bf16" else "fp32"
    if args.rerank_k is None:
        args.rerank_k = 0 if w.name == "serve2m" else 100
    args.hash_bf16 = args.hash == "bf16" or (args.hash == "auto" and w.name == "precision1m")
    if w.name == "batch10m" and not args.no_graph:
        args.graph = True   # the batching workload runs each call as one captured graph
    if args.impl == "reference":
        run_reference(args, w)
        return
    if w.name == "serve2m":
        run_serve(args, w)
        return
    import torch
    import paper_2206_01382_gb300 as F
    from paper_2206_01382_gb300 import _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    _build.build()
    F.load()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    X, Q = W.dataset(w)
    Xd = torch.from_numpy(X).to(dev)
    Qd = torch.from_numpy(Q).to(dev)
    torch.cuda.synchronize()
    tb = time.perf_counter()
    prec = {"fp32": F.FPP_FP32, "bf16": F.FPP_BF16, "fp8": F.FPP_FP8E4M3}[args.precision]
    hp = F.FPP_BF16 if (args.hash_bf16 and prec != F.FPP_FP32) else F.FPP_FP32
    ix = F.Index(Xd, w.L, w.D, w.alpha, seed=w.rot_seed, precision=prec, rerank_k=args.rerank_k,
                 hash_precision=hp)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - tb
    info = ix.info()

    m = Q.shape[0]
    per_query = w.name == "batch10m"
    if per_query:
        # uneven work: per-query k in {1, 10, 100} and probes in {2, 8, 32, 128}
        kpq, ppq = W.per_query_draws(w, m)
        k = int(kpq.max())
        P = "per-query"
        kpq_d = torch.from_numpy(kpq).to(dev)
        ppq_d = torch.from_numpy(ppq).to(dev)
        search_kw = dict(k=k, probes=1, k_per_query=kpq_d, probes_per_query=ppq_d, k_max=k)
        recalls, mcal = {}, min(CALIB_QUERIES, m)
    else:
        # probe budget: smallest of the sweep with recall@10 >= 0.90 on a sample
        k = w.k
        P, recalls, mcal = calibrate_probes(F, ix, Xd, Qd, k,
                                            [args.probes] if args.probes else list(w.probes))
        kpq = ppq = None
        search_kw = dict(k=k, probes=P)
    if args.score_range_rows:
        search_kw["score_range_rows"] = args.score_range_rows
    # the library's autotuner picks the scoring kernel's launch shape on the
    # workload's first batch (results do not depend on it)
    tune = None
    if not args.no_autotune:
        tune = F.fpp_autotune(ix.handle, Qd, k if not per_query else 10,
                              P if not per_query else 8)
    ids = torch.empty((m, k), dtype=torch.int64, device=dev)
    sc = torch.empty((m, k), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    # consecutive steps are pipelined (FPP_SEARCH_PIPELINE: the index
    # alternates two workspaces on two internal streams, so one step's
    # projections overlap the previous step's gather and scoring); a flush
    # orders every step's results before the timed region ends
    pipe = not args.graph and not args.no_pipeline
    for _ in range(args.warmup):
        F.fpp_search_ex(ix.handle, Qd, stream=stream, ids=ids, scores=sc, want_stats=False,
                        graph=args.graph, pipeline=pipe, **search_kw)
    F.fpp_search_flush(ix.handle, stream)
    barrier()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 2)]
    launches0 = F.fpp_launch_count()
    phase = {"ms_project": 0.0, "ms_probe": 0.0, "ms_probe_exact": 0.0, "ms_gather_score": 0.0,
             "ms_dedup": 0.0, "ms_score": 0.0, "ms_topk": 0.0}
    tot = {"entries": 0, "unique": 0, "probes": 0, "probe_rechecks": 0, "probe_full_rechecks": 0,
           "topk_rechecks": 0, "batches": 0}
    # timed steps: asynchronous on one stream, no host round trip per step
    evs[0].record(stream)
    for s in range(args.steps):
        F.fpp_search_ex(ix.handle, Qd, stream=stream, ids=ids, scores=sc, want_stats=False,
                        graph=args.graph, pipeline=pipe, **search_kw)
        evs[s + 1].record(stream)
    F.fpp_search_flush(ix.handle, stream)
    evs[-1].record(stream)
    barrier()
    launches = F.fpp_launch_count() - launches0
    clocks = sampler.stop()
    # per-kernel breakdown: a few more steps with the library's phase events
    # (these synchronise at the end of every call, so they are not timed)
    PK = min(args.steps, 5)
    for s in range(PK):
        _, _, st = F.fpp_search_ex(ix.handle, Qd, stream=stream, ids=ids, scores=sc, **search_kw)
        for key in phase:
            phase[key] += st[key]
        for key in tot:
            tot[key] += st[key]
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]   # (pipelined: call points)
    elapsed_ms = evs[0].elapsed_time(evs[-1])
    if dist is not None:
        t = torch.tensor([elapsed_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / args.steps
    qps = world * m / (ms_per_step / 1e3)

    # distinct candidate rows of the first query batch (the floor of the
    # score kernel's DRAM reads), outside the timed region
    distinct_rows = None
    if not per_query:
        nb = -(-m // max(1, tot["batches"] // PK))
        cands = F.fpp_debug_candidates(ix.handle, Q[:nb], P)
        distinct_rows = int(np.unique(np.concatenate(cands)).size) if cands else 0
        del cands

    # per-kernel rooflines (device time measured with CUDA events on the
    # launching stream inside the library, summed over the timed steps;
    # "per launch" = one query batch)
    hbm_peak, bf16_peak, peak_src = peaks()
    K = PK
    chunks = tot["batches"] // K
    per = chunks * K
    qpl = m / chunks
    d = w.d
    bf16 = args.precision != "fp32"
    row_bytes = (2 * d if args.precision == "bf16"
                 else d + 4 if args.precision == "fp8" else 4 * d)
    kprime = max(k + 16, args.rerank_k if bf16 else 0)
    probes_pl, entries_pl, unique_pl = (tot["probes"] / per, tot["entries"] / per,
                                        tot["unique"] / per)
    # Algorithmic bytes per launch, as the method defines the traffic of the
    # gather and score steps (per query: 8 B per probed bucket for its offset
    # pair, 4 B per kept id scanned, b d B per distinct candidate row with
    # b = 4 FP32 / 2 BF16 / 1 FP8 plus a 4-byte scale, 12 B per result; the
    # precision path adds the 4 d B FP32 rows of its re-ranked shortlist).
    # The per-kernel splits below count the same terms where each kernel
    # moves them; candidate writes and id/score round trips between kernels
    # are implementation traffic and are not counted.
    rerank_b = 4 * d * args.rerank_k * qpl if bf16 else 0.0
    rows_b = row_bytes * unique_pl
    algo_b = 8 * probes_pl + 4 * entries_pl + rows_b + 12 * k * qpl + rerank_b
    dedup_b = 8 * probes_pl + 4 * entries_pl
    score_b = rows_b
    topk_b = 12 * k * qpl + rerank_b
    # projection: the method's work is 2 d FLOPs per (query, random vector);
    # the tensor cores execute it as BF16 products over K padded to 64, 3 of
    # them per FP32 product when the random vectors are on the BF16 grid
    # (three query pieces times one vector piece), else 6
    kpad = -(-d // 64) * 64
    products = 1 if info["q_pieces"] == 1 else 3 if info["r_pieces"] == 1 else 6
    proj_flops = 2.0 * qpl * d * 2 * w.L * w.D
    exec_flops = 2.0 * qpl * kpad * 2 * w.L * w.D * products
    ms_of = {key: phase[key] / per for key in phase}

    def hbm(name, src, ms, nbytes, note):
        gbs = nbytes / (ms / 1e3) / 1e9
        return {"kernel": name, "ms_per_launch": ms, "launches_per_step": chunks, "bound": "hbm",
                "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
                "algorithmic_bytes_per_launch": nbytes, "note": note,
                "peak_source": peak_src + " (hbm_gbs, STREAM-style copy)",
                "traffic": committed_traffic(name, w.name, src)}

    pj_s = ms_of["ms_project"] / 1e3
    pj_tf = proj_flops / pj_s / 1e12
    kernels = {
        "project": {"kernel": "tc_proj_kernel", "ms_per_launch": ms_of["ms_project"],
                    "launches_per_step": chunks, "bound": "tensor", "achieved": pj_tf,
                    "peak": bf16_peak, "unit": "TFLOP/s", "frac": pj_tf / bf16_peak,
                    "algorithmic_flops_per_launch": proj_flops,
                    "note": "achieved = the method's 2 m d 2LD FLOPs per launch / time",
                    "executed_bf16_flops_per_launch": exec_flops,
                    "executed_tflops": exec_flops / pj_s / 1e12,
                    "executed_frac": exec_flops / pj_s / 1e12 / bf16_peak,
                    "bf16_products_per_fp32_product": products,
                    "peak_source": peak_src + " (bf16_tflops, cuBLAS burst)",
                    "traffic": committed_traffic("tc_proj_kernel", w.name, "gemm_tc.cu")},
        "probe": {"kernel": "probe_small_kernel", "ms_per_launch": ms_of["ms_probe"],
                  "launches_per_step": chunks, "bound": "alu"},
        "probe_exact": {"kernel": "probe_window_kernel + probe_recheck_kernel",
                        "ms_per_launch": ms_of["ms_probe_exact"], "launches_per_step": chunks,
                        "bound": "alu"},
        "dedup": hbm("dedup_hash_kernel", "search_kernels.cu", ms_of["ms_dedup"], dedup_b,
                     "dedup_hash tiers (the small one counts each query's entries itself; "
                     "count_entries runs only when a batch needs its exact total) + flatten + "
                     "item ordering kernels: 8 B per probed bucket + 4 B per kept id scanned"),
        "score": hbm({"fp32": "score_kernel", "bf16": "score_bf16_kernel",
                      "fp8": "score_fp8_kernel"}[args.precision], "search_kernels.cu",
                     ms_of["ms_score"], score_b,
                     "one row per (query, distinct candidate); rows shared by the batch's "
                     "queries come from L2, so frac can exceed 1: see dram_vs_distinct_rows"),
        "topk": hbm("topk_kernel", "search_kernels.cu", ms_of["ms_topk"], topk_b,
                    "12 B per result (+ the re-ranked FP32 shortlist rows)"),
    }
    if distinct_rows is not None:
        sk = kernels["score"]
        sk["distinct_rows_per_launch"] = distinct_rows
        sk["distinct_row_bytes_per_launch"] = distinct_rows * row_bytes
        if sk["traffic"]:
            sk["dram_vs_distinct_rows"] = sk["traffic"] / (distinct_rows * row_bytes)
    gs_ms = ms_of["ms_gather_score"]
    gs_gbs = algo_b / (gs_ms / 1e3) / 1e9
    kernels["gather_score"] = {"kernel": "dedup + score + topk", "ms_per_launch": gs_ms,
                               "bound": "hbm", "achieved": gs_gbs, "peak": hbm_peak,
                               "unit": "GB/s", "frac": gs_gbs / hbm_peak,
                               "algorithmic_bytes_per_launch": algo_b,
                               "peak_source": peak_src + " (hbm_gbs, STREAM-style copy)",
                               "note": "8 L P + 4 E + b d U + 12 k bytes per query "
                                       "over the dedup + score + top-k time"}
    # the roofline line is the single kernel with the largest device time
    dom = max(("project", "dedup", "score", "topk"), key=lambda p: kernels[p]["ms_per_launch"])
    roof = {kk: kernels[dom][kk] for kk in ("kernel", "bound", "achieved", "peak", "unit", "frac",
                                            "traffic", "peak_source")}
    if dom == "project":
        roof["executed_frac"] = kernels[dom]["executed_frac"]
    phases = kernels

    # end to end: host (pinned) queries in, host results out, through the C ABI
    e2e = None
    if not args.no_e2e:
        Qh = torch.from_numpy(Q).pin_memory()
        ih = torch.empty((m, k), dtype=torch.int64).pin_memory()
        sh = torch.empty((m, k), dtype=torch.float32).pin_memory()
        host_kw = dict(search_kw)
        if per_query:   # the per-query budgets come from the host too
            host_kw.update(k_per_query=torch.from_numpy(kpq).pin_memory(),
                           probes_per_query=torch.from_numpy(ppq).pin_memory())
        F.fpp_search_ex(ix.handle, Qh, ids=ih, scores=sh, want_stats=False, stream=stream,
                        pipeline=pipe, **host_kw)
        F.fpp_search_flush(ix.handle, stream)
        barrier()
        # each step copies its queries in and its results out (pinned host
        # memory, ordered on the stream); the calls do not wait, one flush
        # and one synchronisation end the timed region
        t0 = time.perf_counter()
        for _ in range(args.steps):
            F.fpp_search_ex(ix.handle, Qh, ids=ih, scores=sh, want_stats=False, stream=stream,
                            pipeline=pipe, **host_kw)
        F.fpp_search_flush(ix.handle, stream)
        barrier()
        e2e_s = (time.perf_counter() - t0) / args.steps
        if dist is not None:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        e2e = {"value": world * m / e2e_s, "unit": "queries/s",
               "h2d_bytes_per_step": int(m * w.d * 4 + (8 * m if per_query else 0)),
               "d2h_bytes_per_step": int(m * k * 12)}

    # recall (per-query k) and score error of the returned results on the
    # calibration sample: returned ids against the library's exact search,
    # returned scores against FP64 inner products of the returned ids
    gi = ids[:mcal].cpu().numpy()
    gs = sc[:mcal].cpu().numpy().astype(np.float64)
    ti, _ = F.fpp_bruteforce(Xd, Qd[:mcal], k)
    truth = ti.cpu().numpy()
    kq = kpq[:mcal] if per_query else np.full(mcal, k)
    hit = sum(len(set(gi[i, :kq[i]].tolist()) & set(truth[i, :kq[i]].tolist())) / kq[i]
              for i in range(mcal))
    recall_k = hit / mcal
    okm = gi >= 0
    ex = np.zeros_like(gs)
    for i in range(mcal):
        sel = gi[i][okm[i]]
        ex[i, okm[i]] = X[sel].astype(np.float64) @ Q[i].astype(np.float64)
    max_score_err = float(np.abs(gs[okm] - ex[okm]).max()) if okm.any() else 0.0
    if per_query:
        # recall@k of each (k, probes) group of the uneven workload
        groups = {}
        pq = ppq[:mcal]
        for i in range(mcal):
            key = f"k={int(kq[i])},P={int(pq[i])}"
            h = len(set(gi[i, :kq[i]].tolist()) & set(truth[i, :kq[i]].tolist())) / kq[i]
            groups.setdefault(key, []).append(h)
        recalls = {"per-query": recall_k,
                   "by_group": {g: {"recall": float(np.mean(v)), "queries": len(v)}
                                for g, v in sorted(groups.items())}}

    # the serving comparison (BF16 rows against plain FP32 under one request
    # mix, each at recall@10 >= 0.90) on the serving workload, one GPU only
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        ix.close()
        del Xd, Qd, ids, sc
        torch.cuda.empty_cache()
        serving = serving_compare(F, W.WORKLOADS["serve2m"], "bf16", 0, args.slots,
                                  args.serve_seconds_default, hash_bf16=args.hash == "bf16",
                                  max_batch=args.max_batch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, X, Q, ppq if per_query else P, kpq if per_query else k)

    if rank == 0:
        sm = sorted(step_ms)
        line = {
            "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "fp8e4m3"}[args.precision],
            "data": "synthetic",
            "config": {"workload": w.name, "note": w.note, "precision": args.precision,
                       "rerank_k": args.rerank_k if bf16 else None,
                       "query_projection": "bf16 one product" if info["q_pieces"] == 1
                                           else "exact split",
                       "n": w.n, "d": w.d, "m": m, "L": w.L,
                       "D": w.D, "alpha": w.alpha, "k": k, "probes": P,
                       "recall_at_10": recalls[P], "recall_sweep": recalls,
                       "recall_at_k_timed": recall_k, "max_abs_score_error": max_score_err,
                       "recall_sample": mcal, "l2": "inputs larger than L2 (X is "
                       f"{w.n * w.d * 4 / 2**20:.0f} MiB), no flush",
                       "build_s": build_s, "index_kept_ids": info["kept_total"],
                       "max_bucket_kept": info["max_bucket_kept"], "cuda_graph": args.graph,
                       "pipelined_steps": pipe,
                       "autotune": tune,
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"batch_p50": sm[len(sm) // 2], "batch_p99": sm[min(len(sm) - 1, int(0.99 * len(sm)))]},
            "roofline": roof,
            "phases": phases,
            "search_stats_per_step": {kk: v / K for kk, v in tot.items()},
            "serving": serving,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
