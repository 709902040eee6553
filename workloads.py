"""Seeded synthetic workloads shaped like the Falconn++ evaluation data.

This module is shared by the tests, the benchmark and the oracle's callers.
It holds only input generation and the workload parameters; none of the
method's arithmetic (projection, hashing, filtering, probing, scoring) lives
here.

The paper evaluates on Glove200, Glove300 and NYTimes (Section 4), unit-norm
word/document embeddings whose density is strongly clustered.  Those datasets
are not available, so every workload here is a Gaussian mixture on the unit
sphere: ``K`` centres drawn as normalised N(0, I_d) vectors, each point a
centre plus N(0, sigma^2 I_d) noise, then L2-normalised.  Queries come from
the same process and are held out (the last ``m`` rows of one draw of
``n + m`` points), as the paper extracts its query sets from the data
(Section 4).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One search workload: data shape, index parameters and query budget."""

    name: str
    n: int            # base vectors
    d: int            # dimension
    K: int            # mixture components
    sigma: float      # per-coordinate noise std-dev
    m: int            # queries
    L: int            # hash tables
    D: int            # random vectors per cross-polytope hash
    alpha: float      # fraction of each bucket kept by the filter
    probes: tuple     # probes per table (swept)
    k: int            # results per query
    data_seed: int
    rot_seed: int
    query_seed: int
    storage: str = "f32"   # stored vector precision of the search path
    note: str = ""


# The five workloads.  Seeds follow one rule: data 1000+i, rotations 2000+i,
# per-query draws 3000+i for workload index i.
WORKLOADS = {
    "tiny": Workload(
        "tiny", n=10_000, d=64, K=256, sigma=0.3 / math.sqrt(64), m=100,
        L=10, D=64, alpha=0.2, probes=(4,), k=10,
        data_seed=1000, rot_seed=2000, query_seed=3000,
        note="n=10k d=64 FP32, L=10 D=64 alpha=0.2, 4 probes/table, k=10"),
    "plain1m": Workload(
        "plain1m", n=1_000_000, d=128, K=4096, sigma=0.25 / math.sqrt(128),
        m=10_000, L=100, D=256, alpha=0.1, probes=(1, 4, 16, 64), k=10,
        data_seed=1001, rot_seed=2001, query_seed=3001,
        note="n=1M d=128 FP32, L=100 D=256 alpha=0.1, probes {1,4,16,64}, k=10"),
    "precision1m": Workload(
        "precision1m", n=1_000_000, d=960, K=1024, sigma=0.35 / math.sqrt(960),
        m=1_000, L=50, D=1024, alpha=0.1, probes=(1, 2, 4, 8, 16), k=10,
        data_seed=1002, rot_seed=2002, query_seed=3002, storage="bf16",
        note="n=1M d=960 BF16 storage + rotations, FP32 accumulate, FP32 "
             "re-rank of a top-100 shortlist, L=50 D=1024 alpha=0.1, k=10"),
    "batch10m": Workload(
        "batch10m", n=10_000_000, d=96, K=16384, sigma=0.3 / math.sqrt(96),
        m=100_000, L=50, D=128, alpha=0.05, probes=(2, 8, 32, 128), k=100,
        data_seed=1003, rot_seed=2003, query_seed=3003,
        note="n=10M d=96 FP32, per-query k in {1,10,100} and probes in "
             "{2,8,32,128}, L=50 D=128 alpha=0.05"),
    "serve2m": Workload(
        "serve2m", n=2_000_000, d=256, K=8192, sigma=0.3 / math.sqrt(256),
        m=100_000, L=64, D=256, alpha=0.1, probes=(1, 2, 4, 8, 16), k=10,
        data_seed=1004, rot_seed=2004, query_seed=3004, storage="bf16",
        note="n=2M d=256 BF16, L=64 D=256 alpha=0.1, Poisson arrivals, "
             "request sizes 1-4096, k in {10,100}"),
}


def gaussian_mixture(n_total: int, d: int, K: int, sigma: float, seed: int,
                     chunk: int = 1 << 20) -> np.ndarray:
    """``n_total`` unit vectors (float32, row-major ``[n_total][d]``) from a
    ``K``-component Gaussian mixture on the sphere.

    Centres: normalised N(0, I_d).  Points: centre[z] + N(0, sigma^2 I_d)
    with z uniform over the K components, then L2-normalised.  Generation is
    chunked so that large workloads do not need a float64 copy of the whole
    matrix.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.standard_normal((K, d))
    centres /= np.linalg.norm(centres, axis=1, keepdims=True)
    out = np.empty((n_total, d), dtype=np.float32)
    for s in range(0, n_total, chunk):
        e = min(n_total, s + chunk)
        z = rng.integers(0, K, size=e - s)
        pts = centres[z] + sigma * rng.standard_normal((e - s, d))
        pts /= np.linalg.norm(pts, axis=1, keepdims=True)
        out[s:e] = pts.astype(np.float32)
    return out


def dataset(w: Workload, n: int | None = None, m: int | None = None):
    """Base vectors ``X`` ``[n][d]`` and held-out queries ``Q`` ``[m][d]``.

    One draw of ``w.n + w.m`` points; the last ``w.m`` rows are the queries.
    Passing a smaller ``n`` or ``m`` takes a prefix of each part of the same
    draw, so reduced-size cases are sub-samples of the full workload.
    """
    allpts = gaussian_mixture(w.n + w.m, w.d, w.K, w.sigma, w.data_seed)
    X = allpts[: w.n]
    Q = allpts[w.n:]
    if n is not None:
        X = X[:n]
    if m is not None:
        Q = Q[:m]
    return np.ascontiguousarray(X), np.ascontiguousarray(Q)


def small_mixture(n: int, m: int, d: int, K: int, sigma: float, seed: int):
    """A small mixture draw split into base and query parts (test helper)."""
    allpts = gaussian_mixture(n + m, d, K, sigma, seed)
    return np.ascontiguousarray(allpts[:n]), np.ascontiguousarray(allpts[n:])


def per_query_draws(w: Workload, m: int, ks=(1, 10, 100), probes=(2, 8, 32, 128)):
    """Per-query ``k`` and probe budgets drawn uniformly from the given sets
    (the uneven-work batching workload)."""
    rng = np.random.Generator(np.random.PCG64(w.query_seed))
    k = rng.choice(np.asarray(ks, dtype=np.int32), size=m)
    p = rng.choice(np.asarray(probes, dtype=np.int32), size=m)
    return k.astype(np.int32), p.astype(np.int32)


SERVE_RATES = (10_000, 100_000, 1_000_000)   # offered queries per second


def serve_arrivals(rate_index: int, rate: float, duration_s: float, max_size: int = 4096,
                   ks=(10, 100)):
    """Poisson request arrivals for the serving workload: arrival times (s),
    request sizes (log-uniform integers in [1, max_size]) and k per request,
    seeded with 4000 + rate_index.  The request rate is the offered query
    rate divided by the mean request size."""
    rng = np.random.Generator(np.random.PCG64(4000 + rate_index))
    mean_size = (max_size - 1) / math.log(max_size)      # mean of the log-uniform law
    req_rate = rate / mean_size
    n = max(1, int(math.ceil(req_rate * duration_s * 1.2)) + 16)
    t = np.cumsum(rng.exponential(1.0 / req_rate, size=n))
    t = t[t < duration_s]
    if t.size == 0:
        t = np.zeros(1)
    sizes = np.floor(np.exp(rng.uniform(0.0, math.log(max_size + 1), size=t.size))).astype(np.int64)
    sizes = np.clip(sizes, 1, max_size)
    k = rng.choice(np.asarray(ks, dtype=np.int32), size=t.size)
    return t, sizes, k
