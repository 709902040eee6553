"""Falconn++ CPU oracle: plain, slow, FP64 restatement of the method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
it is used by ``tests/``, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  It shares no
code with the CUDA library (``paper_2206_01382_gb300``): the two meet only
through the seeded input generators in ``workloads.py`` and through the
published definitions of the random-rotation generator, which each side
implements on its own.

Contents
  rotations.py  SplitMix64 counter streams + Box-Muller Gaussian rotations.
  falconn.py    cross-polytope hashing (Eq. 1), the alpha-fraction filter
                (Section 3.4), multi-probe indexing (Algorithm 1), probe
                ranking (Section 3.4, "a new criteria"), candidate union,
                exact scoring and top-k, brute-force search, near-tie flags.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against brute-force enumeration, invariants the paper fixes and published
test vectors.  Readings of passages the paper leaves open are listed in the
docstrings where they are taken.
"""
from .rotations import splitmix64, gaussian_rotations  # noqa: F401
from .falconn import (  # noqa: F401
    NEAR_TIE,
    OracleIndex,
    brute_force,
    build_index,
    center_points,
    cross_polytope_hash,
    keep_count,
    probe_buckets,
    probe_global,
    recall_at,
    search,
    search_batch,
    simhash_select,
    simhash_signatures,
    hamming,
)
