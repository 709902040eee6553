"""Seeded Gaussian random vectors for the cross-polytope hashes (oracle side).

The paper draws every coordinate of every random vector r_i from N(0, 1)
(Section 2.2) and says nothing about the generator.  Both the oracle and the
CUDA library regenerate the same vectors from a seed, each with its own code,
from two published definitions:

* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the output
  mix z ^= z>>30; z *= 0xBF58476D1CE4E5B9; z ^= z>>27; z *= 0x94D049BB133111EB;
  z ^= z>>31.  Output number j (0-based) of a stream whose initial state is
  s0 is mix(s0 + (j+1) * 0x9E3779B97F4A7C15), so a stream is counter-based.
* Box-Muller (Box and Muller, 1958), cosine branch only:
  z = sqrt(-2 ln u1) * cos(2 pi u2).

Layout: R[t][j][i][c] for table t < L, hash j < 2, vector i < D, coordinate
c < d.  Stream id = 2t + j with initial state seed XOR (golden * (id + 1)).
Coordinate (i, c) uses the stream's outputs 2(i d + c) and 2(i d + c) + 1 as
(u1, u2): u1 = (top 53 bits + 1) / 2^53 in (0, 1], u2 = top 53 bits / 2^53 in
[0, 1).  The FP64 value is rounded to FP32 and that to the nearest BF16 value
(ties to even); the resulting FP32 array (every element on the BF16 grid) is
the canonical R, promoted exactly to FP64 by the oracle.  The paper fixes
only the N(0, 1) distribution; 8 significant bits per coordinate keep the
vectors as random for the hash.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(state0: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream whose
    initial state is ``state0``."""
    with np.errstate(over="ignore"):
        j = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(np.uint64(state0) + j * GOLDEN)


def stream_state(seed: int, stream_id: int) -> int:
    """Initial state of stream ``stream_id``: seed XOR golden*(id+1) mod 2^64."""
    return (int(seed) ^ ((0x9E3779B97F4A7C15 * (stream_id + 1)) & 0xFFFFFFFFFFFFFFFF)) \
        & 0xFFFFFFFFFFFFFFFF


def box_muller(u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    """Box-Muller, cosine branch, in FP64: sqrt(-2 ln u1) cos(2 pi u2)."""
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(6.283185307179586 * u2)


def uniform_pair(raw: np.ndarray):
    """(u1, u2) from consecutive 64-bit outputs: top 53 bits / 2^53, with u1
    shifted to (0, 1] so that its logarithm is finite."""
    top1 = (raw[0::2] >> np.uint64(11)).astype(np.float64)
    top2 = (raw[1::2] >> np.uint64(11)).astype(np.float64)
    return (top1 + 1.0) / 9007199254740992.0, top2 / 9007199254740992.0


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Finite FP32 values rounded to the nearest BF16 value (ties to even),
    returned as FP32: add 0x7FFF plus the lowest kept bit, clear 16 bits."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)) \
        << np.uint64(16)
    return u.astype(np.uint32).view(np.float32)


def gaussian_stream(seed: int, stream_id: int, count: int) -> np.ndarray:
    """``count`` standard normals of one stream, on the BF16 grid (FP32)."""
    raw = splitmix64(stream_state(seed, stream_id), 2 * count)
    u1, u2 = uniform_pair(raw)
    return round_bf16(box_muller(u1, u2).astype(np.float32))


def gaussian_rotations(seed: int, L: int, D: int, d: int) -> np.ndarray:
    """The canonical random vectors ``R[L][2][D][d]`` (FP32 holding BF16 values)."""
    R = np.empty((L, 2, D, d), dtype=np.float32)
    for t in range(L):
        for j in range(2):
            R[t, j] = gaussian_stream(seed, 2 * t + j, D * d).reshape(D, d)
    return R
