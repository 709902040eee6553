// Warp- and block-level selection helpers shared by the search kernels.
//
// Scores travel as packed 64-bit keys: (order-preserving bits of the FP32
// score) << 32 | (0xFFFFFFFF - id), so that a larger key is a better entry
// under the order (score desc, id asc), and key 0 is an empty slot.
#pragma once

#include "common.cuh"

namespace fpp {

#ifdef __CUDACC__

__device__ __forceinline__ uint64_t pack_key(float s, uint32_t id) {
  return ((uint64_t)float_key(s) << 32) | (uint64_t)(0xFFFFFFFFu - id);
}
__device__ __forceinline__ uint32_t key_id(uint64_t k) { return 0xFFFFFFFFu - (uint32_t)k; }
__device__ __forceinline__ float key_score(uint64_t k) {
  uint32_t u = (uint32_t)(k >> 32);
  u = (u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u;
  return __uint_as_float(u);
}

__host__ __device__ constexpr int pow2_ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Bitonic sort of a[0..N) (N a power of two), larger keys first, by one warp.
__device__ __forceinline__ void warp_sort_desc(uint64_t* a, int N) {
  const int lane = threadIdx.x & 31;
  if (N <= 64) {
    // up to 64 keys sorted in registers, key i in e[i / 32] of lane i % 32:
    // a compare-exchange of (i, i ^ j) keeps the larger key at the lower
    // index where (i & k) == 0 and at the upper one otherwise; partners
    // j < 32 sit in other lanes (shuffles), j = 32 in the same lane
    __syncwarp();
    uint64_t e0 = lane < N ? a[lane] : 0ull;
    uint64_t e1 = lane + 32 < N ? a[lane + 32] : 0ull;
    for (int k = 2; k <= N; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        if (j == 32) {   // k = 64: descending over the whole sequence
          const uint64_t hi = e0 > e1 ? e0 : e1, lo = e0 > e1 ? e1 : e0;
          e0 = hi;
          e1 = lo;
        } else {
          const bool lower = (lane & j) == 0;
          const uint64_t y0 = __shfl_xor_sync(0xffffffffu, e0, j);
          const bool big0 = lower == ((lane & k) == 0);
          e0 = big0 ? (e0 > y0 ? e0 : y0) : (e0 < y0 ? e0 : y0);
          if (N > 32) {
            const uint64_t y1 = __shfl_xor_sync(0xffffffffu, e1, j);
            const bool big1 = lower == (((lane + 32) & k) == 0);
            e1 = big1 ? (e1 > y1 ? e1 : y1) : (e1 < y1 ? e1 : y1);
          }
        }
      }
    }
    if (lane < N) a[lane] = e0;
    if (lane + 32 < N) a[lane + 32] = e1;
    __syncwarp();
    return;
  }
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < N; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const uint64_t x = a[i], y = a[l];
          const bool first = (i & k) == 0;
          if (first ? (y > x) : (x > y)) { a[i] = y; a[l] = x; }
        }
      }
      __syncwarp();
    }
  }
}

// Same, by the whole block.
__device__ __forceinline__ void block_sort_desc(uint64_t* a, int N) {
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const uint64_t x = a[i], y = a[l];
          const bool first = (i & k) == 0;
          if (first ? (y > x) : (x > y)) { a[i] = y; a[l] = x; }
        }
      }
      __syncthreads();
    }
  }
}

// An exactly scored entry: FP64-accurate score and id; order (s desc, id asc).
struct SD {
  double s;
  uint32_t id;
  uint32_t pad;
};
__device__ __forceinline__ bool sd_before(const SD& x, const SD& y) {
  return x.s > y.s || (x.s == y.s && x.id < y.id);
}

__device__ __forceinline__ void warp_sort_sd(SD* a, int N) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < N; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const SD x = a[i], y = a[l];
          const bool first = (i & k) == 0;
          if (first ? sd_before(y, x) : sd_before(x, y)) { a[i] = y; a[l] = x; }
        }
      }
      __syncwarp();
    }
  }
}

__device__ __forceinline__ void block_sort_sd(SD* a, int N) {
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const SD x = a[i], y = a[l];
          const bool first = (i & k) == 0;
          if (first ? sd_before(y, x) : sd_before(x, y)) { a[i] = y; a[l] = x; }
        }
      }
      __syncthreads();
    }
  }
}

// Per-warp running top-K' buffer in shared memory.  Entries better than the
// current threshold are appended; when the buffer is nearly full it is
// sorted and cut back to K'.  buf has capacity cap (a power of two >= 2K'+32).
struct WarpTop {
  uint64_t* buf;
  int cap;
  int kp;        // K'
  int cnt;       // entries in buf (warp-uniform)
  uint64_t thr;  // keys <= thr cannot enter (warp-uniform)

  __device__ __forceinline__ void init(uint64_t* b, int c, int k) {
    buf = b; cap = c; kp = k; cnt = 0; thr = 0;
  }
  __device__ __forceinline__ void compact() {
    const int lane = threadIdx.x & 31;
    for (int i = cnt + lane; i < cap; i += 32) buf[i] = 0;
    __syncwarp();
    warp_sort_desc(buf, cap);
    // a candidate offered twice (lists that were not de-duplicated) has the
    // same key both times: keep one copy of each key
    int n = 0;
    for (int i0 = 0; i0 < cnt; i0 += 32) {
      const int i = i0 + lane;
      const uint64_t v = i < cnt ? buf[i] : 0ull;
      const bool keep = i < cnt && (i == 0 || buf[i - 1] != v);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      __syncwarp();
      if (keep) buf[n + __popc(m & ((1u << lane) - 1u))] = v;
      n += __popc(m);
      __syncwarp();
    }
    cnt = n < kp ? n : kp;
    if (cnt == kp) thr = buf[kp - 1];
    __syncwarp();
  }
  // Every lane offers at most one key (valid = false for none).
  __device__ __forceinline__ void offer(bool valid, uint64_t key) {
    const int lane = threadIdx.x & 31;
    const bool take = valid && key > thr;
    const unsigned m = __ballot_sync(0xffffffffu, take);
    if (m == 0) return;
    if (cnt + 32 > cap) compact();
    if (take) buf[cnt + __popc(m & ((1u << lane) - 1u))] = key;
    cnt += __popc(m);
    __syncwarp();
  }
  // Leaves the best min(cnt, K') entries sorted at buf[0..).
  __device__ __forceinline__ int finish() {
    compact();
    return cnt;
  }
};

// An exact-score entry: order key of an FP64 score (larger = better) and id.
struct SK {
  uint64_t k;
  uint32_t id;
  uint32_t pad;
};
__device__ __forceinline__ bool sk_before(const SK& x, const SK& y) {
  return x.k > y.k || (x.k == y.k && x.id < y.id);
}
__device__ __forceinline__ uint64_t double_key(double x) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_double(uint64_t k) {
  const uint64_t u = (k & 0x8000000000000000ull) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)u);
}

__device__ __forceinline__ void warp_sort_sk(SK* a, int N) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < N; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const SK x = a[i], y = a[l];
          const bool first = (i & k) == 0;
          if (first ? sk_before(y, x) : sk_before(x, y)) { a[i] = y; a[l] = x; }
        }
      }
      __syncwarp();
    }
  }
}

// Per-warp running top-k of exact entries (same scheme as WarpTop).
struct WarpTopSK {
  SK* buf;
  int cap, kp, cnt;
  SK thr;
  bool full;
  __device__ __forceinline__ void init(SK* b, int c, int k) {
    buf = b; cap = c; kp = k; cnt = 0; full = false; thr = SK{0ull, 0xFFFFFFFFu, 0u};
  }
  __device__ __forceinline__ void compact() {
    const int lane = threadIdx.x & 31;
    for (int i = cnt + lane; i < cap; i += 32) buf[i] = SK{0ull, 0xFFFFFFFFu, 0u};
    __syncwarp();
    warp_sort_sk(buf, cap);
    cnt = cnt < kp ? cnt : kp;
    if (cnt == kp) { thr = buf[kp - 1]; full = true; }
    __syncwarp();
  }
  __device__ __forceinline__ void offer(bool valid, const SK& e) {
    const int lane = threadIdx.x & 31;
    const bool take = valid && (!full || sk_before(e, thr));
    const unsigned m = __ballot_sync(0xffffffffu, take);
    if (m == 0) return;
    if (cnt + 32 > cap) compact();
    if (take) buf[cnt + __popc(m & ((1u << lane) - 1u))] = e;
    cnt += __popc(m);
    __syncwarp();
  }
  __device__ __forceinline__ int finish() {
    compact();
    return cnt;
  }
};

#endif  // __CUDACC__

}  // namespace fpp
