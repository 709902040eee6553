// Search kernels: probe ranking per (query, table) (Section 3.4, "Multi-
// probing for querying"), candidate gather and de-duplication, scoring and
// top-k (Sections 1 and 4).
#include <algorithm>
#include <atomic>
#include <climits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"
#include "topk.cuh"

namespace fpp {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// ============================================================== probe ranking
//
// One warp per (query, table).  Each hash j gives the signed list v_j over the
// 2D wedges (v_j(i) = q^T r_i, v_j(i + D) = -q^T r_i); its top D entries are
// the |q^T r_i| in the wedge on q's side.  A bucket (h1, h2) scores
// v_1(h1) + v_2(h2) and the P best buckets are probed (ties: lower bucket id).
//
// Fast path, on the FP32 projections of the GEMM: each lane holds its S =
// D/32 projections of a hash as packed keys in registers, sorted; the best
// T = P + 1 entries of the list are pulled out by rounds of warp-wide max.  A
// pair ranked a-th in list 1 and b-th in list 2 is preceded by at least
// (a+1)(b+1) - 1 other pairs, so the pairs with (a+1)(b+1) <= P + 1 contain
// the FP32 top P + 1; those are scored and the top P + 1 selected.  The FP32
// top-P set is the exact one when the gap between the P-th and (P+1)-th FP32
// pair scores exceeds twice their error bound.  Otherwise the (query, table)
// goes on a device-side list that a second kernel re-decides from compensated
// (FP64-accurate) projections.

constexpr int PROBE_WARPS = 8;
constexpr int PMAX = 128;
constexpr int LIST_CAP = PMAX + 1;

// Pair candidates with (a+1)(b+1) <= T over lists of length A (host and device).
__host__ __device__ inline int pair_count(int T, int A) {
  int C = 0;
  for (int a = 0; a < A && a < T; ++a) {
    int nb = T / (a + 1);
    C += nb < A ? nb : A;
  }
  return C;
}

__host__ __device__ inline size_t probe_warp_bytes(int pmax, int D) {
  const int T = pmax + 1;
  const int E = T < D ? T : D;
  const int A = (E == D) ? 2 * D : E;
  const int C = pair_count(T, A);
  const int Cp = ((C + 31) / 32) * 32;
  return (size_t)2 * LIST_CAP * 8 + (size_t)Cp * 8 + (size_t)LIST_CAP * 8;
}

// Sorts each lane's column col[s*32 + lane], s < S, descending, then pulls
// the best T keys of the whole array into out[0..T) in descending order.
__device__ void warp_select(uint64_t* col, int S, int T, uint64_t* out) {
  const int lane = threadIdx.x & 31;
  for (int s = 1; s < S; ++s) {
    const uint64_t x = col[s * 32 + lane];
    int k = s - 1;
    while (k >= 0 && col[k * 32 + lane] < x) {
      col[(k + 1) * 32 + lane] = col[k * 32 + lane];
      --k;
    }
    col[(k + 1) * 32 + lane] = x;
  }
  __syncwarp();
  int hp = 0;
  for (int r = 0; r < T; ++r) {
    const uint64_t my = hp < S ? col[hp * 32 + lane] : 0ull;
    const uint32_t hi = (uint32_t)(my >> 32), lo = (uint32_t)my;
    const uint32_t mh = __reduce_max_sync(FULL, hi);
    const uint32_t ml = __reduce_max_sync(FULL, hi == mh ? lo : 0u);
    if (hi == mh && lo == ml && my != 0ull) ++hp;
    if (lane == 0) out[r] = ((uint64_t)mh << 32) | ml;
  }
  __syncwarp();
}

// Key of a list entry: (bits(|p|) + 1) << 32 | (0xFFFFFFFF - h); larger key =
// larger |p|, then lower wedge.  0 marks an empty slot.
__device__ __forceinline__ uint64_t list_key(float p, uint32_t i, uint32_t D) {
  const uint32_t h = i + (p < 0.f ? D : 0u);
  return ((uint64_t)(__float_as_uint(fabsf(p)) + 1u) << 32) | (uint64_t)(0xFFFFFFFFu - h);
}

struct ListEntry {
  float v;
  uint32_t h;
};

// Signed-list entry a of a list whose E best |p| entries are in keys[0..E);
// positions a >= D (available when E == D) are the antipodal wedges.
__device__ __forceinline__ ListEntry signed_entry(const uint64_t* keys, int a, int D) {
  const uint64_t k = keys[a < D ? a : 2 * D - 1 - a];
  const float v = __uint_as_float((uint32_t)(k >> 32) - 1u);
  uint32_t h = 0xFFFFFFFFu - (uint32_t)k;
  if (a < D) return ListEntry{v, h};
  h = h < (uint32_t)D ? h + D : h - D;
  return ListEntry{-v, h};
}

// Warp-wide bitonic sort, descending, of 32 S keys held S per lane; element
// i = lane S + s is key[s], so the stages with distance below S stay inside a
// lane and the others exchange whole registers between lanes.
template <int S>
__device__ __forceinline__ void warp_bitonic_desc(uint64_t (&key)[S]) {
  const int lane = threadIdx.x & 31;
  constexpr int N = 32 * S;
#pragma unroll
  for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= S) {
        const int lj = j / S;   // the partner lane is lane ^ lj
        const bool lower = (lane & lj) == 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const bool desc = ((lane * S + s) & k) == 0;
          const uint64_t other = __shfl_xor_sync(FULL, key[s], lj);
          // the lower index of a descending run keeps the larger key
          key[s] = (lower == desc) ? (key[s] > other ? key[s] : other)
                                   : (key[s] < other ? key[s] : other);
        }
      } else {
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const int t = s ^ j;
          if (t > s) {
            const bool desc = ((lane * S + s) & k) == 0;
            const uint64_t x = key[s], y = key[t];
            const bool sw = desc ? (x < y) : (x > y);
            key[s] = sw ? y : x;
            key[t] = sw ? x : y;
          }
        }
      }
    }
  }
}

// Best E entries of one list into out[0..E) (out holds LIST_CAP >= 64
// keys).  Lists of up to 128 entries: one warp-wide sort when E > 32, else
// register-resident sorted runs of S keys per lane and E rounds of warp max.
// Longer lists (S >= 16) keep only 32-bit magnitudes in registers: a binary
// search finds a threshold that admits between E and E + 16 of them, those
// are compacted and sorted; heavy ties at the threshold fall back to E rounds
// of warp max over the untaken entries.
template <int S>
__device__ __forceinline__ void list_top(const float* __restrict__ pr, int D, int E, uint64_t* out) {
  const int lane = threadIdx.x & 31;
  if (S >= 16) {
    uint32_t v[S];   // bits(|p|) + 1; 0: no entry
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int i = s * 32 + lane;
      v[s] = i < D ? (__float_as_uint(pr[i]) & 0x7FFFFFFFu) + 1u : 0u;
    }
    uint32_t vmin = 0xFFFFFFFFu, vmax = 0u;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (v[s]) vmin = min(vmin, v[s]);
      vmax = max(vmax, v[s]);
    }
    uint32_t lo = __reduce_min_sync(FULL, vmin), hi = __reduce_max_sync(FULL, vmax);
    // count(v >= lo) >= E holds throughout (E <= D entries exist)
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo + 1u) / 2u;
      unsigned c = 0;
#pragma unroll
      for (int s = 0; s < S; ++s) c += v[s] >= mid ? 1u : 0u;
      c = __reduce_add_sync(FULL, c);
      if (c >= (unsigned)E) {
        lo = mid;
        if (c <= (unsigned)E + 16u) break;
      } else {
        hi = mid - 1u;
      }
    }
    unsigned c = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) c += v[s] >= lo ? 1u : 0u;
    const unsigned total = __reduce_add_sync(FULL, c);
    if (total <= 64u) {
      unsigned n = 0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const bool take = v[s] >= lo;
        const unsigned m = __ballot_sync(FULL, take);
        if (take) {
          const int i = s * 32 + lane;
          out[n + __popc(m & ((1u << lane) - 1u))] = list_key(pr[i], (uint32_t)i, (uint32_t)D);
        }
        n += __popc(m);
      }
      const int np2 = pow2_ceil(total > 1u ? (int)total : 1);
      for (int e = (int)total + lane; e < np2; e += 32) out[e] = 0ull;
      __syncwarp();
      warp_sort_desc(out, np2);
      return;
    }
    // heavy ties: E rounds, each taking the best untaken entry
    uint32_t taken = 0u;
    for (int r = 0; r < E; ++r) {
      uint64_t best = 0ull;
      int bs = -1;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const int i = s * 32 + lane;
        if (!((taken >> s) & 1u) && v[s]) {
          const uint32_t h = (uint32_t)i + (pr[i] < 0.f ? (uint32_t)D : 0u);
          const uint64_t key = ((uint64_t)v[s] << 32) | (uint64_t)(0xFFFFFFFFu - h);
          if (key > best) { best = key; bs = s; }
        }
      }
      const uint32_t bh = (uint32_t)(best >> 32), bl = (uint32_t)best;
      const uint32_t mh = __reduce_max_sync(FULL, bh);
      const uint32_t ml = __reduce_max_sync(FULL, bh == mh ? bl : 0u);
      if (bs >= 0 && bh == mh && bl == ml) taken |= 1u << bs;
      if (lane == 0) out[r] = ((uint64_t)mh << 32) | ml;
    }
    __syncwarp();
    return;
  }
  if (S <= 4 && E > 32) {
    uint64_t key[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int i = lane * S + s;
      key[s] = i < D ? list_key(pr[i], (uint32_t)i, (uint32_t)D) : 0ull;
    }
    warp_bitonic_desc<S>(key);
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (lane * S + s < E) out[lane * S + s] = key[s];
    __syncwarp();
    return;
  }
  uint64_t key[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int i = s * 32 + lane;
    key[s] = i < D ? list_key(pr[i], (uint32_t)i, (uint32_t)D) : 0ull;
  }
  // bitonic sort, descending, fully unrolled (register indices are static)
#pragma unroll
  for (int k = 2; k <= S; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int i = 0; i < S; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const bool desc = (i & k) == 0;
          const uint64_t x = key[i], y = key[l];
          if (desc ? (x < y) : (x > y)) { key[i] = y; key[l] = x; }
        }
      }
  for (int r = 0; r < E; ++r) {
    const uint32_t hi = (uint32_t)(key[0] >> 32), lo = (uint32_t)key[0];
    const uint32_t mh = __reduce_max_sync(FULL, hi);
    const uint32_t ml = __reduce_max_sync(FULL, hi == mh ? lo : 0u);
    if (hi == mh && lo == ml) {
#pragma unroll
      for (int s = 0; s + 1 < S; ++s) key[s] = key[s + 1];
      key[S - 1] = 0ull;
    }
    if (lane == 0) out[r] = ((uint64_t)mh << 32) | ml;
  }
  __syncwarp();
}

template <int S>
__global__ void __launch_bounds__(PROBE_WARPS * 32)
probe_kernel(ProbeArgs a, int pmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_cnt, s_base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_cnt = 0u;
  __syncthreads();
  const int64_t w0 = (int64_t)blockIdx.x * PROBE_WARPS + wid;
  const bool live = w0 < a.mq * a.nt;
  const int64_t w = live ? w0 : 0;   // a dead warp works on item 0 and stores nothing
  const int64_t q = w / a.nt;
  const int tl = (int)(w % a.nt);
  const int t = a.tb + tl;
  const int D = a.D;
  const int P = a.probes_pq ? a.probes_pq[q] : a.probes;
  const int64_t NB = 4ll * D * D;
  unsigned char* wsm = smem + (size_t)wid * probe_warp_bytes(pmax, D);
  uint64_t* lists = reinterpret_cast<uint64_t*>(wsm);            // 2 x LIST_CAP
  uint64_t* pout = lists + 2 * LIST_CAP;                          // LIST_CAP
  uint64_t* col = pout + LIST_CAP;                                // pairs

  const int T = P + 1;
  const int E = T < D ? T : D;
  if (a.P) {
    for (int j = 0; j < 2; ++j)
      list_top<S>(a.P + q * a.ldp + (int64_t)(2 * tl + j) * D, D, E, lists + j * LIST_CAP);
  } else {
    // the projection epilogue already kept the EL >= E best keys per hash
    for (int j = 0; j < 2; ++j) {
      const uint64_t* src = a.lists + ((q * a.nt + tl) * 2 + j) * (int64_t)(a.EL + 1);
      for (int e = lane; e < E; e += 32) lists[j * LIST_CAP + e] = src[e];
    }
    __syncwarp();
  }
  const int A = (E == D) ? 2 * D : E;
  int C = 0;
  for (int ai = 0; ai < A && ai < T; ++ai) {
    int nb = T / (ai + 1);
    if (nb > A) nb = A;
    const ListEntry x = signed_entry(lists, ai, D);
    for (int b = lane; b < nb; b += 32) {
      const ListEntry y = signed_entry(lists + LIST_CAP, b, D);
      const uint32_t bucket = x.h * (uint32_t)(2 * D) + y.h;
      col[C + b] = ((uint64_t)float_key(x.v + y.v) << 32) | (uint64_t)(0xFFFFFFFFu - bucket);
    }
    C += nb;
  }
  const int Sc = (C + 31) / 32;
  for (int e = C + lane; e < Sc * 32; e += 32) col[e] = 0ull;
  __syncwarp();
  const bool boundary = (int64_t)P < NB;
  const int Tsel = boundary ? P + 1 : P;
  warp_select(col, Sc, Tsel, pout);

  bool certain = C >= Tsel;
  if (a.argmax_only) {
    // the argmax pass has made each hash's winner exact; the other probes
    // take the ranking of the BF16 values as it stands
    certain = C >= P;
  } else if (certain && boundary) {
    // FP32 arithmetic (the FP64 pipe is slow); every factor is positive and
    // the 1.001 margin covers the few roundings of this expression.  Pair
    // scores from truncated list values may be low by trunc times the two
    // lists' largest values.
    const float sP = key_score(pout[P - 1]), sP1 = key_score(pout[P]);
    const float tr = a.P ? 0.f
                         : a.trunc * (signed_entry(lists, 0, D).v +
                                      signed_entry(lists + LIST_CAP, 0, D).v);
    const float eps = a.gammaf * a.qnorm[q] * (a.rmax[2 * t] + a.rmax[2 * t + 1]) + tr;
    const float need = (2.f * eps + 6.0e-8f * (fabsf(sP) + fabsf(sP1))) * 1.001f + 1e-30f;
    certain = (sP - sP1) > need;
  }
  if (live && certain) {
    uint32_t* dst = a.out + (q * a.nt + tl) * (int64_t)a.probes;
    for (int p = lane; p < P; p += 32) dst[p] = 0xFFFFFFFFu - (uint32_t)pout[p];
  }
  // recheck slots: counted in shared memory, one global reservation per CTA
  const bool rc = live && !certain && lane == 0;
  const unsigned my = rc ? atomicAdd(&s_cnt, 1u) : 0u;
  __syncthreads();
  if (threadIdx.x == 0 && s_cnt) {
    s_base = atomicAdd(a.recheck_count, s_cnt);
    if (a.rechecks) atomicAdd(a.rechecks, (unsigned long long)s_cnt);
  }
  __syncthreads();
  if (rc) {
    const unsigned slot = s_base + my;
    a.recheck[slot] = (uint32_t)(q * a.nt + tl);
    if (a.recheck_s) {   // the boundary the window pass re-decides (NaN: none)
      const bool have = boundary && C >= Tsel;
      a.recheck_s[4 * slot] = have ? key_score(pout[P - 1]) : __int_as_float(0x7fc00000);
      a.recheck_s[4 * slot + 1] = have ? key_score(pout[P]) : __int_as_float(0x7fc00000);
      // each hash's largest abs(p) (its first list entry)
      a.recheck_s[4 * slot + 2] = signed_entry(lists, 0, D).v;
      a.recheck_s[4 * slot + 3] = signed_entry(lists + LIST_CAP, 0, D).v;
    }
  }
}

// Argmax pass of the one-piece BF16 query projections (argmax_only): each
// hash's winner (the query's own bucket) is made exact, the rest of the
// ranking keeps the BF16 values.  A winner is certain when its BF16 lead
// over the runner-up exceeds twice the window eps = gammaf |q| max|r| (plus
// the list truncation) and its value exceeds eps (its sign); otherwise every
// entry whose BF16 value lies within that margin of the top is re-computed
// exactly (compensated dot products on the FP32 rows) and written back in
// place.  Entries left out have BF16 values below the top's by more than
// 2 eps, so exact values below the top entry's: the largest exact value is
// the winner.  List mode re-sorts the corrected list; a window that reaches
// past the list (its cut) re-computes all D entries and rebuilds the list.
constexpr int SMALL_E = 8;   // longest per-hash list of the projection epilogue

__device__ __forceinline__ float list_val(uint64_t k) {
  return k ? __uint_as_float((uint32_t)(k >> 32) - 1u) : 0.f;
}

__device__ __forceinline__ uint64_t exact_key(float v, uint32_t i, int D) {
  const uint32_t h = i + (v < 0.f ? (uint32_t)D : 0u);
  return ((uint64_t)(__float_as_uint(fabsf(v)) + 1u) << 32) | (uint64_t)(0xFFFFFFFFu - h);
}

// the warp's exact projection of query row qv onto random vector row (2t + j) D + i
__device__ __forceinline__ float exact_proj(const ProbeArgs& a, const float* qv, int t, int j,
                                            uint32_t i) {
  const float* rows[1] = {a.R + ((int64_t)(2 * t + j) * a.D + i) * a.ldr};
  FF v[1];
  warp_dot2_gather_ff<1>(qv, rows, (int)(a.ldr / 4), v);
  return v[0].hi;   // the exact value rounded to FP32
}

// List mode, first kernel, thread per (query, table): the certainty test of
// both hashes; an uncertain hash is listed as a pair (item, hash) for the
// second kernel, and an item whose window reaches past a list (its cut) is
// listed for the exact passes, which re-decide its whole probe set from all
// 2D projections.
__global__ void __launch_bounds__(256)
probe_argmax_test_kernel(ProbeArgs a) {
  const int D = a.D, EL = a.EL, LS = EL + 1;
  const int64_t nitems = a.mq * a.nt;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < nitems;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx / a.nt;
    const int t = a.tb + (int)(idx % a.nt);
    uint32_t bad = 0;
    bool past = false;
    for (int j = 0; j < 2; ++j) {
      const uint64_t* L = a.lists + (idx * 2 + j) * (int64_t)LS;
      const float v0 = list_val(L[0]), v1 = D > 1 ? list_val(L[1]) : 0.f;
      const float eps = a.gammaf * a.qnorm[q] * a.rmax[2 * t + j] + a.trunc * v0;
      const float need = (2.f * eps + 6.0e-8f * (v0 + v1)) * 1.001f + 1e-30f;
      if (v0 - v1 > need && v0 > eps * 1.001f) continue;
      bad |= 1u << j;
      if (list_val(L[EL]) >= v0 - need) past = true;
    }
    if (past) {
      a.recheck[atomicAdd(a.recheck_count, 1u)] = (uint32_t)idx;
      if (a.rechecks) atomicAdd(a.rechecks, 1ull);
    } else {
      for (int j = 0; j < 2; ++j)
        if ((bad >> j) & 1u) a.amax_pairs[atomicAdd(a.amax_count, 1u)] = (uint32_t)(idx * 2 + j);
    }
  }
}

// List mode, second kernel: four listed hashes per warp, eight lanes each.
// The window entries (a prefix of the sorted list) are re-computed exactly
// by the lane group (compensated dot products on the FP32 rows, float-float
// sums combined across the group) and the list is re-sorted.
__global__ void __launch_bounds__(256)
probe_argmax_fix_kernel(ProbeArgs a) {
  const int lane = threadIdx.x & 31, g = lane >> 3, gl = lane & 7;
  const unsigned gmask = 0xFFu << (g * 8);
  const int D = a.D, EL = a.EL, LS = EL + 1;
  const unsigned n = *a.amax_count;
  const int nf4 = (int)(a.ldr / 4);
  for (unsigned base = ((unsigned)blockIdx.x * 8 + (threadIdx.x >> 5)) * 4; base < n;
       base += (unsigned)gridDim.x * 32) {
    const unsigned pi = base + (unsigned)g;
    if (pi >= n) continue;   // the whole 8-lane group
    const uint32_t pair = a.amax_pairs[pi];
    const int64_t idx = pair >> 1;
    const int j = (int)(pair & 1u);
    const int64_t q = idx / a.nt;
    const int t = a.tb + (int)(idx % a.nt);
    uint64_t* L = const_cast<uint64_t*>(a.lists) + (idx * 2 + j) * (int64_t)LS;
    const float v0 = list_val(L[0]), v1 = D > 1 ? list_val(L[1]) : 0.f;
    const float eps = a.gammaf * a.qnorm[q] * a.rmax[2 * t + j] + a.trunc * v0;
    const float need = (2.f * eps + 6.0e-8f * (v0 + v1)) * 1.001f + 1e-30f;
    const float thr = v0 - need;
    const float4* q4 = reinterpret_cast<const float4*>(a.Q + q * a.ldq);
    uint64_t keys[SMALL_E];
#pragma unroll
    for (int e = 0; e < SMALL_E; ++e) {
      keys[e] = e < EL ? L[e] : 0ull;
      if (e < EL && keys[e] && list_val(keys[e]) >= thr) {   // uniform over the group
        const uint32_t i = (0xFFFFFFFFu - (uint32_t)keys[e]) % (uint32_t)D;
        const float4* r4 = reinterpret_cast<const float4*>(
            a.R + ((int64_t)(2 * t + j) * D + i) * a.ldr);
        float p = 0.f, sc = 0.f;
        for (int c = gl; c < nf4; c += 8) {
          const float4 x = q4[c], y = __ldg(r4 + c);
          dot2_step(x.x, y.x, p, sc);
          dot2_step(x.y, y.y, p, sc);
          dot2_step(x.z, y.z, p, sc);
          dot2_step(x.w, y.w, p, sc);
        }
        FF v{p, sc};
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          FF w{__shfl_xor_sync(gmask, v.hi, o), __shfl_xor_sync(gmask, v.lo, o)};
          v = ff_add(v, w);
        }
        keys[e] = exact_key(ff_norm(v).hi, i, D);
      }
    }
    if (gl == 0) {
      // insertion sort, descending (EL <= 8)
#pragma unroll
      for (int e = 1; e < SMALL_E; ++e) {
#pragma unroll
        for (int f = SMALL_E - 1; f >= 1; --f) {
          if (f <= e && keys[f] > keys[f - 1]) {
            const uint64_t tv = keys[f];
            keys[f] = keys[f - 1];
            keys[f - 1] = tv;
          }
        }
      }
#pragma unroll
      for (int e = 0; e < SMALL_E; ++e)
        if (e < EL) L[e] = keys[e];
    }
  }
}

// Stored projections (D > 256 or long lists): warp per (query, table); the
// corrected values overwrite the projections the probe kernel then ranks.
__global__ void __launch_bounds__(256)
probe_argmax_rows_kernel(ProbeArgs a) {
  const int lane = threadIdx.x & 31;
  const int D = a.D;
  const int64_t nitems = a.mq * a.nt;
  const int64_t stride = (int64_t)gridDim.x * 8;
  for (int64_t it = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5); it < nitems; it += stride) {
    const int64_t q = it / a.nt;
    const int tl = (int)(it % a.nt);
    const int t = a.tb + tl;
    const float* qv = a.Q + q * a.ldq;
    for (int j = 0; j < 2; ++j) {
      float* row = const_cast<float*>(a.P) + q * a.ldp + (int64_t)(2 * tl + j) * D;
      // the two largest |p| of the row (ties: either; values only)
      float b0 = -1.f, b1 = -1.f;
      for (int i = lane; i < D; i += 32) {
        const float v = fabsf(row[i]);
        if (v > b0) { b1 = b0; b0 = v; } else if (v > b1) b1 = v;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float c0 = __shfl_xor_sync(FULL, b0, o), c1 = __shfl_xor_sync(FULL, b1, o);
        const float n0 = fmaxf(b0, c0);
        b1 = fmaxf(fminf(b0, c0), fmaxf(b1, c1));
        b0 = n0;
      }
      const float v0 = b0, v1 = D > 1 ? fmaxf(b1, 0.f) : 0.f;
      const float eps = a.gammaf * a.qnorm[q] * a.rmax[2 * t + j];
      const float need = (2.f * eps + 6.0e-8f * (v0 + v1)) * 1.001f + 1e-30f;
      if (v0 - v1 > need && v0 > eps * 1.001f) continue;   // uniform over the warp
      const float thr = v0 - need;
      for (int i0 = 0; i0 < D; i0 += 32) {
        const int i = i0 + lane;
        const bool cand = i < D && fabsf(row[i]) >= thr;
        unsigned cm = __ballot_sync(FULL, cand);
        while (cm) {
          const int src = __ffs(cm) - 1;
          cm &= cm - 1;
          const float v = exact_proj(a, qv, t, j, (uint32_t)(i0 + src));
          if (lane == src) row[i] = v;
        }
      }
      __syncwarp();
    }
  }
}

// Thread-per-(query, table) variant of the fast pass for small budgets in
// list mode (P + 1 <= EL <= 8): the same candidate pairs, selection and
// margin test on the SE = EL list entries per hash, held in registers (the
// loops are unrolled over SE, so a list of 2 costs 4 candidate pairs).

template <int SE>
__global__ void __launch_bounds__(256)
probe_small_kernel(ProbeArgs a) {
  __shared__ unsigned s_cnt, s_base;
  if (threadIdx.x == 0) s_cnt = 0u;
  __syncthreads();
  const int64_t idx0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = idx0 < a.mq * a.nt;
  const int64_t idx = live ? idx0 : 0;   // a dead thread works on item 0 and stores nothing
  const int64_t q = idx / a.nt;
  const int tl = (int)(idx % a.nt);
  const int t = a.tb + tl;
  const int D = a.D;
  const int P = a.probes_pq ? a.probes_pq[q] : a.probes;
  const int T = P + 1;
  const int E = T < D ? T : D;
  const int64_t NB = 4ll * D * D;
  float va[2][SE];
  uint32_t ha[2][SE];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint64_t* L = a.lists + (idx * 2 + j) * (int64_t)(a.EL + 1);
#pragma unroll
    for (int e = 0; e < SE; ++e) {
      const uint64_t k = e < E ? L[e] : 0ull;
      va[j][e] = __uint_as_float((uint32_t)(k >> 32) - 1u);
      ha[j][e] = 0xFFFFFFFFu - (uint32_t)k;
    }
  }
  // the best T pairs among (a+1)(b+1) <= T, kept sorted in registers
  uint64_t best[SE + 1];
#pragma unroll
  for (int e = 0; e <= SE; ++e) best[e] = 0ull;
  int C = 0;
#pragma unroll
  for (int x = 0; x < SE; ++x) {
#pragma unroll
    for (int y = 0; y < SE; ++y) {
      if (x < E && y < E && (x + 1) * (y + 1) <= T) {
        const uint32_t bucket = ha[0][x] * (uint32_t)(2 * D) + ha[1][y];
        uint64_t key = ((uint64_t)float_key(va[0][x] + va[1][y]) << 32) |
                       (uint64_t)(0xFFFFFFFFu - bucket);
        ++C;
#pragma unroll
        for (int e = 0; e <= SE; ++e) {
          const bool sw = key > best[e];
          const uint64_t tv = best[e];
          best[e] = sw ? key : tv;
          key = sw ? tv : key;
        }
      }
    }
  }
  const bool boundary = (int64_t)P < NB;
  bool certain = C >= (boundary ? P + 1 : P);
  if (a.argmax_only) {
    certain = C >= P;   // each hash's winner made exact by the argmax pass
  } else if (certain && boundary) {
    uint64_t kP = 0, kP1 = 0;
#pragma unroll
    for (int e = 0; e <= SE; ++e) {
      if (e == P - 1) kP = best[e];
      if (e == P) kP1 = best[e];
    }
    const float sP = key_score(kP), sP1 = key_score(kP1);
    // truncated list values: pair scores may be low by trunc (v1 + v2)
    const float eps = a.gammaf * a.qnorm[q] * (a.rmax[2 * t] + a.rmax[2 * t + 1]) +
                      a.trunc * (va[0][0] + va[1][0]);
    const float need = (2.f * eps + 6.0e-8f * (fabsf(sP) + fabsf(sP1))) * 1.001f + 1e-30f;
    certain = (sP - sP1) > need;
  }
  if (live && certain) {
    uint32_t* dst = a.out + idx * (int64_t)a.probes;
#pragma unroll
    for (int e = 0; e < SE; ++e)
      if (e < P) dst[e] = 0xFFFFFFFFu - (uint32_t)best[e];
  }
  // recheck slots: counted in shared memory, one global reservation per CTA
  const bool rc = live && !certain;
  const unsigned my = rc ? atomicAdd(&s_cnt, 1u) : 0u;
  __syncthreads();
  if (threadIdx.x == 0 && s_cnt) {
    s_base = atomicAdd(a.recheck_count, s_cnt);
    if (a.rechecks) atomicAdd(a.rechecks, (unsigned long long)s_cnt);
  }
  __syncthreads();
  if (rc) a.recheck[s_base + my] = (uint32_t)idx;
}

// ---------------------------------------------------------------- exact pass

constexpr int SLOW_PAIRS = 1024;

// Entries with float-float values (normalised pairs; see ff_before).
struct FEntry {
  FF v;
  uint32_t h;
  uint32_t pad;
};

__device__ __forceinline__ void warp_best_ff(FF& v, uint32_t& h) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const FF v2{__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)};
    const uint32_t h2 = __shfl_xor_sync(FULL, h, o);
    if (ff_before(v2, h2, v, h)) { v = v2; h = h2; }
  }
}


// Bitonic sort of N (a power of two) entries by ff_before, one warp.
__device__ __forceinline__ void warp_sort_fe(FEntry* a, int N) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < N; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const FEntry x = a[i], y = a[l];
          const bool first = (i & k) == 0;
          if (first ? ff_before(y.v, y.h, x.v, x.h) : ff_before(x.v, x.h, y.v, y.h)) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Bitonic sort of N (a power of two) entries by ff_before, the whole CTA.
__device__ __forceinline__ void block_sort_fe(FEntry* a, int N) {
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const FEntry x = a[i], y = a[l];
          const bool first = (i & k) == 0;
          if (first ? ff_before(y.v, y.h, x.v, x.h) : ff_before(x.v, x.h, y.v, y.h)) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Re-decides the probe set of one (query, table) from compensated
// projections dv[2D] (FP64-accurate float-float pairs), with the same ranking
// rule: the whole
// CTA sorts each hash's signed list (v desc, wedge asc), forms the pairs of
// the best E = min(P, 2D) entries of each list with (a+1)(b+1) <= P, and
// sorts them (score desc, bucket asc).  wsm holds 2 lists of pow2(2D) and
// the pairs, pow2(pair_count) entries.
__device__ void probe_exact_select(const FF* dv, int D, int P, FEntry* lists, FEntry* pairs,
                                   uint32_t* bucket_out) {
  const int W2 = 2 * D;
  const int NL = pow2_ceil(W2);
  const int E = P < W2 ? P : W2;
  const FEntry none{FF{-INFINITY, 0.f}, 0xFFFFFFFFu, 0};
  for (int j = 0; j < 2; ++j) {
    FEntry* L = lists + j * NL;
    for (int h = threadIdx.x; h < NL; h += blockDim.x) {
      if (h < W2) {
        const FF x = dv[j * D + (h < D ? h : h - D)];
        L[h] = FEntry{h < D ? x : FF{-x.hi, -x.lo}, (uint32_t)h, 0};
      } else {
        L[h] = none;
      }
    }
  }
  __syncthreads();
  block_sort_fe(lists, NL);
  block_sort_fe(lists + NL, NL);
  // pairs (a, b) with (a+1)(b+1) <= P: row a holds min(P / (a+1), E) of them
  int C = 0;
  for (int ai = 0; ai < E; ++ai) C += min(P / (ai + 1), E);
  const int NC = pow2_ceil(C > 1 ? C : 1);
  for (int idx = threadIdx.x; idx < NC; idx += blockDim.x) {
    if (idx < C) {
      int ai = 0, base = 0;
      while (base + min(P / (ai + 1), E) <= idx) { base += min(P / (ai + 1), E); ++ai; }
      const int bi = idx - base;
      const FEntry x = lists[ai], y = lists[NL + bi];
      pairs[idx] = FEntry{ff_sum(x.v, y.v), x.h * (uint32_t)W2 + y.h, 0};
    } else {
      pairs[idx] = none;
    }
  }
  __syncthreads();
  block_sort_fe(pairs, NC);
  for (int r = threadIdx.x; r < P; r += blockDim.x) bucket_out[r] = pairs[r].h;
  __syncthreads();
}

// Small budgets (P <= 16): the same selection by one warp, E rounds of warp
// maximum per list and P rounds over the pairs, all in float-float.
__device__ void probe_exact_select_warp(const FF* dv, int D, int P, unsigned char* wsm,
                                        uint32_t* bucket_out) {
  const int lane = threadIdx.x & 31;
  FEntry* top = reinterpret_cast<FEntry*>(wsm);                              // 2 x LIST_CAP
  FEntry* pairs = reinterpret_cast<FEntry*>(wsm + (size_t)2 * LIST_CAP * 16);  // SLOW_PAIRS
  const int W2 = 2 * D;
  const int E = P < W2 ? P : W2;
  const FF none{-INFINITY, 0.f};
  for (int j = 0; j < 2; ++j) {
    uint64_t taken = 0ull;  // bit s: wedge lane + 32 s already selected
    for (int r = 0; r < E; ++r) {
      FF bv = none;
      uint32_t bh = 0xFFFFFFFFu;
      for (int s = 0; s * 32 + lane < W2; ++s) {
        if (taken & (1ull << s)) continue;
        const uint32_t h = s * 32 + lane;
        const FF x = dv[j * D + (h < (uint32_t)D ? h : h - D)];
        const FF v = h < (uint32_t)D ? x : FF{-x.hi, -x.lo};
        if (ff_before(v, h, bv, bh)) { bv = v; bh = h; }
      }
      warp_best_ff(bv, bh);
      if ((int)(bh & 31) == lane) taken |= 1ull << (bh >> 5);
      if (lane == 0) top[j * LIST_CAP + r] = FEntry{bv, bh, 0};
    }
  }
  __syncwarp();
  int C = 0;
  for (int ai = 0; ai < E; ++ai) {
    int nb = P / (ai + 1);
    if (nb > E) nb = E;
    if (nb <= 0) break;
    for (int b = lane; b < nb; b += 32) {
      const FEntry x = top[ai], y = top[LIST_CAP + b];
      pairs[C + b] = FEntry{ff_sum(x.v, y.v), x.h * (uint32_t)W2 + y.h, 0};
    }
    C += nb;
  }
  __syncwarp();
  unsigned taken = 0u;
  for (int r = 0; r < P; ++r) {
    FF bv = none;
    uint32_t bh = 0xFFFFFFFFu;
    int bs = -1;
    for (int s = 0; s * 32 + lane < C; ++s) {
      if (taken & (1u << s)) continue;
      const FEntry e = pairs[s * 32 + lane];
      if (ff_before(e.v, e.h, bv, bh)) { bv = e.v; bh = e.h; bs = s; }
    }
    // bucket ids of distinct pairs are distinct, so the owner lane is unique
    FF wv = bv;
    uint32_t wh = bh;
    warp_best_ff(wv, wh);
    if (bs >= 0 && bh == wh) taken |= 1u << bs;
    if (lane == 0) bucket_out[r] = wh;
  }
  __syncwarp();
}

// Compensated projections of query q on NR rows of R given by their global
// row index (2t + j) D + i; from the BF16 copy when R is on the BF16 grid
// (the same values in half the bytes).
template <int NR, bool RB>
__device__ __forceinline__ void proj_rows_ff(const ProbeArgs& a, const float* qv,
                                             const int64_t (&row)[NR], FF* out) {
  if (RB) {
    const uint16_t* rp[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) rp[k] = a.Rb + row[k] * a.ldrb;
    warp_dot2_gather_bf_ff<NR>(qv, rp, (int)a.ldq, out);
  } else {
    const float* rp[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) rp[k] = a.R + row[k] * a.ldr;
    warp_dot2_gather_ff<NR>(qv, rp, (int)(a.ldr / 4), out);
  }
}

// The full pass runs 1,024 threads per CTA (eight rows in flight per warp,
// 256 rows per pass) when the budget is small (P <= 16: one warp selects, the
// rows dominate an item's time); larger budgets spend most of an item in the
// CTA-wide sorts, which use 256 threads better, with four CTAs per SM.
constexpr int RECHECK_THREADS = 1024;
constexpr int RECHECK_THREADS_LARGE_P = 256;

// dv [2D] float-float pairs, two sorted signed lists of pow2(2D) entries, and the
// candidate pairs (at most P (1 + ln P) <= 1024 for P <= 128 ... bounded by
// pair_count(P, ...) <= SLOW_PAIRS)
__host__ __device__ inline size_t recheck_smem_bytes(int D) {
  const size_t lists = (size_t)2 * pow2_ceil(2 * D) * sizeof(FEntry);
  const size_t wtop = (size_t)2 * LIST_CAP * sizeof(FEntry);   // the one-warp selection
  return (size_t)8 * 2 * D + (lists > wtop ? lists : wtop) + (size_t)SLOW_PAIRS * sizeof(FEntry);
}

// One CTA per (query, table) item of the recheck list: its warps compute the
// 2D compensated projections (eight rows in flight per warp, coalesced
// float4 loads), then warp 0 re-decides the probe set.
template <bool RB, int NT>
__global__ void __launch_bounds__(NT)
probe_recheck_kernel(ProbeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = NT / 32;
  FF* dv = reinterpret_cast<FF*>(smem);
  unsigned char* wsm = smem + (size_t)8 * 2 * a.D;
  const bool after_window = a.lists || a.recheck_s;
  const unsigned cnt = after_window ? *a.recheck2_count : *a.recheck_count;
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.full_rechecks && cnt)
    atomicAdd(a.full_rechecks, (unsigned long long)cnt);
  const uint32_t* items = after_window ? a.recheck2 : a.recheck;
  const int rows = 2 * a.D;
  for (unsigned it = blockIdx.x; it < cnt; it += gridDim.x) {
    const uint32_t item = items[it];
    const int64_t q = item / a.nt;
    const int tl = (int)(item % a.nt);
    const int t = a.tb + tl;
    const int P = a.probes_pq ? a.probes_pq[q] : a.probes;
    const float* qv = a.Q + q * a.ldq;
    const int64_t r0 = (int64_t)2 * t * a.D;   // first row of the table
    for (int i0 = wid * 8; i0 < rows; i0 += nw * 8) {
      if (i0 + 8 <= rows) {
        FF v[8];
        int64_t row[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) row[k] = r0 + i0 + k;
        proj_rows_ff<8, RB>(a, qv, row, v);
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 8; ++k) dv[i0 + k] = v[k];
        }
      } else {
        for (int i = i0; i < rows; ++i) {
          FF v[1];
          const int64_t row[1] = {r0 + i};
          proj_rows_ff<1, RB>(a, qv, row, v);
          if (lane == 0) dv[i] = v[0];
        }
      }
    }
    __syncthreads();
    uint32_t* dst = a.out + (q * a.nt + tl) * (int64_t)a.probes;
    if (P <= 16) {
      if (wid == 0) probe_exact_select_warp(dv, a.D, P, wsm, dst);
      __syncthreads();
    } else {
      FEntry* lists = reinterpret_cast<FEntry*>(wsm);
      probe_exact_select(dv, a.D, P, lists, lists + 2 * pow2_ceil(2 * a.D), dst);
    }
  }
}

// Window pass (list mode): a (query, table) whose FP32 probe boundary was
// inside the error bound is usually settled by recomputing only the list
// entries that can still be among the P best of their hash.  For hash j with
// FP32 list values v_0 >= v_1 >= ..., every entry whose exact |q^T r| could
// reach the exact P-th largest has v >= v_{P-1} - 2 eps_j; if the largest
// value left out of the list (its cut) is already below that, all
// candidates are in the list.  Their
// compensated projections then decide the P best entries of each hash and
// the P best pairs exactly; otherwise the item goes to the full pass.
constexpr int WIN_MAX = 8;

struct WinShared {
  FF v[2][WIN_MAX];       // exact |q^T r| of each hash's candidates, best first
  uint32_t w[2][WIN_MAX]; // their signed wedges
};

template <bool RB>
__global__ void __launch_bounds__(256)
probe_window_kernel(ProbeArgs a) {
  __shared__ WinShared shm[8];
  const int lane = threadIdx.x & 31;
  WinShared& sh = shm[threadIdx.x >> 5];
  const unsigned cnt = *a.recheck_count;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  // lane 16 j + e holds list entry e of hash j (e <= EL <= 8)
  const int j = lane >> 4, e = lane & 15;
  for (unsigned it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < cnt; it += nwarps) {
    const uint32_t item = a.recheck[it];
    const int64_t q = item / a.nt;
    const int tl = (int)(item % a.nt);
    const int t = a.tb + tl;
    const int P = a.probes_pq ? a.probes_pq[q] : a.probes;
    const int D = a.D;
    if (P > a.EL || P > WIN_MAX) {
      if (lane == 0) a.recheck2[atomicAdd(a.recheck2_count, 1u)] = item;
      continue;
    }
    const uint64_t key =
        e <= a.EL ? a.lists[((q * a.nt + tl) * 2 + j) * (int64_t)(a.EL + 1) + e] : 0ull;
    const float v = key ? __uint_as_float((uint32_t)(key >> 32) - 1u) : -1.f;
    const float v0 = __shfl_sync(FULL, v, 16 * j);
    const float vP = __shfl_sync(FULL, v, 16 * j + P - 1);
    const float vcut = __shfl_sync(FULL, v, 16 * j + a.EL);   // largest |p| left out
    // FP32 error, plus the truncation of the list values (at most trunc times
    // the hash's largest value); the 1e-5 margins cover the roundings of
    // these FP32 expressions, and lim is lowered by one more ulp of vP
    const float eps = a.gammaf * a.qnorm[q] * a.rmax[2 * t + j] * 1.00001f +
                      a.trunc * fmaxf(v0, 0.f) * 1.00001f;
    const float lim = (vP - 2.f * eps) - 1.2e-7f * fabsf(vP) - 1e-30f;
    // every entry that can still be among the P best of its hash is in the list
    if (!__all_sync(FULL, vcut < lim)) {
      if (lane == 0) a.recheck2[atomicAdd(a.recheck2_count, 1u)] = item;
      continue;
    }
    const bool in = e < a.EL && e < WIN_MAX && key != 0ull && v >= lim;
    const unsigned mask = __ballot_sync(FULL, in);
    const int nc = __popc(mask);
    // exact projections of the candidates, four rows in flight per round
    const uint32_t h = 0xFFFFFFFFu - (uint32_t)key;
    FF ev{0.f, 0.f};
    const float* qv = a.Q + q * a.ldq;
    for (int g = 0; g < nc; g += 4) {
      int64_t rows[4];
      int src[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        src[k] = __fns(mask, 0, 1 + min(g + k, nc - 1));   // lane of candidate g + k
        const uint32_t hk = __shfl_sync(FULL, h, src[k]) % (uint32_t)D;
        rows[k] = (int64_t)(2 * t + (src[k] >> 4)) * D + hk;
      }
      FF out[4];
      proj_rows_ff<4, RB>(a, qv, rows, out);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (g + k < nc && lane == src[k]) ev = out[k];
    }
    // rank of each candidate within its hash by (|v| desc, wedge asc)
    const FF av = ff_abs(ev);
    const uint32_t wh = (h % (uint32_t)D) + (ev.hi < 0.f ? (uint32_t)D : 0u);
    int rank = 0;
    for (int o = 0; o < 16; ++o) {
      const int l2 = 16 * j + o;
      const FF av2{__shfl_sync(FULL, av.hi, l2), __shfl_sync(FULL, av.lo, l2)};
      const uint32_t wh2 = __shfl_sync(FULL, wh, l2);
      if (l2 != lane && ((mask >> l2) & 1u) && ff_before(av2, wh2, av, wh)) ++rank;
    }
    if (in) { sh.v[j][rank] = av; sh.w[j][rank] = wh; }
    __syncwarp();
    const int n0 = __popc(mask & 0xFFFFu), n1 = __popc(mask >> 16);
    // the candidate pairs (x, y), (x + 1)(y + 1) <= P: lane l takes pair l
    int x = 0, y = -1, base = 0;
    for (int xx = 0; xx < P && xx < n0; ++xx) {
      const int nb = min(P / (xx + 1), n1);
      if (lane >= base && lane < base + nb) { x = xx; y = lane - base; }
      base += nb;
    }
    const bool has = y >= 0;
    const FF ps = has ? ff_sum(sh.v[0][x], sh.v[1][y]) : FF{-1.f, 0.f};
    const uint32_t pb = has ? sh.w[0][x] * (uint32_t)(2 * D) + sh.w[1][y] : 0xFFFFFFFFu;
    int prank = 0;
    for (int l2 = 0; l2 < base; ++l2) {
      const FF ps2{__shfl_sync(FULL, ps.hi, l2), __shfl_sync(FULL, ps.lo, l2)};
      const uint32_t pb2 = __shfl_sync(FULL, pb, l2);
      if (l2 != lane && ff_before(ps2, pb2, ps, pb)) ++prank;
    }
    if (has && prank < P) a.out[(q * a.nt + tl) * (int64_t)a.probes + prank] = pb;
    __syncwarp();
  }
}

// Pair-window pass (stored projections): a (query, table) whose FP32 probe
// boundary sP (P-th pair score) / sP1 ((P+1)-th) was inside the error bound
// is settled from exact values of only the pairs near the boundary.  With
// every FP32 pair score within delta of the exact one, a pair scoring above
// sP1 + 2 delta is in the exact top-P, a pair below sP - 2 delta is out, and
// the top-P is those above plus the best of the window pairs in between by
// exact score.  Every pair scoring at least tau = sP - 2 delta has both
// entries at least tau minus the other list's maximum, so the candidate
// entries of each list are found by a scan; their pairs are classified, and
// the entries of window pairs get compensated (FP64-accurate) values.  An
// item with more than 32 candidate entries in a list or 64 window pairs goes
// to the full pass.
constexpr int PW_CAND = 32;
constexpr int PW_WIN = 64;

struct PWinShared {
  uint32_t ch[2][PW_CAND];
  float cv[2][PW_CAND];
  FF ev[2][PW_CAND];           // signed exact values (normalised float-float)
  uint32_t need[2];            // bit c: candidate c is in a window pair
  uint16_t wa[PW_WIN], wb[PW_WIN];
  FEntry ws[PW_WIN];
  unsigned nwin, nin;
};

template <bool RB>
__global__ void __launch_bounds__(256)
probe_pwin_kernel(ProbeArgs a) {
  __shared__ PWinShared shm[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  PWinShared& sh = shm[wid];
  const unsigned cnt = *a.recheck_count;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (unsigned it = blockIdx.x * (blockDim.x >> 5) + wid; it < cnt; it += nwarps) {
    const uint32_t item = a.recheck[it];
    const int64_t q = item / a.nt;
    const int tl = (int)(item % a.nt);
    const int t = a.tb + tl;
    const int P = a.probes_pq ? a.probes_pq[q] : a.probes;
    const int D = a.D;
    const float4 rs = reinterpret_cast<const float4*>(a.recheck_s)[it];
    const float sP = rs.x, sP1 = rs.y;
    auto give_up = [&]() {
      if (lane == 0) a.recheck2[atomicAdd(a.recheck2_count, 1u)] = item;
    };
    if (isnan(sP) || isnan(sP1)) { give_up(); continue; }
    const float* pr[2] = {a.P + q * a.ldp + (int64_t)(2 * tl) * D,
                          a.P + q * a.ldp + (int64_t)(2 * tl + 1) * D};
    const float vmax[2] = {rs.z, rs.w};   // each hash's largest abs(p), from the fast pass
    // per-pair bound: the projections' error plus the rounding of the FP32
    // sum (every pair score is at most vmax[0] + vmax[1] in magnitude)
    const float eps = a.gammaf * a.qnorm[q] * (a.rmax[2 * t] + a.rmax[2 * t + 1]);
    const float delta = (eps + 6.0e-8f * (vmax[0] + vmax[1] + fabsf(sP) + fabsf(sP1))) * 1.001f + 1e-30f;
    const float tau = sP - 2.f * delta, hi = sP1 + 2.f * delta;
    // candidate entries (signed wedges h in [0, 2D)) of each list: every
    // value p_i gives the wedges i (value p_i) and i + D (value -p_i); the
    // values are read eight per lane at a time
    int nc[2] = {0, 0};
    bool over = false;
    const unsigned lt = (1u << lane) - 1u;
    for (int j = 0; j < 2 && !over; ++j) {
      const float lim = (tau - vmax[1 - j]) - 1e-6f * (fabsf(tau) + vmax[1 - j]);
      for (int i0 = 0; i0 < D; i0 += 256) {
        float pv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * 32 + lane;
          pv[u] = i < D ? pr[j][i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int i = i0 + u * 32 + lane;
          const bool ok = i < D;
#pragma unroll
          for (int sg = 0; sg < 2; ++sg) {
            const float v = sg ? -pv[u] : pv[u];
            const bool in = ok && v >= lim;
            const unsigned m = __ballot_sync(FULL, in);
            if (in) {
              const int slot = nc[j] + __popc(m & lt);
              if (slot < PW_CAND) {
                sh.ch[j][slot] = (uint32_t)(i + (sg ? D : 0));
                sh.cv[j][slot] = v;
              }
            }
            nc[j] += __popc(m);
          }
        }
      }
      if (nc[j] > PW_CAND) over = true;
    }
    if (over) { give_up(); continue; }
    if (lane == 0) { sh.nwin = 0; sh.nin = 0; sh.need[0] = sh.need[1] = 0u; }
    __syncwarp();
    // classify the pairs of candidates: lane x takes list-1 candidate x
    if (lane < nc[0]) {
      const float x = sh.cv[0][lane];
      unsigned nin = 0;
      for (int y = 0; y < nc[1]; ++y) {
        const float s2 = x + sh.cv[1][y];   // the fast pass's FP32 pair score
        if (s2 > hi) {
          ++nin;
        } else if (s2 >= tau) {
          const unsigned w = atomicAdd(&sh.nwin, 1u);
          if (w < PW_WIN) { sh.wa[w] = (uint16_t)lane; sh.wb[w] = (uint16_t)y; }
          atomicOr(&sh.need[0], 1u << lane);
          atomicOr(&sh.need[1], 1u << y);
        }
      }
      atomicAdd(&sh.nin, nin);
    }
    __syncwarp();
    const unsigned nwin = sh.nwin, nin = sh.nin;
    if (nwin > (unsigned)PW_WIN || nin > (unsigned)P || nin + nwin < (unsigned)P) {
      give_up();
      continue;
    }
    // compensated values of the candidates in window pairs
    const float* qv = a.Q + q * a.ldq;
    for (int j = 0; j < 2; ++j) {
      const unsigned need = sh.need[j];
      for (int c0 = 0; c0 < nc[j]; c0 += 8) {
        int64_t rows[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = min(c0 + u, nc[j] - 1);
          rows[u] = (int64_t)(2 * t + j) * D + (sh.ch[j][c] % (uint32_t)D);
        }
        if (!(need >> c0 & 0xFFu)) continue;
        FF v[8];
        proj_rows_ff<8, RB>(a, qv, rows, v);
        if (lane == 0)
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (c0 + u < nc[j])
              sh.ev[j][c0 + u] = sh.ch[j][c0 + u] < (uint32_t)D ? v[u] : FF{-v[u].hi, -v[u].lo};
      }
    }
    __syncwarp();
    // exact window pair scores, best first (score desc, bucket asc)
    const int NW = 64;
    for (int w = lane; w < NW; w += 32) {
      if (w < (int)nwin) {
        const int x = sh.wa[w], y = sh.wb[w];
        sh.ws[w] = FEntry{ff_sum(sh.ev[0][x], sh.ev[1][y]),
                          sh.ch[0][x] * (uint32_t)(2 * D) + sh.ch[1][y], 0};
      } else {
        sh.ws[w] = FEntry{FF{-INFINITY, 0.f}, 0xFFFFFFFFu, 0};
      }
    }
    __syncwarp();
    warp_sort_fe(sh.ws, NW);
    // output: the certain pairs, then the best P - nin window pairs
    uint32_t* dst = a.out + (q * a.nt + tl) * (int64_t)a.probes;
    if (lane == 0) sh.nin = 0;
    __syncwarp();
    if (lane < nc[0]) {
      const float x = sh.cv[0][lane];
      for (int y = 0; y < nc[1]; ++y)
        if (x + sh.cv[1][y] > hi) {
          const unsigned o = atomicAdd(&sh.nin, 1u);
          dst[o] = sh.ch[0][lane] * (uint32_t)(2 * D) + sh.ch[1][y];
        }
    }
    __syncwarp();
    for (int w = lane; w < P - (int)nin; w += 32) dst[nin + w] = sh.ws[w].h;
    __syncwarp();
  }
}

// Global probe budget (qProbes, Sections 2.2 and 4), one CTA per query:
// the FP32 pair scores of every table's top-P buckets are sorted (score
// desc, then table and bucket asc); when the Qp-th and (Qp+1)-th scores are
// closer than twice the per-pair error bound delta, the pairs in the window
// [s_Qp - 2 delta, s_Qp+1 + 2 delta] are re-scored from compensated
// projections and ranked exactly.  The selected buckets of each table are
// written to the front of its slots, the other slots are marked empty.
constexpr int GP_THREADS = 256;
constexpr int GP_WIN = 64;

__device__ __forceinline__ float pair_value_fp32(const ProbeArgs& a, int64_t q, int tl, uint32_t h,
                                                 int j) {
  const int D = a.D;
  const uint32_t i = h % (uint32_t)D;
  float p;
  if (a.P) {
    p = a.P[q * a.ldp + (int64_t)(2 * tl + j) * D + i];
  } else {
    // list mode: the entry of wedge h is normally among the hash's EL best
    // keys; one the exact pass took from outside the list is projected here
    // (a sequential FP32 dot product: error below gamma |q| |r|)
    const uint64_t* L = a.lists + ((q * a.nt + tl) * 2 + j) * (int64_t)(a.EL + 1);
    bool found = false;
    p = 0.f;
    for (int e = 0; e < a.EL; ++e) {
      const uint64_t k = L[e];
      if (k && (0xFFFFFFFFu - (uint32_t)k) % (uint32_t)D == i) {
        const float v = __uint_as_float((uint32_t)(k >> 32) - 1u);
        p = (0xFFFFFFFFu - (uint32_t)k) < (uint32_t)D ? v : -v;
        found = true;
        break;
      }
    }
    if (!found) {
      const float* qv = a.Q + q * a.ldq;
      const float* rv = a.R + ((int64_t)(2 * (a.tb + tl) + j) * D + i) * a.ldr;
      for (int c = 0; c < a.d; ++c) p = fmaf(qv[c], rv[c], p);
    }
  }
  return h < (uint32_t)D ? p : -p;
}

__global__ void __launch_bounds__(GP_THREADS)
global_probes_kernel(ProbeArgs a, int Qp, int npow2) {
  extern __shared__ __align__(16) uint64_t keys[];   // [npow2]
  __shared__ SD win[GP_WIN];
  __shared__ int s_cnt[1];
  __shared__ float s_sQ, s_sQ1;
  const int tid = threadIdx.x;
  const int64_t q = blockIdx.x;
  const int P = a.probes;
  const int N = a.nt * P;
  const int64_t NB = 4ll * a.D * a.D;
  const uint32_t* src = a.out + q * a.nt * (int64_t)P;
  for (int e = tid; e < npow2; e += GP_THREADS) {
    uint64_t key = 0ull;
    if (e < N) {
      const int tl = e / P;
      const uint32_t b = src[e];
      const uint32_t h1 = b / (uint32_t)(2 * a.D), h2 = b % (uint32_t)(2 * a.D);
      const float f = pair_value_fp32(a, q, tl, h1, 0) + pair_value_fp32(a, q, tl, h2, 1);
      key = ((uint64_t)float_key(f) << 32) | (uint64_t)(0xFFFFFFFFu - (uint32_t)(tl * NB + b));
    }
    keys[e] = key;
  }
  __syncthreads();
  block_sort_desc(keys, npow2);
  const int Qe = min(Qp, N);
  // the boundary and the window
  bool exact_ok = true;
  int lo = Qe, hi_i = Qe;   // window [lo, hi_i) in the sorted order
  if (tid == 0) { s_sQ = key_score(keys[Qe - 1]); s_sQ1 = Qe < N ? key_score(keys[Qe]) : -INFINITY; }
  __syncthreads();
  const float sQ = s_sQ, sQ1 = s_sQ1;
  if (Qe < N) {
    float rmx = 0.f;
    for (int t = 0; t < a.nt; ++t) rmx = fmaxf(rmx, a.rmax[2 * (a.tb + t)] + a.rmax[2 * (a.tb + t) + 1]);
    // truncated list values: a pair score (two non-negative list values)
    // may be low by trunc times itself, at most the largest pair score
    const float tr = a.P ? 0.f : a.trunc * fabsf(key_score(keys[0])) * 1.001f;
    const float eps = a.gammaf * a.qnorm[q] * rmx + tr;
    const float delta = (eps + 6.0e-8f * (fabsf(sQ) + fabsf(sQ1) + 2.f * eps)) * 1.001f + 1e-30f;
    if (sQ - sQ1 <= 2.f * delta) {
      // window: sorted positions whose score lies in [sQ - 2 delta, sQ1 + 2 delta]
      const float top = sQ1 + 2.f * delta, bot = sQ - 2.f * delta;
      if (tid == 0) {
        int l = Qe - 1;
        while (l > 0 && key_score(keys[l - 1]) <= top) --l;
        int h = Qe;
        while (h < N && key_score(keys[h]) >= bot) ++h;
        s_cnt[0] = (h - l <= GP_WIN) ? (l << 16 | (h - l)) : -1;
      }
      __syncthreads();
      if (s_cnt[0] < 0) {
        exact_ok = false;
      } else {
        lo = s_cnt[0] >> 16;
        hi_i = lo + (s_cnt[0] & 0xFFFF);
        // compensated pair scores of the window, one warp per pair
        const int lane = tid & 31, wid = tid >> 5;
        const float* qv = a.Q + q * a.ldq;
        const int nf4 = (int)(a.ldr / 4);
        for (int w = wid; w < hi_i - lo; w += GP_THREADS / 32) {
          const uint32_t code = 0xFFFFFFFFu - (uint32_t)keys[lo + w];
          const int tl = (int)(code / NB);
          const uint32_t b = code - (uint32_t)(tl * NB);
          const uint32_t h1 = b / (uint32_t)(2 * a.D), h2 = b % (uint32_t)(2 * a.D);
          const int t = a.tb + tl;
          const float* rows[2] = {a.R + ((int64_t)(2 * t) * a.D + h1 % (uint32_t)a.D) * a.ldr,
                                  a.R + ((int64_t)(2 * t + 1) * a.D + h2 % (uint32_t)a.D) * a.ldr};
          double v[2];
          warp_dot2_gather<2>(qv, rows, nf4, v);
          if (lane == 0) {
            const double f = (h1 < (uint32_t)a.D ? v[0] : -v[0]) + (h2 < (uint32_t)a.D ? v[1] : -v[1]);
            win[w] = SD{f, code, 0};
          }
        }
        for (int w = tid; w < GP_WIN; w += GP_THREADS)
          if (w >= hi_i - lo) win[w] = SD{-INFINITY, 0xFFFFFFFFu, 0};
        __syncthreads();
        block_sort_sd(win, GP_WIN);
      }
    }
  }
  // write: the first lo sorted pairs, then Qe - lo window pairs by exact rank
  uint32_t* dst = a.out + q * a.nt * (int64_t)P;
  __shared__ int s_tcount[1];
  // per table fill counters live at the end of the key array
  int* tcount = reinterpret_cast<int*>(keys + npow2);
  if (!exact_ok) lo = Qe;   // no exact window: keep the FP32 ranking (flagged below)
  __syncthreads();
  // stage the chosen codes in keys[npow2 - Qe ..] is unsafe; copy first
  for (int t = tid; t < a.nt; t += GP_THREADS) tcount[t] = 0;
  __syncthreads();
  uint32_t* chosen = reinterpret_cast<uint32_t*>(tcount + a.nt);
  for (int e = tid; e < Qe; e += GP_THREADS)
    chosen[e] = e < lo ? 0xFFFFFFFFu - (uint32_t)keys[e] : win[e - lo].id;
  __syncthreads();
  for (int e = tid; e < N; e += GP_THREADS) dst[e] = PROBE_EMPTY;
  __syncthreads();
  for (int e = tid; e < Qe; e += GP_THREADS) {
    const uint32_t code = chosen[e];
    const int tl = (int)(code / NB);
    const int slot = atomicAdd(&tcount[tl], 1);
    dst[tl * P + slot] = code - (uint32_t)(tl * NB);
  }
  if (tid == 0 && !exact_ok && a.rechecks) atomicAdd(a.rechecks + 1, 1ull);
  // The per-table offer of P pairs can only change the selection when a
  // table gave all of them: if the uncapped selection held a pair of table t
  // ranked below t's P offered ones, fewer than Qp pairs precede it, so all P
  // offered pairs of t are selected here too.  Such queries are reported.
  if (a.gcap_flag && (int64_t)P < min((int64_t)Qp, NB)) {
    if (tid == 0) s_tcount[0] = 0;
    __syncthreads();
    for (int t = tid; t < a.nt; t += GP_THREADS)
      if (tcount[t] >= P) s_tcount[0] = 1;
    __syncthreads();
    if (tid == 0 && s_tcount[0]) atomicAdd(a.gcap_flag, 1ull);
  }
}

// SimHash signature bits (Section 4: the signatures reuse the index's
// random projections).  One thread per (row, 32-bit word); a bit whose FP32
// projection lies inside the error bound is taken from a compensated dot
// product, so every bit is the sign of the exact projection (0 counts as +).
__global__ void __launch_bounds__(256)
sign_bits_kernel(SignArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.rows * a.words) return;
  const int64_t r = i / a.words;
  const int w = (int)(i - r * a.words);
  const float eps = (float)(a.gamma * (double)a.vnorm[r] * (double)a.rsig_max * 1.0001);
  const int nf4 = (int)(a.ldv / 4);
  uint32_t bits = 0;
  for (int b = 0; b < 32; ++b) {
    const int c = w * 32 + b;
    const float p = a.P[r * a.ldp + c];
    bool pos;
    if (fabsf(p) > eps) {
      pos = p >= 0.f;
    } else {
      pos = thread_dot2_f4(a.V + r * a.ldv, a.R + (int64_t)c * a.ldr, nf4) >= 0.0;
    }
    bits |= (pos ? 1u : 0u) << b;
  }
  a.out[r * a.words + w] = bits;
}

__global__ void query_norms_kernel(const float* __restrict__ Q, int64_t m, int64_t ldq, int d,
                                   float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= m) return;
  const float* x = Q + r * ldq;
  float s = 0.f;
  for (int i = lane; i < d; i += 32) s = fmaf(x[i], x[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  // the FP32 sum carries relative error <= gamma_d: inflate to an upper bound
  if (lane == 0) out[r] = sqrtf(s) * (1.f + 1e-4f + 2e-7f * d);
}

// ============================================================== gather + score
//
// Candidate gather, de-duplication and scoring run as separate kernels per
// query batch, so that the latency-bound part (walking buckets, hash-set
// inserts) and the bandwidth-bound part (streaming candidate rows) each get
// a launch shaped for them:
//  count_entries  warp per query: bucket entries E_q of its probed buckets;
//                 each CTA takes consecutive regions of E_q slots for its
//                 queries from one global counter;
//  dedup          CTA per query with E_q <= 16,384 (two sizes): walks the
//                 kept ids of its buckets, inserts them into a shared-memory
//                 hash set, writes the ids seen first to its region (grouped
//                 by row range) and appends work items of <= ITEM ids; larger
//                 queries are copied without de-duplication (flatten_kernel);
//  order          the work items sorted by the row range of their ids;
//  score          flat over work items: one row read per (query, candidate)
//                 with coalesced float4 loads, G lanes per row and 16 rows in
//                 flight per warp (FP32 scores, error <= gamma_d);
//  topk           warp per query: best k of its candidates by (score desc,
//                 id asc), with exact re-scoring of the boundary window.

constexpr int DW = 8;                           // warps per flatten CTA
constexpr int HS_SMALL = 4096;                  // hash slots of the small-query CTAs
constexpr int HS_BIG = 32768;                   // hash slots of the larger-query CTAs
constexpr int HMAX_SMALL = 3072;                // entries of the small-query tier (the distinct
                                                // ids, about 40% of them, fill a fraction of it)
constexpr int HMAX_BIG = HS_BIG / 2;            // larger queries are not de-duplicated
constexpr int HU = 8;                           // entry loads in flight per lane
constexpr int PCHUNK = 128;                     // probed buckets resolved per pass
constexpr int PPT = PCHUNK / 32;                // buckets per lane per pass
constexpr int EPT = 8;                          // entries per lane per round
constexpr int ITEM = 128;                       // candidates per score work item
// threads per score CTA: 128 threads (about 9k registers) still fit beside a
// projection CTA (320 x 168 registers) on its SM, so a pipelined call's
// scoring can run on SMs where the other call projects; 256 could not
constexpr int SCORE_T = 128;
constexpr int RANGE_MAX = SCORE_RANGE_MAX;      // row ranges of the grouped scoring

struct WarpWalk {
  const DedupArgs* a;
  int64_t q;
  int Pq, nprobe;
  int64_t NB;
  uint64_t* pbase;   // [PCHUNK] shared
  uint32_t* pstart;  // [PCHUNK + 1] shared
};

// Calls visit(id[EPT], has[EPT]) for every kept id of every probed bucket of
// the warp's query, EPT ids per lane per round (warp-collective).
template <class Visit>
__device__ __forceinline__ void warp_walk(const WarpWalk& w, Visit& visit) {
  const DedupArgs& a = *w.a;
  const int lane = threadIdx.x & 31;
  for (int pc0 = 0; pc0 < w.nprobe; pc0 += PCHUNK) {
    const int nc = min(PCHUNK, w.nprobe - pc0);
    uint32_t cnt[PPT];
    uint32_t tsum = 0;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      const int i = lane * PPT + r;
      uint32_t c = 0;
      if (i < nc) {
        const int pi = pc0 + i;
        const int tl = pi / w.Pq, p = pi - tl * w.Pq;
        const int t = a.tb + tl;
        const uint32_t b = a.probes[(w.q * a.nt + tl) * (int64_t)a.pstride + p];
        const uint32_t* off = a.offsets + (int64_t)t * (w.NB + 1);
        // empty slot: no bucket
        const bool live_b = b != PROBE_EMPTY && FPP_IN_BOUNDS(a.bd, b < (uint32_t)w.NB, 3, b);
        const uint32_t o0 = live_b ? off[b] : 0u;
        c = live_b ? off[b + 1] - o0 : 0u;
        w.pbase[i] = a.table_base[t] + o0;
      }
      cnt[r] = c;
      tsum += c;
    }
    uint32_t inc = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t2 = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc += t2;
    }
    const uint32_t total = __shfl_sync(FULL, inc, 31);
    uint32_t run = inc - tsum;
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      w.pstart[lane * PPT + r] = run;
      run += cnt[r];
    }
    __syncwarp();
    for (uint32_t e0 = 0; e0 < total; e0 += 32 * EPT) {
      uint32_t id[EPT];
      bool has[EPT];
#pragma unroll
      for (int r = 0; r < EPT; ++r) {
        const uint32_t e = e0 + r * 32 + lane;
        has[r] = e < total;
        id[r] = 0u;
        if (has[r]) {
          int lo = 0, hi = nc;   // last bucket whose start <= e (it is non-empty)
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (w.pstart[mid] <= e) lo = mid; else hi = mid;
          }
          const uint64_t gi = w.pbase[lo] + (e - w.pstart[lo]);
          id[r] = FPP_IN_BOUNDS(a.bd, gi < a.bd.kept, 8, gi) ? __ldg(a.ids + gi) : 0u;
        }
      }
      visit(id, has);
    }
    __syncwarp();
  }
}

// Appends query q's ceil(U / ITEM) score work items (at most ITEM candidates
// each) to the item list (one counter atomic per query, warp-collective).
__device__ __forceinline__ void write_items(const DedupArgs& a, int64_t q, uint64_t eo, uint32_t U) {
  if (a.no_items) return;
  const int lane = threadIdx.x & 31;
  const uint32_t nit = (U + ITEM - 1) / ITEM;
  unsigned base = 0;
  if (lane == 0 && nit) base = atomicAdd(a.nitems, nit);
  base = __shfl_sync(FULL, base, 0);
  for (uint32_t k = lane; k < nit; k += 32) {
    ScoreItem it;
    it.q = (uint32_t)q;
    it.len = min((uint32_t)ITEM, U - k * ITEM);
    it.start = eo + (uint64_t)k * ITEM;
    a.items[base + k] = it;
  }
}

__global__ void __launch_bounds__(256)
count_entries_kernel(DedupArgs a) {
  __shared__ uint32_t s_cnt[8];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 8 + wid;
  const bool live = q < a.mq;
  const int Pq = !live ? 0 : a.probes_pq ? a.probes_pq[q] : a.pstride;
  const int64_t NB = 4ll * a.D * a.D;
  const int nprobe = a.nt * Pq;
  uint32_t s = 0;
  // four probes per lane per pass: their bucket ids, then their offsets,
  // are loaded together
  for (int pi0 = 0; pi0 < nprobe; pi0 += 128) {
    uint32_t b[4];
    const uint32_t* off[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int pi = pi0 + r * 32 + lane;
      b[r] = PROBE_EMPTY;
      off[r] = a.offsets;
      if (pi < nprobe) {
        const int tl = pi / Pq, p = pi - tl * Pq;
        b[r] = a.probes[(q * a.nt + tl) * (int64_t)a.pstride + p];
        off[r] = a.offsets + (int64_t)(a.tb + tl) * (NB + 1);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (b[r] != PROBE_EMPTY && FPP_IN_BOUNDS(a.bd, b[r] < (uint32_t)NB, 1, b[r])) {
        const uint32_t o0 = off[r][b[r]], o1 = off[r][b[r] + 1];
        if (FPP_IN_BOUNDS(a.bd, o1 >= o0, 2, b[r])) s += o1 - o0;
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
  // the CTA's eight regions, consecutive, at a base taken from one global
  // counter (regions are not in query order; no scan over the batch)
  if (lane == 0) s_cnt[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < 8; ++w) tot += s_cnt[w];
    s_base = tot ? atomicAdd(a.region_total, tot) : 0ull;
  }
  __syncthreads();
  if (live && lane == 0) {
    unsigned long long off = s_base;
    for (int w = 0; w < wid; ++w) off += s_cnt[w];
    a.eoff[q] = off;
    a.ecount[q] = s;
    if (s == 0) a.ucount[q] = 0u;   // no tier kernel visits an empty query
    // queries above the small tier are listed for the kernels of their tier
    const int tier = s > (uint32_t)HMAX_BIG ? 1 : s > (uint32_t)HMAX_SMALL ? 0 : -1;
    if (tier >= 0) a.tierq[tier * a.mq + atomicAdd(a.tiern + tier, 1u)] = (uint32_t)q;
  }
}

// Under a.fused: whether a region reserved at eo for E slots ends within the
// candidate buffer.  If not, the query gets no candidates (its region is not
// written) and the overflow flag is raised; the caller repeats the call with
// a buffer sized from the exact total.  Sets eoff[q] either way.
__device__ __forceinline__ int region_fits(const DedupArgs& a, int64_t q, uint64_t eo, uint32_t E) {
  if (eo + E <= a.cap) {
    a.eoff[q] = eo;
    return 1;
  }
  a.eoff[q] = 0ull;
  a.ecount[q] = E;
  a.ucount[q] = 0u;
  atomicExch(a.overflow, 1ull);
  return 0;
}

// Queries with more than HMAX_BIG bucket entries keep every entry (no
// de-duplication): with that many probed buckets few ids repeat, and a
// repeated id only costs one more row read; the top-k kernel drops repeated
// (score, id) keys.  One warp per query copies its entries in bucket order.
__global__ void __launch_bounds__(DW * 32, 4)
flatten_kernel(DedupArgs a) {
  __shared__ uint64_t s_pbase[DW][PCHUNK];
  __shared__ uint32_t s_pstart[DW][PCHUNK + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t NB = 4ll * a.D * a.D;
  unsigned long long ent = 0, prb = 0;
  const int64_t nwarps = (int64_t)gridDim.x * DW;
  const int64_t nq = a.tiern[1];   // listed by count_entries
  if ((int64_t)blockIdx.x * DW >= nq) return;   // no listed query for this CTA
  for (int64_t i = (int64_t)blockIdx.x * DW + wid; i < nq; i += nwarps) {
    const int64_t q = a.tierq[a.mq + i];
    const uint64_t E = a.ecount[q];
    const int Pq = a.probes_pq ? a.probes_pq[q] : a.pstride;
    WarpWalk w{&a, q, Pq, a.nt * Pq, NB, s_pbase[wid], s_pstart[wid]};
    unsigned long long eo = 0;   // under a.fused the warp reserves its region of E slots
    if (a.fused) {
      int fits = 1;
      if (lane == 0) {
        eo = atomicAdd(a.region_total, (unsigned long long)E);
        fits = region_fits(a, q, eo, (uint32_t)E);
      }
      eo = __shfl_sync(FULL, eo, 0);
      if (!__shfl_sync(FULL, fits, 0)) continue;   // uniform over the warp
    } else {
      eo = a.eoff[q];
    }
    uint32_t* out = a.cand + eo;
    const uint32_t U = (uint32_t)E;
    // (not grouped by row range: its items are ordered by their first id)
    struct Copy {
      uint32_t* out; uint32_t n;
      __device__ void operator()(const uint32_t (&id)[EPT], const bool (&has)[EPT]) {
        // the valid entries of a round are a prefix of its 32 * EPT slots
        const int lane = threadIdx.x & 31;
        uint32_t valid = 0;
#pragma unroll
        for (int r = 0; r < EPT; ++r) {
          if (has[r]) out[n + r * 32 + lane] = id[r];
          valid += __popc(__ballot_sync(FULL, has[r]));
        }
        n += valid;
      }
    } cp{out, 0u};
    warp_walk(w, cp);
    if (lane == 0) {
      ent += E;
      prb += (unsigned long long)w.nprobe;
      a.ucount[q] = U;
    }
    write_items(a, q, eo, U);
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ent += __shfl_xor_sync(FULL, ent, o);
    prb += __shfl_xor_sync(FULL, prb, o);
  }
  if (lane == 0 && a.stats && ent) {
    atomicAdd(a.stats + 0, ent);
    atomicAdd(a.stats + 1, ent);
    atomicAdd(a.stats + 3, prb);
  }
}

// A query that the fused small tier does not de-duplicate itself: its entry
// count is recorded, an empty query gets no candidates, and the others are
// listed for the tier their count needs (the same rule as count_entries).
__device__ __forceinline__ void hand_off(const DedupArgs& a, int64_t q, uint32_t E) {
  a.ecount[q] = E;
  if (E == 0) {
    a.ucount[q] = 0u;
    a.eoff[q] = 0ull;
    return;
  }
  const int tier = E > (uint32_t)HMAX_BIG ? 1 : 0;
  a.tierq[tier * a.mq + atomicAdd(a.tiern + tier, 1u)] = (uint32_t)q;
}

// Entries of probed bucket pi of query q (0 for an empty probe slot).
__device__ __forceinline__ uint32_t probe_entries(const DedupArgs& a, int64_t q, int pi, int Pq,
                                                  int64_t NB) {
  const int tl = pi / Pq, p = pi - tl * Pq;
  const uint32_t bk = a.probes[(q * a.nt + tl) * (int64_t)a.pstride + p];
  if (bk == PROBE_EMPTY || !FPP_IN_BOUNDS(a.bd, bk < (uint32_t)NB, 1, bk)) return 0u;
  const uint32_t* off = a.offsets + (int64_t)(a.tb + tl) * (NB + 1);
  const uint32_t o0 = off[bk], o1 = off[bk + 1];
  return FPP_IN_BOUNDS(a.bd, o1 >= o0, 2, bk) ? o1 - o0 : 0u;
}

// De-duplication of the queries with (ELO, EHI] bucket entries, one CTA (NT
// threads) per query: an open-addressing hash set of HS ids in shared memory
// (linear probing, insertion by compare-and-swap, so exactly one thread sees
// an id as new), at most EHI / HS full and reset after each query.  TIER < 0
// visits every query; otherwise the queries listed for TIER.  The probed
// buckets are resolved NT at a time; each thread then walks a contiguous run
// of the entries, so the bucket of its next entry is found by stepping
// instead of searching.
//
// Regions: without a.fused, count_entries gave each query its region of E
// slots.  With a.fused there is no count_entries pass: the small tier
// (FUSE = 1) takes each query's entry count from its own resolution of the
// probed buckets (a first pass over them when they do not fit one chunk),
// hands the larger queries to the other tiers, and reserves each of its
// queries' regions of E slots with one atomic; the other tiers reserve
// theirs the same way.
constexpr uint32_t HEMPTY = 0xFFFFFFFFu;

// (1024 / NT CTAs per SM: eight 128-thread CTAs get 64 registers per thread
// and no spills; ten at 48 registers spilled and were 5% slower)
template <int NT, int HS, int LOG2HS, int ELO, int EHI, int TIER, int FUSE>
__global__ void __launch_bounds__(NT, 1024 / NT)
dedup_hash_kernel(DedupArgs a) {
  extern __shared__ __align__(16) uint32_t tab[];
  __shared__ uint64_t pbase[NT];
  __shared__ uint32_t pstart[NT + 1];
  __shared__ uint32_t wsum[NT / 32];
  __shared__ uint32_t s_n, s_base;
  __shared__ unsigned long long s_eb;
  __shared__ int s_fit;
  __shared__ uint32_t s_cnt[RANGE_MAX];   // a grouped query's per-range counts, then cursors
  const bool grouped = a.range_count > 1 && !a.no_items;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t nq = TIER < 0 ? a.mq : (int64_t)a.tiern[TIER];
  if (nq == 0) return;   // uniform over the CTA
  for (int i = tid; i < HS / 4; i += NT)
    reinterpret_cast<uint4*>(tab)[i] = make_uint4(HEMPTY, HEMPTY, HEMPTY, HEMPTY);
  for (int r = tid; r < RANGE_MAX; r += NT) s_cnt[r] = 0u;
  if (tid == 0) s_n = 0;
  __syncthreads();
  const int64_t NB = 4ll * a.D * a.D;
  unsigned long long ent = 0, uni = 0, prb = 0;
  for (int64_t qi = blockIdx.x; qi < nq; qi += gridDim.x) {
    const int64_t q = TIER < 0 ? qi : (int64_t)a.tierq[TIER * a.mq + qi];
    const int Pq = a.probes_pq ? a.probes_pq[q] : a.pstride;
    const int nprobe = a.nt * Pq;
    uint64_t E = 0;
    uint64_t eo = 0;      // start of the query's region
    if (FUSE) {
      if (nprobe > NT) {
        // the entries of every probed bucket first (the walk resolves them again)
        uint32_t s = 0;
        for (int pi = tid; pi < nprobe; pi += NT) s += probe_entries(a, q, pi, Pq, NB);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) wsum[wid] = s;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) E += wsum[w];
        const bool mine = E > (uint64_t)ELO && E <= (uint64_t)EHI;
        if (tid == 0) {
          if (mine) {
            s_eb = atomicAdd(a.region_total, (unsigned long long)E);
            s_fit = region_fits(a, q, s_eb, (uint32_t)E);
          } else {
            hand_off(a, q, (uint32_t)E);
          }
        }
        __syncthreads();   // wsum is rewritten below; s_eb and s_fit are read
        if (!mine || !s_fit) continue;   // uniform
        eo = s_eb;
      }
    } else {
      E = a.ecount[q];
      if (E > (uint64_t)EHI || E <= (uint64_t)ELO) continue;   // uniform over the CTA
      if (a.fused) {   // a larger tier under a.fused: its own region of E slots
        if (tid == 0) {
          s_eb = atomicAdd(a.region_total, (unsigned long long)E);
          s_fit = region_fits(a, q, s_eb, (uint32_t)E);
        }
        __syncthreads();
        if (!s_fit) {   // uniform; s_fit is rewritten for the next query only after this barrier
          __syncthreads();
          continue;
        }
        eo = s_eb;
      } else {
        eo = a.eoff[q];
      }
    }
    uint32_t* out = a.cand + eo;   // (a fused query of one chunk: set below)
    bool skip = false;
    for (int pc0 = 0; pc0 < nprobe; pc0 += NT) {
      const int nc = min(NT, nprobe - pc0);
      uint32_t c = 0;
      if (tid < nc) {
        const int pi = pc0 + tid;
        const int tl = pi / Pq, p = pi - tl * Pq;
        const int t = a.tb + tl;
        const uint32_t bk = a.probes[(q * a.nt + tl) * (int64_t)a.pstride + p];
        const uint32_t* off = a.offsets + (int64_t)t * (NB + 1);
        // empty slot: no bucket
        const bool live_b = bk != PROBE_EMPTY && FPP_IN_BOUNDS(a.bd, bk < (uint32_t)NB, 3, bk);
        const uint32_t o0 = live_b ? off[bk] : 0u;
        c = live_b ? off[bk + 1] - o0 : 0u;
        pbase[tid] = a.table_base[t] + o0;
      }
      // exclusive prefix sum of the bucket sizes over the CTA
      uint32_t inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t2 = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t2;
      }
      if (lane == 31) wsum[wid] = inc;
      __syncthreads();
      uint32_t woff = 0, total = 0;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) {
        const uint32_t v = wsum[w];
        woff += w < wid ? v : 0u;
        total += v;
      }
      if (FUSE && nprobe <= NT) {
        // one pass: the query's entry count is this chunk's
        E = total;
        if (E <= (uint64_t)ELO || E > (uint64_t)EHI) {   // uniform
          if (tid == 0) hand_off(a, q, (uint32_t)E);
          __syncthreads();   // wsum is rewritten by the next query
          skip = true;
          break;
        }
        if (tid == 0) {
          s_eb = atomicAdd(a.region_total, (unsigned long long)E);
          s_fit = region_fits(a, q, s_eb, (uint32_t)E);
        }
      }
      if (tid < nc) pstart[tid] = woff + inc - c;
      if (tid == 0) pstart[nc] = total;   // nc <= NT; entries past nc are never read
      __syncthreads();
      if (FUSE && nprobe <= NT) {
        if (!s_fit) {   // uniform: no region, no candidates
          skip = true;
          break;
        }
        eo = s_eb;
        out = a.cand + eo;
      }
      const uint32_t per = (total + NT - 1) / NT;
      uint32_t e = tid * per;
      const uint32_t eend = min(e + per, total);
      int bk = 0;
      if (e < eend) {
        int lo = 0, hi = nc;   // last bucket whose start is <= e
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (pstart[mid] <= e) lo = mid; else hi = mid;
        }
        bk = lo;
      }
      uint32_t bstart = pstart[bk], bnext = pstart[bk + 1];
      uint64_t bbase = pbase[bk];
      // the thread's next HU entries (has: the entry exists)
      auto walk = [&](uint32_t (&id)[HU], bool (&has)[HU]) {
#pragma unroll
        for (int u = 0; u < HU; ++u) {
          has[u] = e < eend;
          id[u] = 0u;
          if (has[u]) {
            while (e >= bnext) {   // step over finished (or empty) buckets
              ++bk;
              bstart = bnext;
              bnext = pstart[bk + 1];
              bbase = pbase[bk];
            }
            const uint64_t gi = bbase + (e - bstart);
            if (FPP_IN_BOUNDS(a.bd, gi < a.bd.kept, 4, gi)) id[u] = __ldg(a.ids + gi);
            else has[u] = false;
            if (!FPP_IN_BOUNDS(a.bd, id[u] < (uint64_t)a.bd.n, 5, id[u])) has[u] = false;
            ++e;
          }
        }
      };
      // insertion: every pending id tries its current slot each pass, all
      // HU compare-and-swaps in flight together; at load <= 1/4 a second
      // pass is rare (fresh: the id was not in the set)
      auto insert = [&](const uint32_t (&id)[HU], const bool (&has)[HU], bool (&fresh)[HU]) {
        uint32_t hp[HU];
        bool pend[HU];
#pragma unroll
        for (int u = 0; u < HU; ++u) {
          pend[u] = has[u];
          fresh[u] = false;
          hp[u] = (id[u] * 0x9E3779B1u) >> (32 - LOG2HS);
        }
        bool again = true;
        while (again) {
          again = false;
#pragma unroll
          for (int u = 0; u < HU; ++u) {
            if (pend[u]) {
              const uint32_t old = atomicCAS(tab + hp[u], HEMPTY, id[u]);
              if (old == HEMPTY) {
                fresh[u] = true;
                pend[u] = false;
              } else if (old == id[u]) {
                pend[u] = false;
              } else {
                hp[u] = (hp[u] + 1) & (HS - 1);
                again = true;
              }
            }
          }
        }
      };
      for (uint32_t it = 0; it < per; it += HU) {
        uint32_t id[HU];
        bool has[HU], fresh[HU];
        walk(id, has);
        insert(id, has, fresh);
        // the thread's new ids go to consecutive slots: one warp scan and
        // one shared-memory atomic per warp
        uint32_t nf = 0;
#pragma unroll
        for (int u = 0; u < HU; ++u) nf += fresh[u] ? 1u : 0u;
        uint32_t inc = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t2 = __shfl_up_sync(FULL, inc, o);
          if (lane >= o) inc += t2;
        }
        uint32_t wbase = 0;
        if (lane == 31 && inc) wbase = atomicAdd(&s_n, inc);
        wbase = __shfl_sync(FULL, wbase, 31);
        uint32_t pos = wbase + inc - nf;
#pragma unroll
        for (int u = 0; u < HU; ++u)
          if (fresh[u]) {
            if (FPP_IN_BOUNDS(a.bd, pos < E && eo + pos < a.bd.cap, 6, pos)) out[pos] = id[u];
            ++pos;
          }
      }
      __syncthreads();   // pbase / pstart are rewritten by the next chunk
    }
    if (skip) continue;   // uniform
    const uint32_t U = s_n;
    if (grouped) {
      // group the query's distinct ids by row range (id >> range_shift): the
      // ids are staged in the table's slots [0, U), counted per range in
      // s_cnt (zero between queries); the ranges' offsets (R + 1 of them) and
      // their items' offsets sit in the table's last 3 RANGE_MAX slots (U <=
      // 3/4 HS), and s_cnt then holds the cursors
      if (tid == 0) {
        ent += E;
        uni += U;
        prb += (unsigned long long)nprobe;
        a.ucount[q] = U;
        if (FUSE) a.ecount[q] = (uint32_t)E;
      }
      uint32_t* ro = tab + HS - 3 * RANGE_MAX;
      uint32_t* io = ro + RANGE_MAX + 1;
      const int R = a.range_count;
      for (uint32_t i = tid; i < U; i += NT) {
        const uint32_t id = out[i];
        tab[i] = id;
        atomicAdd(s_cnt + (id >> a.range_shift), 1u);
      }
      __syncthreads();
      if (wid == 0) {   // exclusive offsets of the ranges and of their items
        uint32_t carry = 0, icarry = 0;
        for (int r0 = 0; r0 < R; r0 += 32) {
          const int r = r0 + lane;
          const uint32_t c = r < R ? s_cnt[r] : 0u;
          const uint32_t ni = (c + ITEM - 1) / ITEM;
          uint32_t inc = c, iinc = ni;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t2 = __shfl_up_sync(FULL, inc, o);
            const uint32_t t3 = __shfl_up_sync(FULL, iinc, o);
            if (lane >= o) { inc += t2; iinc += t3; }
          }
          if (r < R) {
            ro[r] = carry + inc - c;
            io[r] = icarry + iinc - ni;
            s_cnt[r] = carry + inc - c;   // cursor
          }
          carry += __shfl_sync(FULL, inc, 31);
          icarry += __shfl_sync(FULL, iinc, 31);
        }
        if (lane == 0) {
          ro[R] = carry;
          s_base = icarry ? atomicAdd(a.nitems, icarry) : 0u;   // one reservation
        }
      }
      __syncthreads();
      for (int r = tid; r < R; r += NT) {
        const uint32_t c = ro[r + 1] - ro[r];
        const uint32_t nit = (c + ITEM - 1) / ITEM;
        for (uint32_t k = 0; k < nit; ++k) {
          ScoreItem itm;
          itm.q = (uint32_t)q;
          itm.len = min((uint32_t)ITEM, c - k * ITEM);
          itm.start = eo + ro[r] + (uint64_t)k * ITEM;
          a.items[s_base + io[r] + k] = itm;
        }
      }
      for (uint32_t i = tid; i < U; i += NT) {
        const uint32_t id = tab[i];
        out[atomicAdd(s_cnt + (id >> a.range_shift), 1u)] = id;
      }
      __syncthreads();
      for (int r = tid; r < R; r += NT) s_cnt[r] = 0u;   // for the next query
    } else {
      const uint32_t nit = a.no_items ? 0u : (U + ITEM - 1) / ITEM;
      if (tid == 0) {
        ent += E;
        uni += U;
        prb += (unsigned long long)nprobe;
        a.ucount[q] = U;
        if (FUSE) a.ecount[q] = (uint32_t)E;
        s_base = nit ? atomicAdd(a.nitems, nit) : 0u;
      }
      __syncthreads();
      for (uint32_t k = tid; k < nit; k += NT) {
        ScoreItem itm;
        itm.q = (uint32_t)q;
        itm.len = min((uint32_t)ITEM, U - k * ITEM);
        itm.start = eo + (uint64_t)k * ITEM;
        a.items[s_base + k] = itm;
      }
    }
    for (int i = tid; i < HS / 4; i += NT)
      reinterpret_cast<uint4*>(tab)[i] = make_uint4(HEMPTY, HEMPTY, HEMPTY, HEMPTY);
    if (tid == 0) s_n = 0;
    __syncthreads();
  }
  if (tid == 0 && a.stats) {
    atomicAdd(a.stats + 0, ent);
    atomicAdd(a.stats + 1, uni);
    atomicAdd(a.stats + 3, prb);
  }
}

// SimHash pre-ranking, warp per query (see SimArgs).
__global__ void __launch_bounds__(256)
simhash_filter_kernel(SimArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 8 + wid;
  if (q >= a.mq) return;
  uint64_t* buf = reinterpret_cast<uint64_t*>(smem) + (size_t)wid * a.cap;
  uint32_t* reg = a.cand + a.eoff[q];
  uint32_t U = a.ucount[q];
  if (U > (uint32_t)a.keep) {
    const uint32_t* qs = a.qsig + q * a.words;
    WarpTop wt;
    wt.init(buf, a.cap, a.keep);
    for (uint32_t i0 = 0; i0 < U; i0 += 32) {
      const uint32_t i = i0 + lane;
      const bool ok = i < U;
      uint64_t key = 0ull;
      if (ok) {
        const uint32_t id = reg[i];
        const uint32_t* xs = a.xsig + (int64_t)id * a.words;
        uint32_t h = 0;
        for (int w = 0; w < a.words; ++w) h += __popc(__ldg(xs + w) ^ __ldg(qs + w));
        // larger key = fewer differing bits, then lower id
        key = ((uint64_t)(0xFFFFFFFFu - h) << 32) | (uint64_t)(0xFFFFFFFFu - id);
      }
      wt.offer(ok, key);
    }
    const int nk = wt.finish();
    __syncwarp();
    for (int e = lane; e < nk; e += 32) reg[e] = 0xFFFFFFFFu - (uint32_t)buf[e];
    U = (uint32_t)nk;
    if (lane == 0) a.ucount[q] = U;
    __syncwarp();
  }
  const uint32_t nit = (U + ITEM - 1) / ITEM;
  unsigned base = 0;
  if (lane == 0 && nit) base = atomicAdd(a.nitems, nit);
  base = __shfl_sync(FULL, base, 0);
  for (uint32_t k = lane; k < nit; k += 32) {
    ScoreItem it;
    it.q = (uint32_t)q;
    it.len = min((uint32_t)ITEM, U - k * ITEM);
    it.start = a.eoff[q] + (uint64_t)k * ITEM;
    a.items[base + k] = it;
  }
}

// FP32 scores of the candidates of a work item: G lanes per row, each lane
// CPL float4 chunks of a row, U rows per lane group in flight (all U * CPL
// row loads of a step issued before any is used; ids are read per step,
// which measured faster than holding an item's ids in registers and
// shuffling them out).  The next item's header is fetched while the current
// one is scored.  Every score is within gamma_d ||q|| ||x|| of the exact
// inner product.  EXACT: G * CPL float4 chunks cover a row exactly.

template <int G, int CPL, bool EXACT>
__global__ void __launch_bounds__(SCORE_T)
score_kernel(ScoreArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nslots = (int64_t)*a.nitems;
  constexpr int RPP = 32 / G;
  constexpr int U = 4;
  const int sub = lane % G, grp = lane / G;
  const int nf4 = (int)(a.ldx / 4);
  int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  ScoreItem item = it < nslots ? a.items[it] : ScoreItem{0u, 0u, 0ull};
  for (; it < nslots; it += nw) {
    const ScoreItem nxt = it + nw < nslots ? a.items[it + nw] : ScoreItem{0u, 0u, 0ull};
    if (item.len == 0 ||
        !FPP_IN_BOUNDS(a.bd, item.start + item.len <= a.bd.cap, 9, item.start)) {
      item = nxt;
      continue;
    }
    const uint32_t* ids = a.cand + item.start;
    const float4* q4 = reinterpret_cast<const float4*>(a.Q + (int64_t)item.q * a.ldq);
    float* out = a.scores + item.start;
    for (int r0 = 0; r0 < (int)item.len; r0 += U * RPP) {
      uint32_t id[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = r0 + u * RPP + grp;
        ok[u] = (uint32_t)r < item.len;
        id[u] = ok[u] ? __ldcs(ids + r) : 0u;   // streamed: keep L2 for the rows
        ok[u] = ok[u] && FPP_IN_BOUNDS(a.bd, id[u] < (uint64_t)a.bd.n, 10, id[u]);
      }
      float p[U];
#pragma unroll
      for (int u = 0; u < U; ++u) p[u] = 0.f;
      for (int cb = 0; cb < nf4; cb += CPL * G) {   // a single pass when EXACT
        float4 x[U][CPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int ch = cb + sub + c * G;
            x[u][c] = (ok[u] && (EXACT || ch < nf4))
                          ? __ldg(reinterpret_cast<const float4*>(a.X + (int64_t)id[u] * a.ldx) + ch)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        float4 qq[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int ch = cb + sub + c * G;
          qq[c] = (EXACT || ch < nf4) ? __ldg(q4 + ch) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            p[u] = fmaf(x[u][c].x, qq[c].x, p[u]);
            p[u] = fmaf(x[u][c].y, qq[c].y, p[u]);
            p[u] = fmaf(x[u][c].z, qq[c].z, p[u]);
            p[u] = fmaf(x[u][c].w, qq[c].w, p[u]);
          }
        if (EXACT) break;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float f = p[u];
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) f += __shfl_xor_sync(FULL, f, o);
        if (ok[u] && sub == 0) __stcs(out + r0 + u * RPP + grp, f);
      }
    }
    item = nxt;
  }
}

// BF16 rows (precision path): the same structure, each chunk 8 BF16 values
// (16 bytes) against 8 FP32 query values, FP32 accumulation.
template <int G, int CPL, bool EXACT>
__global__ void __launch_bounds__(SCORE_T)
score_bf16_kernel(ScoreArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nslots = (int64_t)*a.nitems;
  constexpr int RPP = 32 / G;
  constexpr int U = 4;
  const int sub = lane % G, grp = lane / G;
  const int nch = (int)(a.ldxb / 8);
  const uint4* Xb = reinterpret_cast<const uint4*>(a.Xb);
  int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  ScoreItem item = it < nslots ? a.items[it] : ScoreItem{0u, 0u, 0ull};
  for (; it < nslots; it += nw) {
    const ScoreItem nxt = it + nw < nslots ? a.items[it + nw] : ScoreItem{0u, 0u, 0ull};
    if (item.len == 0 ||
        !FPP_IN_BOUNDS(a.bd, item.start + item.len <= a.bd.cap, 9, item.start)) {
      item = nxt;
      continue;
    }
    const uint32_t* ids = a.cand + item.start;
    const float4* q4 = reinterpret_cast<const float4*>(a.Q + (int64_t)item.q * a.ldq);
    float* out = a.scores + item.start;
    for (int r0 = 0; r0 < (int)item.len; r0 += U * RPP) {
      uint32_t id[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = r0 + u * RPP + grp;
        ok[u] = (uint32_t)r < item.len;
        id[u] = ok[u] ? __ldg(ids + r) : 0u;   // (a streaming hint here measured 30% slower)
        ok[u] = ok[u] && FPP_IN_BOUNDS(a.bd, id[u] < (uint64_t)a.bd.n, 10, id[u]);
      }
      float p[U];
#pragma unroll
      for (int u = 0; u < U; ++u) p[u] = 0.f;
      for (int cb = 0; cb < nch; cb += CPL * G) {
        uint4 x[U][CPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int ch = cb + sub + c * G;
            x[u][c] = (ok[u] && (EXACT || ch < nch)) ? __ldg(Xb + (int64_t)id[u] * (a.ldxb / 8) + ch)
                                                     : make_uint4(0u, 0u, 0u, 0u);
          }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int ch = cb + sub + c * G;
          const bool in = EXACT || ch < nch;
          const float4 qa = in ? __ldg(q4 + 2 * ch) : make_float4(0.f, 0.f, 0.f, 0.f);
          // the query row may end 4 floats before the padded BF16 row
          const bool inb = in && 8 * ch + 4 < a.ldq;
          const float4 qb = inb ? __ldg(q4 + 2 * ch + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x[u][c].x));
            const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x[u][c].y));
            const float2 f2 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x[u][c].z));
            const float2 f3 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x[u][c].w));
            p[u] = fmaf(f0.x, qa.x, p[u]); p[u] = fmaf(f0.y, qa.y, p[u]);
            p[u] = fmaf(f1.x, qa.z, p[u]); p[u] = fmaf(f1.y, qa.w, p[u]);
            p[u] = fmaf(f2.x, qb.x, p[u]); p[u] = fmaf(f2.y, qb.y, p[u]);
            p[u] = fmaf(f3.x, qb.z, p[u]); p[u] = fmaf(f3.y, qb.w, p[u]);
          }
        }
        if (EXACT) break;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float f = p[u];
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) f += __shfl_xor_sync(FULL, f, o);
        if (ok[u] && sub == 0) out[r0 + u * RPP + grp] = f;
      }
    }
    item = nxt;
  }
}

// FP8 e4m3 rows times a per-row scale: each 16-byte chunk holds 16 values,
// decoded in pairs to half precision (exact) and accumulated in FP32
// against the FP32 query; the row's scale multiplies the sum.
template <int G, int CPL, bool EXACT>
__global__ void __launch_bounds__(SCORE_T)
score_fp8_kernel(ScoreArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nslots = (int64_t)*a.nitems;
  constexpr int RPP = 32 / G;
  constexpr int U = 4;
  const int sub = lane % G, grp = lane / G;
  const int nch = (int)(a.ldxq / 16);
  const uint4* Xq = reinterpret_cast<const uint4*>(a.Xq);
  int64_t it = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  ScoreItem item = it < nslots ? a.items[it] : ScoreItem{0u, 0u, 0ull};
  for (; it < nslots; it += nw) {
    const ScoreItem nxt = it + nw < nslots ? a.items[it + nw] : ScoreItem{0u, 0u, 0ull};
    if (item.len == 0 ||
        !FPP_IN_BOUNDS(a.bd, item.start + item.len <= a.bd.cap, 9, item.start)) {
      item = nxt;
      continue;
    }
    const uint32_t* ids = a.cand + item.start;
    const float* qrow = a.Q + (int64_t)item.q * a.ldq;
    float* out = a.scores + item.start;
    for (int r0 = 0; r0 < (int)item.len; r0 += U * RPP) {
      uint32_t id[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = r0 + u * RPP + grp;
        ok[u] = (uint32_t)r < item.len;
        id[u] = ok[u] ? __ldg(ids + r) : 0u;
      }
      float p[U];
#pragma unroll
      for (int u = 0; u < U; ++u) p[u] = 0.f;
      for (int cb = 0; cb < nch; cb += CPL * G) {
        uint4 x[U][CPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int ch = cb + sub + c * G;
            x[u][c] = (ok[u] && (EXACT || ch < nch)) ? __ldg(Xq + (int64_t)id[u] * (a.ldxq / 16) + ch)
                                                     : make_uint4(0u, 0u, 0u, 0u);
          }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int ch = cb + sub + c * G;
          if (!(EXACT || ch < nch)) continue;
          // the 16 query values of the chunk (the query row is padded to 4;
          // values past it meet zero FP8 bytes)
          float qv[16];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int col = ch * 16 + v * 4;
            const float4 q4 = col < a.ldq ? __ldg(reinterpret_cast<const float4*>(qrow + col))
                                          : make_float4(0.f, 0.f, 0.f, 0.f);
            qv[4 * v] = q4.x; qv[4 * v + 1] = q4.y; qv[4 * v + 2] = q4.z; qv[4 * v + 3] = q4.w;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const uint32_t w[4] = {x[u][c].x, x[u][c].y, x[u][c].z, x[u][c].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const __half2_raw h0 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] & 0xFFFFu), __NV_E4M3);
              const __half2_raw h1 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] >> 16), __NV_E4M3);
              const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&h0));
              const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&h1));
              p[u] = fmaf(f0.x, qv[4 * k], p[u]);
              p[u] = fmaf(f0.y, qv[4 * k + 1], p[u]);
              p[u] = fmaf(f1.x, qv[4 * k + 2], p[u]);
              p[u] = fmaf(f1.y, qv[4 * k + 3], p[u]);
            }
          }
        }
        if (EXACT) break;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float f = p[u];
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) f += __shfl_xor_sync(FULL, f, o);
        if (ok[u] && sub == 0) out[r0 + u * RPP + grp] = f * __ldg(a.xscale + id[u]);
      }
    }
    item = nxt;
  }
}

// Best k candidates of each query by (score desc, id asc).  The first-pass
// scores pre-select the best K' = max(k + 16, kprime); the entries among them
// within twice the score error of the k-th are re-scored with the
// compensated dot product and sorted.  When that window reaches past the
// K'-th entry, every candidate in the window is re-scored (the slow path,
// rare).
constexpr int TK_SLOW = 2048;
constexpr int SEL_REGS = 16;   // candidates per lane of the register selection
constexpr int SEL_SLACK = 16;  // extra keys the selection threshold may keep

// Best kp of U <= 32 * NREG scored candidates by (score desc, id asc),
// sorted into buf[0..): the score keys sit in registers; a binary search over
// the 32-bit key finds the largest t with at least kp keys >= t, the keys >= t
// are compacted into buf and sorted.  Returns min(U, kp), or -1 when ties at
// t leave more than cap entries (the caller then uses the running buffer).
template <int NREG>
__device__ __forceinline__ int select_small(const float* sc, const uint32_t* cid, uint32_t U,
                                            int kp, uint64_t* buf, int cap) {
  const int lane = threadIdx.x & 31;
  uint32_t key[NREG];
#pragma unroll
  for (int j = 0; j < NREG; ++j) {
    const uint32_t i = (uint32_t)(j * 32 + lane);
    key[j] = i < U ? float_key(sc[i]) : 0u;   // 0: no entry (below every score key)
  }
  uint32_t t = 1u;
  if (U > (uint32_t)kp) {
    // count(key >= lo) >= kp holds throughout; stop early once a threshold
    // keeps at most kp + SEL_SLACK keys (the sort below orders them anyway)
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;
#pragma unroll
    for (int j = 0; j < NREG; ++j) {
      if (key[j]) kmin = min(kmin, key[j]);
      kmax = max(kmax, key[j]);
    }
    uint32_t lo = __reduce_min_sync(FULL, kmin), hi = __reduce_max_sync(FULL, kmax);
    if (kp <= 32) {
      // the 32 lane maxima are keys >= the smallest of them, so it keeps at
      // least kp keys; often it is already a threshold to stop at
      const uint32_t lm = __reduce_min_sync(FULL, kmax);
      if (lm > lo) {
        lo = lm;
        unsigned c = 0;
#pragma unroll
        for (int j = 0; j < NREG; ++j) c += key[j] >= lo ? 1u : 0u;
        if (__reduce_add_sync(FULL, c) <= (unsigned)(kp + SEL_SLACK)) hi = lo;
      }
    }
    while (lo < hi) {
      const uint32_t mid = lo + (hi - lo + 1u) / 2u;
      unsigned c = 0;
#pragma unroll
      for (int j = 0; j < NREG; ++j) c += key[j] >= mid ? 1u : 0u;
      c = __reduce_add_sync(FULL, c);
      if (c >= (unsigned)kp) {
        lo = mid;
        if (c <= (unsigned)(kp + SEL_SLACK)) break;
      } else {
        hi = mid - 1u;
      }
    }
    t = lo;
  }
  unsigned c = 0;
#pragma unroll
  for (int j = 0; j < NREG; ++j) c += key[j] >= t ? 1u : 0u;
  const unsigned total = __reduce_add_sync(FULL, c);
  if (total > (unsigned)cap) return -1;
  const unsigned lt = (1u << lane) - 1u;
  unsigned n = 0;
#pragma unroll
  for (int j = 0; j < NREG; ++j) {
    const bool take = key[j] >= t;
    const unsigned m = __ballot_sync(FULL, take);
    if (take) {
      const uint32_t i = (uint32_t)(j * 32 + lane);
      buf[n + __popc(m & lt)] = pack_key(sc[i], cid[i]);
    }
    n += __popc(m);
  }
  const int np2 = pow2_ceil(total > 1u ? (int)total : 1);
  for (int e = (int)total + lane; e < np2; e += 32) buf[e] = 0ull;
  __syncwarp();
  warp_sort_desc(buf, np2);
  return min((int)total, kp);
}

__global__ void __launch_bounds__(256)
topk_kernel(TopkArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 8 + wid;
  uint64_t* buf = reinterpret_cast<uint64_t*>(smem) + (size_t)wid * a.cap;
  SD* resc = reinterpret_cast<SD*>(smem + (size_t)8 * a.cap * 8) + (size_t)wid * a.rcap;
  FEntry* rf = reinterpret_cast<FEntry*>(resc);   // the same 16-byte slots
  if (q >= a.mq) return;
  const int kq = a.k_pq ? a.k_pq[q] : a.k;
  const int kp = max(kq + 16, a.kprime);   // the FP32 re-ranked shortlist
  const uint64_t start = a.eoff[q];
  const uint32_t U = FPP_IN_BOUNDS(a.bd, start + a.ucount[q] <= a.bd.cap, 11, q) ? a.ucount[q] : 0u;
  const float* sc = a.scores + start;
  const uint32_t* cid = a.cand + start;
  const float* qv = a.Q + q * a.ldq;
  const int nf4 = (int)(a.ldq / 4);
  int nk = -1;
  // the register selection with as few registers per lane as U needs
  if (U <= 128u) nk = select_small<4>(sc, cid, U, kp, buf, a.cap);
  else if (U <= 256u) nk = select_small<8>(sc, cid, U, kp, buf, a.cap);
  else if (U <= 384u) nk = select_small<12>(sc, cid, U, kp, buf, a.cap);
  else if (U <= 32u * SEL_REGS) nk = select_small<SEL_REGS>(sc, cid, U, kp, buf, a.cap);
  if (nk < 0) {   // many candidates (or heavy ties): running buffer with compaction
    WarpTop wt;
    wt.init(buf, a.cap, kp);
    for (uint32_t i0 = 0; i0 < U; i0 += 32) {
      const uint32_t i = i0 + lane;
      const bool ok = i < U;
      wt.offer(ok, ok ? pack_key(sc[i], cid[i]) : 0ull);
    }
    nk = wt.finish();
  }
  // Only entries whose first-pass score is within twice the score error of
  // the k-th first-pass score can be in the exact top-k (every entry below
  // that window is exactly below the k entries above it); the pre-selection
  // is sorted, so those entries are a prefix S of it.  If the window reaches
  // the end of the pre-selection while more candidates exist, the slow path
  // re-scores every candidate in the window.
  // FP32 arithmetic (the FP64 pipe is slow): the 1e-5 factors cover the
  // roundings of these products, and the threshold is lowered by one more
  // ulp of the k-th score, so the window can only grow
  const float qn = a.qnorm[q];
  const float eps_s = a.gammaf * qn * a.xmax * 1.00001f;
  const float du = 5.9604645e-08f * (float)(a.d + 8);
  const float delta = 4.f * du * du * qn * a.xmax * 1.00001f + 1e-30f;
  const int kk = min(kq, nk);
  const float kth = nk > 0 ? key_score(buf[kk - 1]) : 0.f;
  const float thr = nk > 0 ? (kth - 2.f * eps_s - 2.f * delta) - 1.2e-7f * fabsf(kth) - 1e-30f : 0.f;
  int ns = 0;   // |S|
  for (int e0 = 0; e0 < nk; e0 += 32) {
    const int e = e0 + lane;
    ns += __popc(__ballot_sync(FULL, e < nk && key_score(buf[e]) >= thr));
  }
  // a window reaching the end of the pre-selection while more candidates
  // exist sends the query to the slow path, except on the BF16 path, which
  // re-ranks its pre-selection (the best K' first-pass scores) and stops
  // there; the FP8 window is about sixteen times wider and keeps the slow path
  const bool slow = U > (uint32_t)nk && ns == nk && a.approx != 1;
  const int64_t orow = q * a.kmax;
  // exact (float-float) scores of n rows, G lanes per row (a power of two,
  // 32 / G rows per round): eight lanes per row for longer lists, so that
  // each row is read in 128-byte coalesced pieces
  const float4* q4 = reinterpret_cast<const float4*>(qv);
  auto rescore = [&](int n, auto id_of, auto put) {
    const int G = n > 8 ? 8 : 32 / pow2_ceil(n > 1 ? n : 1);
    const int rows_per_round = 32 / G;
    const int sub = lane % G;
    for (int r0 = 0; r0 < n; r0 += rows_per_round) {
      const int r = r0 + lane / G;
      const bool ok = r < n;
      const uint32_t id = id_of(ok ? r : 0);
      const float4* x4 = reinterpret_cast<const float4*>(a.X + (int64_t)id * a.ldx);
      float p = 0.f, sacc = 0.f;
      // four chunks of the lane's part of the row loaded before any is used
      // (zero chunks past the row add exact zeros)
      for (int c0 = sub; c0 < nf4; c0 += 4 * G) {
        float4 x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int c = c0 + u * G;
          x[u] = c < nf4 ? __ldg(x4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
          y[u] = c < nf4 ? __ldg(q4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          dot2_step(x[u].x, y[u].x, p, sacc);
          dot2_step(x[u].y, y[u].y, p, sacc);
          dot2_step(x[u].z, y[u].z, p, sacc);
          dot2_step(x[u].w, y[u].w, p, sacc);
        }
      }
      FF v{p, sacc};
      for (int o = G / 2; o > 0; o >>= 1) {
        FF w{__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)};
        v = ff_add(v, w);
      }
      if (ok && sub == 0) put(r, ff_norm(v), id);
    }
  };
  if (!slow) {
    // exact re-scoring of S
    rescore(ns, [&](int r) { return key_id(buf[r]); },
            [&](int r, FF v, uint32_t id) { rf[r] = FEntry{v, id, 0}; });
    const int np2 = pow2_ceil(ns > 1 ? ns : 1);
    for (int e = ns + lane; e < np2; e += 32) rf[e] = FEntry{FF{-INFINITY, 0.f}, 0xFFFFFFFFu, 0};
    __syncwarp();
    warp_sort_fe(rf, np2);
    // hi of a normalised pair is its sum rounded to FP32
    for (int e = lane; e < a.kmax; e += 32) {
      const bool ok = e < kq && e < ns;
      a.out_ids[orow + e] = ok ? (int64_t)rf[e].h : -1;
      a.out_scores[orow + e] = ok ? rf[e].v.hi : -INFINITY;
    }
    return;
  }
  // slow path: every candidate whose FP32 score may still reach the top-k
  if (lane == 0 && a.stats) atomicAdd(a.stats + 2, 1ull);
  FEntry* list = reinterpret_cast<FEntry*>(a.slow) + (int64_t)(blockIdx.x * 8 + wid) * TK_SLOW;
  unsigned nsl = 0;
  for (uint32_t i0 = 0; i0 < U; i0 += 32) {
    const uint32_t i = i0 + lane;
    const bool take = i < U && sc[i] >= thr;
    const unsigned m = __ballot_sync(FULL, take);
    if (take) {
      const unsigned slot = nsl + __popc(m & ((1u << lane) - 1u));
      if (slot < (unsigned)TK_SLOW) list[slot].h = cid[i];
    }
    nsl += __popc(m);
  }
  if (nsl > (unsigned)TK_SLOW) {
    // exact mode cannot guarantee the result; the BF16 path keeps the best
    // effort (the shortlist order is approximate there anyway)
    if (lane == 0 && a.err && !a.approx) atomicExch(a.err, 1);
    nsl = TK_SLOW;
  }
  __syncwarp();
  rescore((int)nsl, [&](int r) { return list[r].h; },
          [&](int r, FF v, uint32_t) { list[r].v = v; });
  const int np2 = pow2_ceil(nsl > 1 ? (int)nsl : 1);
  for (int e = (int)nsl + lane; e < np2; e += 32) list[e] = FEntry{FF{-INFINITY, 0.f}, 0xFFFFFFFFu, 0};
  __syncwarp();
  warp_sort_fe(list, np2);
  // a candidate listed twice (lists that were not de-duplicated) now sits
  // next to its copy: keep one of each
  int nd = 0;
  for (int i0 = 0; i0 < (int)nsl; i0 += 32) {
    const int i = i0 + lane;
    const FEntry v = i < (int)nsl ? list[i] : FEntry{FF{-INFINITY, 0.f}, 0xFFFFFFFFu, 0};
    const bool keep = i < (int)nsl && (i == 0 || list[i - 1].h != v.h);
    const unsigned m = __ballot_sync(FULL, keep);
    __syncwarp();
    if (keep) list[nd + __popc(m & ((1u << lane) - 1u))] = v;
    nd += __popc(m);
    __syncwarp();
  }
  for (int e = lane; e < a.kmax; e += 32) {
    const bool ok = e < kq && e < nd;
    a.out_ids[orow + e] = ok ? (int64_t)list[e].h : -1;
    a.out_scores[orow + e] = ok ? list[e].v.hi : -INFINITY;
  }
}

// ============================================================== dense top-k
//
// Exact top-k over a dense FP32 score row (brute-force search): the same
// FP32 pre-selection, compensated re-scoring and boundary check as above,
// with every column a candidate.
constexpr int TD_WARPS = 8;
constexpr int TD_SLOW = 2048;
constexpr int KSLACK = 16;

struct DenseLayout {
  int kp, cap, mcap, rcap;
  size_t q_off, wtop_off, merge_off, resc_off, total;
};

__host__ __device__ inline DenseLayout dense_layout(int kmax, int ldq) {
  DenseLayout L;
  L.kp = kmax + KSLACK;
  L.cap = pow2_ceil(2 * L.kp + 32);
  L.mcap = pow2_ceil(TD_WARPS * L.kp);
  L.rcap = pow2_ceil(L.kp);
  size_t o = 0;
  L.q_off = o; o += (size_t)4 * ldq; o = (o + 15) & ~(size_t)15;
  L.wtop_off = o; o += (size_t)TD_WARPS * L.cap * 8;
  L.merge_off = o;
  {
    size_t mb = (size_t)L.mcap * 8;
    if (mb < (size_t)TD_SLOW * 16) mb = (size_t)TD_SLOW * 16;
    o += mb;
  }
  L.resc_off = o; o += (size_t)L.rcap * 16;
  L.total = o;
  return L;
}

__global__ void __launch_bounds__(TD_WARPS * 32)
topk_dense_kernel(const float* __restrict__ S, int64_t lds, int64_t n, int k, const float* Q,
                  int64_t ldq, const float* __restrict__ X, int64_t ldx, int d, float xmax,
                  double gamma, int64_t* out_ids, float* out_scores, int kmax,
                  unsigned long long* rechecks, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned s_nslow;
  __shared__ int s_slow;
  __shared__ double s_thr64;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const DenseLayout Lo = dense_layout(kmax, (int)ldq);
  float* qs = reinterpret_cast<float*>(smem + Lo.q_off);
  uint64_t* wbuf = reinterpret_cast<uint64_t*>(smem + Lo.wtop_off) + (size_t)wid * Lo.cap;
  uint64_t* merge = reinterpret_cast<uint64_t*>(smem + Lo.merge_off);
  SD* slow = reinterpret_cast<SD*>(smem + Lo.merge_off);
  SD* resc = reinterpret_cast<SD*>(smem + Lo.resc_off);
  const int64_t q = blockIdx.x;
  const float* row = S + q * lds;
  for (int i = threadIdx.x; i < (int)ldq; i += blockDim.x) qs[i] = Q[q * ldq + i];
  if (threadIdx.x == 0) { s_nslow = 0; s_slow = 0; }
  __syncthreads();
  float ss = 0.f;
  for (int i = lane; i < d; i += 32) ss = fmaf(qs[i], qs[i], ss);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(FULL, ss, o);
  const double qn = (double)sqrtf(ss) * (1.0 + 1e-4 + 2e-7 * d);
  const double eps_s = gamma * qn * (double)xmax;
  const double du = 5.9604644775390625e-08 * (d + 8);
  const double delta = 4.0 * du * du * qn * (double)xmax + 1e-300;

  WarpTop wt;
  wt.init(wbuf, Lo.cap, Lo.kp);
  for (int64_t c0 = (int64_t)wid * 32; c0 < n; c0 += (int64_t)TD_WARPS * 32) {
    const int64_t c = c0 + lane;
    const bool ok = c < n;
    wt.offer(ok, ok ? pack_key(row[c], (uint32_t)c) : 0ull);
  }
  const int nw = wt.finish();
  for (int e = lane; e < Lo.kp; e += 32) merge[(size_t)wid * Lo.kp + e] = e < nw ? wbuf[e] : 0ull;
  __syncthreads();
  for (int e = TD_WARPS * Lo.kp + threadIdx.x; e < Lo.mcap; e += blockDim.x) merge[e] = 0ull;
  __syncthreads();
  block_sort_desc(merge, Lo.mcap);
  const int Kpp = (int)(n < (int64_t)Lo.kp ? n : (int64_t)Lo.kp);
  for (int e = wid; e < Kpp; e += TD_WARPS) {
    const uint32_t id = key_id(merge[e]);
    const double s = warp_dot2(qs, X + (int64_t)id * ldx, d);
    if (lane == 0) resc[e] = SD{s, id, 0};
  }
  for (int e = Kpp + threadIdx.x; e < Lo.rcap; e += blockDim.x) resc[e] = SD{-INFINITY, 0xFFFFFFFFu, 0};
  __syncthreads();
  if (wid == 0) warp_sort_sd(resc, Lo.rcap);
  __syncthreads();
  if (threadIdx.x == 0 && n > Kpp) {
    const double sK = (double)key_score(merge[Lo.kp - 1]);
    const double need = resc[k - 1].s;
    if (!(sK + eps_s + 2.0 * delta < need)) {
      s_slow = 1;
      s_thr64 = need - eps_s - 2.0 * delta;
      if (rechecks) atomicAdd(rechecks, 1ull);
    }
  }
  __syncthreads();
  const int64_t orow = q * kmax;
  if (!s_slow) {
    for (int e = threadIdx.x; e < kmax; e += blockDim.x) {
      const bool ok = e < k && e < Kpp;
      out_ids[orow + e] = ok ? (int64_t)resc[e].id : -1;
      out_scores[orow + e] = ok ? (float)resc[e].s : -INFINITY;
    }
    return;
  }
  const double thr64 = s_thr64;
  __syncthreads();
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    if ((double)row[c] >= thr64) {
      const unsigned slot = atomicAdd(&s_nslow, 1u);
      if (slot < (unsigned)TD_SLOW) slow[slot].id = (uint32_t)c;
      else if (err) atomicExch(err, 1);
    }
  }
  __syncthreads();
  const int ns = (int)(s_nslow < (unsigned)TD_SLOW ? s_nslow : (unsigned)TD_SLOW);
  for (int e = wid; e < ns; e += TD_WARPS) {
    const uint32_t id = slow[e].id;
    const double s = warp_dot2(qs, X + (int64_t)id * ldx, d);
    if (lane == 0) slow[e].s = s;
  }
  const int np2 = pow2_ceil(ns > 1 ? ns : 1);
  for (int e = ns + threadIdx.x; e < np2; e += blockDim.x) slow[e] = SD{-INFINITY, 0xFFFFFFFFu, 0};
  __syncthreads();
  block_sort_sd(slow, np2);
  for (int e = threadIdx.x; e < kmax; e += blockDim.x) {
    const bool ok = e < k && e < ns;
    out_ids[orow + e] = ok ? (int64_t)slow[e].id : -1;
    out_scores[orow + e] = ok ? (float)slow[e].s : -INFINITY;
  }
}

int choose_g(int nf4) {
  int g = 1;
  while (g < 32 && g * 4 < nf4) g <<= 1;
  return g;
}

// Launch of a score kernel: SCORE_WAVES times as many 256-thread CTAs as fit
// on the GPU at once; the kernels stride over the work items, and the
// hardware scheduler balances the CTAs' uneven loads.
constexpr int SCORE_WAVES = 3;

template <class Kernel>
fpp_status launch_resident(Kernel* k, int sms, const ScoreArgs& a, std::atomic<int>& per_sm,
                           cudaStream_t st) {
  int b = per_sm.load(std::memory_order_relaxed);
  if (!b) {
    FPP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k, SCORE_T, 0));
    b = std::max(1, b);
    per_sm.store(b, std::memory_order_relaxed);
  }
  k<<<b * sms * (a.tune_waves > 0 ? a.tune_waves : SCORE_WAVES), SCORE_T, 0, st>>>(a);
  FPP_LAUNCHED();
  return FPP_OK;
}

template <int G, int CPL, bool EXACT>
fpp_status launch_score_one(const ScoreArgs& a, int sms, cudaStream_t st) {
  static std::atomic<int> per_sm{0};
  return launch_resident(score_kernel<G, CPL, EXACT>, sms, a, per_sm, st);
}

template <int G>
fpp_status launch_score_g(const ScoreArgs& a, int sms, cudaStream_t st) {
  // chunks per lane: ceil(nf4 / G) <= 4 by the choice of G, except G = 32
  // (large d), which loops over chunk groups of 8
  const int nf4 = (int)(a.ldx / 4);
  const int cpl = (nf4 + G - 1) / G;
  if (cpl == 1 && nf4 == G) return launch_score_one<G, 1, true>(a, sms, st);
  if (cpl == 2 && nf4 == 2 * G) return launch_score_one<G, 2, true>(a, sms, st);
  if (cpl == 4 && nf4 == 4 * G) return launch_score_one<G, 4, true>(a, sms, st);
  if (cpl <= 1) return launch_score_one<G, 1, false>(a, sms, st);
  if (cpl <= 2) return launch_score_one<G, 2, false>(a, sms, st);
  if (cpl <= 4) return launch_score_one<G, 4, false>(a, sms, st);
  return launch_score_one<G, 8, false>(a, sms, st);
}

}  // namespace

template <int S>
fpp_status launch_probe_s(const ProbeArgs& a, cudaStream_t st) {
  const size_t smem = (size_t)PROBE_WARPS * probe_warp_bytes(a.probes, a.D);
  FPP_CUDA(cudaFuncSetAttribute(probe_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(smem > 48 * 1024 ? smem : 48 * 1024)));
  probe_kernel<S><<<(unsigned)ceil_div(a.mq * a.nt, PROBE_WARPS), PROBE_WARPS * 32, smem, st>>>(
      a, a.probes);
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_probe(const ProbeArgs& a, cudaStream_t st, cudaEvent_t exact_begin) {
  const int64_t warps = a.mq * a.nt;
  if (warps <= 0) return FPP_OK;
  if (a.probes > PMAX) {
    set_error("probes per table must be <= 128");
    return FPP_EINVAL;
  }
  FPP_CUDA(cudaMemsetAsync(a.recheck_count, 0, sizeof(unsigned), st));
  if (a.lists || a.recheck_s) FPP_CUDA(cudaMemsetAsync(a.recheck2_count, 0, sizeof(unsigned), st));
  const int S = pow2_ceil((a.D + 31) / 32);
  fpp_status s;
  if (a.argmax_only) {
    // one-piece BF16 projections: make every hash's winner exact first
    int dv = 0, nsm = 0;
    FPP_CUDA(cudaGetDevice(&dv));
    FPP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dv));
    if (a.lists) {
      if (a.EL > SMALL_E) {
        set_error("argmax pass: lists longer than 8 entries");
        return FPP_EINTERNAL;
      }
      FPP_CUDA(cudaMemsetAsync(a.amax_count, 0, sizeof(unsigned), st));
      const int64_t need = ceil_div(warps, (int64_t)256);
      probe_argmax_test_kernel<<<(unsigned)std::min<int64_t>(need, (int64_t)nsm * 16), 256, 0, st>>>(a);
      FPP_LAUNCHED();
      probe_argmax_fix_kernel<<<(unsigned)nsm * 8, 256, 0, st>>>(a);
    } else {
      const int64_t need = ceil_div(warps, (int64_t)8);
      probe_argmax_rows_kernel<<<(unsigned)std::min<int64_t>(need, (int64_t)nsm * 8), 256, 0, st>>>(a);
    }
    FPP_LAUNCHED();
  }
  if (a.lists && a.probes + 1 <= a.EL && a.EL <= SMALL_E) {
    const unsigned grid = (unsigned)ceil_div(warps, 256);
    if (a.EL <= 2) probe_small_kernel<2><<<grid, 256, 0, st>>>(a);
    else if (a.EL <= 4) probe_small_kernel<4><<<grid, 256, 0, st>>>(a);
    else probe_small_kernel<SMALL_E><<<grid, 256, 0, st>>>(a);
    FPP_LAUNCHED();
    s = FPP_OK;
  } else switch (S) {
    case 1: s = launch_probe_s<1>(a, st); break;
    case 2: s = launch_probe_s<2>(a, st); break;
    case 4: s = launch_probe_s<4>(a, st); break;
    case 8: s = launch_probe_s<8>(a, st); break;
    case 16: s = launch_probe_s<16>(a, st); break;
    default: s = launch_probe_s<32>(a, st); break;
  }
  if (s != FPP_OK) return s;
  if (exact_begin) FPP_CUDA(cudaEventRecord(exact_begin, st));
  int dev0 = 0, sms0 = 0;
  cudaGetDevice(&dev0);
  cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, dev0);
  if (a.lists) {
    // up to 64 resident warps per SM, one item each
    if (a.Rb) probe_window_kernel<true><<<sms0 * 8, 256, 0, st>>>(a);
    else probe_window_kernel<false><<<sms0 * 8, 256, 0, st>>>(a);
    FPP_LAUNCHED();
  } else if (a.recheck_s) {
    // 80 registers with BF16 rows: three CTAs per SM
    if (a.Rb) probe_pwin_kernel<true><<<sms0 * 3, 256, 0, st>>>(a);
    else probe_pwin_kernel<false><<<sms0 * 2, 256, 0, st>>>(a);
    FPP_LAUNCHED();
  }
  // exact pass over the items the fast pass could not decide; the grid is
  // fixed and the kernel reads the item count on the device
  const size_t smem = recheck_smem_bytes(a.D);
  const bool small_p = a.probes <= 16;
  const void* fn = small_p ? (a.Rb ? (const void*)probe_recheck_kernel<true, RECHECK_THREADS>
                                   : (const void*)probe_recheck_kernel<false, RECHECK_THREADS>)
                           : (a.Rb ? (const void*)probe_recheck_kernel<true, RECHECK_THREADS_LARGE_P>
                                   : (const void*)probe_recheck_kernel<false, RECHECK_THREADS_LARGE_P>);
  FPP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (small_p) {
    if (a.Rb) probe_recheck_kernel<true, RECHECK_THREADS><<<sms, RECHECK_THREADS, smem, st>>>(a);
    else probe_recheck_kernel<false, RECHECK_THREADS><<<sms, RECHECK_THREADS, smem, st>>>(a);
  } else {
    if (a.Rb)
      probe_recheck_kernel<true, RECHECK_THREADS_LARGE_P><<<sms * 4, RECHECK_THREADS_LARGE_P, smem, st>>>(a);
    else
      probe_recheck_kernel<false, RECHECK_THREADS_LARGE_P><<<sms * 4, RECHECK_THREADS_LARGE_P, smem, st>>>(a);
  }
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_global_probes(const ProbeArgs& a, int Qp, cudaStream_t st) {
  if (a.mq <= 0) return FPP_OK;
  const int N = a.nt * a.probes;
  const int npow2 = pow2_ceil(N > 1 ? N : 1);
  const size_t smem = (size_t)npow2 * 8 + (size_t)a.nt * 4 + (size_t)std::min(Qp, N) * 4 + 16;
  if (smem > 200 * 1024) {
    set_error("global probes: tables x per-table budget too large (at most 16,384 pairs)");
    return FPP_EINVAL;
  }
  FPP_CUDA(cudaFuncSetAttribute(global_probes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  global_probes_kernel<<<(unsigned)a.mq, GP_THREADS, smem, st>>>(a, Qp, npow2);
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_sign_bits(const SignArgs& a, cudaStream_t st) {
  const int64_t n = a.rows * a.words;
  if (n <= 0) return FPP_OK;
  sign_bits_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(a);
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_simhash_filter(const SimArgs& a, cudaStream_t st) {
  if (a.mq <= 0) return FPP_OK;
  const size_t smem = (size_t)8 * a.cap * 8;
  FPP_CUDA(cudaFuncSetAttribute(simhash_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)std::max<size_t>(smem, 48 * 1024)));
  simhash_filter_kernel<<<(unsigned)ceil_div(a.mq, 8), 256, smem, st>>>(a);
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_query_norms(const float* Q, int64_t m, int64_t ldq, int d, float* out,
                              cudaStream_t st) {
  if (m <= 0) return FPP_OK;
  query_norms_kernel<<<(unsigned)ceil_div(m, 8), 256, 0, st>>>(Q, m, ldq, d, out);
  FPP_LAUNCHED();
  return FPP_OK;
}

int score_item_len() { return ITEM; }
int64_t score_item_slots(uint64_t cand_total, int64_t mq, int ranges) {
  return (int64_t)(cand_total / ITEM) + mq * (int64_t)(ranges > 1 ? ranges : 1) + 1;
}

// Counting sort of the score work items by the row range of their first
// candidate.  Both kernels stride over the items with the same grid; each CTA
// counts its items per range in shared memory and touches the global
// counters once per range: the histogram kernel adds its counts to hist; the
// scatter kernel takes the range bases from hist, reserves its slots in each
// range with one atomic on cursor and places its items with shared-memory
// atomics (the order inside a range is arbitrary).
constexpr int ORDER_T = 256;

__global__ void __launch_bounds__(ORDER_T)
order_hist_kernel(const ScoreItem* __restrict__ in, const unsigned* nitems,
                  const uint32_t* __restrict__ cand, int shift, int R, unsigned* hist) {
  __shared__ unsigned cnt[RANGE_MAX];
  for (int r = threadIdx.x; r < R; r += blockDim.x) cnt[r] = 0u;
  __syncthreads();
  const unsigned n = *nitems;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(cnt + (cand[in[i].start] >> shift), 1u);
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x)
    if (cnt[r]) atomicAdd(hist + r, cnt[r]);
}

__global__ void __launch_bounds__(ORDER_T)
order_scatter_kernel(const ScoreItem* __restrict__ in, const unsigned* nitems,
                     const uint32_t* __restrict__ cand, int shift, int R, const unsigned* hist,
                     unsigned* cursor, ScoreItem* __restrict__ out) {
  __shared__ unsigned base[RANGE_MAX], cnt[RANGE_MAX];
  if (threadIdx.x < 32) {   // base[r]: the items of the ranges before r
    const int lane = threadIdx.x;
    unsigned carry = 0;
    for (int r0 = 0; r0 < R; r0 += 32) {
      const int r = r0 + lane;
      const unsigned c = r < R ? hist[r] : 0u;
      unsigned inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t2 = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += t2;
      }
      if (r < R) base[r] = carry + inc - c;
      carry += __shfl_sync(FULL, inc, 31);
    }
  }
  for (int r = threadIdx.x; r < R; r += blockDim.x) cnt[r] = 0u;
  __syncthreads();
  const unsigned n = *nitems;
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    atomicAdd(cnt + (cand[in[i].start] >> shift), 1u);
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    if (cnt[r]) base[r] += atomicAdd(cursor + r, cnt[r]);   // this CTA's slots of range r
    cnt[r] = 0u;
  }
  __syncthreads();
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const ScoreItem it = in[i];
    const int r = (int)(cand[it.start] >> shift);
    out[base[r] + atomicAdd(cnt + r, 1u)] = it;
  }
}

fpp_status launch_order_items(const ScoreItem* in, const unsigned* nitems, const uint32_t* cand,
                              int range_shift, int range_count, unsigned* hist, unsigned* cursor,
                              ScoreItem* out, cudaStream_t st) {
  if (range_count > RANGE_MAX) {
    set_error("launch_order_items: too many row ranges");
    return FPP_EINTERNAL;
  }
  int dev = 0, sms = 0;
  FPP_CUDA(cudaGetDevice(&dev));
  FPP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  order_hist_kernel<<<sms * 4, ORDER_T, 0, st>>>(in, nitems, cand, range_shift, range_count, hist);
  FPP_LAUNCHED();
  order_scatter_kernel<<<sms * 4, ORDER_T, 0, st>>>(in, nitems, cand, range_shift, range_count,
                                                    hist, cursor, out);
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_count_entries(const DedupArgs& a, cudaStream_t st) {
  if (a.mq <= 0) return FPP_OK;
  count_entries_kernel<<<(unsigned)ceil_div(a.mq, 8), 256, 0, st>>>(a);
  FPP_LAUNCHED();
  return FPP_OK;
}

template <int NT, int HS, int LOG2HS, int ELO, int EHI, int TIER, int FUSE>
fpp_status launch_hash_tier(const DedupArgs& a, std::atomic<int>& grid_cache, cudaStream_t st) {
  const size_t smem = (size_t)HS * 4;
  int g = grid_cache.load(std::memory_order_relaxed);
  if (!g) {
    FPP_CUDA(cudaFuncSetAttribute(dedup_hash_kernel<NT, HS, LOG2HS, ELO, EHI, TIER, FUSE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, sms = 0;
    FPP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dedup_hash_kernel<NT, HS, LOG2HS, ELO, EHI, TIER, FUSE>,
                                                           NT, smem));
    FPP_CUDA(cudaGetDevice(&dev));
    FPP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    g = std::max(1, per_sm) * sms;
    grid_cache.store(g, std::memory_order_relaxed);
  }
  dedup_hash_kernel<NT, HS, LOG2HS, ELO, EHI, TIER, FUSE><<<(int)std::min<int64_t>(a.mq, g), NT, smem, st>>>(a);
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_dedup(const DedupArgs& a, cudaStream_t st) {
  if (a.mq <= 0) return FPP_OK;
  // three tiers by entry count: 128 threads and 4,096 slots (<= 3,072
  // entries), 256 threads and 32,768 slots (<= 16,384), and no
  // de-duplication above that; a table never holds more distinct ids than
  // three quarters of its slots (one half for the larger one)
  static std::atomic<int> g_small{0}, g_fused{0}, g_big{0};
  if (a.fused)
    FPP_TRY((launch_hash_tier<128, HS_SMALL, 12, 0, HMAX_SMALL, -1, 1>(a, g_fused, st)));
  else
    FPP_TRY((launch_hash_tier<128, HS_SMALL, 12, 0, HMAX_SMALL, -1, 0>(a, g_small, st)));
  FPP_TRY((launch_hash_tier<256, HS_BIG, 15, HMAX_SMALL, HMAX_BIG, 0, 0>(a, g_big, st)));
  int sms = 0, dev = 0;
  FPP_CUDA(cudaGetDevice(&dev));
  FPP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  flatten_kernel<<<(int)std::min<int64_t>(ceil_div(a.mq, DW), (int64_t)sms * 4), DW * 32, 0, st>>>(a);
  FPP_LAUNCHED();
  return FPP_OK;
}

template <int G, int CPL, bool EXACT>
fpp_status launch_score_bf_one(const ScoreArgs& a, int sms, cudaStream_t st) {
  static std::atomic<int> per_sm{0};
  return launch_resident(score_bf16_kernel<G, CPL, EXACT>, sms, a, per_sm, st);
}

template <int G>
fpp_status launch_score_bf(const ScoreArgs& a, int sms, cudaStream_t st) {
  const int nch = (int)(a.ldxb / 8);
  const int cpl = (nch + G - 1) / G;
  if (cpl == 1 && nch == G) return launch_score_bf_one<G, 1, true>(a, sms, st);
  if (cpl == 2 && nch == 2 * G) return launch_score_bf_one<G, 2, true>(a, sms, st);
  if (cpl == 4 && nch == 4 * G) return launch_score_bf_one<G, 4, true>(a, sms, st);
  if (cpl <= 1) return launch_score_bf_one<G, 1, false>(a, sms, st);
  if (cpl <= 2) return launch_score_bf_one<G, 2, false>(a, sms, st);
  return launch_score_bf_one<G, 4, false>(a, sms, st);
}

template <int G, int CPL, bool EXACT>
fpp_status launch_score_f8_one(const ScoreArgs& a, int sms, cudaStream_t st) {
  static std::atomic<int> per_sm{0};
  return launch_resident(score_fp8_kernel<G, CPL, EXACT>, sms, a, per_sm, st);
}

template <int G>
fpp_status launch_score_f8(const ScoreArgs& a, int sms, cudaStream_t st) {
  const int nch = (int)(a.ldxq / 16);
  const int cpl = (nch + G - 1) / G;
  if (cpl == 1 && nch == G) return launch_score_f8_one<G, 1, true>(a, sms, st);
  if (cpl == 2 && nch == 2 * G) return launch_score_f8_one<G, 2, true>(a, sms, st);
  if (cpl <= 1) return launch_score_f8_one<G, 1, false>(a, sms, st);
  return launch_score_f8_one<G, 2, false>(a, sms, st);
}

fpp_status launch_score(const ScoreArgs& a, int sm_count, cudaStream_t st) {
  const int grid = sm_count;
  if (a.Xq) {
    // 16-byte chunks of 16 e4m3 values, at most 2 per lane before G = 32
    int g = 1;
    const int nch = (int)(a.ldxq / 16);
    while (g < 32 && g * 2 < nch) g <<= 1;
    if (a.tune_g) g = a.tune_g;
    switch (g) {
      case 1: return launch_score_f8<1>(a, grid, st);
      case 2: return launch_score_f8<2>(a, grid, st);
      case 4: return launch_score_f8<4>(a, grid, st);
      case 8: return launch_score_f8<8>(a, grid, st);
      case 16: return launch_score_f8<16>(a, grid, st);
      default: return launch_score_f8<32>(a, grid, st);
    }
  }
  if (a.Xb) {
    // 16-byte chunks of 8 BF16; at most 4 chunks per lane before G = 32 (as
    // for FP32 rows: more rows per warp in flight)
    int g = 1;
    const int nch = (int)(a.ldxb / 8);
    while (g < 32 && g * 4 < nch) g <<= 1;
    if (a.tune_g) g = a.tune_g;
    switch (g) {
      case 1: return launch_score_bf<1>(a, grid, st);
      case 2: return launch_score_bf<2>(a, grid, st);
      case 4: return launch_score_bf<4>(a, grid, st);
      case 8: return launch_score_bf<8>(a, grid, st);
      case 16: return launch_score_bf<16>(a, grid, st);
      default: return launch_score_bf<32>(a, grid, st);
    }
  }
  switch (a.tune_g ? a.tune_g : choose_g((int)(a.ldx / 4))) {
    case 1: return launch_score_g<1>(a, grid, st);
    case 2: return launch_score_g<2>(a, grid, st);
    case 4: return launch_score_g<4>(a, grid, st);
    case 8: return launch_score_g<8>(a, grid, st);
    case 16: return launch_score_g<16>(a, grid, st);
    default: return launch_score_g<32>(a, grid, st);
  }
}

fpp_status launch_topk(const TopkArgs& a, cudaStream_t st) {
  if (a.mq <= 0) return FPP_OK;
  const size_t smem = (size_t)8 * a.cap * 8 + (size_t)8 * a.rcap * sizeof(SD);
  static bool attr = false;
  if (!attr) {
    FPP_CUDA(cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
    attr = true;
  }
  topk_kernel<<<(unsigned)ceil_div(a.mq, 8), 256, smem, st>>>(a);
  FPP_LAUNCHED();
  return FPP_OK;
}

int topk_cap(int kprime) { return pow2_ceil(2 * kprime + 32); }
int topk_rcap(int kprime) { return pow2_ceil(kprime); }
int topk_slow_cap() { return TK_SLOW; }

fpp_status launch_topk_dense(const float* S, int64_t lds, int64_t mq, int64_t n, int k,
                             const float* Q, int64_t ldq, const float* X, int64_t ldx, int d,
                             float xmax, double gamma, int64_t* out_ids, float* out_scores,
                             int kmax, unsigned long long* rechecks, cudaStream_t st) {
  if (mq <= 0) return FPP_OK;
  const DenseLayout Lo = dense_layout(kmax, (int)ldq);
  FPP_CUDA(cudaFuncSetAttribute(topk_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                200 * 1024));
  int* err = reinterpret_cast<int*>(rechecks + 1);
  topk_dense_kernel<<<(unsigned)mq, TD_WARPS * 32, Lo.total, st>>>(
      S, lds, n, k, Q, ldq, X, ldx, d, xmax, gamma, out_ids, out_scores, kmax, rechecks, err);
  FPP_LAUNCHED();
  return FPP_OK;
}

}  // namespace fpp
