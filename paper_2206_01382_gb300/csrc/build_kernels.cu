// Index build kernels: cross-polytope hashing of the points (Eq. 1), bucket
// histogram, exclusive scans, a stable LSD radix sort that orders every
// bucket by filter score, and the compaction that keeps the top fraction of
// each bucket (Section 3.4) into CSR.
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace fpp {

namespace {

// Kept count of a bucket of size B (Section 3.4, Algorithm 1), evaluated with
// the same IEEE FP64 operations as the host-side definition.
__device__ __forceinline__ uint32_t keep_dev(uint32_t B, const KeepRule& r) {
  double c = ceil(__ddiv_rn(__dmul_rn(r.alpha, (double)B), (double)r.iprobes));
  uint64_t k = (uint64_t)c;
  if (r.kappa > 0 && k < (uint64_t)r.kappa) k = (uint64_t)r.kappa;
  if (k > B) k = B;
  return (uint32_t)k;
}

// ------------------------------------------------------------------ hashing
//
// One warp per (point, table).  For each of the two hashes the warp finds the
// FP32 argmax of |x^T r_i| and the runner-up.  The FP32 winner is the exact
// winner when its lead exceeds twice the GEMM error bound eps (and its value
// exceeds eps, which fixes the sign); its projection is then recomputed with
// the compensated dot product to give an FP64-accurate filter score.
// Otherwise the entries whose FP32 value is within 2 eps of the FP32 maximum
// (the only ones that can be the exact maximum) are recomputed compensated,
// or all D of them when that window holds more than WIN entries, and the
// argmax is taken on those (lowest index on ties), so bucket ids agree with
// an exact evaluation except for genuine near-ties.
constexpr int WIN = 8;   // window entries recomputed before falling back to all D

__global__ void __launch_bounds__(256)
build_hash_kernel(HashArgs a) {
  __shared__ uint32_t win[8][WIN];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= a.rows * a.nt) return;
  const int64_t r = w / a.nt;
  const int tl = (int)(w % a.nt);
  const int t = a.t0 + tl;
  const int D = a.D;
  const int64_t pid = a.row0 + r;
  const float* x = a.X + pid * a.ldx;

  int h[2];
  double val[2];
  for (int j = 0; j < 2; ++j) {
    float b1 = -1.f, s1 = -1.f;
    int i1 = INT_MAX;
    if (a.P) {
      const float* pr = a.P + r * a.ldp + (int64_t)(2 * tl + j) * D;
      for (int i = lane; i < D; i += 32) {
        const float v = fabsf(pr[i]);
        if (v > b1) {
          s1 = b1; b1 = v; i1 = i;
        } else if (v > s1) {
          s1 = v;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float b2 = __shfl_xor_sync(0xffffffffu, b1, o);
        const float s2 = __shfl_xor_sync(0xffffffffu, s1, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i1, o);
        if (b2 > b1 || (b2 == b1 && i2 < i1)) {
          s1 = fmaxf(b1, s2); b1 = b2; i1 = i2;
        } else {
          s1 = fmaxf(s1, b2);
        }
      }
    } else {
      // best two keys of the hash, kept by the projection epilogue:
      // key = (bits(|p|) + 1) << 32 | (0xFFFFFFFF - h)
      const uint64_t* kk = a.lists + ((r * a.nt + tl) * 2 + j) * (int64_t)(a.EL + 1);
      const uint64_t k0 = kk[0], k1 = kk[1];
      b1 = __uint_as_float((uint32_t)(k0 >> 32) - 1u);
      i1 = (int)((0xFFFFFFFFu - (uint32_t)k0) % (uint32_t)D);
      s1 = D > 1 ? __uint_as_float((uint32_t)(k1 >> 32) - 1u) : -1.f;
    }
    // list values are truncated: every |p| of the hash lies below its list
    // value times (1 + trunc), at most trunc * b1 above it
    const float eps = a.eps_xf * a.rmax[2 * t + j] * 1.0001f + (a.P ? 0.f : a.trunc * b1 * 1.0001f);
    const bool certain = (b1 - s1 > 2.f * eps) && (b1 > eps);
    const float* Rj = a.R + (int64_t)(2 * t + j) * D * a.ldr;
    if (certain) {
      val[j] = warp_dot2(x, Rj + (int64_t)i1 * a.ldr, a.d);
      h[j] = i1 + (val[j] < 0.0 ? D : 0);
    } else {
      if (lane == 0 && a.rechecks) atomicAdd(a.rechecks, 1ull);
      // window: only entries whose FP32 |p| is within 2 eps of the FP32
      // maximum can be the exact maximum; recompute those when they are few
      const float lim = b1 - 2.f * eps;
      int nc = 0;
      bool all = false;
      if (a.P) {
        const float* pr = a.P + r * a.ldp + (int64_t)(2 * tl + j) * D;
        for (int i0 = 0; i0 < D && !all; i0 += 32) {
          const int i = i0 + lane;
          const bool in = i < D && fabsf(pr[i]) >= lim;
          const unsigned m = __ballot_sync(0xffffffffu, in);
          if (in) {
            const int slot = nc + __popc(m & ((1u << lane) - 1u));
            if (slot < WIN) win[wid][slot] = (uint32_t)i;
          }
          nc += __popc(m);
          if (nc > WIN) all = true;
        }
      } else {
        const uint64_t* kk = a.lists + ((r * a.nt + tl) * 2 + j) * (int64_t)(a.EL + 1);
        const float cut = kk[a.EL] ? __uint_as_float((uint32_t)(kk[a.EL] >> 32) - 1u) : -1.f;
        if (!(cut < lim)) {
          all = true;
        } else if (lane == 0) {
          for (int e = 0; e < a.EL; ++e)
            if (kk[e] && __uint_as_float((uint32_t)(kk[e] >> 32) - 1u) >= lim)
              win[wid][nc++] = (0xFFFFFFFFu - (uint32_t)kk[e]) % (uint32_t)D;
        }
        nc = __shfl_sync(0xffffffffu, nc, 0);
      }
      __syncwarp();
      double bv = -1.0, bs = 0.0;
      int bi = INT_MAX;
      const int nf4 = (int)(a.ldr / 4);
      if (!all) {
        // every lane computes the same argmax (lowest index on ties)
        const float* rows[WIN];
        uint32_t ii[WIN];
#pragma unroll
        for (int e = 0; e < WIN; ++e) {
          ii[e] = win[wid][e < nc ? e : 0];
          rows[e] = Rj + (int64_t)ii[e] * a.ldr;
        }
        double v[WIN];
        warp_dot2_gather<WIN>(x, rows, nf4, v);
#pragma unroll
        for (int e = 0; e < WIN; ++e)
          if (e < nc && (fabs(v[e]) > bv || (fabs(v[e]) == bv && (int)ii[e] < bi))) {
            bv = fabs(v[e]); bs = v[e]; bi = (int)ii[e];
          }
      } else {
        int i = 0;
        for (; i + 4 <= D; i += 4) {
          double v[4];
          warp_dot2_rows<4>(x, Rj + (int64_t)i * a.ldr, a.ldr, nf4, v);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (fabs(v[k]) > bv) { bv = fabs(v[k]); bs = v[k]; bi = i + k; }
        }
        for (; i < D; ++i) {
          double v[1];
          warp_dot2_rows<1>(x, Rj + (int64_t)i * a.ldr, a.ldr, nf4, v);
          if (fabs(v[0]) > bv) { bv = fabs(v[0]); bs = v[0]; bi = i; }
        }
      }
      val[j] = bs;
      h[j] = bi + (bs < 0.0 ? D : 0);
    }
  }
  if (lane == 0) {
    const uint32_t bucket = (uint32_t)h[0] * (uint32_t)(2 * D) + (uint32_t)h[1];
    const int64_t NB = 4ll * D * D;
    const uint32_t sk = (uint32_t)(tl * NB + bucket);
    if (a.rec) {
      const double f = fabs(val[0]) + fabs(val[1]);
      Rec rc;
      rc.key = ~(uint64_t)__double_as_longlong(f);
      rc.sk = sk;
      rc.id = (uint32_t)pid;
      a.rec[(int64_t)tl * a.n + pid] = rc;
    }
    if (a.counts) atomicAdd(a.counts + sk, 1u);
    if (a.point_bucket) a.point_bucket[r] = bucket;
  }
}

__global__ void row_norm_max_kernel(const float* __restrict__ X, int64_t n, int64_t ldx, int d,
                                    float* out) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= n) return;
  const float* x = X + r * ldx;
  float s = 0.f;
  for (int i = lane; i < d; i += 32) s = fmaf(x[i], x[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    // the FP32 sum carries relative error <= gamma_d; inflate so the result
    // bounds the true norm from above
    const float nrm = sqrtf(s) * (1.f + 1e-4f + 2e-7f * d);
    atomicMax(reinterpret_cast<unsigned int*>(out), __float_as_uint(nrm));
  }
}

// ------------------------------------------------------------------ scan

constexpr int SCAN_T = 256, SCAN_V = 16, SCAN_BLK = SCAN_T * SCAN_V;

__device__ __forceinline__ uint32_t scan_value(const uint32_t* in, int64_t i, int mode,
                                               const KeepRule& r) {
  const uint32_t v = in[i];
  return mode ? keep_dev(v, r) : v;
}

// Block-wide exclusive scan of one u64 per thread; returns the block total.
__device__ __forceinline__ uint64_t block_exscan(uint64_t v, uint64_t& excl) {
  __shared__ uint64_t wsum[SCAN_T / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  uint64_t wbase = 0, total = 0;
  for (int w = 0; w < SCAN_T / 32; ++w) {
    if (w < wid) wbase += wsum[w];
    total += wsum[w];
  }
  __syncthreads();
  excl = wbase + inc - v;
  return total;
}

__global__ void __launch_bounds__(SCAN_T)
scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t n, int mode, KeepRule rule,
                   uint64_t* __restrict__ part) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLK + threadIdx.x * SCAN_V;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_V; ++i)
    if (base + i < n) s += scan_value(in, base + i, mode, rule);
  uint64_t excl;
  const uint64_t tot = block_exscan(s, excl);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T)
scan_partials_kernel(uint64_t* part, int64_t nb, uint64_t* total_out) {
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c = 0; c < nb; c += SCAN_T) {
    const int64_t i = c + threadIdx.x;
    const uint64_t v = i < nb ? part[i] : 0;
    uint64_t excl;
    const uint64_t tot = block_exscan(v, excl);
    if (i < nb) part[i] = carry + excl;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(SCAN_T)
scan_apply_kernel(const uint32_t* __restrict__ in, int64_t n, int mode, KeepRule rule,
                  const uint64_t* __restrict__ part, uint64_t* __restrict__ out) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLK + threadIdx.x * SCAN_V;
  uint32_t v[SCAN_V];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_V; ++i) {
    v[i] = (base + i < n) ? scan_value(in, base + i, mode, rule) : 0u;
    s += v[i];
  }
  uint64_t excl;
  block_exscan(s, excl);
  uint64_t run = part[blockIdx.x] + excl;
#pragma unroll
  for (int i = 0; i < SCAN_V; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

// ------------------------------------------------------------------ radix sort
//
// Stable LSD radix sort, 8-bit digits.  Per pass: tile histograms (digit-
// major), an exclusive scan of them, and a stable scatter.  A tile is 4096
// records; warp w of the tile owns records [w*512, w*512+512) and walks them
// in 16 rounds of 32, so (warp, round, lane) is the input order and ranking
// within a round with __match_any_sync keeps equal digits in input order.

constexpr int RS_T = 256, RS_ROUNDS = 16, RS_TILE = RS_T * RS_ROUNDS;

__device__ __forceinline__ uint32_t rec_digit(const Rec& r, int field, int shift) {
  return field == 0 ? (uint32_t)((r.key >> shift) & 0xFFu) : ((r.sk >> shift) & 0xFFu);
}

__global__ void __launch_bounds__(RS_T)
radix_hist_kernel(const Rec* __restrict__ in, int64_t n, int field, int shift,
                  uint32_t* __restrict__ hist, int64_t ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_T) {
    const int64_t p = base + i;
    if (p < n) atomicAdd(&h[rec_digit(in[p], field, shift)], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_T)
radix_scatter_kernel(const Rec* __restrict__ in, Rec* __restrict__ out, int64_t n, int field,
                     int shift, const uint64_t* __restrict__ gofs, int64_t ntiles) {
  __shared__ uint32_t wcnt[RS_T / 32][256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < (RS_T / 32) * 256; i += RS_T) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)wid * (32 * RS_ROUNDS);
  const unsigned lt = (1u << lane) - 1u;
  Rec rec[RS_ROUNDS];
  uint32_t dig[RS_ROUNDS], rank[RS_ROUNDS];
#pragma unroll
  for (int k = 0; k < RS_ROUNDS; ++k) {
    const int64_t p = wbase + k * 32 + lane;
    const bool ok = p < n;
    if (ok) rec[k] = in[p];
    dig[k] = ok ? rec_digit(rec[k], field, shift) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, dig[k]);
    const uint32_t before = ok ? wcnt[wid][dig[k]] : 0u;
    rank[k] = before + __popc(peers & lt);
    __syncwarp();
    if (ok && (peers & lt) == 0) wcnt[wid][dig[k]] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // exclusive prefix over warps, per digit
    const int dgt = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < RS_T / 32; ++w) {
      const uint32_t c = wcnt[w][dgt];
      wcnt[w][dgt] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < RS_ROUNDS; ++k) {
    if (dig[k] < 256u) {
      const uint64_t pos = gofs[(int64_t)dig[k] * ntiles + blockIdx.x] + wcnt[wid][dig[k]] + rank[k];
      out[pos] = rec[k];
    }
  }
}

// ------------------------------------------------------------------ compaction

__global__ void compact_kernel(const Rec* __restrict__ sorted, int64_t nrec,
                               const uint64_t* __restrict__ bstart,
                               const uint64_t* __restrict__ kstart,
                               const uint32_t* __restrict__ counts, KeepRule rule,
                               uint32_t* __restrict__ ids_out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nrec) return;
  const Rec r = sorted[p];
  const uint64_t rank = (uint64_t)p - bstart[r.sk];
  if (rank < keep_dev(counts[r.sk], rule)) ids_out[kstart[r.sk] + rank] = r.id;
}

__global__ void make_offsets_kernel(const uint64_t* __restrict__ kstart, int nt, int64_t NB,
                                    uint32_t* __restrict__ offsets) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)nt * (NB + 1)) return;
  const int64_t tl = i / (NB + 1), b = i % (NB + 1);
  offsets[i] = (uint32_t)(kstart[tl * NB + b] - kstart[tl * NB]);
}

}  // namespace

// One warp per (point, table): for each of the point's probed buckets
// (h1, h2), the filter score v1(h1) + v2(h2) from compensated projections
// (v(h) = x^T r_i for h = i, -x^T r_i for h = i + D), and its record.
__global__ void __launch_bounds__(256)
pair_records_kernel(PairArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= a.rows * a.nt) return;
  const int64_t r = w / a.nt;
  const int tl = (int)(w % a.nt);
  const int t = a.t0 + tl;
  const int D = a.D;
  const int64_t pid = a.row0 + r;
  const float* x = a.X + pid * a.ldx;
  const int nf4 = (int)(a.ldx / 4);
  const int64_t NB = 4ll * D * D;
  for (int e = 0; e < a.iprobes; ++e) {
    const uint32_t bucket = a.probes[(r * a.nt + tl) * (int64_t)a.iprobes + e];
    const uint32_t h1 = bucket / (uint32_t)(2 * D), h2 = bucket % (uint32_t)(2 * D);
    const float* rows[2] = {
        a.R + ((int64_t)(2 * t) * D + (h1 % (uint32_t)D)) * a.ldr,
        a.R + ((int64_t)(2 * t + 1) * D + (h2 % (uint32_t)D)) * a.ldr};
    double v[2];
    warp_dot2_gather<2>(x, rows, nf4, v);
    if (lane == 0) {
      const double f = (h1 < (uint32_t)D ? v[0] : -v[0]) + (h2 < (uint32_t)D ? v[1] : -v[1]);
      // order-preserving key of the (possibly negative, for tiny D) score,
      // complemented so that ascending keys are descending scores
      const uint64_t u = (uint64_t)__double_as_longlong(f);
      const uint64_t okey = (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
      const uint32_t sk = (uint32_t)(tl * NB + bucket);
      Rec rc;
      rc.key = ~okey;
      rc.sk = sk;
      rc.id = (uint32_t)pid;
      a.rec[(int64_t)tl * a.n * a.iprobes + pid * a.iprobes + e] = rc;
      atomicAdd(a.counts + sk, 1u);
    }
  }
}

fpp_status launch_pair_records(const PairArgs& a, cudaStream_t st) {
  const int64_t warps = a.rows * a.nt;
  if (warps <= 0) return FPP_OK;
  pair_records_kernel<<<(unsigned)ceil_div(warps, 8), 256, 0, st>>>(a);
  FPP_LAUNCHED();
  return FPP_OK;
}

// Centering (Section 3.4, heuristic (1)).  Column sums in FP64 over row
// blocks of CM_ROWS (one thread per column, rows in order), then the block
// partials summed in order and divided by n; the FP64 mean is rounded to
// FP32.  The order is fixed, so c is the same on every run.
constexpr int CM_ROWS = 4096;

__global__ void column_partials_kernel(const float* __restrict__ X, int64_t n, int64_t ldx, int d,
                                       double* __restrict__ part) {
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= d) return;
  const int64_t r0 = (int64_t)blockIdx.x * CM_ROWS;
  const int64_t r1 = n < r0 + CM_ROWS ? n : r0 + CM_ROWS;
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) s += (double)X[r * ldx + c];
  part[(int64_t)blockIdx.x * d + c] = s;
}

__global__ void column_means_kernel(const double* __restrict__ part, int nblk, int d, int64_t n,
                                    float* __restrict__ c) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * d + j];
  c[j] = __double2float_rn(s / (double)n);
}

// x -> fl(x - c), the padded columns stay zero (c is zero there)
__global__ void center_rows_kernel(const float* __restrict__ X, int64_t total, int64_t ldx,
                                   const float* __restrict__ c, float* __restrict__ Xc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  Xc[i] = __fsub_rn(X[i], c[i % ldx]);
}

fpp_status launch_column_means(const float* X, int64_t n, int64_t ldx, int d, float* c,
                               cudaStream_t st) {
  const int nblk = (int)ceil_div(n, CM_ROWS);
  double* part = nullptr;
  FPP_CUDA(dev_malloc(&part, (size_t)nblk * d * 8));
  column_partials_kernel<<<dim3(nblk, (unsigned)ceil_div(d, 128)), 128, 0, st>>>(X, n, ldx, d, part);
  FPP_LAUNCHED();
  column_means_kernel<<<(unsigned)ceil_div(d, 128), 128, 0, st>>>(part, nblk, d, n, c);
  FPP_LAUNCHED();
  FPP_CUDA(cudaStreamSynchronize(st));
  cudaFree(part);
  return FPP_OK;
}

fpp_status launch_center_rows(const float* X, int64_t n, int64_t ldx, const float* c, float* Xc,
                              cudaStream_t st) {
  const int64_t total = n * ldx;
  if (total <= 0) return FPP_OK;
  center_rows_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(X, total, ldx, c, Xc);
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_build_hash(const HashArgs& a, cudaStream_t st) {
  const int64_t warps = a.rows * a.nt;
  if (warps <= 0) return FPP_OK;
  const int wpb = 8;
  build_hash_kernel<<<(unsigned)ceil_div(warps, wpb), wpb * 32, 0, st>>>(a);
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_row_norm_max(const float* X, int64_t n, int64_t ldx, int d, float* out,
                               cudaStream_t st) {
  FPP_CUDA(cudaMemsetAsync(out, 0, sizeof(float), st));
  if (n <= 0) return FPP_OK;
  row_norm_max_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(X, n, ldx, d, out);
  FPP_LAUNCHED();
  return FPP_OK;
}

int64_t scan_scratch_elems(int64_t n) { return ceil_div(n, SCAN_BLK) + 1; }

// Exclusive scan of at most SCAN1_MAX plain counts in one CTA, in tiles of
// 4 x 1,024 counts: each thread scans four consecutive counts, the CTA scans
// the thread totals, and a running carry joins the tiles; out[n] is the total.
constexpr int SCAN1_T = 1024;
constexpr int64_t SCAN1_MAX = 65536;

__global__ void __launch_bounds__(SCAN1_T)
scan_single_kernel(const uint32_t* __restrict__ in, int64_t n, uint64_t* __restrict__ out) {
  __shared__ uint64_t wsum[SCAN1_T / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  uint64_t carry = 0;
  for (int64_t t0 = 0; t0 < n; t0 += 4 * SCAN1_T) {
    const int64_t b = t0 + 4 * tid;
    uint32_t v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = b + r < n ? in[b + r] : 0u;
    const uint64_t s = (uint64_t)v[0] + v[1] + v[2] + v[3];
    uint64_t inc = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      uint64_t w = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += t;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    uint64_t run = carry + (wid ? wsum[wid - 1] : 0ull) + inc - s;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (b + r < n) out[b + r] = run;
      run += v[r];
    }
    carry += wsum[SCAN1_T / 32 - 1];
    __syncthreads();   // wsum is rewritten by the next tile
  }
  if (tid == 0) out[n] = carry;
}

fpp_status exclusive_scan_u32(const uint32_t* in, int64_t n, uint64_t* out, int mode,
                              KeepRule rule, uint64_t* scratch, cudaStream_t st) {
  if (n <= 0) {
    FPP_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
    return FPP_OK;
  }
  if (mode == 0 && n <= SCAN1_MAX) {
    scan_single_kernel<<<1, SCAN1_T, 0, st>>>(in, n, out);
    FPP_LAUNCHED();
    return FPP_OK;
  }
  const int64_t nb = ceil_div(n, SCAN_BLK);
  scan_reduce_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, mode, rule, scratch);
  FPP_LAUNCHED();
  scan_partials_kernel<<<1, SCAN_T, 0, st>>>(scratch, nb, out + n);
  FPP_LAUNCHED();
  scan_apply_kernel<<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, mode, rule, scratch, out);
  FPP_LAUNCHED();
  return FPP_OK;
}

int64_t radix_hist_elems(int64_t n) { return 256 * ceil_div(n, RS_TILE); }

fpp_status radix_sort_recs(Rec* a, Rec* b, int64_t n, int key_bits, int sk_bits,
                           uint32_t* hist, int64_t hist_elems, uint64_t* scan_buf,
                           uint64_t* scan_scratch, Rec** sorted, cudaStream_t st) {
  const int64_t ntiles = ceil_div(n, RS_TILE);
  if (256 * ntiles > hist_elems) {
    set_error("radix_sort_recs: histogram buffer too small");
    return FPP_EINTERNAL;
  }
  Rec* src = a;
  Rec* dst = b;
  const int kp = (key_bits + 7) / 8, sp = (sk_bits + 7) / 8;
  for (int pass = 0; pass < kp + sp && n > 0; ++pass) {
    const int field = pass < kp ? 0 : 1;
    const int shift = 8 * (pass < kp ? pass : pass - kp);
    radix_hist_kernel<<<(unsigned)ntiles, RS_T, 0, st>>>(src, n, field, shift, hist, ntiles);
    FPP_LAUNCHED();
    FPP_TRY(exclusive_scan_u32(hist, 256 * ntiles, scan_buf, 0, KeepRule{1.0, 1, 0},
                               scan_scratch, st));
    radix_scatter_kernel<<<(unsigned)ntiles, RS_T, 0, st>>>(src, dst, n, field, shift, scan_buf,
                                                           ntiles);
    FPP_LAUNCHED();
    Rec* t = src; src = dst; dst = t;
  }
  *sorted = src;
  return FPP_OK;
}

fpp_status launch_compact(const Rec* sorted, int64_t nrec, const uint64_t* bstart,
                          const uint64_t* kstart, const uint32_t* counts, KeepRule rule,
                          uint32_t* ids_out, cudaStream_t st) {
  if (nrec <= 0) return FPP_OK;
  compact_kernel<<<(unsigned)ceil_div(nrec, 256), 256, 0, st>>>(sorted, nrec, bstart, kstart,
                                                               counts, rule, ids_out);
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status launch_make_offsets(const uint64_t* kstart, int nt, int64_t NB, uint32_t* offsets,
                               cudaStream_t st) {
  const int64_t total = (int64_t)nt * (NB + 1);
  make_offsets_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(kstart, nt, NB, offsets);
  FPP_LAUNCHED();
  return FPP_OK;
}

}  // namespace fpp
