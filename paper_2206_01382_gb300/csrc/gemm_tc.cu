// Tensor-core projection GEMM for sm_103a: C[M][N] = A[M][K] * B[N][K]^T with
// tcgen05.mma (BF16 operands, FP32 accumulators in tensor memory), operands
// staged by TMA into a shared-memory ring with 128-byte swizzle.
//
// This is the projection step of Falconn++ (Section 2.2: every query or point
// is projected onto the D random vectors of both hashes of every table).
//
// Exact-split mode (pieces = 3).  An FP32 value x splits exactly into three
// BF16 values x = hi + mid + lo (each residual x - hi, x - hi - mid is exact
// in FP32 and the last one has at most 8 significant bits).  The product
// a . b is then the sum of the nine piece products; the kernel accumulates
// the five next-order products (hi.mid, mid.hi, hi.lo, mid.mid, lo.hi) and
// then hi.hi into one TMEM accumulator.  The dropped products are below
// 2^-23 |a||b| and the partial sums of the small products stay 2^-7 below
// the final value, so the error bound stays within a small factor of the
// FP32 one (tc_error_bound_factor).
//
// When every element of B is itself a BF16 value (bpieces = 1), B's mid and
// lo pieces are zero and the three products lo.hi, mid.hi, hi.hi (in that
// order, into one accumulator) are the exact sum of all nine: half the
// tensor-core work for the same error bound.
//
// Plain mode (pieces = 1): one BF16 product, for the BF16 precision path.
//
// Roles (320 threads): warp 0 issues TMA loads, warp 1 allocates tensor
// memory and issues the MMAs (one elected lane), warps 2..9 drain the two
// accumulator buffers (warp w reads TMEM lanes 32 (w mod 4) .. +31, i.e. the
// rows it owns, in column half (w - 2) / 4) and store either FP32 results or
// each hash's best keys (the fused list epilogue).  Every mbarrier wait is
// bounded; a wait that runs out records an error code and the CTA drains and
// exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cmath>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace fpp {

namespace {

constexpr int TC_BM = 128, TC_BN = 256, TC_BK = 64;   // BK: 64 BF16 = one 128-byte row
constexpr int TC_STAGES = 4;
constexpr int TC_THREADS = 320;                     // 2 + 8 epilogue warps
constexpr int EPI_WARPS = 8;
constexpr uint32_t A_TILE = TC_BM * TC_BK * 2;         // 16 KB
constexpr uint32_t B_TILE = TC_BN * TC_BK * 2;         // 32 KB
constexpr uint32_t STAGE_BYTES = A_TILE + B_TILE;
constexpr long long WAIT_CYCLES = 4000000000ll;        // ~2 s at 2 GHz

struct __align__(8) TcShared {
  uint64_t full[TC_STAGES];
  uint64_t empty[TC_STAGES];
  uint64_t tfull[2];
  uint64_t tempty[2];
  uint64_t drain;       // the MMA warp's last commit when the CTA aborts
  long long limit;      // cycles a wait may take before the CTA aborts
  uint32_t tmem_base;
  int abort;
  // list mode with D = 256: the second column half of every row hands its
  // partial top list (up to 8 packed keys and the cut) to the first half,
  // per TMEM lane quarter; xfull completes when the second half has
  // written, xempty when the first half has read
  uint64_t xfull[4];
  uint64_t xempty[4];
  uint32_t xk[4][32][9];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity`; returns false (and raises the CTA's abort
// flag and the error code) when it runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, TcShared* sh, int* err,
                                          int code) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity)) {
    if (*(volatile int*)&sh->abort) return false;
    if (clock64() - t0 > sh->limit) {
      atomicExch(&sh->abort, 1);
      if (err) atomicExch(err, code);
      return false;
    }
  }
  return true;
}

// Bounded wait used while an aborting CTA drains its own copies and MMAs
// (the abort flag is already raised, so it is not consulted).
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* b, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)(16 >> 4) << 16;                  // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}

// Instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = 256.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                           ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Issues a 32-column TMEM load without waiting for it; the registers must not
// be read before tmem_wait(r) on the same array.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// Waits for the outstanding TMEM loads; the "+r" operands keep the compiler
// from moving reads of r above the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
        "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
        "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]),
        "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]),
        "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
      :
      : "memory");
}

// 16 consecutive columns of the warp's 32 TMEM lanes (one per thread).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait(uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.wait::ld.sync.aligned;"
      : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
        "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
        "+r"(r[14]), "+r"(r[15])
      :
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Chunk c of a tile's K loop: A piece, B piece and 64-wide K block.  In the
// exact-split mode the five next-order products (hi.mid, mid.hi, hi.lo,
// mid.mid, lo.hi) are accumulated first and hi.hi last, into one
// accumulator: while the small products accumulate, the partial sums (and so
// the rounding errors) stay 2^-7 smaller than the final value, which keeps
// the error bound of the whole sum close to that of hi.hi alone.
// With bpieces = 1 the chunks are lo.hi, mid.hi and hi.hi.
__device__ __forceinline__ void chunk_pieces(int c, int nkb, int pieces, int bpieces, int& pa,
                                             int& pb, int& kb) {
  const int pair = c / nkb;
  kb = c - pair * nkb;
  if (pieces == 1) { pa = pb = 0; return; }
  if (bpieces == 1) { pa = 2 - pair; pb = 0; return; }
  switch (pair) {
    case 0: pa = 0; pb = 1; break;
    case 1: pa = 1; pb = 0; break;
    case 2: pa = 0; pb = 2; break;
    case 3: pa = 1; pb = 1; break;
    case 4: pa = 2; pb = 0; break;
    default: pa = 0; pb = 0; break;
  }
}

// A hash list entry is stored as the key (bits(|p|') + 1) << 32 | (0xFFFFFFFF - h)
// with h = i for p >= 0 and i + D otherwise, and 0 marks an empty slot.
// |p|' is |p| with its lowest log2(2D) bits cleared: the epilogue ranks
// packed 32-bit keys 2^31 | (bits(|p|) with those bits cleared) | h with
// integer max/min, so |p|' >= |p| (1 - tc_list_trunc(D)) and entries whose
// |p| agree in all but those bits are ranked in an arbitrary (but fixed)
// order.  Consumers widen their error bounds accordingly.

// Persistent projection kernel.  Tiles of 128 rows x 256 columns are handed
// out round-robin; the TMEM accumulator is double-buffered so the epilogue of
// one tile overlaps the MMAs of the next.  EL = 0: the epilogue stores the
// FP32 projections.  EL > 0: for every (row, hash) it keeps the EL largest
// keys of the hash's D columns (D divides 256) followed by a "cut" key whose
// value is the largest |p| left out, and stores only those EL + 1 keys.
// mfast = 1 hands out the tiles of one column block for consecutive row
// blocks, so that CTAs running together share B's tiles in L2 (for B larger
// than A); otherwise they share A's.
template <int EL>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_proj_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               float* __restrict__ C, int64_t ldc, uint64_t* __restrict__ lists, int M, int N,
               int Kp, int pieces, int bpieces, int D, int mfast, int* err,
               long long wait_cycles, int withhold) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
  TcShared* sh = reinterpret_cast<TcShared*>(base + TC_STAGES * STAGE_BYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = Kp / TC_BK;
  const int nchunks = (pieces == 1 ? 1 : bpieces == 1 ? 3 : 6) * nkb;
  const int ntn = (N + TC_BN - 1) / TC_BN, ntm = (M + TC_BM - 1) / TC_BM;
  const int ntiles = ntn * ntm;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&sh->full[s], 1);
      mbar_init(&sh->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh->tfull[b], 1);
      mbar_init(&sh->tempty[b], EPI_WARPS);
    }
    for (int qq = 0; qq < 4; ++qq) {
      mbar_init(&sh->xfull[qq], 1);
      mbar_init(&sh->xempty[qq], 1);
    }
    mbar_init(&sh->drain, 1);
    sh->abort = 0;
    sh->limit = wait_cycles > 0 ? wait_cycles : WAIT_CYCLES;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh->tmem_base)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh->tmem_base;

  // the stages whose copies the producer issued, and the last chunk of each
  uint32_t issued = 0;
  uint32_t last_g[TC_STAGES];
  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    uint32_t g = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int m0 = (mfast ? t % ntm : t / ntn) * TC_BM;
      const int n0 = (mfast ? t / ntm : t % ntn) * TC_BN;
      bool ok = true;
      for (int c = 0; c < nchunks; ++c, ++g) {
        const uint32_t s = g % TC_STAGES;
        if (g >= TC_STAGES && !mbar_wait(&sh->empty[s], ((g / TC_STAGES) - 1) & 1, sh, err, 1)) {
          ok = false;
          break;
        }
        int pa, pb, kb;
        chunk_pieces(c, nkb, pieces, bpieces, pa, pb, kb);
        unsigned char* st = base + s * STAGE_BYTES;
        // test hook (withhold = 1): CTA 0 never loads its first chunk, so the
        // MMA warp's wait for it runs out
        if (withhold && blockIdx.x == 0 && g == 0) continue;
        mbar_expect_tx(&sh->full[s], STAGE_BYTES);
        tma_load_2d(st, &mapA, pa * Kp + kb * TC_BK, m0, &sh->full[s]);
        tma_load_2d(st + A_TILE, &mapB, pb * Kp + kb * TC_BK, n0, &sh->full[s]);
        issued |= 1u << s;
        last_g[s] = g;
      }
      if (!ok) break;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    uint32_t g = 0;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = i & 1;
      if (i >= 2 && !mbar_wait(&sh->tempty[b], ((i >> 1) - 1) & 1, sh, err, 4)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + (uint32_t)(b * TC_BN);
      bool ok = true;
      for (int c = 0; c < nchunks; ++c, ++g) {
        const uint32_t s = g % TC_STAGES;
        if (!mbar_wait(&sh->full[s], (g / TC_STAGES) & 1, sh, err, 2)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_addr = smem_u32(base + s * STAGE_BYTES);
        const uint32_t b_addr = a_addr + A_TILE;
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk)
          mma_bf16(d, smem_desc_sw128(a_addr + kk * 32), smem_desc_sw128(b_addr + kk * 32),
                   (c == 0 && kk == 0) ? 0u : 1u);
        mma_commit(&sh->empty[s]);
      }
      mma_commit(&sh->tfull[b]);
      if (!ok) break;
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: warp w owns TMEM lanes (rows) 32 (w mod 4) .. +31
    // and column half (w - 2) / 4 of every tile
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    const int NH = N / D;   // hashes per row (list mode)
    const int LS = EL + 1;  // list stride: EL keys and the cut
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = i & 1;
      const int m0 = (mfast ? t % ntm : t / ntn) * TC_BM;
      const int n0 = (mfast ? t / ntm : t % ntn) * TC_BN;
      if (!mbar_wait(&sh->tfull[b], (i >> 1) & 1, sh, err, 3)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = m0 + quarter * 32 + lane;
      const uint32_t taddr = tmem + (uint32_t)(b * TC_BN) + ((uint32_t)(quarter * 32) << 16);
      const int cbeg = half * (TC_BN / 2), cend = cbeg + TC_BN / 2;
      // the accumulator buffer goes back to the MMA warp once the warp's
      // TMEM loads have completed (the wide list path does so before its
      // last chunk, sign fix-up, merge and stores)
      bool released = false;
      auto release = [&]() {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh->tempty[b]);
        released = true;
      };
      bool ok = true;
      if (EL == 0) {
        for (int c0 = cbeg; c0 < cend; c0 += 32) {
          float v[32];
          tmem_ld32(taddr + (uint32_t)c0, v);
          if (row < M) {
            float* dst = C + (int64_t)row * ldc + n0 + c0;
            if (n0 + c0 + 32 <= N) {
#pragma unroll
              for (int k = 0; k < 32; k += 4)
                *reinterpret_cast<float4*>(dst + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
            } else {
              for (int k = 0; k < 32; ++k)
                if (n0 + c0 + k < N) dst[k] = v[k];
            }
          }
        }
      } else if (D >= 128) {
        // D = 128 or 256: the thread's 128 columns belong to one hash.  Keys
        // are ranked without the sign: (|p| bits with the low log2(2D)
        // cleared) | 2^31 | (column offset o < 128 within the thread's half),
        // one LOP3 per value with o an immediate; the signs are shifted into
        // one mask per 32 columns and put into the kept keys at the end.
        const int ldD = __ffs(D) - 1;
        const uint32_t keep = 0x7FFFFFFFu & ~(2u * (uint32_t)D - 1u);
        const uint32_t colbase = (uint32_t)cbeg & ((uint32_t)D - 1u);   // 0, or 128 when D = 256
        uint32_t tk[EL > 0 ? EL + 1 : 1];
#pragma unroll
        for (int e = 0; e <= EL; ++e) tk[e] = 0u;
        auto insert = [&](uint32_t x) {
#pragma unroll
          for (int e = 0; e < EL; ++e) {
            const uint32_t hi = max(tk[e], x);
            x = min(tk[e], x);
            tk[e] = hi;
          }
          tk[EL] = max(tk[EL], x);
        };
        uint32_t sg[4] = {0u, 0u, 0u, 0u};
        // the keys of 16 columns c0 .. c0 + 15 (c0 = 16 c): one LOP3 per
        // value, the signs shifted into sg[c / 2]
        auto chunk = [&](const uint32_t (&r)[16], const int c) {
          uint32_t m = sg[c >> 1];
          if (EL == 2) {
            // two keys at a time into the running top three (t0 >= t1 >= t2):
            // with hi >= lo the new second is max(t1, min(t0, hi), lo) and
            // the new third max(t2, min(t1, hi), min(t0, lo))
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
              const uint32_t u0 = r[k], u1 = r[k + 1];
              const uint32_t x = (u0 & keep) | (0x80000000u | (uint32_t)(16 * c + k));
              const uint32_t y = (u1 & keep) | (0x80000000u | (uint32_t)(16 * c + k + 1));
              m = __funnelshift_l(u0, m, 1);   // m = (m << 1) | sign(u): bit 31 - k is column k's
              m = __funnelshift_l(u1, m, 1);
              const uint32_t hi = max(x, y), lo = min(x, y);
              const uint32_t t2 = __vimax3_u32(tk[2], min(tk[1], hi), min(tk[0], lo));
              const uint32_t t1 = __vimax3_u32(tk[1], min(tk[0], hi), lo);
              tk[0] = max(tk[0], hi);
              tk[1] = t1;
              tk[2] = t2;
            }
          } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const uint32_t u = r[k];
              insert((u & keep) | (0x80000000u | (uint32_t)(16 * c + k)));
              m = __funnelshift_l(u, m, 1);
            }
          }
          sg[c >> 1] = m;
        };
        // eight chunks through two register buffers, the next load in flight
        // while a chunk is ranked
        uint32_t ra[16], rb[16];
        tmem_ld16_async(taddr + (uint32_t)cbeg, ra);
        tmem_wait(ra);
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
          tmem_ld16_async(taddr + (uint32_t)(cbeg + 16 * c + 16), rb);
          chunk(ra, c);
          tmem_wait(rb);
          if (c < 6) tmem_ld16_async(taddr + (uint32_t)(cbeg + 16 * c + 32), ra);
          else release();
          chunk(rb, c + 1);
          if (c < 6) tmem_wait(ra);
        }
        // signed keys 2^31 | (|p| bits) | h, h = column + D for p < 0
#pragma unroll
        for (int e = 0; e <= EL; ++e) {
          const uint32_t o = tk[e] & 127u, jj = o >> 5;
          const uint32_t msk = jj == 0 ? sg[0] : jj == 1 ? sg[1] : jj == 2 ? sg[2] : sg[3];
          const uint32_t neg = (msk >> (31u - (o & 31u))) & 1u;
          tk[e] = tk[e] ? ((tk[e] & keep) | 0x80000000u | (neg << ldD) | (colbase + o)) : 0u;
        }
        // the cut only needs its value
        const uint32_t cmask = 2u * (uint32_t)D - 1u;
        auto emit = [&]() {
          const int hg = n0 / D + half * (TC_BN / 2) / D;
          if (row < M && hg < NH) {
            uint64_t* dst = lists + ((int64_t)row * NH + hg) * LS;
#pragma unroll
            for (int e = 0; e < EL; ++e)
              dst[e] = tk[e] ? (((uint64_t)((tk[e] & keep) + 1u) << 32) |
                                (uint64_t)(0xFFFFFFFFu - (tk[e] & cmask)))
                             : 0ull;
            dst[EL] = tk[EL] ? ((uint64_t)((tk[EL] & keep) + 1u) << 32) : 0ull;
          }
        };
        if (D == TC_BN) {
          // the hash spans both column halves: the second half hands its
          // list to the first (bounded waits: a wait that runs out ends the
          // CTA's loop like the others)
          if (half == 1) {
            if (i > 0 && !mbar_wait(&sh->xempty[quarter], (i - 1) & 1, sh, err, 5)) {
              ok = false;
            } else {
#pragma unroll
              for (int e = 0; e <= EL; ++e) sh->xk[quarter][lane][e] = tk[e];
              __syncwarp();
              if (lane == 0) mbar_arrive(&sh->xfull[quarter]);
            }
          } else if (!mbar_wait(&sh->xfull[quarter], i & 1, sh, err, 5)) {
            ok = false;
          } else {
#pragma unroll
            for (int f = 0; f <= EL; ++f) insert(sh->xk[quarter][lane][f]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->xempty[quarter]);
            emit();
          }
        } else {
          emit();
        }
      } else {
        // running top-(EL + 1) packed keys of the current hash (descending;
        // 0 = none): entries 0..EL-1 form the list, entry EL is the cut
        const uint32_t dmask = (uint32_t)D - 1u;   // D is a power of two dividing 256
        const int ldD = __ffs(D) - 1;
        const uint32_t cmask = 2u * (uint32_t)D - 1u;
        const uint32_t keep = 0x7FFFFFFFu & ~cmask;
        uint32_t tk[EL > 0 ? EL + 1 : 1];
#pragma unroll
        for (int e = 0; e <= EL; ++e) tk[e] = 0u;
        auto insert = [&](uint32_t x) {
#pragma unroll
          for (int e = 0; e < EL; ++e) {
            const uint32_t hi = max(tk[e], x);
            x = min(tk[e], x);
            tk[e] = hi;
          }
          tk[EL] = max(tk[EL], x);
        };
        auto emit = [&](int col_last) {
          const int hg = (n0 + col_last) / D;
          if (row < M && hg < NH) {
            uint64_t* dst = lists + ((int64_t)row * NH + hg) * LS;
#pragma unroll
            for (int e = 0; e < EL; ++e)
              dst[e] = tk[e] ? (((uint64_t)((tk[e] & keep) + 1u) << 32) |
                                (uint64_t)(0xFFFFFFFFu - (tk[e] & cmask)))
                             : 0ull;
            dst[EL] = tk[EL] ? ((uint64_t)((tk[EL] & keep) + 1u) << 32) : 0ull;
          }
#pragma unroll
          for (int e = 0; e <= EL; ++e) tk[e] = 0u;
        };
        uint32_t ra[32], rb[32];
        tmem_ld32_async(taddr + (uint32_t)cbeg, ra);
        tmem_wait(ra);
#pragma unroll
        for (int c0 = cbeg; c0 < cend; c0 += 32) {
          const bool more = c0 + 32 < cend;
          if (more) tmem_ld32_async(taddr + (uint32_t)(c0 + 32), rb);
          // n0 is a multiple of 256 and c0 of 32, so the column within the
          // hash is (c0 mod D) + k for D >= 32 and k mod D otherwise
          const uint32_t cb = 0x80000000u | (D >= 32 ? ((uint32_t)c0 & dmask) : 0u);
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const uint32_t u = ra[k];
            const uint32_t i_in = (uint32_t)k & dmask;
            insert((u & keep) | (cb + (D >= 32 ? (uint32_t)k : i_in)) | ((u >> 31) << ldD));
            if (D < 32 && i_in == dmask) emit(c0 + k);
          }
          if (D >= 32 && D <= TC_BN / 2 && (((uint32_t)(c0 + 31) & dmask) == dmask)) emit(c0 + 31);
          if (more) {
            tmem_wait(rb);
#pragma unroll
            for (int k = 0; k < 32; ++k) ra[k] = rb[k];
          }
        }
      }
      if (!released) release();
      if (!ok) break;
    }
  }
  // An aborted CTA drains before it frees TMEM and exits: the copies it
  // issued land (each stage's last issued chunk completes its full barrier;
  // a stage is refilled only after that) and its MMAs complete (one commit
  // tracks every MMA the issuing thread started).
  __syncthreads();
  if (*(volatile int*)&sh->abort) {
    if (warp == 0 && lane == 0) {
      for (int s = 0; s < TC_STAGES; ++s)
        if ((issued >> s) & 1u) mbar_wait_drain(&sh->full[s], (last_g[s] / TC_STAGES) & 1, sh->limit);
    } else if (warp == 1 && lane == 0) {
      mma_commit(&sh->drain);
      mbar_wait_drain(&sh->drain, 0, sh->limit);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u)
                 : "memory");
  }
}

// Splits rows of an FP32 matrix into BF16 pieces [rows][pieces * Kp]:
// piece 0 = bf16(x), piece 1 = bf16(x - piece0), piece 2 = bf16(x - p0 - p1);
// columns d..Kp-1 of every piece are zero.
__global__ void split_bf16_kernel(const float* __restrict__ src, int64_t rows, int64_t lds, int d,
                                  int Kp, int pieces, __nv_bfloat16* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * Kp) return;
  const int64_t r = i / Kp;
  const int c = (int)(i - r * Kp);
  float x = c < d ? src[r * lds + c] : 0.f;
  __nv_bfloat16* o = dst + r * (int64_t)pieces * Kp + c;
  for (int p = 0; p < pieces; ++p) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    o[(int64_t)p * Kp] = h;
    x = __fsub_rn(x, __bfloat162float(h));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

fpp_status make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, uint32_t box_rows) {
  auto enc = get_encoder();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is unavailable");
    return FPP_ECUDA;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BK, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
    return FPP_ECUDA;
  }
  return FPP_OK;
}

}  // namespace

int tc_kpad(int d) { return (int)round_up(d, TC_BK); }

double tc_error_bound_factor(int Kp, int pieces) {
  // Relative bound (times ||a|| ||b||) of one tensor-core projection.
  // Exact split: the accumulation error is at most u * (sum of partial-sum
  // magnitudes); the 5 Kp small products keep partial sums below
  // 2^-7 sum|a b|, the Kp main products below (1 + 2^-7) sum|a b|, so the
  // bound is gamma_Kp (1 + 5 2^-7 + 2^-7) doubled to allow truncating
  // accumulation, plus the dropped products (< 2^-23 |a||b|) and the BF16
  // piece residuals.  The three-product form (B on the BF16 grid) drops
  // nothing and its two small products likewise keep the partial sums below
  // 2^-7 sum|a b|, so the same bound holds.  Plain BF16: the input rounding
  // 2 * 2^-8 dominates.
  if (pieces == 1) return 2.0 * 3.90625e-3 + 2.0 * gamma_fp32(Kp) + 1.6e-5;
  return 2.0 * gamma_fp32(Kp) * 1.05 + 2.0e-7;
}

double bf16_window_factor(int d) {
  // Near-tie window of a dot product with one operand rounded to BF16,
  // relative to ||a|| ||b||.  Rounding to BF16 (unit roundoff u = 2^-8)
  // perturbs each product by a relative error of variance at most u^2 / 3,
  // so for vectors whose mass is spread over the d coordinates the error has
  // standard deviation about u ||a|| ||b|| / sqrt(3 d).  The window is nine of
  // those plus the worst-case FP32 accumulation error: a statistical margin,
  // not a bound (the BF16 path is graded by recall and score error).
  return 9.0 * 3.90625e-3 / std::sqrt(3.0 * (double)d) + 2.0 * gamma_fp32(tc_kpad(d));
}

double fp8_window_factor(int d) {
  // e4m3 keeps 3 fraction bits (unit roundoff 2^-4); rows are scaled so their
  // largest magnitude is 448, which keeps every element above the subnormal
  // range unless it is below 2^-6 / 448 of that magnitude.  Nine standard
  // deviations of u ||a|| ||b|| / sqrt(3 d), plus the subnormal spacing
  // (2^-9 of the scale unit) over d elements and the FP32 accumulation bound.
  return 9.0 * 0.0625 / std::sqrt(3.0 * (double)d) + (double)d * std::ldexp(1.0, -9) / 448.0 +
         2.0 * gamma_fp32(tc_kpad(d));
}

namespace {
__global__ void rows_fp8_kernel(const float* __restrict__ src, int64_t rows, int64_t lds, int d,
                                int64_t ldo, __nv_fp8_storage_t* __restrict__ dst,
                                float* __restrict__ scale) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const float* x = src + r * lds;
  float m = 0.f;
  for (int i = lane; i < d; i += 32) m = fmaxf(m, fabsf(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const float sc = m > 0.f ? m / 448.f : 1.f;
  for (int i = lane; i < ldo; i += 32)
    dst[r * ldo + i] = i < d ? __nv_cvt_float_to_fp8(x[i] / sc, __NV_SATFINITE, __NV_E4M3)
                             : (__nv_fp8_storage_t)0;
  if (lane == 0) scale[r] = sc;
}
}  // namespace

fpp_status rows_to_fp8(const float* src, int64_t rows, int64_t lds, int d, int64_t ldo, void* dst,
                       float* scale, cudaStream_t st) {
  if (rows <= 0) return FPP_OK;
  rows_fp8_kernel<<<(unsigned)ceil_div(rows, 8), 256, 0, st>>>(
      src, rows, lds, d, ldo, reinterpret_cast<__nv_fp8_storage_t*>(dst), scale);
  FPP_LAUNCHED();
  return FPP_OK;
}

namespace {
__global__ void rows_bf16_kernel(const float* __restrict__ src, int64_t rows, int64_t lds, int d,
                                 int64_t ldo, __nv_bfloat16* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * ldo) return;
  const int64_t r = i / ldo;
  const int c = (int)(i - r * ldo);
  dst[i] = __float2bfloat16_rn(c < d ? src[r * lds + c] : 0.f);
}
}  // namespace

fpp_status rows_to_bf16(const float* src, int64_t rows, int64_t lds, int d, int64_t ldo, void* dst,
                        cudaStream_t st) {
  if (rows <= 0) return FPP_OK;
  rows_bf16_kernel<<<(unsigned)ceil_div(rows * ldo, 256), 256, 0, st>>>(
      src, rows, lds, d, ldo, reinterpret_cast<__nv_bfloat16*>(dst));
  FPP_LAUNCHED();
  return FPP_OK;
}

fpp_status split_to_bf16(const float* src, int64_t rows, int64_t lds, int d, int pieces,
                         void* dst, cudaStream_t st) {
  if (rows <= 0) return FPP_OK;
  const int Kp = tc_kpad(d);
  const int64_t total = rows * Kp;
  split_bf16_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(
      src, rows, lds, d, Kp, pieces, reinterpret_cast<__nv_bfloat16*>(dst));
  FPP_LAUNCHED();
  return FPP_OK;
}

namespace {

template <int EL>
fpp_status launch_proj(const CUtensorMap& ma, const CUtensorMap& mb, float* C, int64_t ldc,
                       uint64_t* lists, int64_t M, int64_t N, int Kp, int pieces, int bpieces,
                       int D, int* err, cudaStream_t st, long long wait_cycles, int withhold) {
  const size_t smem = 1024 + TC_STAGES * STAGE_BYTES + sizeof(TcShared);
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&]() {
    attr_err = cudaFuncSetAttribute(tc_proj_kernel<EL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
  });
  FPP_CUDA(attr_err);
  int dev = 0, sms = 0;
  FPP_CUDA(cudaGetDevice(&dev));
  FPP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t ntiles = ceil_div(M, TC_BM) * ceil_div(N, TC_BN);
  const int grid = (int)std::min<int64_t>(ntiles, sms);
  const int mfast = N * bpieces > M * pieces ? 1 : 0;   // B's bytes read > A's
  tc_proj_kernel<EL><<<grid, TC_THREADS, smem, st>>>(ma, mb, C, ldc, lists, (int)M, (int)N, Kp,
                                                     pieces, bpieces, D, mfast, err, wait_cycles,
                                                     withhold);
  FPP_LAUNCHED();
  return FPP_OK;
}

}  // namespace

float tc_list_trunc(int D) {
  // |p| - |p|' < 2^(b - 23) |p| with b = log2(2D) cleared mantissa bits;
  // relative to |p|' it is below 2^(b - 23) / (1 - 2^(b - 23)), rounded up
  int b = 0;
  while ((1 << b) < 2 * D) ++b;
  const double t = std::ldexp(1.0, b - 23);
  return (float)(t / (1.0 - t) * 1.0001);
}

int tc_list_len(int want) {
  if (want <= 2) return 2;
  if (want <= 4) return 4;
  if (want <= 8) return 8;
  return 0;
}

fpp_status gemm_tc(const void* A, int64_t M, const void* B, int64_t N, int Kp, int pieces, float* C,
                   int64_t ldc, int* err, cudaStream_t st) {
  return project_tc(A, M, B, N, Kp, pieces, pieces, 0, 0, C, ldc, nullptr, err, st);
}

fpp_status project_tc(const void* A, int64_t M, const void* B, int64_t N, int Kp, int pieces,
                      int bpieces, int D, int EL, float* C, int64_t ldc, uint64_t* lists, int* err,
                      cudaStream_t st, long long wait_cycles, int withhold, int b_row_pieces) {
  if (M <= 0 || N <= 0) return FPP_OK;
  if (!b_row_pieces) b_row_pieces = pieces;
  if (b_row_pieces < pieces) {
    set_error("project_tc: B rows hold fewer pieces than A's");
    return FPP_EINTERNAL;
  }
  if (Kp % TC_BK || (pieces != 1 && pieces != 3) || (bpieces != 1 && bpieces != pieces) ||
      M >= (1ll << 31) || N >= (1ll << 31)) {
    set_error("project_tc: bad shape");
    return FPP_EINTERNAL;
  }
  if (EL == 0 && ((ldc & 3) || ((uintptr_t)C & 15))) {
    set_error("project_tc: C must be 16-byte aligned with ldc a multiple of 4");
    return FPP_EINTERNAL;
  }
  if (EL != 0 && (D < 1 || TC_BN % D != 0 || N % D != 0 || !lists)) {
    set_error("project_tc: list mode needs D dividing 256");
    return FPP_EINTERNAL;
  }
  CUtensorMap ma, mb;
  FPP_TRY(make_map(&ma, A, M, (int64_t)pieces * Kp, TC_BM));
  FPP_TRY(make_map(&mb, B, N, (int64_t)b_row_pieces * Kp, TC_BN));
  switch (EL) {
    case 0: return launch_proj<0>(ma, mb, C, ldc, lists, M, N, Kp, pieces, bpieces, D, err, st,
                                    wait_cycles, withhold);
    case 2: return launch_proj<2>(ma, mb, C, ldc, lists, M, N, Kp, pieces, bpieces, D, err, st,
                                    wait_cycles, withhold);
    case 4: return launch_proj<4>(ma, mb, C, ldc, lists, M, N, Kp, pieces, bpieces, D, err, st,
                                    wait_cycles, withhold);
    case 8: return launch_proj<8>(ma, mb, C, ldc, lists, M, N, Kp, pieces, bpieces, D, err, st,
                                    wait_cycles, withhold);
    default:
      set_error("project_tc: list length must be 0, 2, 4 or 8");
      return FPP_EINTERNAL;
  }
}

}  // namespace fpp
