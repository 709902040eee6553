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
// hi.hi in one TMEM accumulator and the five next-order products (hi.mid,
// mid.hi, hi.lo, mid.mid, lo.hi) in a second one, and the epilogue adds the
// two.  The dropped products are below 2^-23 |a||b|, the correction
// accumulator is 2^-7 smaller than the main one, so the error bound stays
// within a small factor of the FP32 one (see tc_error_bound).
//
// Plain mode (pieces = 1): one BF16 product, for the BF16 precision path.
//
// Roles (192 threads): warp 0 issues TMA loads, warp 1 allocates tensor
// memory and issues the MMAs (one elected lane), warps 2..5 drain the
// accumulators (warp w reads TMEM lanes 32 (w mod 4) .. +31, i.e. the rows it
// owns) and store FP32 results.  Every mbarrier wait is bounded; a wait that
// runs out records an error code and the CTA drains and exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace fpp {

namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64;   // BK: 64 BF16 = one 128-byte row
constexpr int TC_STAGES = 3;
constexpr int TC_THREADS = 192;
constexpr uint32_t TILE_BYTES = TC_BM * TC_BK * 2;     // 16 KB (A and B tiles alike)
constexpr long long WAIT_CYCLES = 4000000000ll;        // ~2 s at 2 GHz

struct __align__(8) TcShared {
  uint64_t full[TC_STAGES];
  uint64_t empty[TC_STAGES];
  uint64_t acc_ready;
  uint32_t tmem_base;
  int abort;
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
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(&sh->abort, 1);
      if (err) atomicExch(err, code);
      return false;
    }
  }
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

// Instruction descriptor: D = F32, A = B = BF16, both K-major, M = 128, N = 128.
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

// Chunk c of the K loop: which A piece, which B piece, which 64-wide K block,
// and which accumulator.  Exact-split order: hi.hi first (accumulator 0),
// then hi.mid, mid.hi, hi.lo, mid.mid, lo.hi (accumulator 1).
__device__ __forceinline__ void chunk_pieces(int c, int nkb, int pieces, int& pa, int& pb,
                                             int& kb, int& acc, bool& first) {
  const int pair = c / nkb;
  kb = c - pair * nkb;
  if (pieces == 1) {
    pa = pb = 0; acc = 0; first = (kb == 0);
    return;
  }
  const int PA[6] = {0, 0, 1, 0, 1, 2};
  const int PB[6] = {0, 1, 0, 2, 1, 0};
  pa = PA[pair];
  pb = PB[pair];
  acc = pair == 0 ? 0 : 1;
  first = (kb == 0) && (pair <= 1);
}

__global__ void __launch_bounds__(TC_THREADS, 2)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
               float* __restrict__ C, int64_t ldc, int M, int N, int Kp, int pieces, int* err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  // 1024-byte alignment of the tile ring (required by the 128-byte swizzle)
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dsm) + 1023) & ~(uintptr_t)1023);
  unsigned char* tilesA = base;
  unsigned char* tilesB = base + TC_STAGES * TILE_BYTES;
  TcShared* sh = reinterpret_cast<TcShared*>(base + 2 * TC_STAGES * TILE_BYTES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * TC_BN, m0 = blockIdx.y * TC_BM;
  const int nkb = Kp / TC_BK;
  const int nchunks = (pieces == 1 ? 1 : 6) * nkb;
  const uint32_t ncols = pieces == 1 ? 128u : 256u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&sh->full[s], 1);
      mbar_init(&sh->empty[s], 1);
    }
    mbar_init(&sh->acc_ready, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh->tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sh->tmem_base;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % TC_STAGES;
      const uint32_t round = (uint32_t)(c / TC_STAGES);
      if (c >= TC_STAGES && !mbar_wait(&sh->empty[s], (round - 1) & 1, sh, err, 1)) break;
      int pa, pb, kb, acc;
      bool first;
      chunk_pieces(c, nkb, pieces, pa, pb, kb, acc, first);
      mbar_expect_tx(&sh->full[s], 2 * TILE_BYTES);
      tma_load_2d(tilesA + s * TILE_BYTES, &mapA, pa * Kp + kb * TC_BK, m0, &sh->full[s]);
      tma_load_2d(tilesB + s * TILE_BYTES, &mapB, pb * Kp + kb * TC_BK, n0, &sh->full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % TC_STAGES;
      const uint32_t round = (uint32_t)(c / TC_STAGES);
      if (!mbar_wait(&sh->full[s], round & 1, sh, err, 2)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int pa, pb, kb, acc;
      bool first;
      chunk_pieces(c, nkb, pieces, pa, pb, kb, acc, first);
      const uint32_t a_addr = smem_u32(tilesA + s * TILE_BYTES);
      const uint32_t b_addr = smem_u32(tilesB + s * TILE_BYTES);
      const uint32_t d = tmem + (uint32_t)(acc * TC_BN);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        // K step of 16 BF16 = 32 bytes inside the swizzled 128-byte row
        mma_bf16(d, smem_desc_sw128(a_addr + kk * 32), smem_desc_sw128(b_addr + kk * 32),
                 (first && kk == 0) ? 0u : 1u);
      }
      mma_commit(&sh->empty[s]);
    }
    mma_commit(&sh->acc_ready);
  } else if (warp >= 2) {
    // ---------------- epilogue: TMEM -> registers -> global
    const int quarter = warp & 3;
    const bool ok = mbar_wait(&sh->acc_ready, 0, sh, err, 3);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int row = m0 + quarter * 32 + lane;
      const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
      for (int c0 = 0; c0 < TC_BN; c0 += 32) {
        float v[32];
        tmem_ld32(lane_addr + (uint32_t)c0, v);
        if (pieces != 1) {
          float w[32];
          tmem_ld32(lane_addr + (uint32_t)(TC_BN + c0), w);
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = __fadd_rn(v[i], w[i]);
        }
        if (row < M) {
          float* dst = C + (int64_t)row * ldc + n0 + c0;
          if (n0 + c0 + 32 <= N) {
#pragma unroll
            for (int i = 0; i < 32; i += 4)
              *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
          } else {
            for (int i = 0; i < 32; ++i)
              if (n0 + c0 + i < N) dst[i] = v[i];
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
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
  // Relative bound (times ||a|| ||b||) of one exact-split tensor-core
  // projection: main accumulator 2 gamma_Kp (a factor 2 allows truncating
  // accumulation), correction accumulator 2 gamma_{5 Kp} 2^-7, dropped
  // products 2^-23, final addition 2^-24; plain BF16 adds the input rounding.
  if (pieces == 1) return 2.0 * 3.90625e-3 + 2.0 * gamma_fp32(Kp) + 1.5e-5;
  return 2.0 * gamma_fp32(Kp) * 1.01 + 2.0 * gamma_fp32(5ll * Kp) * 7.8125e-3 + 1.2e-7 + 6.0e-8;
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

fpp_status gemm_tc(const void* A, int64_t M, const void* B, int64_t N, int Kp, int pieces, float* C,
                   int64_t ldc, int* err, cudaStream_t st) {
  if (M <= 0 || N <= 0) return FPP_OK;
  if (Kp % TC_BK || (ldc & 3) || ((uintptr_t)C & 15) || (pieces != 1 && pieces != 3)) {
    set_error("gemm_tc: bad shape");
    return FPP_EINTERNAL;
  }
  if (ceil_div(M, TC_BM) > 65535) {
    set_error("gemm_tc: M too large for one launch");
    return FPP_EINTERNAL;
  }
  CUtensorMap ma, mb;
  FPP_TRY(make_map(&ma, A, M, (int64_t)pieces * Kp, TC_BM));
  FPP_TRY(make_map(&mb, B, N, (int64_t)pieces * Kp, TC_BN));
  const size_t smem = 1024 + 2 * TC_STAGES * TILE_BYTES + sizeof(TcShared);
  static std::once_flag attr;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr, [&]() {
    attr_err = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
  });
  FPP_CUDA(attr_err);
  dim3 grid((unsigned)ceil_div(N, TC_BN), (unsigned)ceil_div(M, TC_BM));
  tc_gemm_kernel<<<grid, TC_THREADS, smem, st>>>(ma, mb, C, ldc, (int)M, (int)N, Kp, pieces, err);
  FPP_LAUNCHED();
  return FPP_OK;
}

}  // namespace fpp
