// FP32 SIMT projection GEMM: C[M][N] = A[M][K] * B[N][K]^T.
//
// This is the projection step of Falconn++ (Section 2.2: every point or query
// is projected onto the D random vectors of every hash of every table), in
// plain FP32 on the CUDA cores, so that every projection carries the error
// bound gamma_K * ||a|| * ||b|| that the exact-decision logic downstream relies
// on.  128x128 output tile per CTA, 8x8 outputs per thread, K staged through
// shared memory in slices of 16 with register double buffering.
//
// Requirements (checked by the launcher): K, lda, ldb, ldc multiples of 4;
// A, B, C 16-byte aligned.  M, N arbitrary.
#include "common.cuh"
#include "kernels.h"

namespace fpp {

namespace {

constexpr int BM = 128, BN = 128, BK = 16, PAD = 4;

__global__ void __launch_bounds__(256, 2)
sgemm_nt_kernel(const float* __restrict__ A, int64_t lda, const float* __restrict__ B,
                int64_t ldb, float* __restrict__ C, int64_t ldc, int M, int N, int K) {
  __shared__ __align__(16) float As[2][BK][BM + PAD];
  __shared__ __align__(16) float Bs[2][BK][BN + PAD];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  // Loader mapping: thread -> (row = tid & 127, k-quad = tid >> 7 and +2).
  const int lrow = tid & 127;
  const int lkq = tid >> 7;  // 0 or 1
  const bool a_ok = (m0 + lrow) < M;
  const bool b_ok = (n0 + lrow) < N;
  const float* Ap = A + (int64_t)(m0 + (a_ok ? lrow : 0)) * lda;
  const float* Bp = B + (int64_t)(n0 + (b_ok ? lrow : 0)) * ldb;

  float4 ra[2], rb[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int kk = k0 + (lkq + 2 * h) * 4;
      const bool kin = kk < K;
      ra[h] = (a_ok && kin) ? *reinterpret_cast<const float4*>(Ap + kk) : make_float4(0, 0, 0, 0);
      rb[h] = (b_ok && kin) ? *reinterpret_cast<const float4*>(Bp + kk) : make_float4(0, 0, 0, 0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int kq = (lkq + 2 * h) * 4;
      As[buf][kq + 0][lrow] = ra[h].x;
      As[buf][kq + 1][lrow] = ra[h].y;
      As[buf][kq + 2][lrow] = ra[h].z;
      As[buf][kq + 3][lrow] = ra[h].w;
      Bs[buf][kq + 0][lrow] = rb[h].x;
      Bs[buf][kq + 1][lrow] = rb[h].y;
      Bs[buf][kq + 2][lrow] = rb[h].z;
      Bs[buf][kq + 3][lrow] = rb[h].w;
    }
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  const int nk = (K + BK - 1) / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[8], b[8];
      float4 t0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
      float4 t1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4 + 64]);
      float4 u0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
      float4 u1 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4 + 64]);
      a[0] = t0.x; a[1] = t0.y; a[2] = t0.z; a[3] = t0.w;
      a[4] = t1.x; a[5] = t1.y; a[6] = t1.z; a[7] = t1.w;
      b[0] = u0.x; b[1] = u0.y; b[2] = u0.z; b[3] = u0.w;
      b[4] = u1.x; b[5] = u1.y; b[6] = u1.z; b[7] = u1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) {
      store(buf ^ 1);
      __syncthreads();
    }
  }

  // Epilogue: rows ty*4+i (+64), columns tx*4+j (+64).
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
    if (r >= M) continue;
    float* Cr = C + (int64_t)r * ldc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = n0 + tx * 4 + h * 64;
      if (c + 3 < N) {
        *reinterpret_cast<float4*>(Cr + c) =
            make_float4(acc[i][h * 4 + 0], acc[i][h * 4 + 1], acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c + j < N) Cr[c + j] = acc[i][h * 4 + j];
      }
    }
  }
}

}  // namespace

fpp_status gemm_f32_nt(const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                       int64_t ldc, int64_t M, int64_t N, int K, cudaStream_t st) {
  if (M <= 0 || N <= 0) return FPP_OK;
  if ((K & 3) || (lda & 3) || (ldb & 3) || (ldc & 3) ||
      ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)C & 15)) {
    set_error("gemm_f32_nt: K, lda, ldb, ldc must be multiples of 4 and pointers 16-byte aligned");
    return FPP_EINTERNAL;
  }
  if (ceil_div(M, BM) > 65535) {
    set_error("gemm_f32_nt: M too large for one launch");
    return FPP_EINTERNAL;
  }
  dim3 grid((unsigned)ceil_div(N, BN), (unsigned)ceil_div(M, BM));
  sgemm_nt_kernel<<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, (int)M, (int)N, K);
  FPP_LAUNCHED();
  return FPP_OK;
}

}  // namespace fpp
