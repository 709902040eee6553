// Shared device/host helpers of libfpp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <string>

#include "../../include/fpp.h"

namespace fpp {

// ---------------------------------------------------------------- errors

void set_error(const std::string& msg);
std::atomic<uint64_t>& launch_counter();
// Device allocations made by the library (every cudaMalloc goes through
// dev_malloc), for callers that check that a phase allocates nothing.
std::atomic<uint64_t>& alloc_counter();
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  alloc_counter().fetch_add(1, std::memory_order_relaxed);
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

struct Status {
  fpp_status code = FPP_OK;
  bool ok() const { return code == FPP_OK; }
};

#define FPP_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      ::fpp::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));   \
      return e_ == cudaErrorMemoryAllocation ? FPP_ENOMEM : FPP_ECUDA;        \
    }                                                                         \
  } while (0)

#define FPP_LAUNCHED()                                                        \
  do {                                                                        \
    ::fpp::launch_counter().fetch_add(1, std::memory_order_relaxed);          \
    cudaError_t e_ = cudaGetLastError();                                      \
    if (e_ != cudaSuccess) {                                                  \
      ::fpp::set_error(std::string("kernel launch: ") + cudaGetErrorString(e_)); \
      return FPP_ECUDA;                                                       \
    }                                                                         \
  } while (0)

#define FPP_TRY(expr)                                                         \
  do {                                                                        \
    fpp_status s_ = (expr);                                                   \
    if (s_ != FPP_OK) return s_;                                              \
  } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// ---------------------------------------------------------------- error bounds
//
// gamma_n = n u / (1 - n u) bounds the relative error of any n-term FP32
// dot product evaluated with rounding to nearest, whatever the order of the
// additions (Higham, "Accuracy and Stability of Numerical Algorithms", 3.1):
// |fl(x^T y) - x^T y| <= gamma_n sum |x_i y_i| <= gamma_n ||x|| ||y||.
inline double gamma_fp32(int64_t n) {
  const double u = 5.9604644775390625e-08;  // 2^-24
  return (n * u) / (1.0 - n * u);
}

// ---------------------------------------------------------------- device math

#ifdef __CUDACC__

// Error-free transformations (Knuth's TwoSum; TwoProduct with a fused
// multiply-add).  Explicit _rn intrinsics keep the compiler from fusing or
// reassociating them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// A float-float value hi + lo.
struct FF {
  float hi, lo;
};

// Accumulates a * b into (p, s) as in the compensated dot product "Dot2" of
// Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci.
// Comput. 26(6), 2005, Algorithm 5.3): p carries the running sum, s the
// running sum of the rounding errors.  The result p + s is as accurate as a
// dot product computed in twice the working precision.
__device__ __forceinline__ void dot2_step(float a, float b, float& p, float& s) {
  float h, r, q;
  two_prod(a, b, h, r);
  two_sum(p, h, p, q);
  s = __fadd_rn(s, __fadd_rn(q, r));
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  return FF{s, __fadd_rn(__fadd_rn(x.lo, y.lo), e)};
}

__device__ __forceinline__ double ff_value(FF x) { return (double)x.hi + (double)x.lo; }

// hi + lo renormalised so that hi = fl(hi + lo) (an error-free TwoSum): such
// pairs order like their exact sums by comparing hi, then lo, which keeps
// exact comparisons off the (slow) FP64 pipe.
__device__ __forceinline__ FF ff_norm(FF x) {
  float s, e;
  two_sum(x.hi, x.lo, s, e);
  return FF{s, e};
}

// |x| of a normalised pair (hi carries the sign of the sum; hi = 0 means 0).
__device__ __forceinline__ FF ff_abs(FF x) { return x.hi < 0.f ? FF{-x.hi, -x.lo} : x; }

// a before b: larger value (normalised pairs), ties by lower id.
__device__ __forceinline__ bool ff_before(FF a, uint32_t ia, FF b, uint32_t ib) {
  if (a.hi != b.hi) return a.hi > b.hi;
  if (a.lo != b.lo) return a.lo > b.lo;
  return ia < ib;
}

// Normalised sum of two normalised pairs (relative error about 2^-46).
__device__ __forceinline__ FF ff_sum(FF x, FF y) { return ff_norm(ff_add(x, y)); }

// Warp-cooperative compensated dot product of two length-n FP32 vectors;
// every lane returns the result.  Lanes take strided elements; the 32 partial
// float-float sums are combined with error-free additions.
__device__ __forceinline__ double warp_dot2(const float* __restrict__ a,
                                            const float* __restrict__ b, int n) {
  const int lane = threadIdx.x & 31;
  float p = 0.f, s = 0.f;
  for (int i = lane; i < n; i += 32) dot2_step(a[i], b[i], p, s);
  FF v{p, s};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    FF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = ff_add(v, w);
  }
  return ff_value(v);
}

// Warp-cooperative compensated dot products of q with NR rows r_0..r_{NR-1}
// (row stride ldr floats); q and the rows are 16-byte aligned with nf4 float4
// per row.  Lanes read float4 chunks (coalesced); the NR rows are in flight
// together.  Every lane returns all NR results as normalised pairs.
template <int NR>
__device__ __forceinline__ void warp_dot2_rows_ff(const float* __restrict__ q,
                                                  const float* __restrict__ r0, int64_t ldr,
                                                  int nf4, FF* out) {
  const int lane = threadIdx.x & 31;
  float p[NR], s[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) { p[k] = 0.f; s[k] = 0.f; }
  const float4* q4 = reinterpret_cast<const float4*>(q);
  for (int c = lane; c < nf4; c += 32) {
    const float4 a = q4[c];
    float4 b[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) b[k] = __ldg(reinterpret_cast<const float4*>(r0 + k * ldr) + c);
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      dot2_step(a.x, b[k].x, p[k], s[k]);
      dot2_step(a.y, b[k].y, p[k], s[k]);
      dot2_step(a.z, b[k].z, p[k], s[k]);
      dot2_step(a.w, b[k].w, p[k], s[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    FF v{p[k], s[k]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      FF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
      v = ff_add(v, w);
    }
    out[k] = ff_norm(v);
  }
}

template <int NR>
__device__ __forceinline__ void warp_dot2_rows(const float* __restrict__ q,
                                               const float* __restrict__ r0, int64_t ldr,
                                               int nf4, double* out) {
  FF v[NR];
  warp_dot2_rows_ff<NR>(q, r0, ldr, nf4, v);
#pragma unroll
  for (int k = 0; k < NR; ++k) out[k] = ff_value(v[k]);
}

// Same, for NR rows at arbitrary addresses (16-byte aligned).
template <int NR>
__device__ __forceinline__ void warp_dot2_gather_ff(const float* __restrict__ q,
                                                    const float* const* rows, int nf4, FF* out) {
  const int lane = threadIdx.x & 31;
  float p[NR], s[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) { p[k] = 0.f; s[k] = 0.f; }
  const float4* q4 = reinterpret_cast<const float4*>(q);
  for (int c = lane; c < nf4; c += 32) {
    const float4 a = q4[c];
    float4 b[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) b[k] = __ldg(reinterpret_cast<const float4*>(rows[k]) + c);
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      dot2_step(a.x, b[k].x, p[k], s[k]);
      dot2_step(a.y, b[k].y, p[k], s[k]);
      dot2_step(a.z, b[k].z, p[k], s[k]);
      dot2_step(a.w, b[k].w, p[k], s[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    FF v{p[k], s[k]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      FF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
      v = ff_add(v, w);
    }
    out[k] = ff_norm(v);
  }
}

// Same, for rows stored as BF16 bit patterns (uint16, a BF16 value is exact
// in FP32: its bits shifted up by 16).  q has dq floats (a multiple of 4);
// each row holds at least round_up(dq, 8) values, zero past the vector, and
// is 16-byte aligned.  Lanes read 8-value chunks; a last 4-value chunk is
// taken by lane 0.
__device__ __forceinline__ void dot2_bf2(float a0, float a1, uint32_t w, float& p, float& s) {
  dot2_step(a0, __uint_as_float(w << 16), p, s);
  dot2_step(a1, __uint_as_float(w & 0xFFFF0000u), p, s);
}

template <int NR>
__device__ __forceinline__ void warp_dot2_gather_bf_ff(const float* __restrict__ q,
                                                       const uint16_t* const* rows, int dq,
                                                       FF* out) {
  const int lane = threadIdx.x & 31;
  float p[NR], s[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) { p[k] = 0.f; s[k] = 0.f; }
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const int n8 = dq >> 3;
  for (int c = lane; c < n8; c += 32) {
    const float4 a0 = q4[2 * c], a1 = q4[2 * c + 1];
    uint4 b[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) b[k] = __ldg(reinterpret_cast<const uint4*>(rows[k]) + c);
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      dot2_bf2(a0.x, a0.y, b[k].x, p[k], s[k]);
      dot2_bf2(a0.z, a0.w, b[k].y, p[k], s[k]);
      dot2_bf2(a1.x, a1.y, b[k].z, p[k], s[k]);
      dot2_bf2(a1.z, a1.w, b[k].w, p[k], s[k]);
    }
  }
  if ((dq & 4) && lane == 0) {
    const float4 a0 = q4[2 * n8];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      const uint2 b = __ldg(reinterpret_cast<const uint2*>(rows[k] + 8 * n8));
      dot2_bf2(a0.x, a0.y, b.x, p[k], s[k]);
      dot2_bf2(a0.z, a0.w, b.y, p[k], s[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < NR; ++k) {
    FF v{p[k], s[k]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      FF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
      v = ff_add(v, w);
    }
    out[k] = ff_norm(v);
  }
}

template <int NR>
__device__ __forceinline__ void warp_dot2_gather(const float* __restrict__ q,
                                                 const float* const* rows, int nf4, double* out) {
  FF v[NR];
  warp_dot2_gather_ff<NR>(q, rows, nf4, v);
#pragma unroll
  for (int k = 0; k < NR; ++k) out[k] = ff_value(v[k]);
}

// Single-thread compensated dot product of two 16-byte aligned rows of nf4
// float4 chunks (four chunk loads in flight at a time).
__device__ __forceinline__ double thread_dot2_f4(const float* __restrict__ a,
                                                 const float* __restrict__ b, int nf4) {
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  float p = 0.f, s = 0.f;
  int c = 0;
  for (; c + 4 <= nf4; c += 4) {
    float4 x[4], y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { x[u] = __ldg(a4 + c + u); y[u] = __ldg(b4 + c + u); }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      dot2_step(x[u].x, y[u].x, p, s);
      dot2_step(x[u].y, y[u].y, p, s);
      dot2_step(x[u].z, y[u].z, p, s);
      dot2_step(x[u].w, y[u].w, p, s);
    }
  }
  for (; c < nf4; ++c) {
    const float4 x = __ldg(a4 + c), y = __ldg(b4 + c);
    dot2_step(x.x, y.x, p, s);
    dot2_step(x.y, y.y, p, s);
    dot2_step(x.z, y.z, p, s);
    dot2_step(x.w, y.w, p, s);
  }
  return ff_value(FF{p, s});
}

// Single-thread compensated dot product.
__device__ __forceinline__ double thread_dot2(const float* __restrict__ a,
                                              const float* __restrict__ b, int n) {
  float p = 0.f, s = 0.f;
  for (int i = 0; i < n; ++i) dot2_step(a[i], b[i], p, s);
  return ff_value(FF{p, s});
}

// Order-preserving map of a float to uint32 (larger float -> larger uint).
__device__ __forceinline__ uint32_t float_key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

#endif  // __CUDACC__

// Device checks of the FPP_DEBUG_BOUNDS build (a second library built from
// the same sources, in place of a memory checker): FPP_IN_BOUNDS(bd, cond,
// site, index) records the first failed condition in *bd.flag and returns
// false, so that the guarded access is skipped; in the product build it is
// the constant true and the condition is not evaluated.
#ifdef FPP_DEBUG_BOUNDS
template <class B>
__device__ __forceinline__ bool fpp_bounds_ok(const B& bd, bool cond, unsigned site,
                                              unsigned long long index) {
  if (cond) return true;
  if (bd.flag) atomicCAS(bd.flag, 0ull, ((unsigned long long)site << 48) | (index & 0xFFFFFFFFFFFFull));
  return false;
}
#define FPP_IN_BOUNDS(bd, cond, site, index) \
  ::fpp::fpp_bounds_ok((bd), (cond), (site), (unsigned long long)(index))
#else
#define FPP_IN_BOUNDS(bd, cond, site, index) true
#endif

}  // namespace fpp
