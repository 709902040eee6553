// Exact search without any device allocation.
//
// Some callers cannot allocate device memory at the moment they search: a
// framework that has already reserved the whole GPU for its own caching
// allocator (so cudaMalloc fails), or a latency-critical path that cannot
// afford the implicit device synchronisation of cudaMalloc/cudaFree.
// fpp_bruteforce_static serves them: it runs
// the same projection GEMM and dense top-k kernels as fpp_bruteforce, but its
// scratch (the score tile and a few counters) lives in the file-scope array
// below, which every GPU that loads this library holds until the process exits.
#include <algorithm>
#include <array>
#include <mutex>
#include <string>

#include "common.cuh"
#include "kernels.h"

namespace fpp {

namespace {

constexpr size_t kStaticScratchBytes = (size_t)FPP_STATIC_SCRATCH_BYTES;
constexpr size_t kMiscBytes = 256;  // xmax (float) at 0, recheck counter + error flag at 16

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_scratch_mu;
std::array<void*, 128> g_scratch_addr{};  // device address of the array, per device

// In host code g_static_scratch names a host-side stand-in, not device memory:
// the device address is looked up once per device, with that device current.
fpp_status scratch_address(void** out) {
  int dev = 0;
  FPP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= (int)g_scratch_addr.size()) {
    set_error("fpp_bruteforce_static: device ordinal out of range");
    return FPP_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    FPP_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return FPP_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace fpp

extern "C" fpp_status fpp_bruteforce_static(const float* X, int64_t n, int32_t d, const float* Q,
                                            int64_t m, int32_t k, int64_t* ids, float* scores,
                                            void* stream) {
  using namespace fpp;
  set_error("");
  if (!X || !Q || !ids || !scores || n < 1 || n >= (1ll << 32) || d < 1 || m < 0 || k < 1 ||
      k > 256) {
    set_error("fpp_bruteforce_static: bad arguments");
    return FPP_EINVAL;
  }
  if ((d & 3) || ((uintptr_t)X & 15) || ((uintptr_t)Q & 15)) {
    set_error("fpp_bruteforce_static: d must be a multiple of 4 and X, Q 16-byte aligned");
    return FPP_EINVAL;
  }
  if (!on_device(X) || !on_device(Q) || !on_device(ids) || !on_device(scores)) {
    set_error("fpp_bruteforce_static: X, Q, ids and scores must be device memory");
    return FPP_EINVAL;
  }
  const int64_t lds = round_up(n, 4);
  const int64_t mc_cap = (int64_t)((kStaticScratchBytes - kMiscBytes) / ((size_t)lds * sizeof(float)));
  if (mc_cap < 1) {
    set_error("fpp_bruteforce_static: n exceeds the static scratch (" +
              std::to_string((kStaticScratchBytes - kMiscBytes) / sizeof(float)) + " scores)");
    return FPP_EINVAL;
  }
  if (m == 0) return FPP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  void* base = nullptr;
  FPP_TRY(scratch_address(&base));
  unsigned char* b = static_cast<unsigned char*>(base);
  float* xmax_dev = reinterpret_cast<float*>(b);
  unsigned long long* misc = reinterpret_cast<unsigned long long*>(b + 16);
  float* S = reinterpret_cast<float*>(b + kMiscBytes);
  // the array keeps the previous call's contents: clear the counters
  FPP_CUDA(cudaMemsetAsync(misc, 0, 2 * sizeof(unsigned long long), st));
  FPP_TRY(launch_row_norm_max(X, n, d, d, xmax_dev, st));
  float xmax = 0.f;
  FPP_CUDA(cudaMemcpyAsync(&xmax, xmax_dev, sizeof(float), cudaMemcpyDeviceToHost, st));
  FPP_CUDA(cudaStreamSynchronize(st));
  const double gamma = gamma_fp32(d);
  for (int64_t q0 = 0; q0 < m; q0 += mc_cap) {
    const int64_t c = std::min<int64_t>(mc_cap, m - q0);
    FPP_TRY(gemm_f32_nt(Q + q0 * d, d, X, d, S, lds, c, n, d, st));
    FPP_TRY(launch_topk_dense(S, lds, c, n, k, Q + q0 * d, d, X, d, d, xmax, gamma, ids + q0 * k,
                              scores + q0 * k, k, misc, st));
  }
  unsigned long long hm[2] = {0, 0};
  FPP_CUDA(cudaMemcpyAsync(hm, misc, sizeof(hm), cudaMemcpyDeviceToHost, st));
  FPP_CUDA(cudaStreamSynchronize(st));
  if (hm[1]) {
    set_error("fpp_bruteforce_static: top-k re-check capacity exceeded");
    return FPP_EINTERNAL;
  }
  return FPP_OK;
}
