// C ABI of libfpp: index object, build and search orchestration.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "kernels.h"

#ifndef FPP_PIPE_SLOTS
#define FPP_PIPE_SLOTS 2
#endif

namespace fpp {

void generate_rotations(uint64_t seed, int L, int D, int d, float* R);

namespace {
thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};
}  // namespace

void set_error(const std::string& msg) { g_err = msg; }
std::atomic<uint64_t>& launch_counter() { return g_launches; }
std::atomic<uint64_t> g_dev_allocs{0};
std::atomic<uint64_t>& alloc_counter() { return g_dev_allocs; }

namespace {

// Page-locked (pinned) host memory: device copies to it are asynchronous.
bool is_pinned_host(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Grow-only device buffer.
// Every (re)allocation of a workspace buffer bumps g_alloc_gen, so that a
// captured search graph (which holds buffer addresses) is re-captured.
std::atomic<uint64_t> g_alloc_gen{0};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  fpp_status ensure(size_t need, bool zero = false, cudaStream_t st = 0) {
    if (need <= bytes && p) return FPP_OK;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    const size_t sz = std::max<size_t>(need, 256);
    g_alloc_gen.fetch_add(1);
    FPP_CUDA(dev_malloc(&p, sz));
    bytes = sz;
    if (zero) FPP_CUDA(cudaMemsetAsync(p, 0, sz, st));
    return FPP_OK;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

struct Workspace {
  DevBuf qpad, qpad_alt, qsplit, proj, probes, qnorm, recheck, recheck2, recheck_s, kpq, ppq,
      out_ids, out_scores, sigproj, qsig,
      ecount, eoff, cand, cscores, items, items2, rhist, tkslow, stats;
  const ScoreItem* score_items = nullptr;   // the item list the last batch scored
  // query tiles: qpad (slot 0) and qpad_alt (slot 1).  Asynchronous calls
  // with page-locked host queries fill the two in turn on an internal copy
  // stream, so that a batch's upload overlaps the previous batch's search;
  // qfree[s] marks the end of the last search that read slot s
  cudaStream_t cstream = nullptr;
  cudaEvent_t qready[2] = {nullptr, nullptr}, qfree[2] = {nullptr, nullptr};
  bool qused[2] = {false, false};
  int qslot = 0;
  fpp_status ensure_copy_stream() {
    if (cstream) return FPP_OK;
    FPP_CUDA(cudaStreamCreateWithFlags(&cstream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      FPP_CUDA(cudaEventCreateWithFlags(&qready[i], cudaEventDisableTiming));
      FPP_CUDA(cudaEventCreateWithFlags(&qfree[i], cudaEventDisableTiming));
    }
    return FPP_OK;
  }
  // completion of the last call that used this workspace: a call on another
  // stream waits for it before touching the buffers
  cudaEvent_t done = nullptr;
  fpp_status order_after_last(cudaStream_t st) {
    if (!done) {
      FPP_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
      return FPP_OK;
    }
    FPP_CUDA(cudaStreamWaitEvent(st, done, 0));
    return FPP_OK;
  }
  fpp_status mark_done(cudaStream_t st) {
    FPP_CUDA(cudaEventRecord(done, st));
    return FPP_OK;
  }
  uint64_t cand_cap = 0;    // candidate slots in cand / cscores
  void release() {
    for (DevBuf* b : {&qpad, &qpad_alt, &qsplit, &proj, &probes, &qnorm, &recheck, &recheck2,
                      &recheck_s, &sigproj, &qsig, &kpq, &ppq,
                      &out_ids, &out_scores, &ecount, &eoff, &cand, &cscores,
                      &items, &items2, &rhist, &tkslow, &stats})
      b->release();
    if (done) cudaEventDestroy(done);
    done = nullptr;
    if (cstream) {
      cudaStreamSynchronize(cstream);
      cudaStreamDestroy(cstream);
      cstream = nullptr;
    }
    for (int i = 0; i < 2; ++i) {
      if (qready[i]) cudaEventDestroy(qready[i]);
      if (qfree[i]) cudaEventDestroy(qfree[i]);
      qready[i] = qfree[i] = nullptr;
      qused[i] = false;
    }
  }
};

}  // namespace
}  // namespace fpp

struct fpp_index {
  int64_t n = 0;
  int d = 0, dpad = 0, L = 0, D = 0, iprobes = 1, kappa = 0, precision = 0;
  double alpha = 1.0;
  float* X = nullptr;          // [n][dpad]
  float* Xc = nullptr;         // [n][dpad] centered points (center = 1), else NULL
  float* c = nullptr;          // [dpad] the center (center = 1)
  int center = 0;
  uint32_t* sig = nullptr;     // [n][sig_words] SimHash signatures, or NULL
  int sig_words = 0;
  float rsig_max = 0.f;        // largest norm of the signature vectors (inflated)
  float* R = nullptr;          // [2 L D][dpad]
  void* Rs = nullptr;          // [2 L D][pieces Kp] BF16 pieces of R (tensor-core operand)
  int Kp = 0;
  int pieces = 3;              // BF16 pieces of a projected row: 3 (exact split)
  int bpieces = 3;             // 1: every coordinate of R is a BF16 value (three products)
  int qpieces = 3;             // pieces of the search's query projections: 3, or 1 with
                               // hash_precision FPP_BF16 (one BF16 product)
  double qgamma = 0.0;         // error factor of the query projections the probe
                               // decisions use (a bound for 3 pieces, a window for 1)
  void* Xb = nullptr;          // [n][ldxb] BF16 copy of X (FPP_BF16 only)
  int64_t ldxb = 0;
  uint8_t* Xq = nullptr;       // [n][ldxq] FP8 e4m3 copy of X (FPP_FP8E4M3 only)
  int64_t ldxq = 0;
  float* xscale = nullptr;     // [n] scales of the FP8 rows
  int rerank_k = 0;            // FPP_BF16: shortlist re-ranked on the FP32 rows
  double score_gamma = 0.0;    // candidate score error factor
  uint64_t cand_budget_entries = 0;  // candidate slots a batch may provision without a read-back
  // captured search graph (FPP_SEARCH_GRAPH) and the call it was captured for
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<uint64_t> graph_key;
  uint64_t graph_kernels = 0;  // kernel nodes of the graph
  uint64_t graph_overflows = 0;  // optimistic replays repeated without the graph
  int tune_score_g = 0, tune_score_waves = 0;   // fpp_autotune's choice (0: built-in)
  float* rmax = nullptr;       // [2L]
  float xmax = 0.f;            // largest point norm (inflated)
  float xhmax = 0.f;           // largest norm of the hashed rows (the centered points when centering)
  uint32_t* offsets = nullptr; // [L][4D^2 + 1]
  uint64_t* table_base = nullptr;  // [L]
  uint32_t* ids = nullptr;
  uint64_t kept_total = 0;
  uint32_t max_bucket_kept = 0;
  std::vector<uint64_t> h_table_base;
  int device = 0, sm_count = 0;
  double gamma = 0.0;
  uint64_t device_bytes = 0;
  float build_ms = 0.f;
  uint64_t build_rechecks = 0;
  std::mutex mu;
  fpp::Workspace ws;
  // FPP_SEARCH_PIPELINE: PIPE_SLOTS workspaces used in turn on as many
  // internal streams, so that a call's projection overlaps the previous
  // calls' gather and scoring; pdone[c] marks the end of the last call on
  // slot c (slot 0 uses ws, slot c > 0 ws_pipe[c - 1])
  static constexpr int PIPE_SLOTS = FPP_PIPE_SLOTS;
  fpp::Workspace ws_pipe[PIPE_SLOTS - 1];
  cudaStream_t pstream[PIPE_SLOTS] = {};
  cudaEvent_t pdone[PIPE_SLOTS] = {};
  cudaEvent_t pin = nullptr;
  bool ppending[PIPE_SLOTS] = {};
  int pnext = 0;
};

using namespace fpp;

namespace fpp_api {

int64_t nbuckets(int D) { return 4ll * D * D; }

fpp_status to_device_padded(const float* src, int64_t rows, int d, int dpad, float** dst,
                            cudaStream_t st, uint64_t* bytes) {
  FPP_CUDA(dev_malloc(dst, (size_t)std::max<int64_t>(rows, 1) * dpad * sizeof(float)));
  if (bytes) *bytes += (uint64_t)rows * dpad * sizeof(float);
  if (dpad != d) FPP_CUDA(cudaMemsetAsync(*dst, 0, (size_t)rows * dpad * sizeof(float), st));
  if (rows > 0)
    FPP_CUDA(cudaMemcpy2DAsync(*dst, dpad * sizeof(float), src, d * sizeof(float), d * sizeof(float),
                               rows, cudaMemcpyDefault, st));
  return FPP_OK;
}

void free_index_memory(fpp_index* ix) {
  cudaFree(ix->X);
  cudaFree(ix->Xc);
  cudaFree(ix->c);
  cudaFree(ix->sig);
  cudaFree(ix->R);
  cudaFree(ix->Rs);
  cudaFree(ix->Xb);
  cudaFree(ix->Xq);
  cudaFree(ix->xscale);
  cudaFree(ix->rmax);
  cudaFree(ix->offsets);
  cudaFree(ix->table_base);
  cudaFree(ix->ids);
  if (ix->graph_exec) cudaGraphExecDestroy(ix->graph_exec);
  ix->graph_exec = nullptr;
  for (int c = 0; c < fpp_index::PIPE_SLOTS; ++c) {
    if (ix->pstream[c]) {
      cudaStreamSynchronize(ix->pstream[c]);
      cudaStreamDestroy(ix->pstream[c]);
    }
    if (ix->pdone[c]) cudaEventDestroy(ix->pdone[c]);
    ix->pstream[c] = nullptr;
    ix->pdone[c] = nullptr;
  }
  if (ix->pin) cudaEventDestroy(ix->pin);
  ix->pin = nullptr;
  ix->ws.release();
  for (auto& w : ix->ws_pipe) w.release();
}

__global__ void gather_u64_kernel(const uint64_t* src, int64_t stride, int cnt, uint64_t* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) dst[i] = src[(int64_t)i * stride];
}

__global__ void max_keep_kernel(const uint32_t* counts, int64_t n, double alpha, int iprobes,
                                int kappa, unsigned* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t B = counts[i];
  double c = ceil(__ddiv_rn(__dmul_rn(alpha, (double)B), (double)iprobes));
  uint64_t k = (uint64_t)c;
  if (kappa > 0 && k < (uint64_t)kappa) k = kappa;
  if (k > B) k = B;
  if (k) atomicMax(out, (unsigned)k);
}

int sig_bits(uint64_t v) {
  int b = 0;
  while (v) { ++b; v >>= 1; }
  return b;
}

// The rows the tables hash and filter: the centered points when the index
// centers (Section 3.4, heuristic (1)), else the points.
const float* hashed_rows(const fpp_index* ix) { return ix->Xc ? ix->Xc : ix->X; }

// Builds tables [t0, t0 + nt) and appends their kept ids.
struct BuildScratch {
  DevBuf proj, xsplit, recA, recB, counts, bstart, kstart, hist, scanbuf, scanscratch, small, rechecks;
  DevBuf norms, pout, rc1, rc2, pcount;   // multi-probe indexing: the points' probe sets
};

// Projection of rows [r0, r0 + rc) of a padded FP32 matrix onto the random
// vectors of tables [t0, t0 + nt): split into BF16 pieces, tensor-core GEMM.
fpp_status project_rows(const fpp_index* ix, const float* src, int64_t rc, DevBuf& split, int t0,
                        int nt, float* out, int64_t ldp, int* err, cudaStream_t st,
                        uint64_t* lists = nullptr, int EL = 0, long long wait_cycles = 0,
                        int withhold = 0, int pieces = 0) {
  // pieces: the rows' BF16 pieces (0: the index's exact split); R keeps its
  // pieces layout and only its first piece is read for one-piece rows
  if (!pieces) pieces = ix->pieces;
  FPP_TRY(split.ensure((size_t)rc * pieces * ix->Kp * 2));
  FPP_TRY(split_to_bf16(src, rc, ix->dpad, ix->d, pieces, split.p, st));
  const char* rb =
      static_cast<const char*>(ix->Rs) + (size_t)2 * t0 * ix->D * ix->pieces * ix->Kp * 2;
  return project_tc(split.p, rc, rb, 2ll * nt * ix->D, ix->Kp, pieces,
                    pieces == 1 ? 1 : ix->bpieces, ix->D, EL, out, ldp, lists, err, st,
                    wait_cycles, withhold, ix->pieces);
}

// Test hook of fpp_debug_projections (fpp_debug_wait_test).
std::atomic<int> g_wait_test_withhold{0};
std::atomic<long long> g_wait_test_cycles{0};

// List length of the fused projection epilogue for a probe budget, or 0
// when the projections must be stored (D must divide 256, and the P + 1
// best entries of a list must lie on q's side of every hash).  One probe
// per table still takes two keys: the window pass re-scores both when the
// first two are closer than the error bound (with one key and the cut,
// every such item went to the full pass).
int fused_list_len(const fpp_index* ix, int pmax) {
  if (256 % ix->D != 0 || pmax + 1 > ix->D) return 0;
  return tc_list_len(pmax + 1);
}

fpp_status build_tables(fpp_index* ix, int t0, int nt, BuildScratch& B, cudaStream_t st,
                        std::vector<std::pair<uint32_t*, uint64_t>>& chunks,
                        uint64_t& global_base) {
  const int64_t n = ix->n;
  const int D = ix->D;
  const int64_t NB = nbuckets(D);
  const int64_t nsk = nt * NB;
  const int64_t ldp = round_up(2ll * nt * D, 4);
  const int ip = ix->iprobes;
  // list length of the projection epilogue: the best two keys (and the cut)
  // per hash for iProbes = 1; the best iProbes + 1 for multi-probe indexing
  // (0: store the projections)
  const int EL = (256 % D != 0) ? 0 : (ip == 1 ? 2 : (ip + 1 <= D ? tc_list_len(ip + 1) : 0));
  int64_t rows = std::max<int64_t>(128, (1ll << 28) / ldp);
  rows = std::min<int64_t>(rows, n);
  // projections (4 B per column) or the EL + 1 best keys per hash (8 B each)
  FPP_TRY(B.proj.ensure(std::max((size_t)rows * ldp * 4, (size_t)rows * 2 * nt * (EL + 1) * 8)));
  const int64_t nrec = (int64_t)nt * n * ip;
  FPP_TRY(B.recA.ensure((size_t)nrec * sizeof(Rec)));
  FPP_TRY(B.recB.ensure((size_t)nrec * sizeof(Rec)));
  FPP_TRY(B.counts.ensure((size_t)nsk * 4));
  FPP_TRY(B.bstart.ensure((size_t)(nsk + 1) * 8));
  FPP_TRY(B.kstart.ensure((size_t)(nsk + 1) * 8));
  if (ip > 1) {
    FPP_TRY(B.norms.ensure((size_t)rows * 4));
    FPP_TRY(B.pout.ensure((size_t)rows * nt * ip * 4));
    FPP_TRY(B.rc1.ensure((size_t)rows * nt * 4));
    FPP_TRY(B.rc2.ensure((size_t)rows * nt * 4));
    FPP_TRY(B.pcount.ensure(16, true, st));
  }
  const int64_t he = radix_hist_elems(nrec);
  FPP_TRY(B.hist.ensure((size_t)he * 4));
  FPP_TRY(B.scanbuf.ensure((size_t)(he + 1) * 8));
  FPP_TRY(B.scanscratch.ensure((size_t)scan_scratch_elems(std::max(he, nsk)) * 8));
  FPP_TRY(B.small.ensure((size_t)(nt + 2) * 8));
  FPP_CUDA(cudaMemsetAsync(B.counts.p, 0, (size_t)nsk * 4, st));

  for (int64_t r0 = 0; r0 < n; r0 += rows) {
    const int64_t rc = std::min<int64_t>(rows, n - r0);
    FPP_TRY(project_rows(ix, hashed_rows(ix) + r0 * ix->dpad, rc, B.xsplit, t0, nt, B.proj.as<float>(), ldp,
                         reinterpret_cast<int*>(B.rechecks.as<unsigned long long>() + 1), st,
                         EL ? B.proj.as<uint64_t>() : nullptr, EL));
    if (ip > 1) {
      // Algorithm 1 with iProbes > 1: each point goes into the iProbes
      // buckets it ranks highest, by the same exact ranking as a query
      const float* xr = hashed_rows(ix) + r0 * ix->dpad;
      FPP_TRY(launch_query_norms(xr, rc, ix->dpad, ix->d, B.norms.as<float>(), st));
      ProbeArgs pa{};
      pa.P = EL ? nullptr : B.proj.as<float>(); pa.ldp = ldp; pa.mq = rc;
      pa.lists = EL ? B.proj.as<uint64_t>() : nullptr; pa.EL = EL;
      pa.trunc = EL ? tc_list_trunc(D) : 0.f;
      pa.Q = xr; pa.ldq = ix->dpad; pa.qnorm = B.norms.as<float>();
      pa.R = ix->R; pa.ldr = ix->dpad; pa.d = ix->d; pa.D = D; pa.tb = t0; pa.nt = nt;
      pa.rmax = ix->rmax; pa.gamma = ix->gamma; pa.gammaf = (float)(ix->gamma * 1.0001);
      pa.probes_pq = nullptr; pa.probes = ip;
      pa.out = B.pout.as<uint32_t>();
      pa.recheck = B.rc1.as<uint32_t>();
      pa.recheck_count = B.pcount.as<unsigned>();
      pa.recheck2 = B.rc2.as<uint32_t>();
      pa.recheck2_count = B.pcount.as<unsigned>() + 1;
      pa.rechecks = B.rechecks.as<unsigned long long>();
      FPP_TRY(launch_probe(pa, st));
      PairArgs pr{};
      pr.probes = B.pout.as<uint32_t>(); pr.iprobes = ip; pr.rows = rc; pr.row0 = r0;
      pr.t0 = t0; pr.nt = nt; pr.D = D; pr.X = hashed_rows(ix); pr.ldx = ix->dpad;
      pr.R = ix->R; pr.ldr = ix->dpad; pr.n = n;
      pr.rec = B.recA.as<Rec>(); pr.counts = B.counts.as<uint32_t>();
      FPP_TRY(launch_pair_records(pr, st));
      continue;
    }
    HashArgs h{};
    h.P = EL ? nullptr : B.proj.as<float>(); h.ldp = ldp; h.rows = rc; h.row0 = r0;
    h.lists = EL ? B.proj.as<uint64_t>() : nullptr; h.EL = EL;
    h.trunc = EL ? tc_list_trunc(D) : 0.f;
    h.t0 = t0; h.nt = nt; h.D = D;
    h.X = hashed_rows(ix); h.ldx = ix->dpad; h.R = ix->R; h.ldr = ix->dpad; h.d = ix->d;
    h.rmax = ix->rmax; h.xmax = ix->xhmax; h.gamma = ix->gamma; h.n = n;
    h.eps_xf = (float)(ix->gamma * (double)ix->xhmax * 1.0001);
    h.rec = B.recA.as<Rec>(); h.counts = B.counts.as<uint32_t>(); h.point_bucket = nullptr;
    h.rechecks = B.rechecks.as<unsigned long long>();
    FPP_TRY(launch_build_hash(h, st));
  }
  Rec* sorted = nullptr;
  FPP_TRY(radix_sort_recs(B.recA.as<Rec>(), B.recB.as<Rec>(), nrec, 64, sig_bits(nsk - 1),
                          B.hist.as<uint32_t>(), he, B.scanbuf.as<uint64_t>(),
                          B.scanscratch.as<uint64_t>(), &sorted, st));
  const KeepRule rule{ix->alpha, ix->iprobes, ix->kappa};
  FPP_TRY(exclusive_scan_u32(B.counts.as<uint32_t>(), nsk, B.bstart.as<uint64_t>(), 0, rule,
                             B.scanscratch.as<uint64_t>(), st));
  FPP_TRY(exclusive_scan_u32(B.counts.as<uint32_t>(), nsk, B.kstart.as<uint64_t>(), 1, rule,
                             B.scanscratch.as<uint64_t>(), st));
  // per-table starts (relative to the chunk) and the chunk total
  gather_u64_kernel<<<(unsigned)ceil_div(nt + 1, 128), 128, 0, st>>>(B.kstart.as<uint64_t>(), NB,
                                                                    nt + 1, B.small.as<uint64_t>());
  FPP_LAUNCHED();
  std::vector<uint64_t> starts(nt + 1);
  FPP_CUDA(cudaMemcpyAsync(starts.data(), B.small.p, (nt + 1) * 8, cudaMemcpyDeviceToHost, st));
  unsigned* mk = reinterpret_cast<unsigned*>(B.small.as<uint64_t>() + nt + 1);
  FPP_CUDA(cudaMemsetAsync(mk, 0, 4, st));
  max_keep_kernel<<<(unsigned)ceil_div(nsk, 256), 256, 0, st>>>(B.counts.as<uint32_t>(), nsk,
                                                                ix->alpha, ix->iprobes, ix->kappa, mk);
  FPP_LAUNCHED();
  unsigned hmk = 0;
  FPP_CUDA(cudaMemcpyAsync(&hmk, mk, 4, cudaMemcpyDeviceToHost, st));
  FPP_CUDA(cudaStreamSynchronize(st));
  ix->max_bucket_kept = std::max(ix->max_bucket_kept, hmk);
  const uint64_t total = starts[nt];
  uint32_t* cids = nullptr;
  FPP_CUDA(dev_malloc(&cids, std::max<uint64_t>(total, 1) * 4));
  chunks.emplace_back(cids, total);
  FPP_TRY(launch_compact(sorted, nrec, B.bstart.as<uint64_t>(), B.kstart.as<uint64_t>(),
                         B.counts.as<uint32_t>(), rule, cids, st));
  FPP_TRY(launch_make_offsets(B.kstart.as<uint64_t>(), nt, NB, ix->offsets + (int64_t)t0 * (NB + 1), st));
  for (int tl = 0; tl < nt; ++tl) ix->h_table_base[t0 + tl] = global_base + starts[tl];
  global_base += total;
  return FPP_OK;
}

fpp_status validate_params(int64_t n, int32_t d, const fpp_params* p) {
  if (!p) { set_error("params is NULL"); return FPP_EINVAL; }
  if (n < 1 || n >= (1ll << 32)) { set_error("n must be in [1, 2^32)"); return FPP_EINVAL; }
  if (d < 1 || d > 16384) { set_error("d must be in [1, 16384]"); return FPP_EINVAL; }
  if (p->L < 1 || p->L > 4096) { set_error("L must be in [1, 4096]"); return FPP_EINVAL; }
  if (p->D < 1 || p->D > 1024) { set_error("D must be in [1, 1024]"); return FPP_EINVAL; }
  if (!(p->alpha > 0.0 && p->alpha <= 1.0)) { set_error("alpha must be in (0, 1]"); return FPP_EINVAL; }
  if (p->iprobes < 1 || p->iprobes > 16 || p->iprobes > 4ll * p->D * p->D) {
    set_error("iprobes must be in [1, min(4D^2, 16)]");
    return FPP_EINVAL;
  }
  if (p->kappa < 0) { set_error("kappa must be >= 0"); return FPP_EINVAL; }
  if (p->precision != FPP_FP32 && p->precision != FPP_BF16 && p->precision != FPP_FP8E4M3) {
    set_error("precision must be FPP_FP32, FPP_BF16 or FPP_FP8E4M3");
    return FPP_EINVAL;
  }
  if (p->hash_precision != FPP_FP32 && p->hash_precision != FPP_BF16) {
    set_error("hash_precision must be FPP_FP32 or FPP_BF16");
    return FPP_EINVAL;
  }
  if (p->hash_precision == FPP_BF16 && (p->precision == FPP_FP32 || p->simhash_bits)) {
    set_error("hash_precision FPP_BF16 needs precision FPP_BF16 or FPP_FP8E4M3 and no simhash_bits");
    return FPP_EINVAL;
  }
  if (p->simhash_bits < 0 || p->simhash_bits % 256 || p->simhash_bits > 1024 ||
      p->simhash_bits > 2ll * p->L * p->D) {
    set_error("simhash_bits must be 0 or a multiple of 256 up to min(1024, 2 L D)");
    return FPP_EINVAL;
  }
  if (p->precision != FPP_FP32 && (p->rerank_k < 0 || p->rerank_k > 256)) {
    set_error("rerank_k must be in [0, 256]");
    return FPP_EINVAL;
  }
  return FPP_OK;
}

fpp_status build_impl(const float* X, int64_t n, int32_t d, const fpp_params* p, fpp_index** out) {
  const auto wall0 = std::chrono::steady_clock::now();
  if (!X || !out) { set_error("X and out must be non-NULL"); return FPP_EINVAL; }
  FPP_TRY(validate_params(n, d, p));
  cudaStream_t st = (cudaStream_t)p->stream;
  fpp_index* ix = new fpp_index();
  auto fail = [&](fpp_status s) { free_index_memory(ix); delete ix; return s; };
  fpp_status s;
  ix->n = n; ix->d = d; ix->dpad = (int)round_up(d, 4);
  ix->L = p->L; ix->D = p->D; ix->iprobes = p->iprobes; ix->kappa = p->kappa;
  ix->alpha = p->alpha; ix->precision = p->precision;
  ix->Kp = tc_kpad(d);
  {
    // candidate buffers (8 bytes per slot) up to min(8 GiB, 1/16 of the
    // device) are provisioned from the worst-case bound without a read-back
    size_t fr = 0, tot = 0;
    const uint64_t lim = cudaMemGetInfo(&fr, &tot) == cudaSuccess ? std::min<uint64_t>(8ull << 30, tot / 16)
                                                                 : (1ull << 31);
    ix->cand_budget_entries = lim / 8;
  }
  // Projections use the exact three-piece split in both precisions: the
  // projection kernel is bound by its epilogue (the per-hash top lists), not
  // by the tensor cores, so one BF16 product is no faster there, while its
  // rounding error would send far more probe decisions to the exact pass.
  ix->pieces = 3;
  ix->gamma = tc_error_bound_factor(ix->Kp, 3);
  ix->qpieces = p->hash_precision == FPP_BF16 ? 1 : 3;
  ix->qgamma = ix->qpieces == 1 ? bf16_window_factor(d) : ix->gamma;
  if (p->precision == FPP_BF16) {
    ix->rerank_k = p->rerank_k;
    ix->score_gamma = bf16_window_factor(d);
  } else if (p->precision == FPP_FP8E4M3) {
    ix->rerank_k = p->rerank_k;
    ix->score_gamma = fp8_window_factor(d);
  } else {
    ix->score_gamma = gamma_fp32(ix->dpad);
  }
  if (cudaGetDevice(&ix->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ix->sm_count, cudaDevAttrMultiProcessorCount, ix->device) != cudaSuccess) {
    set_error("no CUDA device");
    delete ix;
    return FPP_ECUDA;
  }
  const int L = p->L, D = p->D;
  const int64_t rrows = 2ll * L * D;
  // random vectors (host copy needed for the row norms)
  std::vector<float> hR((size_t)rrows * d);
  if (p->R) {
    if (cudaMemcpy(hR.data(), p->R, hR.size() * 4, cudaMemcpyDefault) != cudaSuccess) {
      set_error("copying params->R failed");
      return fail(FPP_EINVAL);
    }
  } else {
    generate_rotations(p->seed, L, D, d, hR.data());
  }
  // R on the BF16 grid (the seeded generator's): three projection products
  ix->bpieces = 1;
  for (size_t e = 0; e < hR.size() && ix->bpieces == 1; ++e) {
    uint32_t u;
    std::memcpy(&u, &hR[e], 4);
    if (u & 0xFFFFu) ix->bpieces = ix->pieces;
  }
  std::vector<float> hrmax(2 * L, 0.f);
  for (int64_t r = 0; r < rrows; ++r) {
    double s = 0.0;
    for (int c = 0; c < d; ++c) s += (double)hR[r * d + c] * hR[r * d + c];
    const int tj = (int)(r / D);
    hrmax[tj] = std::max(hrmax[tj], (float)(std::sqrt(s) * (1.0 + 1e-6)));
  }
  if ((s = to_device_padded(X, n, d, ix->dpad, &ix->X, st, &ix->device_bytes)) != FPP_OK) return fail(s);
  if (p->center) {
    // c: the given vector, or the FP64 column means rounded to FP32; the
    // tables are built over fl(x - c)
    ix->center = 1;
    if (dev_malloc(&ix->c, (size_t)ix->dpad * 4) != cudaSuccess ||
        dev_malloc(&ix->Xc, (size_t)n * ix->dpad * 4) != cudaSuccess) {
      set_error("cudaMalloc (centering)");
      return fail(FPP_ENOMEM);
    }
    ix->device_bytes += (uint64_t)n * ix->dpad * 4 + (uint64_t)ix->dpad * 4;
    if (cudaMemsetAsync(ix->c, 0, (size_t)ix->dpad * 4, st) != cudaSuccess) return fail(FPP_ECUDA);
    if (p->center_vec) {
      if (cudaMemcpyAsync(ix->c, p->center_vec, (size_t)d * 4, cudaMemcpyDefault, st) != cudaSuccess) {
        set_error("copying params->center_vec failed");
        return fail(FPP_EINVAL);
      }
    } else if ((s = launch_column_means(ix->X, n, ix->dpad, d, ix->c, st)) != FPP_OK) {
      return fail(s);
    }
    if ((s = launch_center_rows(ix->X, n, ix->dpad, ix->c, ix->Xc, st)) != FPP_OK) return fail(s);
  }
  if ((s = to_device_padded(hR.data(), rrows, d, ix->dpad, &ix->R, st, &ix->device_bytes)) != FPP_OK)
    return fail(s);
  if (dev_malloc(&ix->Rs, (size_t)rrows * ix->pieces * ix->Kp * 2) != cudaSuccess) {
    set_error("cudaMalloc Rs");
    return fail(FPP_ENOMEM);
  }
  ix->device_bytes += (uint64_t)rrows * ix->pieces * ix->Kp * 2;
  if ((s = split_to_bf16(ix->R, rrows, ix->dpad, d, ix->pieces, ix->Rs, st)) != FPP_OK) return fail(s);
  if (ix->precision == FPP_BF16) {
    ix->ldxb = round_up(d, 8);
    if (dev_malloc(&ix->Xb, (size_t)n * ix->ldxb * 2) != cudaSuccess) {
      set_error("cudaMalloc Xb");
      return fail(FPP_ENOMEM);
    }
    ix->device_bytes += (uint64_t)n * ix->ldxb * 2;
    if ((s = rows_to_bf16(ix->X, n, ix->dpad, d, ix->ldxb, ix->Xb, st)) != FPP_OK) return fail(s);
  }
  if (ix->precision == FPP_FP8E4M3) {
    ix->ldxq = round_up(d, 16);
    if (dev_malloc(&ix->Xq, (size_t)n * ix->ldxq) != cudaSuccess ||
        dev_malloc(&ix->xscale, (size_t)n * 4) != cudaSuccess) {
      set_error("cudaMalloc Xq");
      return fail(FPP_ENOMEM);
    }
    ix->device_bytes += (uint64_t)n * ix->ldxq + (uint64_t)n * 4;
    if ((s = rows_to_fp8(ix->X, n, ix->dpad, d, ix->ldxq, ix->Xq, ix->xscale, st)) != FPP_OK)
      return fail(s);
  }
  if (dev_malloc(&ix->rmax, 2 * L * 4) != cudaSuccess) { set_error("cudaMalloc rmax"); return fail(FPP_ENOMEM); }
  if (cudaMemcpyAsync(ix->rmax, hrmax.data(), 2 * L * 4, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    set_error("copy rmax");
    return fail(FPP_ECUDA);
  }
  {
    // largest norm of the points (score bounds) and of the hashed rows
    // (projection bounds of the build); equal unless the index centers
    float* dxm = nullptr;
    if (dev_malloc(&dxm, 8) != cudaSuccess) { set_error("cudaMalloc"); return fail(FPP_ENOMEM); }
    s = launch_row_norm_max(ix->X, n, ix->dpad, d, dxm, st);
    if (s == FPP_OK) s = launch_row_norm_max(hashed_rows(ix), n, ix->dpad, d, dxm + 1, st);
    float hm[2] = {0.f, 0.f};
    if (s == FPP_OK && cudaMemcpyAsync(hm, dxm, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) s = FPP_ECUDA;
    if (s == FPP_OK && cudaStreamSynchronize(st) != cudaSuccess) s = FPP_ECUDA;
    cudaFree(dxm);
    if (s != FPP_OK) return fail(s);
    ix->xmax = hm[0];
    ix->xhmax = hm[1];
  }
  const int64_t NB = nbuckets(D);
  if (dev_malloc(&ix->offsets, (size_t)L * (NB + 1) * 4) != cudaSuccess) {
    set_error("cudaMalloc offsets");
    return fail(FPP_ENOMEM);
  }
  ix->device_bytes += (uint64_t)L * (NB + 1) * 4;
  ix->h_table_base.assign(L, 0);

  const int64_t rcap = 1ll << 28;   // records per table chunk
  int nt_chunk = (int)std::max<int64_t>(1, rcap / (n * p->iprobes));
  nt_chunk = (int)std::min<int64_t>(nt_chunk, (int64_t)(0xFFFFFFFFll / NB));
  nt_chunk = std::max(1, std::min(nt_chunk, L));
  BuildScratch B;
  std::vector<std::pair<uint32_t*, uint64_t>> chunks;
  uint64_t base = 0;
  auto cleanup = [&]() {
    for (DevBuf* b : {&B.proj, &B.xsplit, &B.recA, &B.recB, &B.counts, &B.bstart, &B.kstart, &B.hist,
                      &B.scanbuf, &B.scanscratch, &B.small, &B.rechecks, &B.norms, &B.pout, &B.rc1,
                      &B.rc2, &B.pcount})
      b->release();
    for (auto& c : chunks) cudaFree(c.first);
  };
  if ((s = B.rechecks.ensure(16, true, st)) != FPP_OK) { cleanup(); return fail(s); }
  for (int t0 = 0; t0 < L; t0 += nt_chunk) {
    const int nt = std::min(nt_chunk, L - t0);
    if ((s = build_tables(ix, t0, nt, B, st, chunks, base)) != FPP_OK) { cleanup(); return fail(s); }
  }
  ix->kept_total = base;
  if (dev_malloc(&ix->ids, std::max<uint64_t>(base, 1) * 4) != cudaSuccess) {
    set_error("cudaMalloc ids");
    cleanup();
    return fail(FPP_ENOMEM);
  }
  ix->device_bytes += base * 4;
  uint64_t at = 0;
  for (auto& c : chunks) {
    if (c.second && cudaMemcpyAsync(ix->ids + at, c.first, c.second * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      set_error("concatenating ids");
      cleanup();
      return fail(FPP_ECUDA);
    }
    at += c.second;
  }
  if (dev_malloc(&ix->table_base, L * 8) != cudaSuccess ||
      cudaMemcpyAsync(ix->table_base, ix->h_table_base.data(), L * 8, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    set_error("table_base");
    cleanup();
    return fail(FPP_ECUDA);
  }
  unsigned long long rech[2] = {0, 0};
  cudaMemcpyAsync(rech, B.rechecks.p, 16, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    set_error(std::string("build: ") + cudaGetErrorString(cudaGetLastError()));
    cleanup();
    return fail(FPP_ECUDA);
  }
  if (rech[1]) {
    set_error("build: a bounded wait in the projection kernel ran out");
    cleanup();
    return fail(FPP_ETIMEOUT);
  }
  ix->build_rechecks = rech[0];
  if (p->simhash_bits > 0) {
    // SimHash signatures of the points over the first simhash_bits random
    // vectors (the rows of R in table order)
    const int bits = p->simhash_bits;
    ix->sig_words = bits / 32;
    for (int j = 0; j * D < bits; ++j) ix->rsig_max = std::max(ix->rsig_max, hrmax[j]);
    if (dev_malloc(&ix->sig, (size_t)n * ix->sig_words * 4) != cudaSuccess) {
      set_error("cudaMalloc (signatures)");
      cleanup();
      return fail(FPP_ENOMEM);
    }
    ix->device_bytes += (uint64_t)n * ix->sig_words * 4;
    const int64_t rows = std::min<int64_t>(n, 1 << 16);
    if ((s = B.proj.ensure((size_t)rows * bits * 4)) != FPP_OK ||
        (s = B.norms.ensure((size_t)rows * 4)) != FPP_OK) {
      cleanup();
      return fail(s);
    }
    for (int64_t r0 = 0; r0 < n && s == FPP_OK; r0 += rows) {
      const int64_t rc = std::min<int64_t>(rows, n - r0);
      const float* xr = ix->X + r0 * ix->dpad;
      s = B.xsplit.ensure((size_t)rc * ix->pieces * ix->Kp * 2);
      if (s == FPP_OK) s = split_to_bf16(xr, rc, ix->dpad, d, ix->pieces, B.xsplit.p, st);
      if (s == FPP_OK)
        s = project_tc(B.xsplit.p, rc, ix->Rs, bits, ix->Kp, ix->pieces, ix->bpieces, 0, 0, B.proj.as<float>(),
                       bits, nullptr, reinterpret_cast<int*>(B.rechecks.as<unsigned long long>() + 1), st);
      if (s == FPP_OK) s = launch_query_norms(xr, rc, ix->dpad, d, B.norms.as<float>(), st);
      if (s == FPP_OK) {
        SignArgs sa{};
        sa.P = B.proj.as<float>(); sa.ldp = bits; sa.rows = rc; sa.words = ix->sig_words;
        sa.V = xr; sa.ldv = ix->dpad; sa.vnorm = B.norms.as<float>();
        sa.R = ix->R; sa.ldr = ix->dpad; sa.gamma = ix->gamma; sa.rsig_max = ix->rsig_max;
        sa.out = ix->sig + r0 * ix->sig_words;
        s = launch_sign_bits(sa, st);
      }
    }
    if (s == FPP_OK && cudaStreamSynchronize(st) != cudaSuccess) s = FPP_ECUDA;
    if (s != FPP_OK) {
      cleanup();
      return fail(s);
    }
  }
  cleanup();
  ix->build_ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - wall0).count();
  *out = ix;
  return FPP_OK;
}

// ------------------------------------------------------------------ search

struct SearchPlan {
  int64_t m;
  int kmax, pmax, tb, te;
  int global_q = 0;     // > 0: global probe budget (pmax = the per-table cap)
  int sim_keep = 0;     // > 0: SimHash pre-ranking keeps this many candidates
  int range_shift = 0;  // range_count > 1: candidates grouped by id >> range_shift
  int range_count = 1;
  bool no_grow = false; // serving: never grow the candidate buffers; a batch
                        // whose candidates do not fit returns FPP_EBUSY
  bool optimistic = false;  // captured graph whose worst case exceeds the buffer:
                            // no read-back, the tiers check each region against
                            // the buffer and raise the overflow flag (slot 4)
  const int32_t* kpq;   // user arrays (host or device) or NULL
  const int32_t* ppq;
  bool kpq_dev, ppq_dev;
  int k, probes;
};

fpp_status validate_search(const fpp_index* ix, const float* Q, int64_t m, const fpp_search_opts* o,
                           int64_t* ids, float* scores, SearchPlan& pl) {
  if (!ix) { set_error("index is NULL"); return FPP_EINVAL; }
  if (!o) { set_error("opts is NULL"); return FPP_EINVAL; }
  if (m < 0) { set_error("m must be >= 0"); return FPP_EINVAL; }
  if (m > 0 && (!Q || !ids || !scores)) { set_error("Q, ids and scores must be non-NULL"); return FPP_EINVAL; }
  pl.m = m;
  pl.tb = o->table_begin;
  pl.te = (o->table_end == 0) ? ix->L : o->table_end;
  if (pl.tb < 0 || pl.te > ix->L || pl.tb >= pl.te) { set_error("bad table range"); return FPP_EINVAL; }
  const int64_t NB = nbuckets(ix->D);
  const int pcap = (int)std::min<int64_t>(NB, 128);
  pl.kpq = o->k_per_query;
  pl.ppq = o->probes_per_query;
  pl.kpq_dev = is_device_ptr(pl.kpq);
  pl.ppq_dev = is_device_ptr(pl.ppq);
  pl.k = o->k;
  pl.probes = o->probes;
  int kmax_seen = pl.kpq ? 0 : pl.k, pmax_seen = pl.ppq ? 0 : pl.probes;
  auto check_arr = [&](const int32_t* a, int lo, int hi, int& mx, const char* what) -> fpp_status {
    std::vector<int32_t> h(m);
    if (m && cudaMemcpy(h.data(), a, m * 4, cudaMemcpyDefault) != cudaSuccess) {
      set_error(std::string("reading ") + what);
      return FPP_EINVAL;
    }
    for (int64_t i = 0; i < m; ++i) {
      if (h[i] < lo || h[i] > hi) {
        set_error(std::string(what) + " out of range at query " + std::to_string(i));
        return FPP_EINVAL;
      }
      mx = std::max(mx, (int)h[i]);
    }
    return FPP_OK;
  };
  if (pl.kpq) FPP_TRY(check_arr(pl.kpq, 1, 256, kmax_seen, "k_per_query"));
  else if (pl.k < 1 || pl.k > 256) { set_error("k must be in [1, 256]"); return FPP_EINVAL; }
  if (pl.ppq) FPP_TRY(check_arr(pl.ppq, 1, pcap, pmax_seen, "probes_per_query"));
  else if (o->global_probes <= 0 && (pl.probes < 1 || pl.probes > pcap)) {
    set_error("probes must be in [1, min(4D^2, 128)]");
    return FPP_EINVAL;
  }
  if (o->global_probes < 0) { set_error("global_probes must be >= 0"); return FPP_EINVAL; }
  if (o->global_probes > 0) {
    if (pl.ppq) { set_error("global_probes excludes probes_per_query"); return FPP_EINVAL; }
    pl.global_q = o->global_probes;
    pl.probes = (int)std::min<int64_t>(std::min<int64_t>(o->global_probes, 128), NB);
    pmax_seen = pl.probes;
    if ((int64_t)(pl.te - pl.tb) * pl.probes > 16384) {
      set_error("global_probes: tables x per-table cap must be <= 16384");
      return FPP_EINVAL;
    }
  }
  if (o->simhash_keep < 0 || o->simhash_keep > 512) {
    set_error("simhash_keep must be in [0, 512]");
    return FPP_EINVAL;
  }
  if (o->simhash_keep > 0 && !ix->sig) {
    set_error("simhash_keep needs an index built with simhash_bits");
    return FPP_EINVAL;
  }
  pl.sim_keep = o->simhash_keep;
  if (o->score_range_rows < 0) { set_error("score_range_rows must be >= 0"); return FPP_EINVAL; }
  if (pl.sim_keep == 0) {
    // rows per range: 32,768 (measured fastest for 512-byte FP32 rows and
    // for 1,920-byte BF16 rows alike), or the caller's count, rounded to a
    // power of two; at most SCORE_RANGE_MAX ranges
    const uint64_t want = o->score_range_rows > 0 ? (uint64_t)o->score_range_rows : 32768ull;
    int sh = 0;
    while ((1ull << (sh + 1)) <= want) ++sh;
    if (o->score_range_rows > 0 && (1ull << sh) < want) ++sh;
    while ((uint64_t)((ix->n + (1ll << sh) - 1) >> sh) > (uint64_t)SCORE_RANGE_MAX) ++sh;
    const int64_t R = (ix->n + (1ll << sh) - 1) >> sh;
    if (R > 1) { pl.range_shift = sh; pl.range_count = (int)R; }
  }
  pl.kmax = o->k_max > 0 ? o->k_max : kmax_seen;
  if (pl.kmax < kmax_seen || pl.kmax > 256) { set_error("k_max must cover every k and be <= 256"); return FPP_EINVAL; }
  pl.pmax = std::max(1, pmax_seen);
  return FPP_OK;
}

// Entries the top-k kernel re-scores exactly: k + 16, or the FP32 shortlist
// of the BF16 path when that is longer.
int topk_kprime(const fpp_index* ix, int kmax) {
  return std::max(kmax + 16, ix->precision != FPP_FP32 ? ix->rerank_k : 0);
}

// Runs projection + probe ranking (and, unless probes_only, gather/score) for
// queries [q0, q0 + mc).
enum Stage { kFull = 0, kProbesOnly = 1, kCandidatesOnly = 2 };

fpp_status search_chunk(fpp_index* ix, Workspace& ws, const float* Q, int64_t q0, int64_t mc,
                        const SearchPlan& pl, int64_t* ids_dev, float* scores_dev, cudaStream_t st,
                        int stage, cudaEvent_t* ev, bool ahead = false) {
  const int nt = pl.te - pl.tb;
  const int64_t ldp = round_up(2ll * nt * ix->D, 4);
  // queries, padded: on the call's stream, or (ahead) on the copy stream
  // into the tile the search before last has finished reading
  const int slot = ahead ? (ws.qslot ^= 1) : 0;
  float* const qp = slot ? ws.qpad_alt.as<float>() : ws.qpad.as<float>();
  if (ahead) {
    if (ws.qused[slot]) FPP_CUDA(cudaStreamWaitEvent(ws.cstream, ws.qfree[slot], 0));
    FPP_CUDA(cudaMemcpy2DAsync(qp, ix->dpad * 4, Q + q0 * ix->d, ix->d * 4, ix->d * 4, mc,
                               cudaMemcpyHostToDevice, ws.cstream));
    FPP_CUDA(cudaEventRecord(ws.qready[slot], ws.cstream));
    FPP_CUDA(cudaStreamWaitEvent(st, ws.qready[slot], 0));
  } else {
    FPP_CUDA(cudaMemcpy2DAsync(qp, ix->dpad * 4, Q + q0 * ix->d, ix->d * 4, ix->d * 4, mc,
                               cudaMemcpyDefault, st));
  }
  // the end of the reads of this tile (every return below)
  auto tile_read = [&]() -> fpp_status {
    if (ws.qfree[slot]) {
      FPP_CUDA(cudaEventRecord(ws.qfree[slot], st));
      ws.qused[slot] = true;
    }
    return FPP_OK;
  };
  const int32_t* kpq = nullptr;
  const int32_t* ppq = nullptr;
  if (pl.kpq) {
    if (pl.kpq_dev) kpq = pl.kpq + q0;
    else {
      FPP_CUDA(cudaMemcpyAsync(ws.kpq.p, pl.kpq + q0, mc * 4, cudaMemcpyHostToDevice, st));
      kpq = ws.kpq.as<int32_t>();
    }
  }
  if (pl.ppq) {
    if (pl.ppq_dev) ppq = pl.ppq + q0;
    else {
      FPP_CUDA(cudaMemcpyAsync(ws.ppq.p, pl.ppq + q0, mc * 4, cudaMemcpyHostToDevice, st));
      ppq = ws.ppq.as<int32_t>();
    }
  }
  if (ev) FPP_CUDA(cudaEventRecord(ev[0], st));
  const int EL = fused_list_len(ix, pl.pmax);
  FPP_TRY(project_rows(ix, qp, mc, ws.qsplit, pl.tb, nt, ws.proj.as<float>(), ldp,
                       reinterpret_cast<int*>(ws.stats.as<unsigned long long>() + 9), st,
                       EL ? ws.proj.as<uint64_t>() : nullptr, EL, 0, 0, ix->qpieces));
  if (ev) FPP_CUDA(cudaEventRecord(ev[1], st));
  FPP_TRY(launch_query_norms(qp, mc, ix->dpad, ix->d, ws.qnorm.as<float>(), st));
  if (pl.sim_keep > 0) {
    // the queries' SimHash signatures from their split pieces
    const int bits = ix->sig_words * 32;
    FPP_TRY(project_tc(ws.qsplit.p, mc, ix->Rs, bits, ix->Kp, ix->pieces, ix->bpieces, 0, 0,
                       ws.sigproj.as<float>(), bits, nullptr,
                       reinterpret_cast<int*>(ws.stats.as<unsigned long long>() + 9), st));
    SignArgs sg{};
    sg.P = ws.sigproj.as<float>(); sg.ldp = bits; sg.rows = mc; sg.words = ix->sig_words;
    sg.V = qp; sg.ldv = ix->dpad; sg.vnorm = ws.qnorm.as<float>();
    sg.R = ix->R; sg.ldr = ix->dpad; sg.gamma = ix->gamma; sg.rsig_max = ix->rsig_max;
    sg.out = ws.qsig.as<uint32_t>();
    FPP_TRY(launch_sign_bits(sg, st));
  }
  ProbeArgs pa{};
  pa.P = EL ? nullptr : ws.proj.as<float>(); pa.ldp = ldp; pa.mq = mc;
  pa.lists = EL ? ws.proj.as<uint64_t>() : nullptr; pa.EL = EL;
  pa.trunc = EL ? tc_list_trunc(ix->D) : 0.f;
  pa.Q = qp; pa.ldq = ix->dpad; pa.qnorm = ws.qnorm.as<float>();
  pa.R = ix->R; pa.ldr = ix->dpad; pa.d = ix->d; pa.D = ix->D; pa.tb = pl.tb; pa.nt = nt;
  if (ix->bpieces == 1) {   // R on the BF16 grid: its first BF16 piece is R itself
    pa.Rb = static_cast<const uint16_t*>(ix->Rs);
    pa.ldrb = (int64_t)ix->pieces * ix->Kp;
  }
  pa.rmax = ix->rmax; pa.gamma = ix->qgamma; pa.gammaf = (float)(ix->qgamma * 1.0001);
  pa.argmax_only = ix->qpieces == 1 ? 1 : 0;
  // the argmax pass's pair list (list mode) reuses the pair-window buffer,
  // which list mode does not use: 4 words per item hold 2 pairs
  pa.amax_pairs = ws.recheck_s.as<uint32_t>();
  pa.amax_count = reinterpret_cast<unsigned*>(ws.stats.as<unsigned long long>() + 14);
  pa.probes_pq = ppq; pa.probes = pl.pmax;
  pa.out = ws.probes.as<uint32_t>();
  pa.recheck = ws.recheck.as<uint32_t>();
  pa.recheck_count = reinterpret_cast<unsigned*>(ws.stats.as<unsigned long long>() + 8);
  pa.recheck2 = ws.recheck2.as<uint32_t>();
  pa.recheck2_count = reinterpret_cast<unsigned*>(ws.stats.as<unsigned long long>() + 8) + 1;
  pa.recheck_s = EL ? nullptr : ws.recheck_s.as<float>();   // pair-window pass (stored projections)
  pa.rechecks = ws.stats.as<unsigned long long>() + 6;
  pa.full_rechecks = ws.stats.as<unsigned long long>() + 7;
  pa.gcap_flag = ws.stats.as<unsigned long long>() + 13;
  FPP_TRY(launch_probe(pa, st, ev ? ev[4] : nullptr));
  if (pl.global_q > 0) FPP_TRY(launch_global_probes(pa, pl.global_q, st));
  if (ev) FPP_CUDA(cudaEventRecord(ev[2], st));
  if (stage == kProbesOnly) return tile_read();
  // ---- candidates: count bucket entries, give each query a region, dedup,
  // score, top-k
  unsigned long long* stv = ws.stats.as<unsigned long long>();
  DedupArgs da{};
  da.probes = ws.probes.as<uint32_t>(); da.pstride = pl.pmax; da.mq = mc;
  da.tb = pl.tb; da.nt = nt; da.D = ix->D; da.probes_pq = ppq;
  da.offsets = ix->offsets; da.table_base = ix->table_base; da.ids = ix->ids;
  da.ecount = ws.ecount.as<uint32_t>(); da.eoff = ws.eoff.as<uint64_t>();
  da.ucount = ws.ecount.as<uint32_t>() + mc;
  da.nitems = reinterpret_cast<unsigned*>(stv + 10);
  da.tierq = ws.ecount.as<uint32_t>() + 2 * mc;
  da.tiern = da.nitems + 1;
  da.region_total = stv + 12;
  da.no_items = pl.sim_keep > 0 ? 1 : 0;
  da.range_shift = pl.range_shift; da.range_count = pl.range_count;
  da.stats = stv;
  // the FPP_DEBUG_BOUNDS build's limits (slot 15 takes the first violation)
  da.bd.flag = stv + 15; da.bd.n = ix->n; da.bd.kept = ix->kept_total;
  da.bd.cap = ws.cand_cap; da.bd.nb = nbuckets(ix->D);
  // items, tier counts (slots 10 and 11) and the slots handed out (slot 12)
  FPP_CUDA(cudaMemsetAsync(stv + 10, 0, 3 * sizeof(unsigned long long), st));
  // candidate slots: the bound from the largest kept bucket when the
  // workspace holds it or can be grown to it within the sync-free budget
  // (no host round trip, so the batch can be captured in a graph; the
  // de-duplication tiers then count the entries and reserve the regions
  // themselves); otherwise count_entries' exact total, read back
  const uint64_t bound = (uint64_t)mc * nt * pl.pmax * std::max<uint32_t>(ix->max_bucket_kept, 1);
  uint64_t need = bound;
  const bool exact = !pl.optimistic && bound > ws.cand_cap &&
                     (pl.no_grow || bound > ix->cand_budget_entries);
  da.fused = exact ? 0 : 1;
  da.overflow = stv + 4;
  if (exact) {
    FPP_TRY(launch_count_entries(da, st));
    FPP_CUDA(cudaMemcpyAsync(&need, stv + 12, 8, cudaMemcpyDeviceToHost, st));
    FPP_CUDA(cudaStreamSynchronize(st));
  }
  if (need > ws.cand_cap && pl.no_grow) {
    set_error("the batch's candidates exceed the candidate buffer");
    return FPP_EBUSY;
  }
  if (need > ws.cand_cap && !pl.optimistic) {
    ws.cand.release(); ws.cscores.release(); ws.items.release();
    const uint64_t cap = exact ? need + need / 4 + 1024 : need;
    FPP_TRY(ws.cand.ensure((size_t)cap * 4));
    FPP_TRY(ws.cscores.ensure((size_t)cap * 4));
    ws.cand_cap = cap;
  }
  const size_t item_bytes =
      (size_t)score_item_slots(ws.cand_cap, mc, pl.range_count) * sizeof(ScoreItem);
  if (pl.no_grow && (ws.items.bytes < item_bytes || (pl.range_count > 1 && ws.items2.bytes < item_bytes))) {
    set_error("serving workspace: score items not provisioned");
    return FPP_EINTERNAL;
  }
  FPP_TRY(ws.items.ensure(item_bytes));
  if (pl.range_count > 1) FPP_TRY(ws.items2.ensure(item_bytes));
  da.cand = ws.cand.as<uint32_t>();
  da.items = ws.items.as<ScoreItem>();
  da.bd.cap = ws.cand_cap;
  da.cap = ws.cand_cap;
  FPP_TRY(launch_dedup(da, st));
  // the work items in order of their row range (the scoring reads them so)
  const ScoreItem* score_items = ws.items.as<ScoreItem>();
  if (pl.range_count > 1) {
    unsigned* rh = reinterpret_cast<unsigned*>(ws.rhist.p);
    FPP_CUDA(cudaMemsetAsync(rh, 0, 2 * SCORE_RANGE_MAX * sizeof(unsigned), st));   // hist, cursors
    FPP_TRY(launch_order_items(ws.items.as<ScoreItem>(), da.nitems, ws.cand.as<uint32_t>(),
                               pl.range_shift, pl.range_count, rh, rh + SCORE_RANGE_MAX,
                               ws.items2.as<ScoreItem>(), st));
    score_items = ws.items2.as<ScoreItem>();
  }
  ws.score_items = score_items;
  if (pl.sim_keep > 0) {
    SimArgs sm{};
    sm.mq = mc; sm.eoff = ws.eoff.as<uint64_t>(); sm.cand = ws.cand.as<uint32_t>();
    sm.ucount = da.ucount; sm.xsig = ix->sig; sm.qsig = ws.qsig.as<uint32_t>();
    sm.words = ix->sig_words; sm.keep = pl.sim_keep; sm.cap = topk_cap(pl.sim_keep);
    sm.items = ws.items.as<ScoreItem>(); sm.nitems = da.nitems;
    FPP_TRY(launch_simhash_filter(sm, st));
  }
  if (ev) FPP_CUDA(cudaEventRecord(ev[5], st));
  if (stage == kCandidatesOnly) return tile_read();
  ScoreArgs sa{};
  sa.items = score_items; sa.nitems = da.nitems;
  sa.eoff = ws.eoff.as<uint64_t>(); sa.mq = mc;
  sa.cand = ws.cand.as<uint32_t>();
  sa.X = ix->X; sa.ldx = ix->dpad; sa.Q = qp; sa.ldq = ix->dpad;
  sa.Xb = ix->Xb; sa.ldxb = ix->ldxb;
  sa.Xq = ix->Xq; sa.ldxq = ix->ldxq; sa.xscale = ix->xscale;
  sa.scores = ws.cscores.as<float>();
  sa.tune_g = ix->tune_score_g; sa.tune_waves = ix->tune_score_waves;
  sa.bd = da.bd;
  FPP_TRY(launch_score(sa, ix->sm_count, st));
  if (ev) FPP_CUDA(cudaEventRecord(ev[6], st));
  TopkArgs ta{};
  ta.mq = mc; ta.eoff = ws.eoff.as<uint64_t>(); ta.ucount = da.ucount; ta.cand = ws.cand.as<uint32_t>();
  ta.scores = ws.cscores.as<float>(); ta.k_pq = kpq; ta.k = pl.k; ta.kmax = pl.kmax;
  ta.X = ix->X; ta.ldx = ix->dpad; ta.Q = qp; ta.ldq = ix->dpad; ta.d = ix->d;
  ta.qnorm = ws.qnorm.as<float>(); ta.xmax = ix->xmax; ta.gamma = ix->score_gamma;
  ta.gammaf = (float)(ix->score_gamma * 1.0001);
  ta.kprime = topk_kprime(ix, pl.kmax);
  ta.approx = ix->precision == FPP_BF16 ? 1 : ix->precision == FPP_FP8E4M3 ? 2 : 0;
  ta.cap = topk_cap(ta.kprime); ta.rcap = topk_rcap(ta.kprime);
  ta.slow = ws.tkslow.p; ta.err = reinterpret_cast<int*>(stv + 5); ta.stats = stv;
  ta.out_ids = ids_dev; ta.out_scores = scores_dev;
  ta.bd = da.bd;
  FPP_TRY(launch_topk(ta, st));
  if (ev) FPP_CUDA(cudaEventRecord(ev[3], st));
  return tile_read();
}

// Queries per batch: bounded by the projection workspace (the FP32 tile, or
// the per-hash lists in fused mode) of about 1 GB.
int64_t chunk_rows(const fpp_index* ix, int nt, int pmax, bool allow_fused = true) {
  const int EL = allow_fused ? fused_list_len(ix, pmax) : 0;
  const int64_t per_query = EL ? 2ll * nt * (EL + 1) * 8 : round_up(2ll * nt * ix->D, 4) * 4;
  int64_t mc = (1ll << 30) / per_query;
  mc = std::max<int64_t>(128, std::min<int64_t>(mc, 65536));
  return mc;
}

fpp_status prepare_workspace(fpp_index* ix, Workspace& ws, const SearchPlan& pl, int64_t mc,
                             bool host_out, cudaStream_t st, bool allow_fused = true,
                             bool two_tiles = false) {
  const int nt = pl.te - pl.tb;
  const int64_t ldp = round_up(2ll * nt * ix->D, 4);
  // query tiles; the pad columns stay zero (the uploads write d columns)
  if (two_tiles) FPP_TRY(ws.ensure_copy_stream());
  bool zeroed = false;
  for (DevBuf* qb : {&ws.qpad, &ws.qpad_alt}) {
    if (qb == &ws.qpad_alt && !two_tiles) break;
    const bool qz = qb->bytes < (size_t)mc * ix->dpad * 4;
    FPP_TRY(qb->ensure((size_t)mc * ix->dpad * 4, false, st));
    if (qz && ix->dpad != ix->d) {
      FPP_CUDA(cudaMemsetAsync(qb->p, 0, qb->bytes, st));
      zeroed = true;
    }
  }
  if (zeroed && ws.cstream) {
    // uploads on the copy stream start after the zeroing
    for (int i = 0; i < 2; ++i) {
      FPP_CUDA(cudaEventRecord(ws.qfree[i], st));
      ws.qused[i] = true;
    }
  }
  const int EL = allow_fused ? fused_list_len(ix, pl.pmax) : 0;
  const size_t tile = EL ? (size_t)mc * 2 * nt * (EL + 1) * 8 : (size_t)mc * ldp * 4;
  FPP_TRY(ws.proj.ensure(tile, false, st));
  FPP_TRY(ws.qsplit.ensure((size_t)mc * ix->pieces * ix->Kp * 2));   // the queries' BF16 pieces
  FPP_TRY(ws.probes.ensure((size_t)mc * nt * pl.pmax * 4, false, st));
  FPP_TRY(ws.qnorm.ensure((size_t)mc * 4, false, st));
  FPP_TRY(ws.recheck.ensure((size_t)mc * nt * 4, false, st));
  FPP_TRY(ws.recheck2.ensure((size_t)mc * nt * 4, false, st));
  FPP_TRY(ws.recheck_s.ensure((size_t)mc * nt * 16, false, st));   // sP, sP1, two list maxima
  if (pl.sim_keep > 0) {
    FPP_TRY(ws.sigproj.ensure((size_t)mc * ix->sig_words * 32 * 4, false, st));
    FPP_TRY(ws.qsig.ensure((size_t)mc * ix->sig_words * 4, false, st));
  }
  FPP_TRY(ws.kpq.ensure((size_t)mc * 4, false, st));
  FPP_TRY(ws.ppq.ensure((size_t)mc * 4, false, st));
  FPP_TRY(ws.stats.ensure(16 * 8, true, st));
  FPP_TRY(ws.rhist.ensure(2 * SCORE_RANGE_MAX * sizeof(unsigned), false, st));
  if (host_out) {
    FPP_TRY(ws.out_ids.ensure((size_t)mc * pl.kmax * 8, false, st));
    FPP_TRY(ws.out_scores.ensure((size_t)mc * pl.kmax * 4, false, st));
  }
  FPP_TRY(ws.ecount.ensure((size_t)4 * mc * 4, false, st));   // counts, distinct counts, 2 tiers
  FPP_TRY(ws.eoff.ensure((size_t)mc * 8, false, st));
  FPP_TRY(ws.tkslow.ensure((size_t)(ceil_div(mc, 8) * 8) * topk_slow_cap() * 16, false, st));
  return FPP_OK;
}

// FPP_SEARCH_GRAPH: the whole call (every batch) as one CUDA graph, captured
// on first use and replayed while the call's arguments and the workspace
// stay the same.  There is no read-back inside a graph.  When the
// candidate buffers can be provisioned from the worst-case bound, the graph
// runs without waiting.  Otherwise (a bound past the sync-free budget) the
// buffers are provisioned up to that budget and the graph is optimistic:
// the de-duplication tiers check every region against the buffer, a query
// whose region would not fit gets no candidates and raises the overflow flag,
// and the call waits for the flag; if it is set, search_graph returns false
// and the caller repeats the call without the graph, sized from the exact
// totals.  Returns false (nothing done) as well when the graph cannot be used.
bool search_graph(fpp_index* ix, const float* Q, int64_t m, const fpp_search_opts* o,
                  const SearchPlan& pl0, int64_t mc, int64_t* ids, float* scores, cudaStream_t st,
                  fpp_status& out) {
  Workspace& ws = ix->ws;
  const int nt = pl0.te - pl0.tb;
  const uint64_t bound = (uint64_t)mc * nt * pl0.pmax * std::max<uint32_t>(ix->max_bucket_kept, 1);
  SearchPlan pl = pl0;
  pl.optimistic = bound > ws.cand_cap && bound > ix->cand_budget_entries;
  const uint64_t want = pl.optimistic ? std::max<uint64_t>(ws.cand_cap, ix->cand_budget_entries) : bound;
  out = FPP_OK;
  auto fail = [&](fpp_status s) { out = s; return true; };
  if (want > ws.cand_cap) {
    ws.cand.release(); ws.cscores.release(); ws.items.release();
    if ((out = ws.cand.ensure((size_t)want * 4)) != FPP_OK) return true;
    if ((out = ws.cscores.ensure((size_t)want * 4)) != FPP_OK) return true;
    ws.cand_cap = want;
  }
  const size_t item_bytes =
      (size_t)score_item_slots(ws.cand_cap, mc, pl.range_count) * sizeof(ScoreItem);
  if ((out = ws.items.ensure(item_bytes)) != FPP_OK) return true;
  if (pl.range_count > 1 && (out = ws.items2.ensure(item_bytes)) != FPP_OK) return true;
  const std::vector<uint64_t> key = {
      (uint64_t)(uintptr_t)Q, (uint64_t)m, (uint64_t)(uintptr_t)ids, (uint64_t)(uintptr_t)scores,
      (uint64_t)(uintptr_t)pl.kpq, (uint64_t)(uintptr_t)pl.ppq, (uint64_t)pl.k,
      (uint64_t)pl.probes, (uint64_t)pl.kmax, (uint64_t)pl.pmax, (uint64_t)pl.tb, (uint64_t)pl.te,
      (uint64_t)(uintptr_t)st, (uint64_t)pl.global_q, (uint64_t)pl.sim_keep,
      (uint64_t)pl.range_shift, (uint64_t)pl.range_count, (uint64_t)pl.optimistic, g_alloc_gen.load()};
  if (!ix->graph_exec || ix->graph_key != key) {
    if (ix->graph_exec) cudaGraphExecDestroy(ix->graph_exec);
    ix->graph_exec = nullptr;
    ix->graph_key.clear();
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      set_error("search graph: stream capture could not start");
      return fail(FPP_ECUDA);
    }
    fpp_status s = FPP_OK;
    const uint64_t k0 = launch_counter().load();
    if (cudaMemsetAsync(ws.stats.p, 0, 16 * 8, st) != cudaSuccess) s = FPP_ECUDA;
    for (int64_t q0 = 0; q0 < m && s == FPP_OK; q0 += mc) {
      const int64_t c = std::min<int64_t>(mc, m - q0);
      s = search_chunk(ix, ws, Q, q0, c, pl, ids + q0 * pl.kmax, scores + q0 * pl.kmax, st, kFull,
                       nullptr);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (s == FPP_OK && ce != cudaSuccess) {
      set_error(std::string("search graph: capture failed: ") + cudaGetErrorString(ce));
      s = FPP_ECUDA;
    }
    if (s == FPP_OK && cudaGraphInstantiate(&ix->graph_exec, g, 0) != cudaSuccess) {
      set_error("search graph: instantiation failed");
      ix->graph_exec = nullptr;
      s = FPP_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    // the capture counted the kernels it recorded; they run at each replay
    ix->graph_kernels = launch_counter().load() - k0;
    launch_counter().fetch_sub(ix->graph_kernels);
    if (s != FPP_OK) return fail(s);
    ix->graph_key = key;
  }
  if (cudaGraphLaunch(ix->graph_exec, st) != cudaSuccess) {
    set_error("search graph: launch failed");
    return fail(FPP_ECUDA);
  }
  launch_counter().fetch_add(ix->graph_kernels, std::memory_order_relaxed);
  if (pl.optimistic) {
    unsigned long long ov = 0;
    if (cudaMemcpyAsync(&ov, ws.stats.as<unsigned long long>() + 4, 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_error("search graph: reading the overflow flag failed");
      return fail(FPP_ECUDA);
    }
    if (ov) {   // some region did not fit: the call is repeated without the graph
      ix->graph_overflows += 1;
      return false;
    }
  }
  return true;
}

// FPP_SEARCH_PIPELINE: call c of the index runs on internal stream c % 2
// with workspace c % 2.  It starts once the caller's stream reaches the call
// (its inputs are then final) and the previous call on the same slot has
// ended; the caller's stream then waits for the previous call of the other
// slot, so at most two calls are in flight and each call's results are
// complete when the caller's stream reaches the next pipelined call (or
// fpp_search_flush).  Device-side error flags are not read.
fpp_status search_pipelined(fpp_index* ix, const float* Q, int64_t m, const SearchPlan& pl,
                            int64_t mc, int64_t* ids, float* scores, cudaStream_t st,
                            bool dev_out) {
  constexpr int NS = fpp_index::PIPE_SLOTS;
  const int c = ix->pnext;
  ix->pnext = (c + 1) % NS;
  if (!ix->pin) FPP_CUDA(cudaEventCreateWithFlags(&ix->pin, cudaEventDisableTiming));
  if (!ix->pstream[c]) {
    FPP_CUDA(cudaStreamCreateWithFlags(&ix->pstream[c], cudaStreamNonBlocking));
    FPP_CUDA(cudaEventCreateWithFlags(&ix->pdone[c], cudaEventDisableTiming));
  }
  cudaStream_t ps = ix->pstream[c];
  Workspace& W = c ? ix->ws_pipe[c - 1] : ix->ws;
  FPP_CUDA(cudaEventRecord(ix->pin, st));
  FPP_CUDA(cudaStreamWaitEvent(ps, ix->pin, 0));
  FPP_TRY(prepare_workspace(ix, W, pl, mc, !dev_out, ps, true, false));
  FPP_TRY(W.order_after_last(ps));
  FPP_CUDA(cudaMemsetAsync(W.stats.p, 0, 16 * 8, ps));
  for (int64_t q0 = 0; q0 < m; q0 += mc) {
    const int64_t cq = std::min<int64_t>(mc, m - q0);
    int64_t* oid = dev_out ? ids + q0 * pl.kmax : W.out_ids.as<int64_t>();
    float* osc = dev_out ? scores + q0 * pl.kmax : W.out_scores.as<float>();
    FPP_TRY(search_chunk(ix, W, Q, q0, cq, pl, oid, osc, ps, kFull, nullptr, false));
    if (!dev_out) {
      FPP_CUDA(cudaMemcpyAsync(ids + q0 * pl.kmax, oid, cq * pl.kmax * 8, cudaMemcpyDeviceToHost, ps));
      FPP_CUDA(cudaMemcpyAsync(scores + q0 * pl.kmax, osc, cq * pl.kmax * 4, cudaMemcpyDeviceToHost, ps));
    }
  }
  FPP_TRY(W.mark_done(ps));
  FPP_CUDA(cudaEventRecord(ix->pdone[c], ps));
  ix->ppending[c] = true;
  // the caller's stream waits for the oldest call still in flight, so that
  // NS calls overlap and the call NS - 1 back is complete at this point
  const int old = (c + 1) % NS;
  if (ix->ppending[old]) {
    FPP_CUDA(cudaStreamWaitEvent(st, ix->pdone[old], 0));
    ix->ppending[old] = false;
  }
  return FPP_OK;
}

fpp_status search_impl(const fpp_index* cix, const float* Q, int64_t m, const fpp_search_opts* o,
                       int64_t* ids, float* scores, fpp_search_stats* stats) {
  SearchPlan pl{};
  FPP_TRY(validate_search(cix, Q, m, o, ids, scores, pl));
  fpp_index* ix = const_cast<fpp_index*>(cix);
  std::lock_guard<std::mutex> lock(ix->mu);
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (m == 0) return FPP_OK;
  cudaStream_t st = (cudaStream_t)o->stream;
  const bool dev_out = is_device_ptr(ids) && is_device_ptr(scores);
  const int nt = pl.te - pl.tb;
  const int64_t mc = std::min<int64_t>(chunk_rows(ix, nt, pl.pmax), m);
  const bool out_pinned = is_pinned_host(ids) && is_pinned_host(scores);
  if ((o->flags & FPP_SEARCH_PIPELINE) && st && !stats && pl.global_q == 0 &&
      (dev_out || out_pinned) && (is_device_ptr(Q) || is_pinned_host(Q)) &&
      (!pl.kpq || pl.kpq_dev) && (!pl.ppq || pl.ppq_dev))
    return search_pipelined(ix, Q, m, pl, mc, ids, scores, st, dev_out);
  // page-locked host queries on a caller's stream: the uploads run ahead on
  // the workspace's copy stream, two query tiles in turn
  const bool ahead = st != nullptr && !is_device_ptr(Q) && is_pinned_host(Q);
  FPP_TRY(prepare_workspace(ix, ix->ws, pl, mc, !dev_out, st, true, ahead));
  FPP_TRY(ix->ws.order_after_last(st));
  if ((o->flags & FPP_SEARCH_GRAPH) && st && dev_out && !stats && is_device_ptr(Q) && pl.global_q == 0 &&
      (!pl.kpq || pl.kpq_dev) && (!pl.ppq || pl.ppq_dev)) {
    fpp_status gs = FPP_OK;
    if (search_graph(ix, Q, m, o, pl, mc, ids, scores, st, gs)) {
      if (gs == FPP_OK) gs = ix->ws.mark_done(st);
      return gs;
    }
  }
  FPP_CUDA(cudaMemsetAsync(ix->ws.stats.p, 0, 16 * 8, st));
  cudaEvent_t ev[7] = {};
  bool timing = stats != nullptr;
  if (timing)
    for (auto& e : ev) FPP_CUDA(cudaEventCreate(&e));
  float ms[7] = {0, 0, 0, 0, 0, 0, 0};
  uint64_t batches = 0;
  for (int64_t q0 = 0; q0 < m; q0 += mc, ++batches) {
    const int64_t c = std::min<int64_t>(mc, m - q0);
    int64_t* oid = dev_out ? ids + q0 * pl.kmax : ix->ws.out_ids.as<int64_t>();
    float* osc = dev_out ? scores + q0 * pl.kmax : ix->ws.out_scores.as<float>();
    FPP_TRY(search_chunk(ix, ix->ws, Q, q0, c, pl, oid, osc, st, kFull, timing ? ev : nullptr,
                         ahead));
    if (!dev_out) {
      FPP_CUDA(cudaMemcpyAsync(ids + q0 * pl.kmax, oid, c * pl.kmax * 8, cudaMemcpyDeviceToHost, st));
      FPP_CUDA(cudaMemcpyAsync(scores + q0 * pl.kmax, osc, c * pl.kmax * 4, cudaMemcpyDeviceToHost, st));
    }
    if (timing) {
      FPP_CUDA(cudaEventSynchronize(ev[3]));
      float t[7];
      cudaEventElapsedTime(&t[0], ev[0], ev[1]);
      cudaEventElapsedTime(&t[1], ev[1], ev[4]);
      cudaEventElapsedTime(&t[2], ev[4], ev[2]);
      cudaEventElapsedTime(&t[3], ev[2], ev[3]);
      cudaEventElapsedTime(&t[4], ev[2], ev[5]);
      cudaEventElapsedTime(&t[5], ev[5], ev[6]);
      cudaEventElapsedTime(&t[6], ev[6], ev[3]);
      for (int i = 0; i < 7; ++i) ms[i] += t[i];
    }
  }
  FPP_TRY(ix->ws.mark_done(st));
  // with a stream and no stats the call returns without waiting when the
  // outputs are device memory or page-locked host memory (the copies back
  // are ordered on the stream); error flags are then not read
  const bool out_async = dev_out || (is_pinned_host(ids) && is_pinned_host(scores));
  // a global probe budget always waits: its cap flag decides the status
  const bool need_sync = !out_async || o->stream == nullptr || stats != nullptr || pl.global_q > 0;
  unsigned long long hs[16] = {0};
  if (need_sync) {
    // counters, the top-k flag (slot 5) and the projection's wait flag (slot 9)
    FPP_CUDA(cudaMemcpyAsync(hs, ix->ws.stats.p, 16 * 8, cudaMemcpyDeviceToHost, st));
    FPP_CUDA(cudaStreamSynchronize(st));
    if (hs[5]) {
      set_error("search: top-k re-check capacity exceeded");
      return FPP_EINTERNAL;
    }
    if (hs[9]) {
      set_error("search: a bounded wait in the projection kernel ran out");
      return FPP_ETIMEOUT;
    }
    if (hs[15]) {
      set_error("bounds check failed at site " + std::to_string(hs[15] >> 48) + ", index " +
                std::to_string(hs[15] & 0xFFFFFFFFFFFFull));
      return FPP_EINTERNAL;
    }
    if (hs[13]) {
      set_error("global_probes: " + std::to_string(hs[13]) +
                " queries would take more than 128 buckets from one table; the results are not the "
                "uncapped selection (use a smaller budget or per-table probes)");
      return FPP_EINVAL;
    }
  }
  if (timing)
    for (auto& e : ev) cudaEventDestroy(e);
  if (stats) {
    stats->queries = m;
    stats->entries = hs[0];
    stats->unique = hs[1];
    stats->topk_rechecks = hs[2];
    stats->probes = hs[3];
    stats->probe_rechecks = hs[6];
    stats->probe_full_rechecks = hs[7];
    stats->batches = batches;
    stats->ms_project = ms[0];
    stats->ms_probe = ms[1];
    stats->ms_probe_exact = ms[2];
    stats->ms_gather_score = ms[3];
    stats->ms_dedup = ms[4];
    stats->ms_score = ms[5];
    stats->ms_topk = ms[6];
    stats->ms_total = ms[0] + ms[1] + ms[2] + ms[3];
  }
  return FPP_OK;
}


// ------------------------------------------------------------------ serving
//
// Continuous batching: every slot is a worker thread with its own stream,
// workspace and pinned staging buffers.  A free worker takes the oldest
// queued requests (FIFO) while the batch stays within max_batch queries and
// its estimated candidate-buffer memory within the slot's budget, runs the
// search pipeline on them with per-query k and probe budgets, and completes
// the requests.  Each query's result depends only on the query and its own
// k and probes, never on the rest of its batch.

struct ServerRequest {
  uint64_t id = 0;
  int32_t nq = 0, k = 0, probes = 0;
  std::vector<float> q;          // [nq][d]
  std::vector<int64_t> ids;      // [nq][k]
  std::vector<float> scores;     // [nq][k]
  int state = 0;                 // 0 queued, 1 running, 2 done
  fpp_status status = FPP_OK;
  std::string error;
  std::chrono::steady_clock::time_point t_submit, t_done;
};

struct ServerSlot {
  Workspace ws;
  cudaStream_t st = nullptr;
  float* hq = nullptr;           // pinned [max_batch][d]
  int32_t* hk = nullptr;         // pinned [max_batch]
  int32_t* hp = nullptr;
  int64_t* hids = nullptr;       // pinned [max_batch][k_max]
  float* hsc = nullptr;
  unsigned long long* hstats = nullptr;   // pinned [16]
  std::thread worker;
};

}  // namespace fpp_api

struct fpp_server {
  fpp_index* ix = nullptr;
  fpp_server_cfg cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<fpp_api::ServerRequest*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<fpp_api::ServerRequest>> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::vector<std::unique_ptr<fpp_api::ServerSlot>> slots;
  double entries_per_probe = 0.0;   // running estimate for admission
  fpp_server_stats stats{};
};

namespace fpp_api {

// Candidate-buffer entries a request is expected to need.
double request_entries(const fpp_server* s, const ServerRequest& r) {
  return (double)r.nq * s->ix->L * r.probes * s->entries_per_probe;
}

// A run of consecutive queries of one request.
struct Seg {
  ServerRequest* r;
  int32_t q0, nq;
};

// One search over the segments' queries with the slot's pre-sized
// workspace; results go straight into the requests.  FPP_EBUSY: the
// candidates do not fit the slot's buffer (nothing was written).
fpp_status server_search(fpp_server* s, ServerSlot& sl, const std::vector<Seg>& segs,
                         unsigned long long* entries, unsigned long long* probes) {
  fpp_index* ix = s->ix;
  const int d = ix->d;
  int64_t m = 0;
  int pmax = 1;
  for (const Seg& g : segs) {
    std::memcpy(sl.hq + m * d, g.r->q.data() + (size_t)g.q0 * d, (size_t)g.nq * d * 4);
    for (int i = 0; i < g.nq; ++i) {
      sl.hk[m + i] = g.r->k;
      sl.hp[m + i] = g.r->probes;
    }
    pmax = std::max(pmax, g.r->probes);
    m += g.nq;
  }
  SearchPlan pl{};
  pl.m = m;
  pl.kmax = s->cfg.k_max;
  pl.pmax = pmax;
  pl.tb = 0;
  pl.te = ix->L;
  pl.kpq = sl.hk;
  pl.ppq = sl.hp;
  pl.kpq_dev = pl.ppq_dev = false;
  pl.k = s->cfg.k_max;
  pl.probes = pmax;
  pl.no_grow = true;
  FPP_TRY(prepare_workspace(ix, sl.ws, pl, m, true, sl.st));
  FPP_CUDA(cudaMemsetAsync(sl.ws.stats.p, 0, 16 * 8, sl.st));
  FPP_TRY(search_chunk(ix, sl.ws, sl.hq, 0, m, pl, sl.ws.out_ids.as<int64_t>(),
                       sl.ws.out_scores.as<float>(), sl.st, kFull, nullptr));
  FPP_CUDA(cudaMemcpyAsync(sl.hids, sl.ws.out_ids.p, (size_t)m * pl.kmax * 8,
                           cudaMemcpyDeviceToHost, sl.st));
  FPP_CUDA(cudaMemcpyAsync(sl.hsc, sl.ws.out_scores.p, (size_t)m * pl.kmax * 4,
                           cudaMemcpyDeviceToHost, sl.st));
  FPP_CUDA(cudaMemcpyAsync(sl.hstats, sl.ws.stats.p, 16 * 8, cudaMemcpyDeviceToHost, sl.st));
  FPP_CUDA(cudaStreamSynchronize(sl.st));
  if (sl.hstats[5]) { set_error("search: top-k re-check capacity exceeded"); return FPP_EINTERNAL; }
  if (sl.hstats[9]) { set_error("search: a bounded wait in the projection kernel ran out"); return FPP_ETIMEOUT; }
  if (sl.hstats[15]) { set_error("search: a bounds check failed"); return FPP_EINTERNAL; }
  int64_t row = 0;
  for (const Seg& g : segs) {
    ServerRequest* r = g.r;
    for (int i = 0; i < g.nq; ++i) {
      std::memcpy(r->ids.data() + (size_t)(g.q0 + i) * r->k, sl.hids + (row + i) * pl.kmax, (size_t)r->k * 8);
      std::memcpy(r->scores.data() + (size_t)(g.q0 + i) * r->k, sl.hsc + (row + i) * pl.kmax, (size_t)r->k * 4);
    }
    row += g.nq;
  }
  *entries += sl.hstats[0];
  *probes += sl.hstats[3];
  return FPP_OK;
}

// Runs the segments, splitting them in half by queries (and again) while
// their candidates do not fit the slot's buffer.  A single query always
// fits: fpp_server_create checks its worst case against the buffer.
fpp_status server_run_segs(fpp_server* s, ServerSlot& sl, const std::vector<Seg>& segs,
                           unsigned long long* entries, unsigned long long* probes,
                           uint64_t* splits) {
  const fpp_status st = server_search(s, sl, segs, entries, probes);
  if (st != FPP_EBUSY) return st;
  int64_t m = 0;
  for (const Seg& g : segs) m += g.nq;
  if (m <= 1) {
    set_error("server: one query's candidates exceed the slot's buffer");
    return FPP_EINTERNAL;
  }
  ++*splits;
  const int64_t half = m / 2;
  std::vector<Seg> a, b;
  int64_t at = 0;
  for (const Seg& g : segs) {
    if (at + g.nq <= half) a.push_back(g);
    else if (at >= half) b.push_back(g);
    else {
      const int32_t na = (int32_t)(half - at);
      a.push_back({g.r, g.q0, na});
      b.push_back({g.r, g.q0 + na, g.nq - na});
    }
    at += g.nq;
  }
  FPP_TRY(server_run_segs(s, sl, a, entries, probes, splits));
  return server_run_segs(s, sl, b, entries, probes, splits);
}

void server_run_batch(fpp_server* s, ServerSlot& sl, std::vector<ServerRequest*>& batch) {
  std::vector<Seg> segs;
  int64_t m = 0;
  for (ServerRequest* r : batch) {
    segs.push_back({r, 0, r->nq});
    m += r->nq;
  }
  unsigned long long entries = 0, probes = 0;
  uint64_t splits = 0;
  const uint64_t allocs0 = alloc_counter().load();
  const fpp_status st = server_run_segs(s, sl, segs, &entries, &probes, &splits);
  const uint64_t allocs = alloc_counter().load() - allocs0;
  const auto now = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  s->stats.splits += splits;
  s->stats.serving_allocs += allocs;
  for (ServerRequest* r : batch) {
    r->state = 2;
    r->t_done = now;
    if (st != FPP_OK) {
      r->status = st;
      r->error = g_err;
    }
  }
  if (st != FPP_OK) {
    s->stats.failed += batch.size();
    s->cv_done.notify_all();
    return;
  }
  s->stats.completed += batch.size();
  s->stats.batches += 1;
  s->stats.queries += (uint64_t)m;
  s->stats.entries += entries;
  s->stats.probes += probes;
  if (probes) {
    const double epp = (double)entries / (double)probes;
    s->entries_per_probe = 0.8 * s->entries_per_probe + 0.2 * epp * 1.25;
  }
  s->cv_done.notify_all();
}

void server_worker(fpp_server* s, ServerSlot* sl) {
  cudaSetDevice(s->ix->device);
  const double budget = (double)s->cfg.candidate_budget_bytes / 8.0;   // cand + score per entry
  std::vector<ServerRequest*> batch;
  while (true) {
    batch.clear();
    {
      std::unique_lock<std::mutex> lock(s->mu);
      s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) return;
      int64_t nq = 0;
      double ent = 0.0;
      while (!s->queue.empty()) {
        ServerRequest* r = s->queue.front();
        const double e = request_entries(s, *r);
        if (!batch.empty() && (nq + r->nq > s->cfg.max_batch || ent + e > budget)) break;
        batch.push_back(r);
        s->queue.pop_front();
        r->state = 1;
        nq += r->nq;
        ent += e;
      }
      s->stats.queued = s->queue.size();
    }
    server_run_batch(s, *sl, batch);
  }
}

void server_release(fpp_server* s) {
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& sl : s->slots)
    if (sl->worker.joinable()) sl->worker.join();
  for (auto& sl : s->slots) {
    sl->ws.release();
    if (sl->st) cudaStreamDestroy(sl->st);
    cudaFreeHost(sl->hq);
    cudaFreeHost(sl->hk);
    cudaFreeHost(sl->hp);
    cudaFreeHost(sl->hids);
    cudaFreeHost(sl->hsc);
    cudaFreeHost(sl->hstats);
  }
  s->slots.clear();
}

fpp_status server_create_impl(const fpp_index* cix, const fpp_server_cfg* cfg, fpp_server** out) {
  if (!cix || !cfg || !out) { set_error("NULL argument"); return FPP_EINVAL; }
  const int64_t NB = nbuckets(cix->D);
  const int pcap = (int)std::min<int64_t>(NB, 128);
  if (cfg->max_batch < 1 || cfg->max_batch > 65536) { set_error("max_batch must be in [1, 65536]"); return FPP_EINVAL; }
  if (cfg->slots < 1 || cfg->slots > 16) { set_error("slots must be in [1, 16]"); return FPP_EINVAL; }
  if (cfg->k_max < 1 || cfg->k_max > 256) { set_error("k_max must be in [1, 256]"); return FPP_EINVAL; }
  if (cfg->probes_max < 1 || cfg->probes_max > pcap) {
    set_error("probes_max must be in [1, min(4D^2, 128)]");
    return FPP_EINVAL;
  }
  if (cfg->max_queue < 1) { set_error("max_queue must be >= 1"); return FPP_EINVAL; }
  if (cfg->candidate_budget_bytes < ((uint64_t)1 << 20)) {
    set_error("candidate_budget_bytes must be >= 1 MiB");
    return FPP_EINVAL;
  }
  // the worst case of one query (every probed bucket as large as the largest
  // kept bucket) must fit a slot's buffer, so that splitting a batch always
  // ends in batches that fit
  const uint64_t one_query = (uint64_t)cix->L * cfg->probes_max * std::max<uint32_t>(cix->max_bucket_kept, 1);
  if (one_query > cfg->candidate_budget_bytes / 8) {
    set_error("candidate_budget_bytes must hold one query's worst case, 8 L probes_max max_bucket_kept = " +
              std::to_string(one_query * 8) + " bytes");
    return FPP_EINVAL;
  }
  auto s = std::make_unique<fpp_server>();
  s->ix = const_cast<fpp_index*>(cix);
  s->cfg = *cfg;
  // initial admission estimate: the mean kept bucket size, doubled
  s->entries_per_probe = 2.0 * (double)cix->kept_total / ((double)cix->L * (double)NB) + 1.0;
  if (cudaSetDevice(cix->device) != cudaSuccess) { set_error("cudaSetDevice failed"); return FPP_ECUDA; }
  SearchPlan pl{};
  pl.m = cfg->max_batch;
  pl.kmax = cfg->k_max;
  pl.pmax = cfg->probes_max;
  pl.tb = 0;
  pl.te = cix->L;
  const int d = cix->d;
  for (int i = 0; i < cfg->slots; ++i) {
    auto sl = std::make_unique<ServerSlot>();
    fpp_status st = FPP_OK;
    if (cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&sl->hq, (size_t)cfg->max_batch * d * 4) != cudaSuccess ||
        cudaMallocHost(&sl->hk, (size_t)cfg->max_batch * 4) != cudaSuccess ||
        cudaMallocHost(&sl->hp, (size_t)cfg->max_batch * 4) != cudaSuccess ||
        cudaMallocHost(&sl->hids, (size_t)cfg->max_batch * cfg->k_max * 8) != cudaSuccess ||
        cudaMallocHost(&sl->hsc, (size_t)cfg->max_batch * cfg->k_max * 4) != cudaSuccess ||
        cudaMallocHost(&sl->hstats, 16 * 8) != cudaSuccess) {
      set_error("server: allocating a slot's stream or pinned buffers failed");
      st = FPP_ENOMEM;
    }
    if (st == FPP_OK) st = prepare_workspace(s->ix, sl->ws, pl, cfg->max_batch, true, sl->st);
    if (st == FPP_OK) {
      const uint64_t cap = cfg->candidate_budget_bytes / 8;
      if ((st = sl->ws.cand.ensure((size_t)cap * 4)) == FPP_OK &&
          (st = sl->ws.cscores.ensure((size_t)cap * 4)) == FPP_OK)
        sl->ws.cand_cap = cap;
      // the score work items for a full buffer: serving allocates nothing
      if (st == FPP_OK)
        st = sl->ws.items.ensure((size_t)score_item_slots(cap, cfg->max_batch, 1) * sizeof(ScoreItem));
    }
    if (st == FPP_OK && cudaStreamSynchronize(sl->st) != cudaSuccess) st = FPP_ECUDA;
    s->slots.push_back(std::move(sl));
    if (st != FPP_OK) {
      server_release(s.get());
      return st;
    }
  }
  for (auto& sl : s->slots) sl->worker = std::thread(server_worker, s.get(), sl.get());
  *out = s.release();
  return FPP_OK;
}

}  // namespace fpp_api

using namespace fpp_api;

// ====================================================================== C ABI

extern "C" {

void fpp_default_params(fpp_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->L = 10;
  p->D = 64;
  p->iprobes = 1;
  p->kappa = 0;
  p->alpha = 0.1;
  p->seed = 0;
  p->R = nullptr;
  p->precision = FPP_FP32;
  p->rerank_k = 100;
  p->stream = nullptr;
}

void fpp_default_search_opts(fpp_search_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->k = 10;
  o->probes = 1;
}

const char* fpp_last_error(void) { return g_err.c_str(); }

fpp_status fpp_search_flush(const fpp_index* cix, void* stream) {
  g_err.clear();
  if (!cix) { set_error("index is NULL"); return FPP_EINVAL; }
  fpp_index* ix = const_cast<fpp_index*>(cix);
  std::lock_guard<std::mutex> lock(ix->mu);
  for (int c = 0; c < fpp_index::PIPE_SLOTS; ++c) {
    if (!ix->ppending[c]) continue;
    FPP_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, ix->pdone[c], 0));
    ix->ppending[c] = false;
  }
  return FPP_OK;
}

uint64_t fpp_launch_count(void) { return g_launches.load(); }
uint64_t fpp_alloc_count(void) { return alloc_counter().load(); }

uint64_t fpp_keep_count(uint64_t B, double alpha, int32_t iprobes, int32_t kappa) {
  if (iprobes < 1) iprobes = 1;
  const double c = std::ceil((alpha * (double)B) / (double)iprobes);
  uint64_t k = (uint64_t)c;
  if (kappa > 0 && k < (uint64_t)kappa) k = (uint64_t)kappa;
  return k > B ? B : k;
}

fpp_status fpp_rotations(uint64_t seed, int32_t L, int32_t D, int32_t d, float* R) {
  g_err.clear();
  if (!R || L < 1 || D < 1 || d < 1) {
    set_error("fpp_rotations: L, D, d must be >= 1 and R non-NULL");
    return FPP_EINVAL;
  }
  generate_rotations(seed, L, D, d, R);
  return FPP_OK;
}

fpp_status fpp_build(const float* X, int64_t n, int32_t d, const fpp_params* p, fpp_index** out) {
  g_err.clear();
  try {
    return build_impl(X, n, d, p, out);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return FPP_ENOMEM;
  } catch (...) {
    set_error("unexpected exception in fpp_build");
    return FPP_EINTERNAL;
  }
}

fpp_status fpp_search_ex(const fpp_index* ix, const float* Q, int64_t m, const fpp_search_opts* opts,
                         int64_t* ids, float* scores, fpp_search_stats* stats) {
  g_err.clear();
  try {
    return search_impl(ix, Q, m, opts, ids, scores, stats);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return FPP_ENOMEM;
  } catch (...) {
    set_error("unexpected exception in fpp_search_ex");
    return FPP_EINTERNAL;
  }
}

fpp_status fpp_search(const fpp_index* ix, const float* Q, int64_t m, int32_t k, int32_t probes,
                      int64_t* ids, float* scores) {
  fpp_search_opts o;
  fpp_default_search_opts(&o);
  o.k = k;
  o.probes = probes;
  o.k_max = k;
  return fpp_search_ex(ix, Q, m, &o, ids, scores, nullptr);
}

void fpp_free(fpp_index* ix) {
  if (!ix) return;
  free_index_memory(ix);
  delete ix;
}

fpp_status fpp_index_get_info(const fpp_index* ix, fpp_index_info* info) {
  g_err.clear();
  if (!ix || !info) { set_error("NULL argument"); return FPP_EINVAL; }
  info->n = ix->n; info->d = ix->d; info->L = ix->L; info->D = ix->D;
  info->iprobes = ix->iprobes; info->kappa = ix->kappa; info->precision = ix->precision;
  info->alpha = ix->alpha; info->kept_total = ix->kept_total;
  info->max_bucket_kept = ix->max_bucket_kept; info->device_bytes = ix->device_bytes;
  info->build_ms = ix->build_ms;
  info->rerank_k = ix->rerank_k;
  info->center = ix->center;
  info->simhash_bits = ix->sig_words * 32;
  info->r_pieces = ix->bpieces;
  info->score_error_factor = ix->score_gamma;
  info->q_pieces = ix->qpieces;
  info->graph_fallbacks = (uint32_t)ix->graph_overflows;
  return FPP_OK;
}

fpp_status fpp_set_candidate_budget(fpp_index* ix, uint64_t bytes) {
  g_err.clear();
  if (!ix) { set_error("index is NULL"); return FPP_EINVAL; }
  if (bytes < 4096) { set_error("the candidate budget must be at least 4,096 bytes"); return FPP_EINVAL; }
  std::lock_guard<std::mutex> lock(ix->mu);
  ix->cand_budget_entries = bytes / 8;
  return FPP_OK;
}

fpp_status fpp_debug_point_buckets(const fpp_index* cix, int32_t t, uint32_t* out) {
  g_err.clear();
  if (!cix || !out) { set_error("NULL argument"); return FPP_EINVAL; }
  if (t < 0 || t >= cix->L) { set_error("table out of range"); return FPP_EINVAL; }
  fpp_index* ix = const_cast<fpp_index*>(cix);
  std::lock_guard<std::mutex> lock(ix->mu);
  cudaStream_t st = 0;
  const int ip = ix->iprobes;
  const int64_t ldp = round_up(2ll * ix->D, 4);
  const int64_t rows = std::min<int64_t>(ix->n, std::max<int64_t>(128, (1ll << 27) / ldp));
  DevBuf proj, pb, split, err, norms, rc1, rc2;
  auto done = [&](fpp_status s) {
    for (DevBuf* b : {&proj, &pb, &split, &err, &norms, &rc1, &rc2}) b->release();
    return s;
  };
  fpp_status s;
  if ((s = err.ensure(16, true, st)) != FPP_OK) return done(s);
  if ((s = proj.ensure((size_t)rows * ldp * 4)) != FPP_OK) return done(s);
  if ((s = pb.ensure((size_t)ix->n * ip * 4)) != FPP_OK) return done(s);
  if (ip > 1 && ((s = norms.ensure((size_t)rows * 4)) != FPP_OK ||
                 (s = rc1.ensure((size_t)rows * 4)) != FPP_OK ||
                 (s = rc2.ensure((size_t)rows * 4)) != FPP_OK))
    return done(s);
  for (int64_t r0 = 0; r0 < ix->n; r0 += rows) {
    const int64_t rc = std::min<int64_t>(rows, ix->n - r0);
    if ((s = project_rows(ix, hashed_rows(ix) + r0 * ix->dpad, rc, split, t, 1, proj.as<float>(), ldp,
                          err.as<int>(), st)) != FPP_OK)
      return done(s);
    if (ip > 1) {
      // the point's iProbes best buckets, ranked as for a query
      const float* xr = hashed_rows(ix) + r0 * ix->dpad;
      if ((s = launch_query_norms(xr, rc, ix->dpad, ix->d, norms.as<float>(), st)) != FPP_OK)
        return done(s);
      ProbeArgs pa{};
      pa.P = proj.as<float>(); pa.ldp = ldp; pa.mq = rc;
      pa.Q = xr; pa.ldq = ix->dpad; pa.qnorm = norms.as<float>();
      pa.R = ix->R; pa.ldr = ix->dpad; pa.d = ix->d; pa.D = ix->D; pa.tb = t; pa.nt = 1;
      pa.rmax = ix->rmax; pa.gamma = ix->gamma; pa.gammaf = (float)(ix->gamma * 1.0001);
      pa.probes = ip; pa.out = pb.as<uint32_t>() + r0 * ip;
      pa.recheck = rc1.as<uint32_t>(); pa.recheck_count = err.as<unsigned>() + 2;
      pa.recheck2 = rc2.as<uint32_t>(); pa.recheck2_count = err.as<unsigned>() + 3;
      if ((s = launch_probe(pa, st)) != FPP_OK) return done(s);
      continue;
    }
    HashArgs h{};
    h.P = proj.as<float>(); h.ldp = ldp; h.rows = rc; h.row0 = r0; h.t0 = t; h.nt = 1; h.D = ix->D;
    h.X = hashed_rows(ix); h.ldx = ix->dpad; h.R = ix->R; h.ldr = ix->dpad; h.d = ix->d;
    h.rmax = ix->rmax; h.xmax = ix->xhmax; h.gamma = ix->gamma; h.n = ix->n;
    h.eps_xf = (float)(ix->gamma * (double)ix->xhmax * 1.0001);
    h.point_bucket = pb.as<uint32_t>() + r0;
    if ((s = launch_build_hash(h, st)) != FPP_OK) return done(s);
  }
  if (cudaMemcpy(out, pb.p, (size_t)ix->n * ip * 4, cudaMemcpyDefault) != cudaSuccess) {
    set_error("copy point buckets");
    return done(FPP_ECUDA);
  }
  return done(FPP_OK);
}

fpp_status fpp_debug_table(const fpp_index* ix, int32_t t, uint32_t* offsets, uint32_t* ids) {
  g_err.clear();
  if (!ix || !offsets) { set_error("NULL argument"); return FPP_EINVAL; }
  if (t < 0 || t >= ix->L) { set_error("table out of range"); return FPP_EINVAL; }
  const int64_t NB = nbuckets(ix->D);
  FPP_CUDA(cudaMemcpy(offsets, ix->offsets + (int64_t)t * (NB + 1), (NB + 1) * 4, cudaMemcpyDefault));
  if (ids) {
    uint32_t cnt = 0;
    FPP_CUDA(cudaMemcpy(&cnt, ix->offsets + (int64_t)t * (NB + 1) + NB, 4, cudaMemcpyDeviceToHost));
    if (cnt) FPP_CUDA(cudaMemcpy(ids, ix->ids + ix->h_table_base[t], (size_t)cnt * 4, cudaMemcpyDefault));
  }
  return FPP_OK;
}

fpp_status fpp_debug_probes(const fpp_index* cix, const float* Q, int64_t m, int32_t probes,
                            int32_t table_begin, int32_t table_end, uint32_t* out) {
  g_err.clear();
  fpp_search_opts o;
  fpp_default_search_opts(&o);
  o.probes = probes;
  o.k = 1;
  o.table_begin = table_begin;
  o.table_end = table_end;
  SearchPlan pl{};
  int64_t dummy_i = 0;
  float dummy_s = 0;
  FPP_TRY(validate_search(cix, Q, m, &o, &dummy_i, &dummy_s, pl));
  if (!out && m) { set_error("out is NULL"); return FPP_EINVAL; }
  fpp_index* ix = const_cast<fpp_index*>(cix);
  std::lock_guard<std::mutex> lock(ix->mu);
  if (m == 0) return FPP_OK;
  const int nt = pl.te - pl.tb;
  const int64_t mc = std::min<int64_t>(chunk_rows(ix, nt, pl.pmax), m);
  FPP_TRY(prepare_workspace(ix, ix->ws, pl, mc, false, 0));
  FPP_TRY(ix->ws.order_after_last(0));
  for (int64_t q0 = 0; q0 < m; q0 += mc) {
    const int64_t c = std::min<int64_t>(mc, m - q0);
    FPP_TRY(search_chunk(ix, ix->ws, Q, q0, c, pl, nullptr, nullptr, 0, kProbesOnly, nullptr));
    FPP_CUDA(cudaMemcpy(out + q0 * nt * probes, ix->ws.probes.p, (size_t)c * nt * probes * 4,
                        cudaMemcpyDefault));
  }
  return FPP_OK;
}

fpp_status fpp_debug_candidates(const fpp_index* cix, const float* Q, int64_t m, int32_t probes,
                                int64_t* cand_off, uint32_t* cand) {
  g_err.clear();
  fpp_search_opts o;
  fpp_default_search_opts(&o);
  o.probes = probes;
  o.k = 1;
  SearchPlan pl{};
  int64_t dummy_i = 0;
  float dummy_s = 0;
  FPP_TRY(validate_search(cix, Q, m, &o, &dummy_i, &dummy_s, pl));
  if (!cand_off) { set_error("cand_off is NULL"); return FPP_EINVAL; }
  fpp_index* ix = const_cast<fpp_index*>(cix);
  std::lock_guard<std::mutex> lock(ix->mu);
  cand_off[0] = 0;
  if (m == 0) return FPP_OK;
  const int nt = pl.te - pl.tb;
  const int64_t mc = std::min<int64_t>(chunk_rows(ix, nt, pl.pmax), m);
  FPP_TRY(prepare_workspace(ix, ix->ws, pl, mc, false, 0));
  FPP_TRY(ix->ws.order_after_last(0));
  std::vector<uint64_t> eoff;
  std::vector<uint32_t> ucount, buf;
  for (int64_t q0 = 0; q0 < m; q0 += mc) {
    const int64_t c = std::min<int64_t>(mc, m - q0);
    FPP_TRY(search_chunk(ix, ix->ws, Q, q0, c, pl, nullptr, nullptr, 0, kCandidatesOnly, nullptr));
    eoff.resize(c);
    ucount.resize(c);
    uint64_t total = 0;   // slots handed out to the batch's regions
    FPP_CUDA(cudaMemcpy(eoff.data(), ix->ws.eoff.p, c * 8, cudaMemcpyDeviceToHost));
    FPP_CUDA(cudaMemcpy(ucount.data(), ix->ws.ecount.as<uint32_t>() + c, c * 4,
                        cudaMemcpyDeviceToHost));
    FPP_CUDA(cudaMemcpy(&total, ix->ws.stats.as<unsigned long long>() + 12, 8,
                        cudaMemcpyDeviceToHost));
    if (cand) {
      buf.resize(total);
      if (total)
        FPP_CUDA(cudaMemcpy(buf.data(), ix->ws.cand.p, total * 4, cudaMemcpyDeviceToHost));
    }
    for (int64_t i = 0; i < c; ++i) {
      const int64_t g = q0 + i;
      cand_off[g + 1] = cand_off[g] + ucount[i];
      if (cand) {
        uint32_t* dst = cand + cand_off[g];
        std::copy(buf.begin() + eoff[i], buf.begin() + eoff[i] + ucount[i], dst);
        std::sort(dst, dst + ucount[i]);
      }
    }
  }
  return FPP_OK;
}

fpp_status fpp_debug_projections(const fpp_index* cix, const float* Q, int64_t m, int32_t table_begin,
                                 int32_t table_end, float* out) {
  g_err.clear();
  fpp_search_opts o;
  fpp_default_search_opts(&o);
  o.table_begin = table_begin;
  o.table_end = table_end;
  SearchPlan pl{};
  int64_t dummy_i = 0;
  float dummy_s = 0;
  FPP_TRY(validate_search(cix, Q, m, &o, &dummy_i, &dummy_s, pl));
  if (!out && m) { set_error("out is NULL"); return FPP_EINVAL; }
  fpp_index* ix = const_cast<fpp_index*>(cix);
  std::lock_guard<std::mutex> lock(ix->mu);
  if (m == 0) return FPP_OK;
  const int nt = pl.te - pl.tb;
  const int64_t N = 2ll * nt * ix->D;
  const int64_t ldp = round_up(N, 4);
  const int64_t mc = std::min<int64_t>(chunk_rows(ix, nt, pl.pmax, false), m);
  FPP_TRY(prepare_workspace(ix, ix->ws, pl, mc, false, 0, false));
  FPP_TRY(ix->ws.order_after_last(0));
  FPP_CUDA(cudaMemset(ix->ws.stats.p, 0, 16 * 8));
  for (int64_t q0 = 0; q0 < m; q0 += mc) {
    const int64_t c = std::min<int64_t>(mc, m - q0);
    FPP_CUDA(cudaMemcpy2D(ix->ws.qpad.p, ix->dpad * 4, Q + q0 * ix->d, ix->d * 4, ix->d * 4, c,
                          cudaMemcpyDefault));
    FPP_TRY(project_rows(ix, ix->ws.qpad.as<float>(), c, ix->ws.qsplit, pl.tb, nt,
                         ix->ws.proj.as<float>(), ldp,
                         reinterpret_cast<int*>(ix->ws.stats.as<unsigned long long>() + 9), 0,
                         nullptr, 0, g_wait_test_cycles.load(), g_wait_test_withhold.load(),
                         ix->qpieces));
    FPP_CUDA(cudaMemcpy2D(out + q0 * N, N * 4, ix->ws.proj.p, ldp * 4, N * 4, c, cudaMemcpyDefault));
  }
  unsigned long long flag = 0;
  FPP_CUDA(cudaMemcpy(&flag, ix->ws.stats.as<unsigned long long>() + 9, 8, cudaMemcpyDeviceToHost));
  if (flag) {
    set_error("projection: a bounded wait ran out (code " + std::to_string(flag & 0xFFFFFFFFull) + ")");
    return FPP_ETIMEOUT;
  }
  return FPP_OK;
}

fpp_status fpp_debug_wait_test(int32_t withhold, int64_t wait_cycles) {
  g_err.clear();
  if (withhold < 0 || withhold > 1 || wait_cycles < 0) {
    set_error("withhold must be 0 or 1 and wait_cycles >= 0");
    return FPP_EINVAL;
  }
  g_wait_test_withhold.store(withhold);
  g_wait_test_cycles.store(wait_cycles);
  return FPP_OK;
}

fpp_status fpp_projection_error_bound(const fpp_index* ix, double* factor) {
  g_err.clear();
  if (!ix || !factor) { set_error("NULL argument"); return FPP_EINVAL; }
  *factor = ix->qgamma;
  return FPP_OK;
}

fpp_status fpp_bruteforce(const float* X, int64_t n, int32_t d, const float* Q, int64_t m, int32_t k,
                          int64_t* ids, float* scores, void* stream) {
  g_err.clear();
  if (!X || n < 1 || n >= (1ll << 32) || d < 1 || m < 0 || k < 1 || k > 256 ||
      (m > 0 && (!Q || !ids || !scores))) {
    set_error("fpp_bruteforce: bad arguments");
    return FPP_EINVAL;
  }
  if (m == 0) return FPP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int dpad = (int)round_up(d, 4);
  float* dX = nullptr;
  float* dQ = nullptr;
  DevBuf S, oi, os, misc, xm;
  auto done = [&](fpp_status s) {
    cudaStreamSynchronize(st);
    cudaFree(dX); cudaFree(dQ);
    S.release(); oi.release(); os.release(); misc.release(); xm.release();
    return s;
  };
  fpp_status s;
  if ((s = to_device_padded(X, n, d, dpad, &dX, st, nullptr)) != FPP_OK) return done(s);
  if ((s = to_device_padded(Q, m, d, dpad, &dQ, st, nullptr)) != FPP_OK) return done(s);
  if ((s = xm.ensure(4)) != FPP_OK) return done(s);
  if ((s = launch_row_norm_max(dX, n, dpad, d, xm.as<float>(), st)) != FPP_OK) return done(s);
  float xmax = 0.f;
  if (cudaMemcpyAsync(&xmax, xm.p, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("bruteforce: norm");
    return done(FPP_ECUDA);
  }
  const int64_t lds = round_up(n, 4);
  int64_t mc = std::max<int64_t>(1, std::min<int64_t>(m, (1ll << 28) / lds));
  if ((s = S.ensure((size_t)mc * lds * 4)) != FPP_OK) return done(s);
  if ((s = oi.ensure((size_t)mc * k * 8)) != FPP_OK) return done(s);
  if ((s = os.ensure((size_t)mc * k * 4)) != FPP_OK) return done(s);
  if ((s = misc.ensure(16, true, st)) != FPP_OK) return done(s);
  const double gamma = gamma_fp32(dpad);
  for (int64_t q0 = 0; q0 < m; q0 += mc) {
    const int64_t c = std::min<int64_t>(mc, m - q0);
    if ((s = gemm_f32_nt(dQ + q0 * dpad, dpad, dX, dpad, S.as<float>(), lds, c, n, dpad, st)) != FPP_OK)
      return done(s);
    if ((s = launch_topk_dense(S.as<float>(), lds, c, n, k, dQ + q0 * dpad, dpad, dX, dpad, d, xmax,
                               gamma, oi.as<int64_t>(), os.as<float>(), k,
                               misc.as<unsigned long long>(), st)) != FPP_OK)
      return done(s);
    if (cudaMemcpyAsync(ids + q0 * k, oi.p, c * k * 8, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(scores + q0 * k, os.p, c * k * 4, cudaMemcpyDefault, st) != cudaSuccess) {
      set_error("bruteforce: copy out");
      return done(FPP_ECUDA);
    }
  }
  unsigned long long hm[2] = {0, 0};
  if (cudaMemcpyAsync(hm, misc.p, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error(std::string("bruteforce: ") + cudaGetErrorString(cudaGetLastError()));
    return done(FPP_ECUDA);
  }
  if (hm[1]) {
    set_error("bruteforce: top-k re-check capacity exceeded");
    return done(FPP_EINTERNAL);
  }
  return done(FPP_OK);
}


fpp_status fpp_autotune(fpp_index* ix, const float* Q, int64_t m, int32_t k, int32_t probes,
                        fpp_tune_report* report) {
  g_err.clear();
  fpp_search_opts o;
  fpp_default_search_opts(&o);
  o.k = k;
  o.probes = probes;
  o.k_max = k;
  SearchPlan pl{};
  int64_t dummy_i = 0;
  float dummy_s = 0;
  FPP_TRY(validate_search(ix, Q, m, &o, &dummy_i, &dummy_s, pl));
  if (m < 1) { set_error("fpp_autotune needs at least one query"); return FPP_EINVAL; }
  std::lock_guard<std::mutex> lock(ix->mu);
  const int nt = pl.te - pl.tb;
  const int64_t mc = std::min<int64_t>(chunk_rows(ix, nt, pl.pmax), m);
  Workspace& ws = ix->ws;
  FPP_TRY(prepare_workspace(ix, ws, pl, mc, true, 0));
  FPP_TRY(ws.order_after_last(0));
  // one batch through the whole path leaves its candidates in the workspace
  FPP_CUDA(cudaMemsetAsync(ws.stats.p, 0, 16 * 8, 0));
  FPP_TRY(search_chunk(ix, ws, Q, 0, mc, pl, ws.out_ids.as<int64_t>(), ws.out_scores.as<float>(), 0,
                       kFull, nullptr));
  FPP_CUDA(cudaDeviceSynchronize());
  ScoreArgs sa{};
  sa.items = ws.score_items;
  sa.nitems = reinterpret_cast<unsigned*>(ws.stats.as<unsigned long long>() + 10);
  sa.eoff = ws.eoff.as<uint64_t>(); sa.mq = mc;
  sa.cand = ws.cand.as<uint32_t>();
  sa.X = ix->X; sa.ldx = ix->dpad; sa.Q = ws.qpad.as<float>(); sa.ldq = ix->dpad;
  sa.Xb = ix->Xb; sa.ldxb = ix->ldxb;
  sa.Xq = ix->Xq; sa.ldxq = ix->ldxq; sa.xscale = ix->xscale;
  sa.scores = ws.cscores.as<float>();
  cudaEvent_t e0, e1;
  FPP_CUDA(cudaEventCreate(&e0));
  FPP_CUDA(cudaEventCreate(&e1));
  auto time_shape = [&](int g, int waves, float* ms) -> fpp_status {
    sa.tune_g = g;
    sa.tune_waves = waves;
    float best = 1e30f;
    for (int r = 0; r < 4; ++r) {   // the first run warms up, the best of the rest counts
      FPP_CUDA(cudaEventRecord(e0, 0));
      FPP_TRY(launch_score(sa, ix->sm_count, 0));
      FPP_CUDA(cudaEventRecord(e1, 0));
      FPP_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      FPP_CUDA(cudaEventElapsedTime(&t, e0, e1));
      if (r > 0) best = std::min(best, t);
    }
    *ms = best;
    return FPP_OK;
  };
  fpp_tune_report rep{};
  fpp_status st = time_shape(0, 0, &rep.ms_default);
  int best_g = 0, best_w = 0;
  float best_ms = rep.ms_default;
  const int chunks = ix->precision == FPP_BF16      ? (int)(ix->ldxb / 8)
                     : ix->precision == FPP_FP8E4M3 ? (int)(ix->ldxq / 16)
                                                    : ix->dpad / 4;
  for (int g = 1; g <= 32 && st == FPP_OK; g <<= 1) {
    if (g * 8 < chunks || g > 2 * chunks) continue;   // shapes the kernels instantiate well
    for (int w : {1, 2, 3, 4, 6, 8}) {
      float ms = 0.f;
      if ((st = time_shape(g, w, &ms)) != FPP_OK) break;
      ++rep.shapes_tried;
      if (ms < best_ms * 0.98f) { best_ms = ms; best_g = g; best_w = w; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FPP_OK) return st;
  ix->tune_score_g = best_g;
  ix->tune_score_waves = best_w;
  rep.score_lanes = best_g;
  rep.score_waves = best_w;
  rep.ms_best = best_ms;
  if (report) *report = rep;
  return FPP_OK;
}

fpp_status fpp_merge_topk(const int64_t* ids, const float* scores, int32_t parts, int64_t m,
                          int32_t k, int64_t* out_ids, float* out_scores) {
  g_err.clear();
  if (!ids || !scores || !out_ids || !out_scores || parts < 1 || m < 0 || k < 1) {
    set_error("fpp_merge_topk: bad arguments");
    return FPP_EINVAL;
  }
  std::vector<std::pair<float, int64_t>> e;
  e.reserve((size_t)parts * k);
  for (int64_t q = 0; q < m; ++q) {
    e.clear();
    for (int p = 0; p < parts; ++p) {
      const size_t row = ((size_t)p * m + q) * k;
      for (int j = 0; j < k; ++j)
        if (ids[row + j] >= 0) e.emplace_back(scores[row + j], ids[row + j]);
    }
    std::sort(e.begin(), e.end(), [](const std::pair<float, int64_t>& x,
                                     const std::pair<float, int64_t>& y) {
      return x.first > y.first || (x.first == y.first && x.second < y.second);
    });
    int n = 0;
    for (size_t i = 0; i < e.size() && n < k; ++i) {
      bool dup = false;
      for (int j = 0; j < n && !dup; ++j) dup = out_ids[q * k + j] == e[i].second;
      if (dup) continue;
      out_ids[q * k + n] = e[i].second;
      out_scores[q * k + n] = e[i].first;
      ++n;
    }
    for (; n < k; ++n) {
      out_ids[q * k + n] = -1;
      out_scores[q * k + n] = -INFINITY;
    }
  }
  return FPP_OK;
}

void fpp_default_server_cfg(fpp_server_cfg* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->max_batch = 4096;
  c->slots = 2;
  c->k_max = 100;
  c->probes_max = 16;
  c->max_queue = 1 << 16;
  c->candidate_budget_bytes = 256ull << 20;
}

fpp_status fpp_server_create(const fpp_index* ix, const fpp_server_cfg* cfg, fpp_server** out) {
  g_err.clear();
  try {
    return server_create_impl(ix, cfg, out);
  } catch (const std::exception& e) {
    set_error(std::string("fpp_server_create: ") + e.what());
    return FPP_EINTERNAL;
  }
}

fpp_status fpp_server_submit_many(fpp_server* s, const float* q, int32_t nreq, const int32_t* nq,
                                  const int32_t* k, const int32_t* probes, uint64_t* req_ids) {
  g_err.clear();
  if (!s || !q || !nq || !k || !probes || !req_ids || nreq < 0) {
    set_error("NULL argument or nreq < 0");
    return FPP_EINVAL;
  }
  // copy every request first, then queue them under one lock with one
  // wake-up, so that a free slot sees the whole group at once
  std::vector<std::unique_ptr<ServerRequest>> rs;
  fpp_status st = FPP_OK;
  int32_t bad = nreq;
  try {
    int64_t row = 0;
    const bool dev = is_device_ptr(q);
    for (int32_t r = 0; r < nreq; ++r) {
      if (nq[r] < 1 || nq[r] > s->cfg.max_batch || k[r] < 1 || k[r] > s->cfg.k_max ||
          probes[r] < 1 || probes[r] > s->cfg.probes_max) {
        set_error("request " + std::to_string(r) + ": nq, k or probes out of range");
        st = FPP_EINVAL;
        bad = r;
        break;
      }
      auto x = std::make_unique<ServerRequest>();
      x->nq = nq[r];
      x->k = k[r];
      x->probes = probes[r];
      const size_t nel = (size_t)nq[r] * s->ix->d;
      x->q.resize(nel);
      const float* src = q + row * s->ix->d;
      if (dev) {
        if (cudaMemcpy(x->q.data(), src, nel * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
          set_error("copying the queries failed");
          st = FPP_ECUDA;
          bad = r;
          break;
        }
      } else {
        std::memcpy(x->q.data(), src, nel * 4);
      }
      x->ids.resize((size_t)nq[r] * k[r]);
      x->scores.resize((size_t)nq[r] * k[r]);
      rs.push_back(std::move(x));
      row += nq[r];
    }
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    st = FPP_ENOMEM;
    bad = (int32_t)rs.size();
  }
  {
    std::lock_guard<std::mutex> lock(s->mu);
    const auto now = std::chrono::steady_clock::now();
    for (size_t r = 0; r < rs.size(); ++r) {
      if (s->stop || (int64_t)s->queue.size() >= s->cfg.max_queue) {
        set_error(s->stop ? "server is shutting down" : "queue full");
        st = FPP_EBUSY;
        bad = (int32_t)r;
        break;
      }
      ServerRequest* x = rs[r].get();
      x->t_submit = now;
      x->id = s->next_id++;
      req_ids[r] = x->id;
      s->queue.push_back(x);
      s->reqs.emplace(x->id, std::move(rs[r]));
      s->stats.submitted += 1;
    }
    s->stats.queued = s->queue.size();
  }
  for (int32_t x = bad; x < nreq; ++x) req_ids[x] = 0;
  s->cv_work.notify_all();
  return st;
}

fpp_status fpp_server_submit(fpp_server* s, const float* q, int32_t nq, int32_t k, int32_t probes,
                             uint64_t* req_id) {
  g_err.clear();
  if (!s || !q || !req_id) { set_error("NULL argument"); return FPP_EINVAL; }
  if (nq < 1 || nq > s->cfg.max_batch) { set_error("nq must be in [1, max_batch]"); return FPP_EINVAL; }
  if (k < 1 || k > s->cfg.k_max) { set_error("k must be in [1, k_max]"); return FPP_EINVAL; }
  if (probes < 1 || probes > s->cfg.probes_max) {
    set_error("probes must be in [1, probes_max]");
    return FPP_EINVAL;
  }
  try {
    auto r = std::make_unique<ServerRequest>();
    r->nq = nq;
    r->k = k;
    r->probes = probes;
    const size_t nel = (size_t)nq * s->ix->d;
    r->q.resize(nel);
    if (is_device_ptr(q)) {
      if (cudaMemcpy(r->q.data(), q, nel * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("copying the queries failed");
        return FPP_ECUDA;
      }
    } else {
      std::memcpy(r->q.data(), q, nel * 4);
    }
    r->ids.resize((size_t)nq * k);
    r->scores.resize((size_t)nq * k);
    r->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->stop) { set_error("server is shutting down"); return FPP_EBUSY; }
    if ((int64_t)s->queue.size() >= s->cfg.max_queue) {
      set_error("queue full");
      return FPP_EBUSY;
    }
    r->id = s->next_id++;
    *req_id = r->id;
    s->queue.push_back(r.get());
    s->reqs.emplace(r->id, std::move(r));
    s->stats.submitted += 1;
    s->stats.queued = s->queue.size();
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return FPP_ENOMEM;
  }
  s->cv_work.notify_one();
  return FPP_OK;
}

fpp_status fpp_server_poll(fpp_server* s, uint64_t req_id, int64_t* ids, float* scores,
                           int32_t timeout_us, float* latency_ms) {
  g_err.clear();
  if (!s) { set_error("server is NULL"); return FPP_EINVAL; }
  std::unique_ptr<ServerRequest> r;
  {
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) { set_error("unknown request id"); return FPP_EINVAL; }
    ServerRequest* rp = it->second.get();
    auto done = [&] { return rp->state == 2; };
    if (timeout_us < 0) s->cv_done.wait(lock, done);
    else if (!s->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), done)) {
      set_error("request not complete yet");
      return FPP_ETIMEOUT;
    }
    r = std::move(it->second);
    s->reqs.erase(it);
  }
  if (latency_ms)
    *latency_ms = std::chrono::duration<float, std::milli>(r->t_done - r->t_submit).count();
  if (r->status != FPP_OK) {
    set_error(r->error);
    return r->status;
  }
  const size_t ni = r->ids.size();
  if (ids && cudaMemcpy(ids, r->ids.data(), ni * 8, cudaMemcpyDefault) != cudaSuccess) {
    set_error("copying ids failed");
    return FPP_ECUDA;
  }
  if (scores && cudaMemcpy(scores, r->scores.data(), ni * 4, cudaMemcpyDefault) != cudaSuccess) {
    set_error("copying scores failed");
    return FPP_ECUDA;
  }
  return FPP_OK;
}

fpp_status fpp_server_get_stats(fpp_server* s, fpp_server_stats* out) {
  g_err.clear();
  if (!s || !out) { set_error("NULL argument"); return FPP_EINVAL; }
  std::lock_guard<std::mutex> lock(s->mu);
  *out = s->stats;
  return FPP_OK;
}

void fpp_server_destroy(fpp_server* s) {
  if (!s) return;
  server_release(s);
  delete s;
}
}  // extern "C"
