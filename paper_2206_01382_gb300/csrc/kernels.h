// Internal launchers of libfpp (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fpp.h"

namespace fpp {

// One bucket entry of a table during the build: sorted by (sk asc, key asc,
// id asc) where key = ~bits(filter score) so that ascending key order is
// descending filter score.  sk = table-in-chunk * 4D^2 + bucket.
struct __align__(16) Rec {
  uint64_t key;
  uint32_t sk;
  uint32_t id;
};

// Projection GEMM (gemm_f32.cu).
fpp_status gemm_f32_nt(const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                       int64_t ldc, int64_t M, int64_t N, int K, cudaStream_t st);

// Tensor-core projection GEMM (gemm_tc.cu).  Operands are BF16 piece
// arrays [rows][pieces * Kp] made by split_to_bf16; C is FP32 [M][ldc].
int tc_kpad(int d);
double tc_error_bound_factor(int Kp, int pieces);
// Near-tie window (relative to ||a|| ||b||) of dot products with BF16 rows.
double bf16_window_factor(int d);
// Near-tie window (relative to ||a|| ||b||) of dot products with rows in FP8
// e4m3 times a per-row scale.
double fp8_window_factor(int d);
// FP32 rows [rows][lds] (d used) -> e4m3 rows [rows][ldo] (zero padded) and
// per-row scales (largest magnitude / 448, 1 for a zero row).
fpp_status rows_to_fp8(const float* src, int64_t rows, int64_t lds, int d, int64_t ldo, void* dst,
                       float* scale, cudaStream_t st);
// FP32 rows [rows][lds] (d used) -> BF16 rows [rows][ldo], zero padded.
fpp_status rows_to_bf16(const float* src, int64_t rows, int64_t lds, int d, int64_t ldo, void* dst,
                        cudaStream_t st);
fpp_status split_to_bf16(const float* src, int64_t rows, int64_t lds, int d, int pieces,
                         void* dst, cudaStream_t st);
fpp_status gemm_tc(const void* A, int64_t M, const void* B, int64_t N, int Kp, int pieces,
                   float* C, int64_t ldc, int* err, cudaStream_t st);
// Projection with the per-(row, hash) top-EL list epilogue (EL in {2, 4, 8};
// D must divide 256); EL = 0 stores the projections like gemm_tc.
int tc_list_len(int want);
// Relative bound t of the list values' truncation: |p|' <= |p| < |p|' (1 + t).
float tc_list_trunc(int D);
// bpieces = 1: every element of B is a BF16 value (its mid and lo pieces are
// zero), three products per K block instead of six; else bpieces = pieces.
// wait_cycles > 0 replaces the default limit (about 2 s) of every bounded
// wait; withhold = 1 makes CTA 0 skip its first chunk's loads (a test of the
// bounded waits: the launch then reports a run-out wait in *err).
fpp_status project_tc(const void* A, int64_t M, const void* B, int64_t N, int Kp, int pieces,
                      int bpieces, int D, int EL, float* C, int64_t ldc, uint64_t* lists, int* err,
                      cudaStream_t st, long long wait_cycles = 0, int withhold = 0,
                      int b_row_pieces = 0);

// Build (build_kernels.cu).
struct HashArgs {
  const float* P;        // projections [rows][ldp] for tables [t0, t0 + nt), or NULL
  int64_t ldp;
  const uint64_t* lists; // [rows][2 nt][EL + 1] per-hash top-EL keys + cut when P is NULL
  int EL;
  float trunc;           // list values: |p|' <= |p| < |p|' (1 + trunc) (tc_list_trunc)
  int64_t rows;          // points in this chunk
  int64_t row0;          // id of the chunk's first point
  int t0, nt, D;
  const float* X;        // [n][ldx] padded points
  int64_t ldx;
  const float* R;        // [2 L D][ldr] padded random vectors
  int64_t ldr;
  int d;                 // true dimension (padded columns are zero)
  const float* rmax;     // [2L] max row norm per (table, hash), inflated
  float xmax;            // max point norm, inflated
  double gamma;          // error factor of the projection
  float eps_xf;          // gamma * xmax, rounded up to FP32 with margin
  int64_t n;             // points in the index (record stride per table)
  Rec* rec;              // [nt][n] records, or NULL
  uint32_t* counts;      // [nt][4D^2] bucket sizes, or NULL
  uint32_t* point_bucket;// [rows] (nt must be 1), or NULL
  unsigned long long* rechecks;  // counter of FP64-accurate re-decisions, or NULL
};
fpp_status launch_build_hash(const HashArgs& a, cudaStream_t st);

// SimHash signature bits (Section 4): bit i of row r is [v_r^T r_i >= 0]
// for the first 32 W random vectors, from the FP32 projections P [rows][ldp]
// where |p| exceeds eps_r = gamma ||v_r|| rsig_max, else from a compensated
// dot product.  out: [rows][W] uint32, little-endian bits.
struct SignArgs {
  const float* P;
  int64_t ldp, rows;
  int words;
  const float* V;            // [rows][ldv] padded vectors
  int64_t ldv;
  const float* vnorm;        // [rows] norm upper bounds
  const float* R;            // signature vectors [32 W][ldr]
  int64_t ldr;
  double gamma;
  float rsig_max;
  uint32_t* out;
};
fpp_status launch_sign_bits(const SignArgs& a, cudaStream_t st);

// Multi-probe indexing (Algorithm 1, iProbes > 1): the records of the
// iProbes buckets each point was ranked into (probe kernels run on the
// points), with the exact pair score v1(h1) + v2(h2) as filter score.
struct PairArgs {
  const uint32_t* probes;    // [rows][nt][iprobes] bucket ids in rank order
  int iprobes;
  int64_t rows, row0;
  int t0, nt, D;
  const float* X;            // [n][ldx] padded points
  int64_t ldx;
  const float* R;            // [2 L D][ldr]
  int64_t ldr;
  int64_t n;
  Rec* rec;                  // [nt][n * iprobes]
  uint32_t* counts;          // [nt][4D^2]
};
fpp_status launch_pair_records(const PairArgs& a, cudaStream_t st);

fpp_status launch_row_norm_max(const float* X, int64_t n, int64_t ldx, int d, float* out,
                               cudaStream_t st);
// Centering: c [d] = FP32 rounding of the FP64 column means of X; Xc = fl(X - c).
fpp_status launch_column_means(const float* X, int64_t n, int64_t ldx, int d, float* c,
                               cudaStream_t st);
fpp_status launch_center_rows(const float* X, int64_t n, int64_t ldx, const float* c, float* Xc,
                              cudaStream_t st);

// Exclusive scan of n values into out[0..n] (out[n] = total).  mode 0: the
// values are in[i]; mode 1: the values are keep_count(in[i]).
struct KeepRule {
  double alpha;
  int iprobes;
  int kappa;
};
fpp_status exclusive_scan_u32(const uint32_t* in, int64_t n, uint64_t* out, int mode,
                              KeepRule rule, uint64_t* scratch, cudaStream_t st);
int64_t scan_scratch_elems(int64_t n);

// Stable LSD radix sort of records by (sk, key) with 8-bit digits;
// key_bits / sk_bits give the number of significant low bits of each field.
fpp_status radix_sort_recs(Rec* a, Rec* b, int64_t n, int key_bits, int sk_bits,
                           uint32_t* hist, int64_t hist_elems, uint64_t* scan_buf,
                           uint64_t* scan_scratch, Rec** sorted, cudaStream_t st);
int64_t radix_hist_elems(int64_t n);

// Kept-CSR compaction: records sorted by (sk, key, id); bstart = exclusive
// scan of counts, kstart = exclusive scan of keep counts (both [nsk + 1]).
fpp_status launch_compact(const Rec* sorted, int64_t nrec, const uint64_t* bstart,
                          const uint64_t* kstart, const uint32_t* counts, KeepRule rule,
                          uint32_t* ids_out, cudaStream_t st);
fpp_status launch_make_offsets(const uint64_t* kstart, int nt, int64_t NB, uint32_t* offsets,
                               cudaStream_t st);

// Search (search_kernels.cu).
struct ProbeArgs {
  const float* P;            // [mq][ldp] query projections for tables [tb, te), or NULL
  int64_t ldp;
  const uint64_t* lists;     // [mq][2 nt][EL + 1] per-hash top-EL keys and cut (P NULL)
  int EL;
  float trunc;               // list values: |p|' <= |p| < |p|' (1 + trunc) (tc_list_trunc)
  int64_t mq;
  const float* Q;            // [mq][ldq] padded queries
  int64_t ldq;
  const float* qnorm;        // [mq] upper bounds of the query norms
  const float* R;            // [2 L D][ldr]
  int64_t ldr;
  const uint16_t* Rb;        // R as BF16 bits, row stride ldrb (R on the BF16 grid), or NULL
  int64_t ldrb;
  int d, D, tb, nt;
  const float* rmax;         // [2L]
  double gamma;
  float gammaf;              // gamma, rounded up to FP32 with margin
  const int32_t* probes_pq;  // [mq] or NULL
  int probes;                // scalar probes / max over queries (row stride of out)
  uint32_t* out;             // [mq][nt][probes] bucket ids
  uint32_t* recheck;         // [mq * nt] (query, table) items for the exact pass
  unsigned* recheck_count;   // device counter of recheck items
  uint32_t* recheck2;        // [mq * nt] items the window pass could not settle
  unsigned* recheck2_count;
  float* recheck_s;          // [mq * nt][4] the FP32 P-th and (P+1)-th pair scores of each
                             // recheck item and its two hashes' largest abs(p) (stored
                             // projections; 16-byte aligned), or NULL
  unsigned long long* rechecks;  // statistics counter or NULL
  unsigned long long* full_rechecks;  // items of the full pass (statistics) or NULL
  uint32_t* amax_pairs;      // argmax pass, list mode: the uncertain (item, hash) pairs
  unsigned* amax_count;      //   [2 mq nt] and their device counter
  int argmax_only;            // 1 (one-piece BF16 query projections): only each hash's
                             // argmax must be certain; the other probes take the FP32
                             // ranking of the BF16 values
  unsigned long long* gcap_flag;  // global budget: queries whose per-table cap may have
                                  // bound (some table gave all its `probes` slots), or NULL
};
fpp_status launch_probe(const ProbeArgs& a, cudaStream_t st, cudaEvent_t exact_begin = nullptr);

// Global probe budget: out of the probe kernels' per-table top-P lists
// (a.out, P = a.probes), keeps the Qp best (table, bucket) pairs of every
// query by pair score (ties: lower table, lower bucket) and marks the rest
// of each table's slots empty (PROBE_EMPTY).  Exact: a boundary inside the
// error bound is re-decided from compensated projections.  The selection
// equals the uncapped one over all 4D^2 buckets of every table unless some
// table had all of its P offered pairs selected while P < min(Qp, 4D^2);
// such queries are counted in a.gcap_flag.
constexpr uint32_t PROBE_EMPTY = 0xFFFFFFFFu;
fpp_status launch_global_probes(const ProbeArgs& a, int Qp, cudaStream_t st);
fpp_status launch_query_norms(const float* Q, int64_t m, int64_t ldq, int d, float* out,
                              cudaStream_t st);

// Candidate gather / de-duplication / scoring / top-k (search_kernels.cu).
// Bounds of the FPP_DEBUG_BOUNDS build's device checks (kernels.h users
// fill it in both builds; only that build reads it): *flag receives the
// first violation as (site << 48) | index, and the access is skipped.
struct Bounds {
  unsigned long long* flag = nullptr;
  int64_t n = 0;             // points: every candidate id is below n
  uint64_t kept = 0;         // kept ids of all tables (the ids array)
  uint64_t cap = 0;          // candidate slots of the workspace
  int64_t nb = 0;            // buckets per table
};

struct ScoreItem {
  uint32_t q;        // query in the batch
  uint32_t len;      // candidates in this item
  uint64_t start;    // first candidate slot
};

struct DedupArgs {
  const uint32_t* probes;    // [mq][nt][pstride] probed bucket ids
  int pstride;
  int64_t mq;
  int tb, nt, D;
  const int32_t* probes_pq;  // [mq] or NULL (then pstride probes each)
  const uint32_t* offsets;   // [L][4D^2 + 1]
  const uint64_t* table_base;// [L]
  const uint32_t* ids;       // kept ids
  uint32_t* ecount;          // [mq] bucket entries per query (count_entries, or the
                             // fused small tier)
  uint64_t* eoff;            // [mq] start of each query's region (regions are not in
                             // query order)
  unsigned long long* region_total;  // slots handed out (zeroed before count_entries)
  uint32_t* cand;            // candidate ids, query q at eoff[q] ..
  uint32_t* ucount;          // [mq] distinct candidates per query
  ScoreItem* items;          // score work items, appended (any order)
  unsigned* nitems;          // items appended (zeroed before count_entries)
  uint32_t* tierq;           // [2][mq] queries listed by count_entries for the 32,768-slot
                             // tier and for the no-de-duplication tier
  unsigned* tiern;           // [2] their counts (zeroed before count_entries)
  int no_items;              // 1: leave the items to the SimHash filter
  int fused;                 // 1: no count_entries pass; the small tier counts each
                             // query's entries, lists the larger ones in tierq, and
                             // every tier reserves its queries' regions itself
  uint64_t cap;              // candidate slots: under fused, a query whose reserved
                             // region would end past cap gets no candidates and
                             // sets *overflow (the caller then repeats the call)
  unsigned long long* overflow;
  int range_shift;           // range_count > 1: each query's ids are grouped by row
  int range_count;           // range (id >> range_shift), one or more items per range
  unsigned long long* stats; // entries, unique, -, probes
  Bounds bd;
};

// SimHash pre-ranking: for every query with more than keep candidates,
// the keep with the fewest differing signature bits (ties: lower id) are
// moved to the front of its region and become its candidates; then the
// score work items of every query are appended (the de-duplication kernels
// skip that step when this runs).
struct SimArgs {
  int64_t mq;
  const uint64_t* eoff;
  uint32_t* cand;
  uint32_t* ucount;
  const uint32_t* xsig;      // [n][W]
  const uint32_t* qsig;      // [mq][W]
  int words, keep, cap;
  ScoreItem* items;
  unsigned* nitems;
};
fpp_status launch_simhash_filter(const SimArgs& a, cudaStream_t st);

struct ScoreArgs {
  const ScoreItem* items;    // [*nitems] work items
  const unsigned* nitems;
  const uint64_t* eoff;
  int64_t mq;
  const uint32_t* cand;
  const float* X;            // [n][ldx]
  int64_t ldx;
  const float* Q;            // [mq][ldq] (ldq == ldx)
  int64_t ldq;
  const void* Xb;            // BF16 rows [n][ldxb] (precision path) or NULL
  int64_t ldxb;
  const uint8_t* Xq;         // FP8 e4m3 rows [n][ldxq] or NULL
  int64_t ldxq;
  const float* xscale;       // [n] scales of the FP8 rows
  float* scores;             // FP32 scores, parallel to cand
  int tune_g;                // lanes per row (power of two) or 0: heuristic
  int tune_waves;            // CTAs per resident slot or 0: default
  Bounds bd;
};

struct TopkArgs {
  int64_t mq;
  const uint64_t* eoff;
  const uint32_t* ucount;
  const uint32_t* cand;
  const float* scores;
  const float* X;            // [n][ldx] for the compensated re-scoring
  int64_t ldx;
  const float* Q;            // [mq][ldq]
  int64_t ldq;
  int d;
  const float* qnorm;        // [mq]
  float xmax;
  double gamma;              // FP32 score error factor gamma_d
  float gammaf;              // gamma rounded up to FP32 with margin
  const int32_t* k_pq;       // [mq] or NULL
  int k, kmax, cap, rcap;
  int kprime;                // shortlist re-scored exactly (>= k + 16)
  int approx;                // 0 exact; 1 BF16 (the pre-selection is re-ranked, no slow
                             // path); 2 FP8 (slow-list overflow is not an error)
  void* slow;                // [ceil(mq / 8) * 8][topk_slow_cap()] 16-byte entries
  int* err;
  unsigned long long* stats; // stats[2] counts slow-path queries
  int64_t* out_ids;          // [mq][kmax]
  float* out_scores;
  Bounds bd;
};

int score_item_len();
// Work-item slots for cand_total candidates of mq queries whose ids are
// grouped into at most `ranges` row ranges.
int64_t score_item_slots(uint64_t entries_total, int64_t mq, int ranges);
constexpr int SCORE_RANGE_MAX = 256;   // row ranges of the grouped scoring
int topk_cap(int kprime);
int topk_rcap(int kprime);
int topk_slow_cap();
fpp_status launch_count_entries(const DedupArgs& a, cudaStream_t st);
// Orders the score work items by the row range of their first candidate
// (counting sort; hist and cursor are [range_count] zeroed counters), so that
// the CTAs scoring at the same time read rows of one range, which stays in L2.
fpp_status launch_order_items(const ScoreItem* in, const unsigned* nitems, const uint32_t* cand,
                              int range_shift, int range_count, unsigned* hist, unsigned* cursor,
                              ScoreItem* out, cudaStream_t st);
fpp_status launch_dedup(const DedupArgs& a, cudaStream_t st);
fpp_status launch_score(const ScoreArgs& a, int sm_count, cudaStream_t st);
fpp_status launch_topk(const TopkArgs& a, cudaStream_t st);

// Brute force top-k over a dense score matrix S [mq][lds] (n columns).
fpp_status launch_topk_dense(const float* S, int64_t lds, int64_t mq, int64_t n, int k,
                             const float* Q, int64_t ldq, const float* X, int64_t ldx, int d,
                             float qxmax, double gamma, int64_t* out_ids, float* out_scores,
                             int kmax, unsigned long long* rechecks, cudaStream_t st);

}  // namespace fpp
