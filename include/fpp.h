/*
 * fpp.h -- C ABI of libfpp, a GB300 (sm_103a) implementation of the
 * Falconn++ search path (Pham & Liu, "Falconn++: A Locality-sensitive
 * Filtering Approach for Approximate Nearest Neighbor Search", NeurIPS 2022).
 *
 * The method: L hash tables, each the concatenation of l = 2 cross-polytope
 * hashes over D Gaussian random vectors (Section 2.2, Eq. 1), so a table has
 * 4D^2 buckets.  Each bucket keeps only the fraction alpha of its points with
 * the largest projection magnitude, the locality-sensitive filter (Section
 * 3.4).  A query probes the P highest-ranked buckets of every table, ranked by
 * projection value (Section 3.4, "Multi-probing for querying"), takes the
 * union of their kept points, scores them by exact inner product and returns
 * the top-k (the problem statement of Section 1: top-k by x^T q on the unit
 * sphere).
 *
 * Conventions shared by every call:
 *  - Every call returns fpp_status; no exception or abort crosses the ABI.
 *    On failure fpp_last_error() returns a message owned by the library and
 *    valid until the calling thread's next libfpp call.
 *  - Matrices are row-major, FP32, with rows of exactly d elements.
 *  - A pointer argument may point to host memory (pageable or pinned) or to
 *    device memory of the current CUDA device; the library detects which
 *    with cudaPointerGetAttributes and copies as needed.  Device pointers
 *    must be 4-byte aligned.
 *  - Results are complete when the call returns, except when the caller
 *    passes a non-NULL stream in fpp_search_opts, no stats, and both result
 *    pointers are device memory or page-locked (pinned) host memory: then
 *    the results are complete once that stream has reached the call's point
 *    (the call itself does not synchronise, and device-side error flags are
 *    not reported).
 *  - Page-locked host queries Q with a non-NULL stream are uploaded on an
 *    internal copy stream into one of two device query tiles used in turn,
 *    so that a call's upload overlaps the previous call's search.  That
 *    upload is not ordered after earlier work on the caller's stream: the
 *    contents of Q must be final when the call is made and must not change
 *    until the call's results are complete.  Other host inputs are copied on
 *    the caller's stream.
 *  - An fpp_index is immutable after fpp_build.  Concurrent searches on one
 *    index from several host threads are serialised by a per-index lock.
 *  - With precision FPP_FP32, decisions (bucket ids, probe sets, candidate
 *    sets, top-k ids) equal those of an exact FP64 evaluation of the method
 *    except where an FP64 margin below 1e-6 makes two answers equally valid;
 *    returned scores are FP64-accurate inner products rounded to FP32.  With
 *    FPP_BF16 the top-k ids may differ where a BF16 rounding error exceeds
 *    the statistical window described at fpp_precision or a true top-k
 *    candidate falls outside the shortlist; returned scores are still
 *    FP64-accurate.
 */
#ifndef FPP_H_
#define FPP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fpp_status {
  FPP_OK = 0,
  FPP_EINVAL = 1,    /* an argument is out of range or a pointer is NULL */
  FPP_ENOMEM = 2,    /* device or host allocation failed */
  FPP_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  FPP_ETIMEOUT = 4,  /* a bounded device wait ran out */
  FPP_EBUSY = 5,     /* resource in use (serving slots, admission) */
  FPP_EINTERNAL = 6  /* a device-side consistency check failed */
} fpp_status;

typedef enum fpp_precision {
  FPP_FP32 = 0,      /* FP32 storage and projections, FP64-exact decisions */
  FPP_BF16 = 1,      /* Candidate scores are read from a BF16 copy of X
                        (FP32 accumulation); the best max(rerank_k, k + 16)
                        of them form the shortlist, and every shortlisted
                        candidate within twice the BF16 error window
                        (nine estimated standard deviations of the rounding
                        error, score_error_factor) of the k-th is re-scored
                        exactly on the FP32 rows before the final top-k
                        (when the window spans the whole shortlist, the
                        shortlist is re-ranked and nothing beyond it).
                        Hashing and probing are as for FPP_FP32.  The index
                        holds X in both precisions (6 bytes per element).
                        Graded by recall and score error. */
  FPP_FP8E4M3 = 2    /* As FPP_BF16 (but a window reaching past the
                        shortlist re-scores every candidate inside it) with
                        candidate rows stored in FP8 e4m3
                        (one byte per element) times a per-row FP32 scale
                        (the row's largest magnitude / 448); the window is
                        nine estimated standard deviations of the e4m3
                        rounding error (unit roundoff 2^-4).  5 bytes per
                        element with the FP32 rows.  Graded by recall and
                        score error. */
} fpp_precision;

/* Index parameters.  Initialise with fpp_default_params(). */
typedef struct fpp_params {
  int32_t L;           /* hash tables, >= 1 (Section 2.1: L tables)          */
  int32_t D;           /* random vectors per hash, 1..1024 (Section 2.2)     */
  int32_t iprobes;     /* indexing probes per point, >= 1 (Algorithm 1)      */
  int32_t kappa;       /* limit scaling floor, 0 = off (Section 3.4)         */
  double alpha;        /* kept fraction per bucket, 0 < alpha <= 1 (3.4)     */
  uint64_t seed;       /* seed of the rotation generator (fpp_rotations)     */
  const float* R;      /* optional explicit random vectors [L][2][D][d],
                          host or device; NULL = generate from seed. Copied. */
  int32_t precision;   /* fpp_precision                                      */
  int32_t rerank_k;    /* FPP_BF16: shortlist length (default 100), 0..256  */
  void* stream;        /* cudaStream_t for the build, or NULL (legacy)       */
  int32_t center;      /* 1: build the tables over the centered points x - c
                          (Section 3.4, heuristic (1)); queries are not
                          centered and scores stay x^T q (default 0)        */
  int32_t simhash_bits; /* SimHash signature bits per point, 0 (none) or a
                          multiple of 256 up to min(1024, 2 L D): bit i is
                          [x^T r_i >= 0] for the i-th random vector in table
                          order (Section 4); needed by simhash_keep        */
  const float* center_vec; /* optional c [d] (host or device); NULL = the
                          FP64 column means of X rounded to FP32            */
  int32_t hash_precision; /* query projections of the search: FPP_FP32
                          (default) = the exact three-piece split, decisions
                          exact; FPP_BF16 = one BF16 product per projection
                          (queries rounded to BF16, FP32 accumulation), only
                          with precision FPP_BF16 or FPP_FP8E4M3 and without
                          simhash_bits.  Then each hash's argmax (the query's
                          own bucket) is re-decided exactly whenever its BF16
                          lead is inside a window of nine estimated standard
                          deviations of the rounding error (the factor
                          bf16_window of Section 2.2's projections, see
                          fpp_precision), and the other probes are ranked by
                          the BF16 values: graded by recall.  The index's
                          own hashing stays exact.                         */
} fpp_params;

/* Per-call search options.  Initialise with fpp_default_search_opts(). */
typedef struct fpp_search_opts {
  int32_t k;                  /* results per query when k_per_query is NULL  */
  int32_t probes;             /* probes per table when probes_per_query is NULL */
  const int32_t* k_per_query; /* optional [m] (host or device), each 1..k_max */
  const int32_t* probes_per_query; /* optional [m], each 1..min(4D^2, 128)   */
  int32_t k_max;              /* row stride of ids/scores; >= every k         */
  int32_t table_begin;        /* search tables [table_begin, table_end)     */
  int32_t table_end;          /* 0 or L = all tables                          */
  int32_t flags;              /* FPP_SEARCH_* bits                            */
  void* stream;               /* cudaStream_t or NULL                         */
  int32_t global_probes;      /* > 0: probe this many buckets per query over
                                 all tables together (qProbes, Sections 2.2
                                 and 4): the best (table, bucket) pairs by
                                 pair score over all 4D^2 buckets of every
                                 table (ties: lower table, lower bucket).
                                 Each table offers its best
                                 min(global_probes, 128, 4D^2) buckets; a
                                 query that would take more than 128 from one
                                 table makes the call return FPP_EINVAL (the
                                 outputs are then not the uncapped selection).
                                 Such a call always waits for its results and
                                 never runs as a graph.  probes and
                                 probes_per_query are then unused
                                 (probes_per_query must be NULL).  0: probes
                                 per table.                                   */
  int32_t simhash_keep;       /* > 0: score only the simhash_keep candidates
                                 whose signatures differ least from the
                                 query's (ties: lower id), 1..512; needs an
                                 index built with simhash_bits (Section 4).
                                 An approximation: graded by recall.  0: off */
  int32_t score_range_rows;   /* candidate scoring groups each query's ids by
                                 row range so that the rows of one range are
                                 read by the whole GPU at once and stay in L2.
                                 0: ranges of 32,768 rows, more when 256
                                 ranges do not cover the index (none when all
                                 rows fit one range); > 0: at
                                 least this many rows per range (rounded up to
                                 a power of two, at most 256 ranges).  Results
                                 do not depend on it.                          */
  int32_t reserved0;
} fpp_search_opts;

/* FPP_SEARCH_GRAPH: run the call as one CUDA graph, captured on the first
 * call and replayed by later calls with the same Q, ids, scores, per-query
 * arrays, k, probes, k_max, table range and stream (the data they point to
 * may change between calls).  Taken only when stream is non-NULL, Q, ids,
 * scores and the per-query arrays are device memory and stats is NULL;
 * otherwise the call runs normally.  When the candidate buffers can hold the
 * batch's worst case (L x probes x the largest kept bucket per query) within
 * the candidate budget (fpp_set_candidate_budget), the call returns without
 * waiting: results are complete once the stream reaches the call's point.
 * Otherwise the graph is optimistic: the buffers are provisioned up to the
 * budget, every query's candidate region is checked against them on the
 * device, and the call waits for the check; if some region did not fit, the
 * call is repeated without the graph (sized from the exact totals) and
 * fpp_index_info.graph_fallbacks counts it.  Error flags raised inside the
 * graph are not reported. */
#define FPP_SEARCH_GRAPH 1

/* FPP_SEARCH_PIPELINE: consecutive calls on one index overlap on the
 * device.  The index alternates two workspaces on two internal streams: a
 * call starts once the caller's stream reaches it (its inputs must be final
 * there) and the call before last has ended, so one call's projections run
 * while the previous call gathers and scores.  Taken only with a non-NULL
 * stream, NULL stats, no global_probes, device or page-locked host Q and
 * outputs, and device per-query arrays; otherwise the call runs normally.
 * A pipelined call's results are complete once the caller's stream reaches
 * the next pipelined call on the index, or after fpp_search_flush(ix,
 * stream); device-side error flags are not reported.  The index holds a
 * second workspace while pipelining. */
#define FPP_SEARCH_PIPELINE 2

/* Counters of one search call (summed over queries). */
typedef struct fpp_search_stats {
  uint64_t queries;
  uint64_t probes;            /* buckets probed                               */
  uint64_t entries;           /* bucket entries scanned, with duplicates      */
  uint64_t unique;            /* candidates scored: distinct ids, except for
                                 queries with more than 16,384 bucket entries,
                                 whose entries are scored without
                                 de-duplication (repeats dropped at top-k)    */
  uint64_t probe_rechecks;    /* (query, table) probe sets re-decided in
                                 FP64-accurate arithmetic                     */
  uint64_t topk_rechecks;     /* queries whose top-k boundary was re-decided  */
  uint64_t batches;           /* query batches the call was split into (each
                                 batch is one launch of every search kernel)  */
  uint64_t probe_full_rechecks; /* of the probe_rechecks, those re-decided from
                                 all 2D projections of the table (the window
                                 passes could not settle them)                 */
  float ms_project;           /* device time per phase, milliseconds          */
  float ms_probe;             /* fast probe ranking                            */
  float ms_probe_exact;       /* exact re-decision of near-tie probe sets      */
  float ms_gather_score;      /* candidate gather, scoring and top-k, of which: */
  float ms_dedup;             /*   bucket walk and hash-set de-duplication     */
  float ms_score;             /*   candidate scoring                            */
  float ms_topk;              /*   per-query top-k                              */
  float ms_total;
} fpp_search_stats;

typedef struct fpp_index_info {
  int64_t n;
  int32_t d, L, D, iprobes, kappa, precision;
  double alpha;
  uint64_t kept_total;        /* ids stored over all tables                   */
  uint32_t max_bucket_kept;   /* largest kept bucket                          */
  uint64_t device_bytes;      /* device memory held by the index              */
  float build_ms;             /* wall time of fpp_build                        */
  int32_t rerank_k;           /* FPP_BF16 shortlist length (0 for FPP_FP32)    */
  int32_t center;             /* 1: the tables hash the centered points        */
  int32_t simhash_bits;       /* SimHash signature bits per point (0: none)    */
  int32_t r_pieces;           /* BF16 pieces of R in the projection: 1 when
                                 every coordinate of R is a BF16 value (the
                                 seeded generator's), else 3                  */
  double score_error_factor;  /* c: a candidate's first-pass score is within
                                 c ||q|| ||x|| of x^T q (FPP_FP32: the FP32
                                 bound gamma_d; FPP_BF16: the statistical
                                 window of BF16 rows) before exact re-scoring */
  int32_t q_pieces;           /* BF16 pieces of the search's query
                                 projections: 3 (exact split) or 1
                                 (hash_precision FPP_BF16)                    */
  uint32_t graph_fallbacks;   /* FPP_SEARCH_GRAPH calls whose optimistic
                                 graph found a candidate region past the
                                 buffer and were repeated without the graph  */
} fpp_index_info;

typedef struct fpp_index fpp_index;

void fpp_default_params(fpp_params* p);
void fpp_default_search_opts(fpp_search_opts* o);

/* Builds the index over X [n][d] (Section 3.4 and Algorithm 1): generates or
 * copies the random vectors, hashes every point into one bucket per table
 * (iprobes buckets with multi-probe indexing), keeps in each bucket of size
 * B the min(B, max(kappa, ceil(alpha * B / iprobes))) points with the
 * largest filter score |x^T r_i1| + |x^T r_i2| (ties: lower point id), and
 * stores each table as CSR.  X is copied; the caller keeps ownership.
 * Errors: FPP_EINVAL for n < 1, d < 1, L < 1, D outside 1..1024,
 * alpha outside (0, 1], iprobes outside 1..min(4D^2, 16), kappa < 0,
 * n >= 2^32, precision not
 * an fpp_precision, rerank_k outside 0..256 with FPP_BF16.
 * *out is set only on success; release it with fpp_free. */
fpp_status fpp_build(const float* X, int64_t n, int32_t d, const fpp_params* p,
                     fpp_index** out);

/* Searches m queries Q [m][d] (the Falconn++ query, Section 3.4): projects
 * each query onto every table's random vectors (Section 2.2), takes the
 * cross-polytope hash of each of its two hashes (Eq. 1), probes the `probes`
 * buckets of every table with the highest pair score v1(h1) + v2(h2)
 * (Section 3.4, multi-probing: the first is the query's own bucket), takes
 * the union of their kept points, scores it by exact inner product and
 * returns the top-k (the problem of Section 1: top-k by x^T q).
 * Writes ids [m][k] (int64, -1 padding) and scores [m][k] (FP32, -inf
 * padding), best first (score desc, id asc).  Q, ids and scores are
 * caller-owned, host or device memory.  probes = buckets probed per table,
 * 1..min(4D^2, 128); k = 1..256.  m = 0 is a no-op.  Errors: FPP_EINVAL
 * for a NULL pointer or an argument out of range, FPP_ENOMEM, FPP_ECUDA,
 * FPP_ETIMEOUT (a bounded device wait ran out), FPP_EINTERNAL. */
fpp_status fpp_search(const fpp_index* ix, const float* Q, int64_t m, int32_t k,
                      int32_t probes, int64_t* ids, float* scores);

/* fpp_search (Section 3.4's query) with per-query k and probe budgets, a
 * table range (the slice a table-sharded rank searches), the global probe
 * budget qProbes over all tables (Sections 2.2 and 4), SimHash pre-ranking
 * of the candidates (Section 4), a stream and counters.  ids/scores have row
 * stride opts->k_max; entries past a query's own k are set to -1 / -inf.
 * stats may be NULL.  Same errors as fpp_search, plus FPP_EINVAL for a
 * global budget that a table's 128 offered buckets cannot serve. */
fpp_status fpp_search_ex(const fpp_index* ix, const float* Q, int64_t m,
                         const fpp_search_opts* opts, int64_t* ids,
                         float* scores, fpp_search_stats* stats);

/* Makes `stream` wait for every pipelined call of the index (see
 * FPP_SEARCH_PIPELINE): their results are complete once the stream reaches
 * this point.  A no-op when none is pending.  Errors: FPP_EINVAL for a NULL
 * index, FPP_ECUDA. */
fpp_status fpp_search_flush(const fpp_index* ix, void* stream);

/* Releases the index and its device memory.  NULL is allowed. */
void fpp_free(fpp_index* ix);

/* Message of the calling thread's last failed call ("" if none). */
const char* fpp_last_error(void);

/* Host-only: the canonical random vectors R[L][2][D][d] for a seed.  Stream
 * 2t+j (table t, hash j) is SplitMix64 (Steele, Lea, Flood 2014) started at
 * seed XOR 0x9E3779B97F4A7C15*(2t+j+1); coordinate (i, c) is the
 * Box-Muller value sqrt(-2 ln u1) cos(2 pi u2) of the stream's outputs
 * 2(i d + c) and 2(i d + c)+1, u1 = (top53 + 1) / 2^53, u2 = top53 / 2^53,
 * rounded to FP32 and then to the nearest BF16 value (ties to even).  The
 * paper fixes only that each coordinate is N(0, 1) (Section 2.2); with R on
 * the BF16 grid the projections take three tensor-core products instead of
 * six (any FP32 R passed in params->R still works, at the six-product cost).
 * R is host memory of L*2*D*d floats owned by the caller.  Needs no GPU. */
fpp_status fpp_rotations(uint64_t seed, int32_t L, int32_t D, int32_t d, float* R);

/* Host-only: kept count of a bucket of size B (Section 3.4, Algorithm 1):
 * min(B, max(kappa, ceil((alpha * B) / iprobes))) in IEEE FP64. */
uint64_t fpp_keep_count(uint64_t B, double alpha, int32_t iprobes, int32_t kappa);

fpp_status fpp_index_get_info(const fpp_index* ix, fpp_index_info* info);

/* Introspection for parity tests (all outputs host or device memory):
 * fpp_debug_point_buckets: bucket ids of every point in table t before
 *   filtering, [n][iprobes]: for iprobes = 1 the point's hash bucket
 *   h1 * 2D + h2 (h = i for +r_i, i + D for -r_i, Eq. 1); for iprobes > 1
 *   its iprobes best buckets in rank order (Algorithm 1).
 * fpp_debug_table: kept CSR of table t: offsets [4D^2 + 1] (relative to the
 *   table) and ids [kept_t], ids ordered by filter score desc, id asc inside
 *   a bucket.  Pass ids = NULL to get only offsets (kept_t = offsets[4D^2]).
 * fpp_debug_probes: probed bucket ids [m][L'][probes] in rank order for the
 *   tables of opts (L' = table_end - table_begin).  probes <= 128.
 * fpp_debug_candidates: the de-duplicated candidate set of every query (the
 *   union of the kept ids of its probed buckets over all tables, Section
 *   3.4), ascending per query, host memory: cand_off [m + 1] (cand_off[0] =
 *   0) and cand [cand_off[m]].  Pass cand = NULL to get only cand_off, then
 *   call again with a buffer of cand_off[m] entries.  */
fpp_status fpp_debug_point_buckets(const fpp_index* ix, int32_t t, uint32_t* out);
fpp_status fpp_debug_table(const fpp_index* ix, int32_t t, uint32_t* offsets,
                           uint32_t* ids);
fpp_status fpp_debug_probes(const fpp_index* ix, const float* Q, int64_t m,
                            int32_t probes, int32_t table_begin, int32_t table_end,
                            uint32_t* out);
fpp_status fpp_debug_candidates(const fpp_index* ix, const float* Q, int64_t m,
                                int32_t probes, int64_t* cand_off, uint32_t* cand);

/* fpp_debug_projections: the projections q^T r [m][2 L' D] of the queries
 *   onto the random vectors of tables [table_begin, table_end) (0, 0 = all),
 *   column (2 t' + j) D + i for table t' of the range, hash j, vector i, as
 *   the search computes them (tensor cores, exact three-piece BF16 split).
 * fpp_projection_error_bound: the factor c such that every such projection
 *   is within c ||q|| ||r_i|| of the exact inner product; the search's
 *   decisions rely on it (Section 2.2's projections, evaluated in pieces).
 *   With hash_precision FPP_BF16 the projections are one BF16 product and c
 *   is the statistical window of their argmax decisions (not a bound). */
fpp_status fpp_debug_projections(const fpp_index* ix, const float* Q, int64_t m,
                                 int32_t table_begin, int32_t table_end, float* out);

/* Test hook of the bounded device waits (the paper has no counterpart).
 * Every wait inside the projection kernel gives up after a limit (about 2 s
 * by default): the CTA raises an error code, lets the copies and tensor-core
 * operations it issued complete, frees its tensor memory and exits, and the
 * call returns FPP_ETIMEOUT with the context still usable.  This setting
 * applies to later fpp_debug_projections calls only (never to builds or
 * searches): wait_cycles > 0 replaces the limit (in SM clock cycles; 0 = the
 * default) and withhold = 1 makes the first CTA skip the loads of its first
 * K chunk, so that its tensor-core warp's wait for them runs out.  Reset
 * with (0, 0).  Errors: FPP_EINVAL for withhold not 0 or 1, or a negative
 * wait_cycles. */
fpp_status fpp_debug_wait_test(int32_t withhold, int64_t wait_cycles);
fpp_status fpp_projection_error_bound(const fpp_index* ix, double* factor);

/* Exact search: top-k of every query over all of X by inner product
 * (ground truth for recall).  Same output conventions as fpp_search.
 * stream may be NULL. */
fpp_status fpp_bruteforce(const float* X, int64_t n, int32_t d, const float* Q,
                          int64_t m, int32_t k, int64_t* ids, float* scores,
                          void* stream);

/* Exact search that allocates nothing.  The paper has no counterpart: this
 * is for callers that cannot allocate device memory when they search, for
 * example because their framework has already reserved the whole GPU for its
 * own allocator (so cudaMalloc fails), or because the implicit device
 * synchronisation of cudaMalloc and cudaFree is too costly on their path.
 * It computes the same result as fpp_bruteforce with the same kernels, but
 * its scratch is a file-scope device array of FPP_STATIC_SCRATCH_BYTES that
 * every GPU which loads libfpp holds until the process exits.
 *  - X [n][d], Q [m][d], ids [m][k], scores [m][k] must all be device memory
 *    of the current device; d must be a multiple of 4 and X, Q 16-byte
 *    aligned; 4 * round_up(n, 4) + 256 bytes must fit the array (n up to
 *    8,388,544), else FPP_EINVAL with a message.  1 <= k <= 256.
 *  - The first call on a device looks up the array's device address for that
 *    device (cudaGetSymbolAddress, with the device current); make that first
 *    call before any stream capture.
 *  - All calls share the one array and each call clears what must start at
 *    zero.  Calls that overlap on the GPU (several host threads or streams)
 *    race on the array and must be serialised by the caller.
 *  - The call synchronises the stream before it returns; results are then
 *    complete.  It calls no cudaMalloc, cudaFree or allocating library
 *    routine. */
#define FPP_STATIC_SCRATCH_BYTES (32ull << 20)
fpp_status fpp_bruteforce_static(const float* X, int64_t n, int32_t d, const float* Q,
                                 int64_t m, int32_t k, int64_t* ids, float* scores,
                                 void* stream);

/* Autotuner: runs the search once on Q [m][d] (host or device) with k and
 * probes, then times the candidate-scoring kernel on the candidates of that
 * batch under each launch shape it supports (lanes per candidate row x CTAs
 * per resident slot) and keeps the fastest for every later search on this
 * index (and on servers over it).  The results of searches do not depend on
 * the shape.  report may be NULL.  Errors as fpp_search_ex. */
typedef struct fpp_tune_report {
  int32_t score_lanes;        /* lanes per candidate row chosen               */
  int32_t score_waves;        /* CTAs per resident slot chosen                */
  float ms_default;           /* scoring time with the built-in choice        */
  float ms_best;              /* scoring time with the chosen shape           */
  int32_t shapes_tried;
  int32_t reserved0;
} fpp_tune_report;
fpp_status fpp_autotune(fpp_index* ix, const float* Q, int64_t m, int32_t k, int32_t probes,
                        fpp_tune_report* report);

/* ------------------------------------------------------------ serving
 *
 * A server answers a stream of independent search requests on one index with
 * continuous batching.  It runs `slots` worker threads, each with its own
 * CUDA stream, device workspace and pinned staging buffers; a worker that
 * becomes free takes the oldest queued requests (FIFO) while the batch holds
 * at most max_batch queries and its estimated candidate-buffer memory (bucket
 * entries of the probed buckets, 8 bytes each, estimated from the entries per
 * probe seen so far) stays within candidate_budget_bytes, then runs the whole
 * search on that batch with per-query k and probe budgets.  A request's
 * results are those fpp_search_ex returns for its queries alone (nothing
 * depends on the rest of the batch).  The index must outlive the server and
 * must not be freed while it runs; fpp_search on the same index may run
 * concurrently (it uses the index's own workspace). */
typedef struct fpp_server fpp_server;

typedef struct fpp_server_cfg {
  int32_t max_batch;          /* queries per batch, 1..65536 (default 4096)    */
  int32_t slots;              /* batches in flight, 1..16 (default 2)          */
  int32_t k_max;              /* largest k of a request, 1..256 (default 100)  */
  int32_t probes_max;         /* largest probe budget (default 16)             */
  int32_t max_queue;          /* queued requests before submit returns
                                 FPP_EBUSY (default 65536)                    */
  int32_t reserved0;
  uint64_t candidate_budget_bytes; /* per slot, >= 1 MiB (default 256 MiB)    */
} fpp_server_cfg;

typedef struct fpp_server_stats {
  uint64_t submitted, completed, failed;  /* requests                        */
  uint64_t queued;                        /* requests waiting now            */
  uint64_t batches, queries;              /* batches run, queries in them    */
  uint64_t entries, probes;               /* bucket entries scanned, buckets */
  uint64_t splits;                        /* batches halved because their
                                             candidates did not fit a slot  */
  uint64_t serving_allocs;                /* device allocations made while
                                             running batches (always 0)     */
} fpp_server_stats;

void fpp_default_server_cfg(fpp_server_cfg* cfg);

/* Starts the worker threads and allocates every slot's workspace for
 * max_batch queries, probes_max probes and k_max results up front, with a
 * candidate buffer of candidate_budget_bytes / 8 entries per slot; running
 * batches allocates no device memory.  A free slot takes the oldest queued
 * requests while the batch stays within max_batch queries and within the
 * buffer by a running estimate of the entries per probed bucket; the exact
 * entry count of the batch, taken after its probes are ranked, decides: a
 * batch that does not fit is halved by queries (again if needed) and each
 * part is searched in turn.  Errors: FPP_EINVAL for a field out of range or
 * a buffer that cannot hold one query's worst case (8 L probes_max
 * max_bucket_kept bytes); FPP_ENOMEM. */
fpp_status fpp_server_create(const fpp_index* ix, const fpp_server_cfg* cfg,
                             fpp_server** out);

/* Queues nq queries q [nq][d] (host or device memory; copied before the call
 * returns) with k results and `probes` probes per table each.  *req_id
 * identifies the request for fpp_server_poll.  Errors: FPP_EINVAL for nq
 * outside 1..max_batch, k outside 1..k_max, probes outside 1..probes_max;
 * FPP_EBUSY when max_queue requests are already waiting. */
fpp_status fpp_server_submit(fpp_server* s, const float* q, int32_t nq, int32_t k,
                             int32_t probes, uint64_t* req_id);

/* Queues nreq requests in one call, as nreq fpp_server_submit calls would:
 * request r has nq[r] consecutive query rows of q (host or device memory;
 * the rows of the requests follow each other), k[r] results and probes[r]
 * probes per table; req_ids [nreq] receives their ids.  On an error the
 * requests before the failing one stay queued, the failing one and the rest
 * get id 0, and the status is that of fpp_server_submit. */
fpp_status fpp_server_submit_many(fpp_server* s, const float* q, int32_t nreq,
                                  const int32_t* nq, const int32_t* k, const int32_t* probes,
                                  uint64_t* req_ids);

/* Waits up to timeout_us microseconds (< 0: without limit, 0: no wait) for
 * request req_id.  When it is complete, writes ids [nq][k] and scores
 * [nq][k] (host or device memory; either may be NULL), the time from submit
 * to completion in *latency_ms (may be NULL), forgets the request and
 * returns its status.  FPP_ETIMEOUT: not complete yet (poll again);
 * FPP_EINVAL: unknown id. */
fpp_status fpp_server_poll(fpp_server* s, uint64_t req_id, int64_t* ids, float* scores,
                           int32_t timeout_us, float* latency_ms);

fpp_status fpp_server_get_stats(fpp_server* s, fpp_server_stats* out);

/* Stops the workers after their current batches and frees the server;
 * requests still queued are dropped.  NULL-safe. */
void fpp_server_destroy(fpp_server* s);

/* Table-sharded search (one index per GPU over a slice of the tables, built
 * from the same seed, searched with fpp_search_ex's table range): merges the
 * parts' top-k lists of every query into the global top-k.  ids, scores:
 * host memory [parts][m][k] (rows padded with -1 / -inf); out_ids,
 * out_scores: host memory [m][k].  Entries are ordered by (score desc, id
 * asc); an id in several parts is kept once.  The exact top-k over the union
 * of the tables' candidates is contained in the union of the parts' top-k
 * lists, so this equals the unsharded search.  Host code only (parts x k
 * entries per query); no device needed.  Errors: FPP_EINVAL for NULL
 * pointers, parts < 1, m < 0, k < 1. */
fpp_status fpp_merge_topk(const int64_t* ids, const float* scores, int32_t parts, int64_t m,
                          int32_t k, int64_t* out_ids, float* out_scores);

/* Candidate buffer a search call may provision from the worst-case bound
 * without reading the exact entry count back (and the size of an optimistic
 * graph's buffers), in bytes: 8 per candidate slot.  Default min(8 GiB,
 * device memory / 16).  Errors: FPP_EINVAL for a NULL index or bytes below
 * 4,096. */
fpp_status fpp_set_candidate_budget(fpp_index* ix, uint64_t bytes);

/* Number of kernels this process has launched through libfpp. */
uint64_t fpp_launch_count(void);
/* Number of device allocations (cudaMalloc) libfpp has made in this process. */
uint64_t fpp_alloc_count(void);

#ifdef __cplusplus
}
#endif
#endif /* FPP_H_ */
