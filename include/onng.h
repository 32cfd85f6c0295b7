/*
 * onng — GB300 (sm_103a) library for degree- and path-adjusted k-nearest-neighbour
 * graph search, after Iwasaki & Miyazaki, "Optimization of Indexing Based on
 * k-Nearest Neighbor Graph for Proximity Search in High-dimensional Data"
 * (arXiv 1810.07355).
 *
 * Conventions shared by every entry point:
 *  - All array pointers are DEVICE pointers owned by the caller.  The library
 *    never frees them and keeps no reference to them after the call returns.
 *    Float arrays must be 16-byte aligned (they are read with 16-byte loads).
 *  - Matrices are row-major.  Vectors X [n, d] and queries Q [nq, d] are float32
 *    with d a multiple of 4 (ONNG_E_UNSUPPORTED otherwise).
 *  - Graphs are CSR: row_ptr [n+1] int64, col [nnz] int32, len [nnz] float32,
 *    every row ordered by (length, id) ascending.  Lengths are Euclidean.
 *  - `ws` / `ws_bytes` is caller-owned device scratch; each call that needs it
 *    has a *_workspace_bytes query.  Too small a workspace gives ONNG_E_WORKSPACE.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) unless the comment says the call synchronises.
 *  - Every call returns an onng_status; on failure onng_last_error() gives a
 *    message (thread-local, valid until the next call on that thread).
 *    Per-query soft failures are flags in the search stats, not call failures.
 */
#ifndef ONNG_H
#define ONNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *onng_stream_t; /* = cudaStream_t */

enum onng_status {
    ONNG_OK = 0,
    ONNG_E_INVAL = 1,       /* bad argument (negative size, k > n - 1, NULL pointer ...) */
    ONNG_E_WORKSPACE = 2,   /* ws_bytes smaller than the *_workspace_bytes query */
    ONNG_E_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    ONNG_E_LIMIT = 4,       /* an iteration cap or a time limit was reached */
    ONNG_E_UNSUPPORTED = 5, /* shape outside what the kernels handle (d % 4, k > 128 ...) */
    ONNG_E_AGAIN = 6        /* onng_serve_poll: not done within timeout_ms (poll again) */
};

/* per-query flags, stats[q*4 + 3] */
#define ONNG_FLAG_S_OVERFLOW 1u      /* candidate spill pool full: candidates dropped (see pool_cap) */
#define ONNG_FLAG_VISIT_OVERFLOW 2u  /* reserved (the visited set cannot overflow) */
#define ONNG_FLAG_LIMIT 4u           /* stopped by max_expansions with an in-bound candidate left */
#define ONNG_FLAG_CHECK 8u           /* bounds-checked builds (-DONNG_CHECK, float32 search only): a graph
                                        id outside [0, n), a row outside col or an overwritten shared-memory
                                        canary was met; the access was skipped */

const char *onng_last_error(void);
int onng_version(void);

/* ------------------------------------------------------------------ kNN graph
 * Exact k nearest neighbours (the exact graph stands in for the approximate
 * kNN graph the paper derives from an ANNG, Sec. 2.6 / Algorithm ConstructGraph).
 *
 * onng_knn: for every query row r < nq, the k base points of X [n, d] nearest to
 * Q[r], as ids nbr [nq, k] int32 and Euclidean lengths len [nq, k] float32,
 * ordered by (length, id).  If self_offset >= 0, query row r is base point
 * self_offset + r and that id is excluded (a duplicate point with another id is
 * still a neighbour).  k <= 256.  Rows with fewer than k candidates are padded
 * with -1 / +inf.  Three sweeps over the base: byte-valued inputs (integers
 * 0-255) at d = 64 / 128 on the tensor cores, ranked exactly (the lists are
 * written as ranked); other non-integer inputs at d >= 32 on the tensor cores
 * with both sets centred on the base mean and split into bfloat16 hi + lo (dot
 * products to about 2^-16 |q| |x|), and the rest by a float32 SIMT sweep
 * (integer-valued inputs with squared norms below 2^23 exactly); these two rank
 * the expanded form |q|^2 + |x|^2 - 2 q.x, keep KC >= k + 16 survivors per row and
 * rescore them by direct difference in float32.  Inputs must be finite.
 *
 * onng_build_knng(X, n, d, k, ...) == onng_knn(X, n, d, X, n, k, 0, ...).
 */
size_t onng_knn_workspace_bytes(int64_t n, int32_t d, int64_t nq, int32_t k);
int onng_knn(const float *X, int64_t n, int32_t d, const float *Q, int64_t nq, int32_t k,
             int64_t self_offset, int32_t *nbr, float *len, void *ws, size_t ws_bytes,
             onng_stream_t stream);
int onng_build_knng(const float *X, int64_t n, int32_t d, int32_t k, int32_t *nbr, float *len,
                    void *ws, size_t ws_bytes, onng_stream_t stream);

/* ---------------------------------------------------- static degree adjustment
 * Algorithm 2 (ConstructAdjustedGraph), set form: the adjusted list of node o is
 *   first_{e_o}(N_k(o))  united with  { x : o in first_{e_i}(N_k(x)) },
 * the loop bound of Algorithm 2 read as p <= max(e_o, e_i).  A reversed edge
 * x->o carries the length stored for o->x; a forward edge keeps its own length
 * when both directions exist.  Rows are ordered by (length, id).
 * Input: the kNN lists nbr / len [n, k] of onng_build_knng.
 *
 * onng_adjust_degree_count writes the exact row_ptr [n+1] of the result and,
 * if nnz_host != NULL, synchronises `stream` and stores the edge count there.
 * onng_adjust_degree then fills col / len_out [nnz] using that row_ptr.
 */
size_t onng_adjust_degree_workspace_bytes(int64_t n, int32_t k);
int onng_adjust_degree_count(const int32_t *nbr, const float *len, int64_t n, int32_t k,
                             int32_t e_o, int32_t e_i, int64_t *row_ptr, int64_t *nnz_host,
                             void *ws, size_t ws_bytes, onng_stream_t stream);
int onng_adjust_degree(const int32_t *nbr, const float *len, int64_t n, int32_t k, int32_t e_o,
                       int32_t e_i, const int64_t *row_ptr, int32_t *col, float *len_out,
                       void *ws, size_t ws_bytes, onng_stream_t stream);

/* --------------------------------------- degree adjustment with constraints
 * Algorithm 3 (ConstructAdjustedGraphWithConstraint, "SAC"), equal edge for
 * edge to its sequential greedy pass: G_t = Algorithm 2 with (0, e_i); nodes o in
 * increasing (|N(G_t, o)|, o) (ties by the smaller id), each taking the members
 * n of N(G_t, o) in increasing (length, id) and adding o->n when n has no
 * in-edge yet or (n has fewer than e_i in-edges and o fewer than e_o edges);
 * then every node with fewer than e_o edges takes its nearest kNN neighbours
 * not yet in its list.  An edge o->n of the first loop carries the stored
 * length of n->o.  Rows are ordered by (length, id).
 * The GPU evaluates the pass per edge: n meets only the nodes of its own first
 * e_i kNN entries, so the in-degree test never fails, and o->n is added exactly
 * when n is among o's first e_o members or o is the first node, in the order
 * above, to meet n.
 *
 * onng_adjust_degree_sac_count writes row_ptr [n+1] (and, if nnz_host != NULL,
 * synchronises and stores the edge count); onng_adjust_degree_sac then fills
 * col / len_out [nnz].  Input: the kNN lists nbr / len [n, k].
 */
size_t onng_adjust_degree_sac_workspace_bytes(int64_t n, int32_t k);
int onng_adjust_degree_sac_count(const int32_t *nbr, const float *len, int64_t n, int32_t k,
                                 int32_t e_o, int32_t e_i, int64_t *row_ptr, int64_t *nnz_host,
                                 void *ws, size_t ws_bytes, onng_stream_t stream);
int onng_adjust_degree_sac(const int32_t *nbr, const float *len, int64_t n, int32_t k, int32_t e_o,
                           int32_t e_i, const int64_t *row_ptr, int32_t *col, float *len_out,
                           void *ws, size_t ws_bytes, onng_stream_t stream);

/* ------------------------------------------------------------ path adjustment
 * Algorithms 4/5 (AdjustPath / HasPath) read order-free: edge (i, j) is dropped
 * when the INPUT graph has i->m and m->j with len(i,m) < len(i,j) and
 * len(m,j) < len(i,j) (stored float32 lengths, strict comparisons).  Kept edges
 * keep their order.  Outputs: row_ptr_out [n+1]; col_out / len_out need room for
 * the input edge count.  If nnz_host != NULL the call synchronises and stores
 * the kept edge count there.  removed_by (optional, [nnz_in] int32) receives, for
 * every input edge, the smallest-position witness m or -1.
 */
size_t onng_adjust_path_workspace_bytes(int64_t n, int64_t nnz);
int onng_adjust_path(const int64_t *row_ptr, const int32_t *col, const float *len, int64_t n,
                     int64_t *row_ptr_out, int32_t *col_out, float *len_out, int64_t *nnz_host,
                     int32_t *removed_by, void *ws, size_t ws_bytes, onng_stream_t stream);

/* Algorithm 4 (AdjustPath) taken literally, a variant beside the order-free rule
 * of onng_adjust_path: in round p every node s with more than p edges decides
 * its p-th input edge (s, t), nodes in ascending id, and keeps it unless
 * Algorithm 5 finds in the partial output a kept edge (s, m) and a kept edge
 * (m, t) with len(m, t) < len(s, t).  Kept edges keep their input order; the
 * result is one round-robin pass of the paper's listing, with node order inside
 * a round (which the paper leaves open) fixed to ascending ids.  Synchronises
 * `stream` once per round and pass (rounds = the largest degree).
 * Outputs as onng_adjust_path (row_ptr_out [n+1]; col_out / len_out sized for
 * the input edge count; nnz_host optional).  n < 2^31 - 2^23. */
size_t onng_adjust_path_literal_workspace_bytes(int64_t n, int64_t nnz);
int onng_adjust_path_literal(const int64_t *row_ptr, const int32_t *col, const float *len, int64_t n,
                             int64_t *row_ptr_out, int32_t *col_out, float *len_out, int64_t *nnz_host,
                             void *ws, size_t ws_bytes, onng_stream_t stream);

/* ------------------------------------------------------------ graph statistics
 * The graph statistics of Table 4 (Sec. 3.1), a diagnostic of a built graph
 * (not on the search path).  With m = ceil(n / 20) (5 % of the nodes, at least
 * one):
 *   mean_out    nnz / n
 *   top5_out    mean outdegree of the m nodes of largest outdegree
 *   bottom5_in  mean indegree of the m nodes of smallest indegree
 *   in_dist10   mean length over the edges of the transposed graph with every
 *               node's incoming list cut to its 10 shortest (NaN without edges)
 *   max_out, max_in, zero_in   largest outdegree and indegree, and the count of
 *               nodes no edge reaches (the 1-NNG indegrees of Sec. 3, Fig. 3(c))
 * row_ptr [n+1] must be a valid CSR (row_ptr[0] = 0, non-decreasing); col ids
 * outside [0, n) give ONNG_E_INVAL (after the kernels ran, ignoring them).
 * `out` is HOST memory; the call synchronises `stream`.  Degrees are counted as
 * 32-bit; the length sum is accumulated in double in no fixed order. */
typedef struct {
    int64_t n, nnz, max_out, max_in, zero_in;
    double mean_out, top5_out, bottom5_in, in_dist10;
} onng_graph_stats_t;
size_t onng_graph_stats_workspace_bytes(int64_t n, int64_t nnz);
int onng_graph_stats(const int64_t *row_ptr, const int32_t *col, const float *len, int64_t n,
                     onng_graph_stats_t *out, void *ws, size_t ws_bytes, onng_stream_t stream);

/* ------------------------------------------------------------------ index files
 * A built index written to disk and read back (the paper keeps its graphs as
 * NGT index files and quotes their memory in Table 7; the format is this
 * library's own).  Little-endian: a 64-byte header (magic "ONNGIDX\0", u32
 * version 1, u32 flags with bit 0 = lengths present, i64 n, i32 d, u32 CRC-32 of
 * the payload, i64 nnz, 24 zero bytes), then row_ptr [n+1] i64, col [nnz] i32,
 * len [nnz] f32 (when present) and X [n, d] f32.  The CRC is the reflected
 * CRC-32 of polynomial 0xEDB88320 (initial value and final xor 0xFFFFFFFF).
 *   onng_index_save: writes the device arrays (len may be NULL) to `path`,
 *                    replacing it; synchronises `stream`.
 *   onng_index_check: reads the header and checks the payload size and CRC
 *                    (host only, no CUDA call); optional outputs n, d, nnz and
 *                    has_len (0 / 1).
 *   onng_index_load: checks the file as onng_index_check does and that it holds
 *                    the given n, d and nnz (and lengths when len != NULL), and
 *                    only then copies it into the caller's device arrays;
 *                    synchronises `stream`.
 * A missing file, a wrong magic, version, size or CRC gives ONNG_E_INVAL with
 * the reason in onng_last_error().
 * onng_crc32: the CRC above over `len` bytes of host memory, continuing `crc`
 * (0 to start). */
int onng_index_save(const char *path, const int64_t *row_ptr, const int32_t *col, const float *len,
                    const float *X, int64_t n, int32_t d, onng_stream_t stream);
int onng_index_check(const char *path, int64_t *n, int32_t *d, int64_t *nnz, int32_t *has_len);
int onng_index_load(const char *path, int64_t n, int32_t d, int64_t nnz, int64_t *row_ptr, int32_t *col,
                    float *len, float *X, onng_stream_t stream);
uint32_t onng_crc32(uint32_t crc, const void *data, size_t len);

/* ---------------------------------------------------------------------- seeds
 * onng_seeds_random: the paper's random seeds (Sec. 3.2, Fig. 5(a)): n_seed
 * distinct ids per query, query q drawing from the SplitMix64 stream that
 * starts at state global_seed + q * 2^32; a draw z maps to floor(z * n / 2^64),
 * repeats are redrawn.  With m = min(n_seed, n): when 2 * m > n the seeds are
 * 0 .. m-1; entries past m are -1.  out [nq, n_seed].
 *
 * onng_seeds_pivot: the n_seed nearest (distance, id) of the P = min(n_pivot, n)
 * pivots floor(t * n / P); stands in for the paper's vp-tree seeds (Sec. 2,
 * Table 5), which reach nodes roughly near the query.  n_seed <= 64; any
 * n_pivot >= 1 (shared memory does not grow with it).
 */
int onng_seeds_random(uint64_t global_seed, int64_t nq, int64_t n, int32_t n_seed, int32_t *out,
                      onng_stream_t stream);
size_t onng_seeds_pivot_workspace_bytes(int64_t n, int32_t d, int32_t n_pivot);
int onng_seeds_pivot(const float *X, int64_t n, int32_t d, const float *Q, int64_t nq,
                     int32_t n_pivot, int32_t n_seed, int32_t *out, void *ws, size_t ws_bytes,
                     onng_stream_t stream);

/* --------------------------------------------------------------------- search
 * KnnSearch, Algorithm 1, one warp per query, with e_p (Eq. 1) given as e_s:
 * best-first expansion from the seeds; only the first min(e_s, degree) list
 * entries of an expanded node are scanned (e_s <= 0: all); a neighbour joins
 * the candidates if d <= r(1+eps) and the results if d <= r; the search ends
 * when the nearest candidate lies beyond r(1+eps).  Seeds are marked visited
 * and counted; R starts as the k nearest seeds with r = +inf until an insertion
 * fills R.  Ties break by (distance, id).  eps = +inf is allowed.  The visited
 * set (Set / IsSet, Sec. 2.5) is exact.
 *
 * The index: row_ptr / col as above (lengths are not needed by the search), X
 * float32 [n, d].  Optional: adj [n, adj_width] int32, each row's first
 * adj_width entries padded with -1 (onng_pad_adjacency), used instead of the
 * CSR lists whenever e_s <= adj_width; X_bf16 [n, d] (bfloat16 bits), used when
 * precision == ONNG_PREC_BF16; X_fp8 [n, d] e4m3 codes with fp8_scale [d]
 * (onng_to_fp8), used when precision == ONNG_PREC_FP8 (distances on the float32
 * products scale_j * e4m3).  In both reduced forms the final list of
 * k_rerank >= k candidates is rescored in float32 against X and the best k are
 * returned.
 *
 * Outputs: out_ids [nq, k] int32 and out_dist [nq, k] float32 (Euclidean), sorted
 * by (distance, id), padded -1 / +inf; stats [nq, 4] int32 (optional):
 * distance computations, expansions, adjacency entries scanned, ONNG_FLAG_* bits.
 * eps_q / es_q (optional, [nq]) override eps / e_s per query.
 * Limits: k, k_rerank <= 128, n_seed <= 64, d <= 1024.  The workspace holds, per
 * warp, a visited bitmap over the n ids (used past the shared-memory table) and
 * a spill pool for candidates beyond the register pool; it grows with n, and a
 * smaller workspace than the query runs fewer warps.
 */
enum onng_precision { ONNG_PREC_FP32 = 0, ONNG_PREC_BF16 = 1, ONNG_PREC_FP8 = 2 };

typedef struct {
    const int64_t *row_ptr;
    const int32_t *col;
    const float *X;
    const uint16_t *X_bf16;
    const int32_t *adj;
    int64_t n;
    int32_t d;
    int32_t adj_width;
    const uint8_t *X_fp8;    /* ONNG_PREC_FP8: e4m3 codes [n, d] from onng_to_fp8 */
    const float *fp8_scale;  /* ONNG_PREC_FP8: per-dimension scales [d] */
} onng_index;

typedef struct {
    int32_t k;
    int32_t e_s;
    float eps;
    int32_t precision;
    int32_t k_rerank;        /* bf16 and FP8: candidates rescored in float32 (>= k) */
    int32_t max_expansions;  /* 0: no cap; else per-query cap -> ONNG_FLAG_LIMIT */
    int32_t pool_cap;        /* candidate spill-pool entries per warp (0: 16384).  A query
                                whose candidates outgrow the pool drops the ones that
                                arrive when it is full (each farther than every
                                candidate kept outside the pool) and is flagged
                                ONNG_FLAG_S_OVERFLOW; larger pools take more workspace */
} onng_search_params;

size_t onng_search_workspace_bytes(int64_t nq, const onng_index *idx, const onng_search_params *p);
int onng_search(const onng_index *idx, const float *Q, int64_t nq, const onng_search_params *p,
                const int32_t *seeds, int32_t n_seed, const float *eps_q, const int32_t *es_q,
                int32_t *out_ids, float *out_dist, int32_t *stats, void *ws, size_t ws_bytes,
                onng_stream_t stream);

/* Probe for the learned parameter predictor: runs the search with
 * p->max_expansions (>= 1) as the number of hops h and writes, per query,
 * features [nq, 16] float32 instead of results:
 *   0 target (copied),  1 log d_s1,  2 log(d_s2/d_s1),  3 log(mean seed dist/d_s1),
 *   4 log(r_1/d_s1),  5 log(r_k/r_1),  6 log(next/r_1),  7 new nodes / nodes scanned,
 *   8 expansions / h,  9 log(1 + distance computations),  10 result insertions /
 *   distance computations,  11 R full,  12 log(r_k/d_s1),  13 log(1 + scanned),
 *   14 capped with an in-bound candidate left,  15 log(d)/8,
 * where d_s1, d_s2 are the two nearest seed distances, r_1 / r_k the first / last
 * of R after the h hops, and `next` the nearest candidate left, capped at
 * r(1+eps) (equal to it when the search ended).  Distances are Euclidean.
 * The paper's counterpart is Eq. 1, a fixed function of eps. */
int onng_search_probe(const onng_index *idx, const float *Q, int64_t nq, const onng_search_params *p,
                      const int32_t *seeds, int32_t n_seed, float target, float *features, int32_t *stats,
                      void *ws, size_t ws_bytes, onng_stream_t stream);

/* onng_search without a caller workspace and without any allocation.  The
 * paper has no counterpart: it is a convenience for callers that cannot
 * allocate device memory per call, such as a query loop that must not stall
 * (cudaMalloc and cudaFree may synchronise the whole device), a process whose
 * device memory is already committed to the index and its batch buffers, or
 * plain C code with no allocator of its own.
 *
 * Arguments, results and errors are those of onng_search; the scratch (query
 * counter, per-warp visited bitmaps, logs and spill pools) lives in one fixed
 * array of ONNG_SEARCH_NOALLOC_SCRATCH_BYTES per device, reserved when the
 * library's search module is loaded and held until the process exits.  One
 * CTA of the search needs 1 KB + 4 * (n/8 rounded up to 1 KB + 192 KB) of it,
 * so indexes up to about n = 65 million fit; a larger n returns
 * ONNG_E_WORKSPACE with the limit in onng_last_error().  Larger query batches
 * are fine: they run on as many CTAs as the array holds (26 at n = 1M), each
 * taking queries until none are left.
 *
 * Every call looks up the array's device address with the caller's device
 * current, so the entry point stays valid after cudaDeviceReset; make the
 * first call on a device before any stream capture, since that lookup may
 * load the module.  Every call clears the parts that must start at zero (the
 * query counter and the bitmaps) on its stream, so a call sees nothing of the
 * previous one.  All calls on a device share the one array: calls whose
 * kernels can overlap on the GPU (other streams, other host threads) race
 * and give wrong results; order them on one stream or with events. */
#define ONNG_SEARCH_NOALLOC_SCRATCH_BYTES (32u << 20)
int onng_search_noalloc(const onng_index *idx, const float *Q, int64_t nq, const onng_search_params *p,
                        const int32_t *seeds, int32_t n_seed, const float *eps_q, const int32_t *es_q,
                        int32_t *out_ids, float *out_dist, int32_t *stats, onng_stream_t stream);

/* adj [n, width]: the first `width` entries of every CSR row, -1 past its end */
int onng_pad_adjacency(const int64_t *row_ptr, const int32_t *col, int64_t n, int32_t width,
                       int32_t *adj, onng_stream_t stream);

/* --------------------------------------------------------------------- serving
 * A search service with continuous batching (the serving pattern of a request
 * stream over a device-resident index; no paper counterpart).  Requests of 1 ..
 * max_queries query vectors (host memory, copied at submit), each with its own k,
 * eps and e_s, are batched by one worker thread: a launch takes the (k, eps, e_s)
 * class of the oldest pending request and, in arrival order, every pending request
 * of that class that fits, copies their queries to the device, runs
 * onng_seeds_pivot (n_pivot, n_seed) and onng_search (precision, k_rerank) on its
 * own stream and copies the results back; up to `slots` launches are in flight.
 * A request's result depends only on its queries and class, never on its batch.
 *   onng_serve_create:  starts the service over `idx` (its arrays stay owned by
 *                       the caller and must outlive the server) on the current
 *                       device; allocates the slots' device and pinned host
 *                       buffers (the one part of the library that allocates).
 *   onng_serve_submit:  queues Q [nq, d] (host) and returns a ticket; thread-safe.
 *   onng_serve_poll:    waits up to timeout_ms for the ticket's results and copies
 *                       ids [nq, k] and dist [nq, k] (host memory); ONNG_E_AGAIN if
 *                       not done yet (poll again); the ticket is consumed once
 *                       the results (or a failure) are returned.
 *   onng_serve_destroy: stops the worker, waits for launches in flight and frees
 *                       every buffer; tickets not polled are dropped.
 * A launch still running after timeout_ms (the watchdog) fails its requests with
 * ONNG_E_LIMIT and stops the server: later submits and polls of pending requests
 * return that status.  A failed launch does the same with its own status. */
typedef struct onng_server onng_server;
typedef struct {
    int32_t precision;        /* ONNG_PREC_* of every launch */
    int32_t k_rerank;         /* reduced precision: candidates rescored in float32 (max with k) */
    int32_t n_pivot, n_seed;  /* the pivot seed rule of onng_seeds_pivot */
    int32_t max_queries;      /* queries per launch (and at most per request) */
    int32_t k_max;            /* the largest k a request may ask */
    int32_t slots;            /* launches in flight, one stream each (1 .. 64) */
    int32_t timeout_ms;       /* watchdog per launch */
} onng_serve_config;
int onng_serve_create(const onng_index *idx, const onng_serve_config *cfg, onng_server **out);
int onng_serve_submit(onng_server *srv, const float *Q, int32_t nq, int32_t k, float eps, int32_t e_s,
                      uint64_t *ticket);
int onng_serve_poll(onng_server *srv, uint64_t ticket, int32_t *ids, float *dist, int32_t timeout_ms);
int onng_serve_destroy(onng_server *srv);

/* ------------------------------------------------------- parameter predictor
 * A 16 -> 64 -> 64 -> 2 network with ReLU hidden layers mapping probe features
 * to (log(eps + 0.01), log e_s) per query (no paper counterpart; it replaces the
 * fixed policy of Eq. 1).  P is the flat float32 parameter vector
 * W1[64][16], b1[64], W2[64][64], b2[64], W3[2][64], b3[2] (onng_mlp_nparam()
 * values); X [B, 16] float32 rows; targets T [B, 2].
 *   onng_mlp_forward:   Y [B, 2] = network(X) in float32.
 *   onng_mlp_loss_grad: loss (1 float) = mean over B of 0.5 * |Y - T|^2, and
 *                       G [nparam] its gradient (G and loss are overwritten).
 *   onng_mlp_adam:      one Adam step (Kingma & Ba 2015) on P with moments M, V
 *                       at step count t >= 1.
 *   onng_mlp_train:     `steps` Adam steps (lr, beta 0.9 / 0.999, eps 1e-8) on
 *                       consecutive mini-batches of `batch` <= 128 rows of X / T
 *                       (wrapping), steps numbered t0 + 1 ...; G is unused
 *                       (may be NULL); losses [steps] (optional) receives each
 *                       loss.  Runs in one CTA.
 *   onng_mlp_predict:   bfloat16 evaluation (weights and inputs rounded to
 *                       bfloat16, float32 accumulation): eps_out = max(0,
 *                       exp(y0) - 0.01) * alpha, es_out = clamp(round(exp(y1)),
 *                       es_min, es_max). */
int onng_mlp_nparam(void);
int onng_mlp_forward(const float *P, const float *X, int64_t B, float *Y, onng_stream_t stream);
int onng_mlp_loss_grad(const float *P, const float *X, const float *T, int64_t B, float *G, float *loss,
                       onng_stream_t stream);
int onng_mlp_adam(float *P, const float *G, float *M, float *V, int64_t t, float lr, float beta1,
                  float beta2, float eps, onng_stream_t stream);
int onng_mlp_train(float *P, float *M, float *V, const float *X, const float *T, int64_t N, int32_t batch,
                   int64_t steps, int64_t t0, float lr, float *G, float *losses, onng_stream_t stream);
int onng_mlp_predict(const float *P, const float *X, int64_t B, float alpha, int32_t es_min,
                     int32_t es_max, float *eps_out, int32_t *es_out, onng_stream_t stream);

/* FP8 e4m3 copy of a vector set X [n, d] for the FP8 search form (no paper
 * counterpart): scale [d] = max_i |x_ij| / 448 in float32 (1 for an all-zero
 * column) and out [n, d] = e4m3(x_ij / scale_j), the nearest finite e4m3 value
 * with ties to even, saturating at 448.  The search dequantises a coordinate as
 * the float32 product scale_j * e4m3(code).  X must be finite. */
int onng_to_fp8(const float *X, int64_t n, int32_t d, float *scale, uint8_t *out, onng_stream_t stream);

/* float32 -> bfloat16 (round to nearest even) copy of a vector set, for X_bf16 */
int onng_to_bf16(const float *X, int64_t count, uint16_t *out, onng_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* ONNG_H */
