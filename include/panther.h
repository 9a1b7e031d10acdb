/*
 * panther.h - C ABI of libpanther, a GB300 (sm_103a) implementation of the
 * hot path of Panther and Panther++ (Zhang et al., "Panther: Fast Top-k
 * Similarity Search in Large Networks", arXiv 1504.02577).
 *
 * The hot path:
 *   panther_sample_size    R of the sample-size guarantee (Sec. 3.2)
 *   panther_build_graph    graph + transition tables t_ij of Eq. (3)
 *   panther_sample_paths   R random T-paths (Algorithm 3)
 *   panther_build_index    vertex -> path inverted index P_v (Sec. 3.1)
 *   panther_topk           per-query co-occurrence counts and top-k
 *                          (Algorithm 1, Eq. (4))
 *   pantherpp_vectors      Panther++ feature vectors theta(v) (Sec. 3.3, Alg. 2)
 *   pantherpp_knn          nearest neighbours of theta under Euclidean
 *                          distance (Sec. 3.3, Alg. 2)
 *   panther_serve_*        a request loop over resident graph/paths/index
 *                          (no counterpart in the paper)
 *
 * Conventions shared by every call:
 *   - Calls return a panther_status and never throw. Arguments are validated
 *     before any launch; on error nothing is launched, *out handles are left
 *     NULL and panther_last_error() describes the problem.
 *   - A context owns one CUDA device and one stream. Work is enqueued on that
 *     stream; a call returns when its work is enqueued unless stated
 *     otherwise. Calls on one context must not run concurrently from several
 *     host threads (the serving loop has its own context and lock).
 *   - Handles (graph, paths, index, vecs) own device memory allocated by the
 *     library; free them with the matching panther_free_* call. Query and
 *     output arrays are caller-owned: device pointers, unless the flag
 *     PANTHER_IO_HOST says they are host pointers (then the call copies and
 *     returns only when the host outputs are written).
 *   - Kernels report data errors they detect (a hash table overfull, an
 *     index out of range, a bounded wait that ran out) in a device status
 *     word; panther_sync() waits for the stream and returns that status.
 *   - Results are integers: counts of shared paths (similarity = count / R)
 *     and exact squared distances. Ties order by vertex id ascending. Rows
 *     with fewer than k candidates are padded with id -1 and count 0
 *     (k-NN: id -1, distance UINT64_MAX).
 */
#ifndef PANTHER_H
#define PANTHER_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PANTHER_API __attribute__((visibility("default")))
#else
#define PANTHER_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PANTHER_OK = 0,
    PANTHER_EINVAL = 1,     /* invalid argument or malformed graph */
    PANTHER_ENOMEM = 2,     /* device or pinned host allocation failed, or budget exceeded */
    PANTHER_ECUDA = 3,      /* a CUDA runtime call failed */
    PANTHER_ETIMEOUT = 4,   /* a bounded device-side or host-side wait ran out */
    PANTHER_EOVERFLOW = 5,  /* a size or value exceeds what the data layout holds */
    PANTHER_EBUSY = 6       /* the serving loop is full or shutting down */
} panther_status;

/* where caller arrays live */
enum { PANTHER_MEM_HOST = 0, PANTHER_MEM_DEVICE = 1 };

/* neighbour selection (Eq. 3); panther_build_graph takes a bit mask of the
 * tables to build, panther_sample_paths one mode. UNWEIGHTED is Eq. (3) with
 * every weight equal, t_ij = 1/deg(i) (the paper's unweighted networks): no
 * table, a step reads one column entry. */
enum { PANTHER_MODE_PREFIX = 1, PANTHER_MODE_ALIAS = 2, PANTHER_MODE_BOTH = 3, PANTHER_MODE_UNWEIGHTED = 4 };

/* panther_topk / pantherpp_knn flags */
enum {
    PANTHER_TOPK_BATCHED = 0,      /* one load-balanced persistent launch for the whole batch */
    PANTHER_TOPK_PLAIN = 1,        /* one launch per query (comparison form) */
    PANTHER_KNN_BF16_SCREEN = 0,   /* tensor-core BF16 screening + exact integer rerank */
    PANTHER_KNN_FP32 = 2,          /* FP32 brute force + exact integer rerank (comparison form) */
    PANTHER_IO_HOST = 0x100        /* queries and outputs are host pointers */
};

typedef struct panther_ctx panther_ctx;
typedef struct panther_graph panther_graph;
typedef struct panther_paths panther_paths;
typedef struct panther_index panther_index;
typedef struct pantherpp_vecs pantherpp_vecs;
typedef struct panther_server panther_server;

/* ------------------------------------------------------------ context --- */

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t
 * to enqueue on (NULL: the library creates and owns a non-blocking stream).
 * Errors: EINVAL (no such device), ECUDA. */
PANTHER_API panther_status panther_create(panther_ctx** out, int device, void* cuda_stream);

/* Synchronises the stream, frees context-owned scratch. Handles created on
 * the context must be freed before it. NULL is ignored. */
PANTHER_API void panther_destroy(panther_ctx* ctx);

/* Human-readable description of the last error on this context ("" if none).
 * The pointer stays valid until the next call on the context. */
PANTHER_API const char* panther_last_error(const panther_ctx* ctx);

/* Wait for all work on the context's stream, then return and clear the
 * device status word (OK, EOVERFLOW, EINVAL or ETIMEOUT) or ECUDA. */
PANTHER_API panther_status panther_sync(panther_ctx* ctx);

/* Scratch budget in bytes for temporary device buffers of one call (top-k
 * hub tables, index sort buffers are sized separately). Default 8 GiB. */
PANTHER_API panther_status panther_set_scratch_budget(panther_ctx* ctx, int64_t bytes);

/* Number of kernel launches this context has enqueued so far. */
PANTHER_API int64_t panther_launch_count(const panther_ctx* ctx);

/* --------------------------------------------------------- Sec. 3.2 --- */

/* Sample size of the guarantee (Theorem 1 with Lemma 1):
 *   R = ceil( c / eps^2 * ( log2 C(T,2) + 1 + ln(1/delta) ) ).
 * Host only, no context. Errors: EINVAL unless 0<eps<1, 0<delta<1, c>0,
 * T>=2; EOVERFLOW if R does not fit in int64. */
PANTHER_API panther_status panther_sample_size(double eps, double delta, double c, int T, int64_t* R);

/* ----------------------------------------------------- graph, Eq. (3) --- */

/* Copy an undirected weighted graph G=(V,E,W) (Definition 1) to the device
 * and build the transition tables of Eq. (3), t_ij = w_ij / sum_k w_ik.
 *   n        number of vertices, 1 <= n < 2^31
 *   m        number of directed CSR entries (2|E|), m < 2^32
 *   row_ptr  int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = m
 *   col      int32[m], neighbours of each row in strictly ascending order
 *   w        uint32[m], weights >= 1; w(u,v) = w(v,u). May be NULL when
 *            modes is PANTHER_MODE_UNWEIGHTED alone (every weight 1).
 *   mem      PANTHER_MEM_HOST or PANTHER_MEM_DEVICE for the three arrays
 *   modes    a combination of PANTHER_MODE_PREFIX, PANTHER_MODE_ALIAS (the
 *            tables to build) and PANTHER_MODE_UNWEIGHTED (keep a device copy
 *            of col, 4 B per entry, for sampling with t_ij = 1/deg; no table)
 * Host arrays are staged in temporary device buffers; device arrays are read
 * in place during the call. The caller keeps ownership and nothing of the
 * CSR is kept afterwards (the tables, or the library's own copy of col for
 * UNWEIGHTED, hold what sampling needs). The call
 * validates the graph on the device (ranges, sorted rows, no self-loops,
 * symmetry with equal weights, every row sum * degree < 2^63) and returns
 * after the tables are built (it synchronises the stream).
 * Errors: EINVAL (bad arguments or graph), EOVERFLOW (m >= 2^32, row sum too
 * large), ENOMEM, ECUDA. */
PANTHER_API panther_status panther_build_graph(panther_ctx* ctx, int64_t n, int64_t m,
                                   const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                                   int mem, int modes, panther_graph** out);

/* ------------------------------------------------------- Algorithm 3 --- */

/* Sample R paths of T steps (T+1 vertices). Path r starts at
 * Uniform[0,n) and moves T times to a neighbour chosen with probability
 * t_ij (Eq. 3); a vertex without neighbours keeps the walk in place.
 * Draws are Philox4x32-10 with key (lo32(seed), hi32(seed)) and counter
 * (lo32(r), hi32(r), t, attempt); Uniform[0,S) is Lemire's multiply-shift
 * with rejection on the 64-bit word (x0 | x1<<32). PREFIX picks the neighbour
 * j with cum(j-1) <= x < cum(j) for x = Uniform[0, sum w); ALIAS picks column
 * c = Uniform[0,deg) (x0,x1) and coin u = Uniform[0, sum w) (x2,x3) of the
 * same draw from the integer Vose table. UNWEIGHTED picks column
 * c = Uniform[0,deg) from (x0,x1), the same words and rejections as PREFIX, so
 * its paths equal PREFIX paths of the same graph with every weight 1. All
 * realise Eq. 3 exactly and the paths are reproducible bit for bit.
 *   R in [1, 2^32-1], T in [1, 127], mode PREFIX, ALIAS or UNWEIGHTED (the
 *   graph must have been built with that mode). The index stores path ids as
 *   uint32; at 32 B of row and 4 B of index per vertex of each path, 2^32
 *   paths already take more than one GPU's memory; R >= 2^32 returns
 *   EOVERFLOW.
 * Rows live on the device as int32[R][stride], stride = 8, 16, 32, 64 or 128
 * (the smallest that holds T+1); entries past T+1 are -1.
 * Errors: EINVAL, EOVERFLOW, ENOMEM, ECUDA. */
PANTHER_API panther_status panther_sample_paths(panther_ctx* ctx, const panther_graph* g, uint64_t seed,
                                    int64_t R, int T, int mode, panther_paths** out);

/* Paths r0 .. r0+R-1 of the same sequence (no counterpart in the paper): row
 * i holds path r0 + i, drawn with counter r0 + i, so a range is bit-identical
 * to the same rows of a run from 0. Use it to resume sampling from any path
 * id or to split the paths between GPUs. Path ids in an index built from this
 * handle are local (i = r - r0). r0 >= 0, r0 + R < 2^63; otherwise as
 * panther_sample_paths. */
PANTHER_API panther_status panther_sample_paths_range(panther_ctx* ctx, const panther_graph* g, uint64_t seed,
                                                      int64_t r0, int64_t R, int T, int mode, panther_paths** out);

/* Device view of the path rows (library-owned; valid until freed). */
PANTHER_API panther_status panther_paths_view(const panther_paths* p, const int32_t** dev_rows,
                                  int64_t* R, int* L, int* stride);

/* Shape of a path handle: n vertices of its graph, R rows, T steps, r0 the
 * global id of row 0. Any output pointer may be NULL. Errors: EINVAL (null p). */
PANTHER_API panther_status panther_paths_info(const panther_paths* p, int64_t* n, int64_t* R, int* T, int64_t* r0);

/* ------------------------------------------------------------ Sec. 3.1 --- */

/* Build the inverted index P_v = { r : v in p_r } with a device LSD radix
 * sort of (vertex, path id) pairs. A path that visits v several times is
 * listed once. Layout: off int64[n+1], pid uint32[nnz] (ids reach 2^32 - 2;
 * a signed 32-bit view shows ids from 2^31 up as negative); P_v is
 * pid[off[v] .. off[v+1]) in ascending path id.
 * Memory: one sort over all pairs needs about 16 B per pair (+ 5% for tile
 * counts) of temporary device memory next to the result (4 B per pair). When
 * that exceeds the index budget (panther_set_index_budget; by default the
 * free device memory less the result), the rows are sorted in chunks of
 * consecutive paths: |P_v| of every vertex is counted first, then each
 * chunk's pairs are sorted and appended to the lists, so the temporary memory
 * follows the chunk and the result is the same. Synchronises once per chunk
 * to size it. Errors: EINVAL, ENOMEM, ECUDA. */
PANTHER_API panther_status panther_build_index(panther_ctx* ctx, const panther_paths* p, panther_index** out);

/* Temporary device bytes one panther_build_index call may use (0: the free
 * device memory less the result, the default; otherwise at least 1 MiB).
 * Errors: EINVAL. */
PANTHER_API panther_status panther_set_index_budget(panther_ctx* ctx, int64_t bytes);

/* Index build that allocates nothing (the paper has no counterpart; this is
 * for callers that cannot call cudaMalloc, such as a host application that
 * owns a fixed share of the GPU and accounts for every byte itself, or a
 * latency-bound loop where an allocation could synchronise the device).
 * Same result as panther_build_index: P_v = pid[off[v] .. off[v+1]),
 * ascending. The caller passes dev_off (int64[n+1]) and dev_pid (uint32,
 * pid_capacity >= R*(T+1) entries); *nnz receives the number of pairs.
 * Temporary buffers come from one static device array of about 86 MiB that
 * every GPU loading the library reserves until the process exits; R*(T+1)
 * may be at most 4,194,304 (EOVERFLOW beyond, before any launch). The first
 * call on a device looks up that array's device address, so make it before
 * any stream capture. Calls share the array: two calls that overlap on the
 * GPU (other contexts or streams) race and must be ordered by the caller.
 * Every call, not only the first, waits once for the context stream (it
 * copies the number of pairs found by the first radix pass to the host to
 * size the later passes), so the call returns only after the work queued
 * before it on that stream has finished.
 * Errors: EINVAL, EOVERFLOW, ECUDA. */
PANTHER_API panther_status panther_build_index_noalloc(panther_ctx* ctx, const panther_paths* p, int64_t* dev_off,
                                                       uint32_t* dev_pid, int64_t pid_capacity, int64_t* nnz);

PANTHER_API panther_status panther_index_view(const panther_index* ix, const int64_t** dev_off,
                                  const uint32_t** dev_pid, int64_t* n, int64_t* nnz);

/* ---------------------------------------------- Algorithm 1, Eq. (4) --- */

/* For each query v = queries[i]: cnt(v,u) = number of paths in P_v that
 * contain u (each path counted once per u), for every u != v; then the k
 * largest by (cnt desc, u asc). Writes out_ids int32[q][k] and
 * out_counts uint32[q][k] (similarity S_RP(v,u) = cnt / R).
 *   q >= 0 (q = 0 is a no-op), 1 <= k <= 128, queries in [0, n). With
 *   k <= 64 every tier runs; with 64 < k <= 128 queries of up to 32 paths
 *   stay in the group tiers and every other query is counted in a per-query
 *   device table and selected with 128-entry lists (slower, same results);
 *   the PLAIN form then runs that path once per query.
 *   flags: PANTHER_TOPK_BATCHED or PANTHER_TOPK_PLAIN, optionally
 *          | PANTHER_IO_HOST (queries/outputs in host memory; the call then
 *          synchronises; batches of 4M queries or more run in four chunks
 *          whose rows are copied to the host while the next chunk computes)
 * Temporary device memory (hub hash tables) is drawn from the context's
 * scratch budget; a batch whose hubs do not fit is processed in several
 * rounds.
 * Host waits: the BATCHED form is not fully asynchronous. After the lane,
 * group and persistent launches it copies the number of hub queries to the
 * host and waits for the context stream (once per call); when there are hub
 * queries it waits again to read their path counts and once per hub round
 * (to read which queries need a second, exact pass). The call therefore
 * returns only after its own work and everything queued before it on the
 * stream has finished, and a serving worker's host thread is held for the
 * whole batch. The PLAIN form only enqueues (one launch per query).
 * Errors: EINVAL, ENOMEM, ECUDA. */
PANTHER_API panther_status panther_topk(panther_ctx* ctx, const panther_index* ix, const panther_paths* p,
                            const int32_t* queries, int64_t q, int k,
                            int32_t* out_ids, uint32_t* out_counts, int flags);

/* Tier sizes of the last panther_topk call on this context (also set by
 * pantherpp_vectors, which counts through the same tiers):
 *   [0] queries, [1] lane tier, [2] group tiers (8/16/32 lanes per query),
 *   [3] warp tier, [4] CTA tier (both persistent passes), [5] hub queries,
 *   [6] hub queries counted through the bucketed two-pass tier (per round),
 *   [7] hub queries counted in per-query device tables (per round),
 *   [8] hub queries whose buckets overflowed (counted again in tables),
 *   [9] hub queries counted a second time because the first-round
 *       threshold could have dropped a top-k candidate.
 * The PLAIN form sets only [0]. Errors: EINVAL. */
PANTHER_API panther_status panther_topk_stats(panther_ctx* ctx, int64_t stats[10]);

/* Autotuner for the batched form: runs the batch once per candidate launch
 * shape of the persistent kernel (threads per CTA, shared-table slots, CTAs
 * per SM), times three more runs of each with CUDA events on the context
 * stream, and keeps the fastest shape in the context for later calls.
 * Arguments as panther_topk (device pointers); the outputs hold the batch's
 * result on return. chosen (may be NULL) receives {threads, slots, ctas/SM}.
 * Synchronises. Errors: EINVAL, ENOMEM, ECUDA. */
PANTHER_API panther_status panther_tune_topk(panther_ctx* ctx, const panther_index* ix, const panther_paths* p,
                                             const int32_t* queries, int64_t q, int k, int32_t* out_ids,
                                             uint32_t* out_counts, int* chosen);

/* Set the batched form's launch shape directly (for example one chosen by
 * panther_tune_topk in an earlier run): threads per CTA in {128, 256, 512, 1024},
 * shared-table slots (a multiple of 32, at least threads/32*512, at most
 * 24,576), CTAs per SM in [1, 8]. Results do not depend on the shape.
 * Errors: EINVAL. */
PANTHER_API panther_status panther_set_topk_shape(panther_ctx* ctx, int threads, int table_slots, int ctas_per_sm);

/* ---------------------------------------------------- Panther++ (3.3) --- */

/* theta(v) = the D largest counts cnt(v,u), u != v, descending, zero padded,
 * for every vertex (Algorithm 2's loop over V), plus the device data the
 * k-NN search needs (for D <= 56 a BF16 copy padded to 64 columns; exact
 * squared norms).
 *   1 <= D <= 128 (D > 64 counts through the top-k path for k > 64).
 *   Errors: EINVAL, ENOMEM, EOVERFLOW (max count^2 * D reaches 2^64, so a
 *   squared distance could overflow 64 bits), ECUDA. Synchronises. */
PANTHER_API panther_status pantherpp_vectors(panther_ctx* ctx, const panther_index* ix, const panther_paths* p,
                                 int D, pantherpp_vecs** out);

/* Device view of theta: uint32[n][D] row-major. */
PANTHER_API panther_status pantherpp_vecs_view(const pantherpp_vecs* v, const uint32_t** dev_theta,
                                   int64_t* n, int* D);

/* For each query v: the k vertices u != v with the smallest
 * ||theta(v) - theta(u)||^2, ties by id ascending (the order of
 * S_RP++ = 1/||.|| descending, Sec. 3.3, without forming the reciprocal).
 * Writes out_ids int32[q][k] and out_dist2 uint64[q][k] (exact).
 *   1 <= k <= 32, queries in [0, n)
 *   flags: PANTHER_KNN_BF16_SCREEN (tensor cores, BF16 inputs, FP32
 *          accumulation, a proven error bound, exact uint64 rerank of every
 *          candidate the bound cannot rule out) or PANTHER_KNN_FP32 (FP32
 *          CUDA-core brute force with the same bound and rerank), optionally
 *          | PANTHER_IO_HOST.
 * Vectors wider than the BF16 screen's 56 columns (D > 56) take the FP32
 * screen (64 or 128 columns) under either flag, with the same exact rerank.
 * Every form returns the exact answer. Errors: EINVAL, ENOMEM, ECUDA. */
PANTHER_API panther_status pantherpp_knn(panther_ctx* ctx, const pantherpp_vecs* v, const int32_t* queries,
                             int64_t q, int k, int32_t* out_ids, uint64_t* out_dist2, int flags);

/* Panther++ across two networks (the paper's identity-resolution use of
 * S_RP++ between vertices of different graphs, Sec. 3.3 / Fig. 1a): queries
 * are vertices of vq, candidates every vertex of vc, none excluded; both
 * vector sets have the same D. Output ids are vertices of vc. Otherwise as
 * pantherpp_knn. Errors: EINVAL (also different D), ENOMEM, ECUDA. */
PANTHER_API panther_status pantherpp_knn_cross(panther_ctx* ctx, const pantherpp_vecs* vq, const pantherpp_vecs* vc,
                                               const int32_t* queries, int64_t q, int k, int32_t* out_ids,
                                               uint64_t* out_dist2, int flags);

/* Screening statistics of the last pantherpp_knn call on this context:
 * [0] pairs screened, [1] pairs sent to exact rerank, [2] max |d_hat - d|
 * observed over reranked pairs, [3] pairs whose bound was zero (exact). */
PANTHER_API panther_status pantherpp_knn_stats(panther_ctx* ctx, int64_t stats[4]);

/* BF16 screening values, for measuring the screening error (no counterpart
 * in the paper). Runs the tensor-core screen of pantherpp_knn for q queries
 * (1 <= q <= 128, device int32 vertex ids) against every vertex and writes
 * each screened value: out_y (device float[q][npad]) receives
 * y_hat = |b|^2 - 2 a_hat.b_hat (FP32 accumulation of BF16 inputs) for query
 * i and the candidate at position p, out_cid (device int32[npad]) the vertex
 * at each position (-1: padding, whose values are meaningless). The exact
 * value is |b|^2 - 2 a.b, so d_hat = |a|^2 + y_hat. With out_y and out_cid
 * both NULL the call only sets *npad (the candidate positions, a multiple of
 * 256). Synchronises. Errors: EINVAL (also D > 56), ENOMEM, ECUDA. */
PANTHER_API panther_status pantherpp_debug_screen(panther_ctx* ctx, const pantherpp_vecs* v, const int32_t* queries,
                                                  int64_t q, float* out_y, int32_t* out_cid, int64_t* npad);

/* ------------------------------------------------------ test support --- */

/* Copies of the graph's transition tables, for tests: dev_alias16 receives
 * m entries {thr_lo, thr_hi, col[c], col[alias[c]]} (uint32 x4) and
 * dev_prefix m entries {cum, col} (uint32 x2, or x4 with a 64-bit cum when
 * *prefix_wide is 1). Either pointer may be NULL. Synchronises. */
PANTHER_API panther_status panther_debug_graph_tables(const panther_graph* g, void* dev_alias16, void* dev_prefix,
                                                      int* prefix_wide);

/* Philox4x32-10 words for `count` counters (lo32(r0+i), hi32(r0+i), c2, c3)
 * under key (k0, k1), written to dev_out[i][0..3], and the same counters
 * through curand's Philox4_32_10 (curand_init(k0 | k1<<32, subsequence =
 * c2 | c3<<32, offset = 4*(r0+i)), one curand4) to dev_ref[i][0..3].
 * Synchronises. */
PANTHER_API panther_status panther_debug_philox(panther_ctx* ctx, uint32_t k0, uint32_t k1, uint64_t r0,
                                                uint32_t c2, uint32_t c3, int64_t count, uint32_t* dev_out,
                                                uint32_t* dev_ref);

/* Hub-tier routing (test-only; no counterpart in the paper): from now on
 * queries whose candidate bound min(|P_v| * T, n-1) exceeds hub_min_cap
 * (when > 0, at least 256) are hub queries, and route selects how hub
 * queries are counted: 0 as usual, 1 every one through the bucketed
 * two-pass tier, 2 every one in a per-query device table. Results do not
 * change; tests use it to reach every hub kernel on small inputs.
 * (0, 0) restores the default. Errors: EINVAL. */
PANTHER_API panther_status panther_debug_topk_route(panther_ctx* ctx, int64_t hub_min_cap, int route);

/* Fault injection (test-only; no counterpart in the paper). The nth device
 * allocation of this context from now on (0-based) fails once with ENOMEM,
 * as if the device were out of memory; nth < 0 cancels. The call that meets
 * it returns ENOMEM, frees what it had allocated and leaves the context
 * usable. Errors: EINVAL (null ctx). */
PANTHER_API panther_status panther_debug_fail_alloc(panther_ctx* ctx, int64_t nth);

/* Bounded device wait (test-only; no counterpart in the paper): one warp
 * waits for a device flag that nothing sets, gives up after limit_cycles
 * SM clock cycles (1 <= limit_cycles <= 2^31), records a timeout in the
 * context's status word and returns; the synchronisation at the end reports
 * it. Returns ETIMEOUT when the wait ran out (always, by construction); the
 * context stays usable. Errors: EINVAL. */
PANTHER_API panther_status panther_debug_wait_timeout(panther_ctx* ctx, int64_t limit_cycles);

/* --------------------------------------------------------- free calls --- */
PANTHER_API void panther_free_graph(panther_graph* g);
PANTHER_API void panther_free_paths(panther_paths* p);
PANTHER_API void panther_free_index(panther_index* ix);
PANTHER_API void pantherpp_free_vecs(pantherpp_vecs* v);

/* ---------------------------------------------------------- checkpoint --- */
/* (No counterpart in the paper.) Write sampled paths or an index to a file
 * and read them back, for example to serve from a saved index after a
 * restart. File: a 64-byte header (magic "PNTHPATH"/"PNTHINDX", version 1,
 * T, L, stride, mode, n, R, r0 or nnz, seed), then the device arrays as they
 * are laid out in memory (little-endian). Loading validates the header and,
 * for an index, the offsets (monotone from 0 to nnz) and path ids (< R) on
 * the device before returning the handle. Synchronous.
 * Errors: EINVAL (null arguments, unreadable or inconsistent file), ENOMEM,
 * ECUDA. */
PANTHER_API panther_status panther_save_paths(const panther_paths* p, const char* path);
PANTHER_API panther_status panther_load_paths(panther_ctx* ctx, const char* path, panther_paths** out);
PANTHER_API panther_status panther_save_index(const panther_index* ix, const char* path);
PANTHER_API panther_status panther_load_index(panther_ctx* ctx, const char* path, panther_index** out);

/* ------------------------------------------------------------ serving --- */
/* (No counterpart in the paper.) A request loop over resident paths, index
 * and vectors. Requests arrive from any host thread. `streams` worker
 * threads each own a context (one CUDA stream) and device buffers sized from
 * mem_budget_bytes. A free worker takes the oldest pending request and every
 * later pending request of the same kind whose queries still fit its buffers
 * (FIFO), runs them as ONE batched call with k = the largest k among them,
 * and hands each request the first k entries of its rows. Ranking is a total
 * order, so a result in the mix is identical to the same request made alone.
 * Up to `streams` batches run at once, so new requests start while earlier
 * ones are on the GPU.
 *
 * panther_serve_create: ix and p must belong together (same n and R), v
 *   (optional, needed for k-NN) must have the same n; streams in [1, 16];
 *   max_inflight_requests >= 1; mem_budget_bytes >= 1 MiB. The handles stay
 *   owned by the caller and must outlive the server. EINVAL on bad
 *   arguments, ENOMEM when the budget or the device cannot hold the buffers.
 * panther_serve_submit: kind 0 = top-k (Algorithm 1, k in [1, 64], out_vals
 *   uint32 counts), 1 = Panther++ k-NN (Sec. 3.3, k in [1, 32], out_vals
 *   uint64 squared distances). queries[q] (ids in [0, n)), out_ids[q][k] and
 *   out_vals[q][k] are HOST pointers owned by the caller; they must stay
 *   valid until panther_serve_wait has returned for the ticket. EINVAL on bad
 *   arguments (checked before queueing); EBUSY when max_inflight_requests
 *   requests are open, when q exceeds one worker's buffers, or after
 *   destroy has begun. */
PANTHER_API panther_status panther_serve_create(int device, const panther_index* ix, const panther_paths* p,
                                    const pantherpp_vecs* v, int64_t mem_budget_bytes,
                                    int max_inflight_requests, int streams, panther_server** out);
PANTHER_API panther_status panther_serve_submit(panther_server* s, int kind, const int32_t* queries, int64_t q,
                                    int k, int32_t* out_ids, void* out_vals, int64_t* ticket);
/* Wait for a request (timeout_s <= 0: no limit); *latency_ms = completion
 * time - submit time. Returns the request's own status and releases the
 * ticket; ETIMEOUT leaves it open (wait again). One thread waits on a given
 * ticket at a time; EINVAL for an unknown or already released ticket. */
PANTHER_API panther_status panther_serve_wait(panther_server* s, int64_t ticket, double timeout_s,
                                  double* latency_ms);
/* [0] submitted, [1] completed, [2] batches launched, [3] max requests in one batch,
 * [4] max batches in flight at once, [5] requests refused (EBUSY) */
PANTHER_API panther_status panther_serve_stats(panther_server* s, int64_t stats[6]);
/* Stops taking requests, finishes the pending ones, joins the workers and
 * frees the server (tickets not yet waited for are released). */
PANTHER_API void panther_serve_destroy(panther_server* s);

#ifdef __cplusplus
}
#endif
#endif /* PANTHER_H */
