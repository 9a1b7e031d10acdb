// Internal declarations shared by the libpanther translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/panther.h"

// ------------------------------------------------------------ status bits ---
// Device status word bits (atomicOr); read back by panther_sync().
enum : uint32_t {
    ST_HASH_FULL = 1u << 0,    // a hash table ran out of slots
    ST_BAD_QUERY = 1u << 1,    // query id outside [0, n)
    ST_GRAPH_BAD = 1u << 2,    // graph validation failed
    ST_OVERFLOW = 1u << 3,     // a value exceeded its layout
    ST_TIMEOUT = 1u << 4,      // a bounded wait ran out
    ST_BAD_INDEX = 1u << 5,    // an index or path entry out of range
};

// ------------------------------------------------------------ host state ---
struct panther_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint32_t* d_status = nullptr;     // [0] flags, [1..3] detail
    uint32_t* h_status = nullptr;     // pinned mirror
    int64_t scratch_budget = int64_t(8) << 30;
    int64_t index_budget = 0;         // temporary bytes of an index build (0: free device memory)
    std::atomic<int64_t> launches{0};
    std::string err;
    int64_t knn_stats[4] = {0, 0, 0, 0};
    // autotuned top-k launch shape (0 = not tuned yet)
    int topk_threads = 0, topk_cta_slots = 0, topk_blocks_per_sm = 0;
    // side streams for independent kernels of one call (fork/join by events
    // on `stream`); null when they could not be created
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
    // copies of host-I/O results that overlap the next chunk's kernels
    cudaStream_t copy = nullptr;
    cudaEvent_t copy_ev = nullptr;
    // slot arena of the hub device tables, kept between calls: all slots are
    // EMPTY whenever hub_arena_clean (the select pass empties what it reads)
    unsigned long long* hub_arena = nullptr;
    int64_t hub_arena_slots = 0;
    bool hub_arena_clean = true;
    // fault injection: the allocation numbered fail_alloc_at fails once (-1: off)
    int64_t fail_alloc_at = -1, alloc_seen = 0;
    // tier sizes of the last top-k call (see panther_topk_stats)
    int64_t topk_stats[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    // test routing of the hub tier (panther_debug_topk_route): queries whose
    // candidate bound exceeds dbg_hub_min_cap (> 0) are hub queries; route 1
    // counts every hub query through the buckets, 2 through device tables
    int64_t dbg_hub_min_cap = 0;
    int dbg_hub_route = 0;
};

struct panther_graph {
    panther_ctx* ctx = nullptr;
    int64_t n = 0, m = 0;
    int modes = 0;
    uint4* vrec = nullptr;           // [n]: {start, deg, S_lo, S_hi}
    void* prefix = nullptr;          // [m]: uint2 {cum, col} or uint4 {cum_lo, cum_hi, col, 0}
    int prefix_wide = 0;             // 1 when a row sum reaches 2^32
    uint4* alias = nullptr;          // [m]: {thr_lo, thr_hi, col_self, col_alias}
    int32_t* col = nullptr;          // [m]: neighbours (UNWEIGHTED mode only)
    uint64_t max_row_sum = 0;
};

struct panther_paths {
    panther_ctx* ctx = nullptr;
    int64_t n = 0, R = 0;
    int T = 0, L = 0, stride = 0, mode = 0;
    uint64_t seed = 0;
    int64_t r0 = 0;                  // global id of local row 0 (draw counters use r0 + row)
    int32_t* rows = nullptr;         // [R][stride]
};

struct panther_index {
    panther_ctx* ctx = nullptr;
    int64_t n = 0, nnz = 0;
    int64_t R = 0;                   // rows of the paths its ids refer to
    int64_t* off = nullptr;          // [n+1]
    uint32_t* pid = nullptr;         // [nnz] path ids (row numbers of the path set, R <= 2^32 - 1)
    uint8_t* cls = nullptr;          // [n] path_code(|P_v|) (|P_v| bounds any count with v)
    int64_t* cls_hist = nullptr;     // [256] vertices per code
};

struct pantherpp_vecs {
    panther_ctx* ctx = nullptr;
    int64_t n = 0;
    int D = 0;
    uint32_t* theta = nullptr;       // [n][D]
    uint64_t* norm2 = nullptr;       // [n] exact squared norms
    float* nrm = nullptr;            // [n] sqrt(norm2) rounded up (for the error bound)
    uint8_t* exact = nullptr;        // [n] 1 if every entry <= 256 (BF16-exact row)
    uint32_t max_val = 0;
    // candidate side of the screening GEMM, exact rows first
    int64_t npad = 0, nexact = 0;    // positions (multiple of 256), exact positions
    uint16_t* B = nullptr;           // [npad][64] bf16 candidate rows
    int32_t* cid = nullptr;          // [npad] vertex at each position (-1 padding)
    float* cnrm = nullptr;           // [npad] |b| rounded up
    float* cncf = nullptr;           // [npad] |b|^2 rounded up
    uint8_t* ctile = nullptr;        // [npad/256] 1 if the tile holds only exact rows
};

// ------------------------------------------------------------ host helpers ---
panther_status set_err(panther_ctx* ctx, panther_status st, const char* fmt, ...);
panther_status cuda_err(panther_ctx* ctx, cudaError_t e, const char* what);

#define PCK(ctx, call)                                                   \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_err((ctx), e_, #call);        \
    } while (0)

// count and check a launch
#define PLAUNCH(ctx)                                                     \
    do {                                                                 \
        (ctx)->launches.fetch_add(1, std::memory_order_relaxed);         \
        cudaError_t e_ = cudaGetLastError();                             \
        if (e_ != cudaSuccess) return cuda_err((ctx), e_, "kernel launch"); \
    } while (0)

panther_status dev_alloc(panther_ctx* ctx, void** p, size_t bytes);
void dev_free(panther_ctx* ctx, void* p);

static inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// stride of a path row for L vertices: 8, 16, 32, 64 or 128 int32
static inline int path_stride(int L) {
    return L <= 8 ? 8 : (L <= 16 ? 16 : (L <= 32 ? 32 : (L <= 64 ? 64 : 128)));
}
constexpr int MAX_T = 127;   // longest path: T + 1 = 128 vertices fill the widest row

// device-wide exclusive scan of int64 values (in place), n >= 1; uses scratch
panther_status scan_exclusive_i64(panther_ctx* ctx, int64_t* data, int64_t n);

// the index's per-vertex path-count classes (cls, cls_hist) from its offsets
panther_status index_classes(panther_ctx* ctx, panther_index* ix);

// One-byte code of a path count x = |P_v|, monotone in x: x itself below 128,
// then 8 steps per doubling (leading bit and the 3 bits after it), 255 from
// 15 * 2^19 on. code(x) >= c exactly when x >= code_floor(c), so a filter
// "code >= c" keeps every vertex with at least code_floor(c) paths and drops
// only vertices with fewer.
__host__ __device__ inline uint32_t path_code(int64_t x) {
    if (x < 128) return x < 0 ? 0u : (uint32_t)x;
    int e = 0;
    while ((x >> (e + 1)) != 0) ++e;          // leading bit, >= 7
    if (e > 22) return 255u;
    return 128u + 8u * (uint32_t)(e - 7) + ((uint32_t)(x >> (e - 3)) & 7u);
}

__host__ __device__ inline int64_t code_floor(uint32_t c) {
    if (c < 128) return c;
    const uint32_t e = 7 + (c - 128) / 8, m = (c - 128) % 8;
    return (int64_t)(8 + m) << (e - 3);
}

// ---------------------------------------------------------- device helpers ---
#ifdef __CUDACC__

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// 4x32 S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key bumps
// 0x9E3779B9 / 0xBB67AE85.
struct pword4 { uint32_t x, y, z, w; };

__device__ __forceinline__ pword4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        uint32_t a = hi1 ^ c1 ^ k0, b = lo1, c = hi0 ^ c3 ^ k1, d = lo0;
        c0 = a; c1 = b; c2 = c; c3 = d;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// draw (r, t, attempt) of the path stream
__device__ __forceinline__ pword4 path_draw(uint64_t seed, uint64_t r, uint32_t t, uint32_t attempt) {
    return philox10((uint32_t)r, (uint32_t)(r >> 32), t, attempt, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Lemire multiply-shift: true and *out = floor(U*S / 2^64) unless rejected.
__device__ __forceinline__ bool lemire64(uint64_t U, uint64_t S, uint64_t* out) {
    uint64_t lo = U * S;
    uint64_t hi = __umul64hi(U, S);
    if (lo < S) {
        uint64_t thr = (0ull - S) % S;
        if (lo < thr) return false;
    }
    *out = hi;
    return true;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ void flag_status(uint32_t* st, uint32_t bit) { atomicOr(st, bit); }

#endif  // __CUDACC__
