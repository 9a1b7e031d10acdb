// Co-occurrence counting and top-k (Algorithm 1, Eq. (4)).
//
// For query v every path r in P_v contributes 1 to cnt(v,u) for each distinct
// u != v on the path. Counts accumulate in an open-addressing hash of 64-bit
// slots (vertex << 32 | count); a slot is claimed with one 64-bit CAS and
// bumped with one 64-bit add. The top-k by (count desc, id asc) is the k
// largest of score = count << 32 | (2^32 - 1 - id), kept as a sorted list
// spread over a warp's registers (rank l in lane l, rank 32+l in lane l's
// second register) and merged across warps through shared memory.
//
// Queries are split by the bound cap = min(n-1, |P_v| * T) on their distinct
// candidates:
//   warp tier  (cap <= 256):      a warp-private 512-slot table in smem
//   CTA tier   (cap <= CTA cap):  one CTA, a table filling most of smem
//   global tier (larger):         a table in device memory, filled by many
//                                 CTAs, read back in chunks, partial top-k
//                                 lists merged per query
// The warp and CTA tiers run in ONE persistent launch whose CTAs pull work
// from device counters (CTA-tier queries first, then warp-tier queries in
// chunks), so skewed |P_v| does not leave SMs idle.
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace {

constexpr uint64_t EMPTY = ~0ull;
// path ids are unsigned 32-bit (R <= 2^32 - 1, so no valid id is all ones);
// lanes without a path pass NO_PATH, which every reader rejects with r >= R
constexpr uint32_t NO_PATH = 0xffffffffu;
constexpr int WSLOTS = 512;      // warp-tier table slots
constexpr int WCAP = 256;        // warp-tier candidate bound
// A query's own path count bounds the work of the tier that takes it: one
// warp (warp tier) or one CTA (CTA tiers) walks every path of P_v, so a query
// with few candidates but more paths than these (a small graph with a large
// R) goes to a wider tier, and beyond CTA_MAX_NP to the hub tier, which
// splits P_v over many CTAs.
constexpr int64_t WARP_MAX_NP = int64_t(1) << 16;
constexpr int64_t CTA_MAX_NP = int64_t(1) << 20;
constexpr int KMAX = 64;
constexpr int WCHUNK = 16;       // warp-tier queries fetched per atomic

__device__ __forceinline__ uint32_t hslot(uint32_t key, uint32_t nslots) {
    return __umulhi(key * 0x9E3779B1u ^ (key >> 15), nslots);
}

// add `amount` to the count of `key`; returns false if the table is full
template <bool SHARED>
__device__ __forceinline__ bool hash_add(unsigned long long* tab, uint32_t nslots, uint32_t key,
                                         uint32_t amount = 1) {
    uint32_t s = hslot(key, nslots);
    for (uint32_t probe = 0; probe < nslots; ++probe) {
        unsigned long long cur = tab[s];
        if ((uint32_t)(cur >> 32) == key && cur != EMPTY) {
            atomicAdd(&tab[s], (unsigned long long)amount);
            return true;
        }
        if (cur == EMPTY) {
            unsigned long long prev = atomicCAS(&tab[s], EMPTY, ((unsigned long long)key << 32) | amount);
            if (prev == EMPTY) return true;
            if ((uint32_t)(prev >> 32) == key) {
                atomicAdd(&tab[s], (unsigned long long)amount);
                return true;
            }
        }
        s = (s + 1 == nslots) ? 0 : s + 1;
    }
    return false;
}

// table size for a query whose distinct candidates are at most cap: about
// twice cap, a multiple of 32, within [lo, hi]
__device__ __forceinline__ uint32_t table_size(int64_t cap, uint32_t lo, uint32_t hi) {
    int64_t t = ((2 * cap + 31) / 32) * 32;
    return (uint32_t)(t < lo ? lo : (t > hi ? hi : t));
}

// ------------------------------------------------------ warp top-k list ---
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }
__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

struct WarpTopK {
    uint64_t a = 0, b = 0;   // ranks lane and 32+lane, descending; 0 = empty
    __device__ __forceinline__ uint64_t kth(int k) const {
        return k <= 32 ? __shfl_sync(0xffffffffu, a, k - 1) : __shfl_sync(0xffffffffu, b, k - 33);
    }
    __device__ __forceinline__ void insert(uint64_t x) {
        unsigned lane = threadIdx.x & 31;
        int pos = __popc(__ballot_sync(0xffffffffu, a > x)) + __popc(__ballot_sync(0xffffffffu, b > x));
        uint64_t au = __shfl_up_sync(0xffffffffu, a, 1);
        uint64_t bu = __shfl_up_sync(0xffffffffu, b, 1);
        uint64_t a31 = __shfl_sync(0xffffffffu, a, 31);
        if (lane == 0) bu = a31;
        int ra = (int)lane, rb = 32 + (int)lane;
        uint64_t na = ra < pos ? a : (ra == pos ? x : au);
        uint64_t nb = rb < pos ? b : (rb == pos ? x : bu);
        a = na;
        b = nb;
    }
    // merge another descending 64-list (xa, xb) in: the top 64 of the union,
    // by one bitonic half-cleaner cascade (keys are distinct or 0)
    __device__ __forceinline__ void merge(uint64_t xa, uint64_t xb) {
        unsigned lane = threadIdx.x & 31;
        uint64_t ra = __shfl_sync(0xffffffffu, xb, 31 - lane);
        uint64_t rb = __shfl_sync(0xffffffffu, xa, 31 - lane);
        uint64_t za = umax64(a, ra), zb = umax64(b, rb);
        a = umax64(za, zb);
        b = umin64(za, zb);
#pragma unroll
        for (int d = 16; d; d >>= 1) {
            uint64_t pa = __shfl_xor_sync(0xffffffffu, a, d);
            uint64_t pb = __shfl_xor_sync(0xffffffffu, b, d);
            bool upper = lane & d;
            a = upper ? umin64(a, pa) : umax64(a, pa);
            b = upper ? umin64(b, pb) : umax64(b, pb);
        }
    }
    // offer one candidate per lane (0 = none)
    __device__ __forceinline__ void offer(uint64_t c, int k) {
        uint64_t thr = kth(k);
        unsigned m = __ballot_sync(0xffffffffu, c > thr);
        if (__popc(m) > 2) {
            // many pass: sort the 32 candidates (descending bitonic sort) and merge
            unsigned lane = threadIdx.x & 31;
#pragma unroll
            for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    uint64_t pc = __shfl_xor_sync(0xffffffffu, c, j);
                    bool desc = (lane & kk) == 0 || kk == 32;
                    bool lower = (lane & j) == 0;
                    c = (lower == desc) ? umax64(c, pc) : umin64(c, pc);
                }
            }
            merge(c, 0);
            return;
        }
        while (m) {
            int src = __ffs(m) - 1;
            uint64_t x = __shfl_sync(0xffffffffu, c, src);
            insert(x);
            m &= m - 1;
            thr = kth(k);
            m &= __ballot_sync(0xffffffffu, c > thr);
        }
    }
};

// Bitonic sort, descending, of the 64 keys (a, b) of a warp: key a of lane l
// has rank l, key b rank 32 + l once sorted.
__device__ __forceinline__ void warp_sort64_desc(uint64_t& a, uint64_t& b) {
    const unsigned lane = threadIdx.x & 31;
#pragma unroll
    for (int kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j == 32) {
                // partners a (index lane) and b (index 32 + lane) in the same lane
                const bool desc = (lane & kk) == 0;     // kk == 64: always
                const uint64_t hi = umax64(a, b), lo = umin64(a, b);
                a = desc ? hi : lo;
                b = desc ? lo : hi;
            } else {
                const uint64_t pa = __shfl_xor_sync(0xffffffffu, a, j);
                const uint64_t pb = __shfl_xor_sync(0xffffffffu, b, j);
                const bool lower = (lane & j) == 0;
                const bool da = kk == 64 || (lane & kk) == 0;
                const bool db = kk == 64 || ((32 + lane) & kk) == 0;
                a = (lower == da) ? umax64(a, pa) : umin64(a, pa);
                b = (lower == db) ? umax64(b, pb) : umin64(b, pb);
            }
        }
    }
}

// merge the lists of all warps of the CTA into warp 0 (log-depth tree);
// `lists` holds 64 entries per warp; every thread of the CTA must call it
__device__ __forceinline__ void cta_merge(WarpTopK& t, unsigned long long* lists) {
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31;
    for (int s = 1; s < nw; s <<= 1) {
        if ((w & (2 * s - 1)) == s) {
            lists[w * KMAX + lane] = t.a;
            lists[w * KMAX + 32 + lane] = t.b;
        }
        __syncthreads();
        if ((w & (2 * s - 1)) == 0 && w + s < nw) t.merge(lists[(w + s) * KMAX + lane], lists[(w + s) * KMAX + 32 + lane]);
        __syncthreads();
    }
}

__device__ __forceinline__ uint64_t slot_score(unsigned long long s) {
    if (s == EMPTY) return 0;
    uint32_t key = (uint32_t)(s >> 32), cnt = (uint32_t)s;
    return ((uint64_t)cnt << 32) | (uint64_t)(0xffffffffu - key);
}

// Top-k of a warp-private table of ns slots (ns a multiple of 32). With at
// most 64 filled slots they are compacted in place and sorted once; otherwise
// every slot is offered to a running list. The table is garbage afterwards.
__device__ __forceinline__ WarpTopK warp_table_topk(unsigned long long* tab, uint32_t ns, int k) {
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    int filled = 0;
    for (uint32_t base = 0; base < ns; base += 32)
        filled += __popc(__ballot_sync(0xffffffffu, tab[base + lane] != EMPTY));
    WarpTopK t;
    if (filled > 64) {
        for (uint32_t base = 0; base < ns; base += 32) t.offer(slot_score(tab[base + lane]), k);
        return t;
    }
    uint64_t mine[2] = {0, 0};
    int pos = 0;
    for (uint32_t base = 0; base < ns; base += 32) {
        const uint64_t sc = slot_score(tab[base + lane]);
        const unsigned m = __ballot_sync(0xffffffffu, sc != 0);
        const int at = pos + __popc(m & lt);
        // every lane read its slot before the ballot, and at < base + 32
        if (sc) tab[at] = sc;
        pos += __popc(m);
    }
    __syncwarp();
    mine[0] = lane < (unsigned)filled ? tab[lane] : 0;
    mine[1] = 32 + lane < (unsigned)filled ? tab[32 + lane] : 0;
    warp_sort64_desc(mine[0], mine[1]);
    t.a = mine[0];
    t.b = mine[1];
    return t;
}

struct OutRef {
    int32_t* ids;       // [q][k] or null
    uint32_t* cnt;      // [q][k]
    int k;
};

__device__ __forceinline__ void write_list(const WarpTopK& t, const OutRef& o, int64_t qi) {
    unsigned lane = threadIdx.x & 31;
    for (int half = 0; half < 2; ++half) {
        int r = (int)lane + 32 * half;
        uint64_t s = half ? t.b : t.a;
        if (r < o.k) {
            int64_t at = qi * o.k + r;
            if (o.ids) o.ids[at] = s ? (int32_t)(0xffffffffu - (uint32_t)s) : -1;
            o.cnt[at] = (uint32_t)(s >> 32);
        }
    }
}

// ------------------------------------------- 128-entry lists (k > 64) ---
// The same descending list with four registers per lane (ranks l, 32+l,
// 64+l, 96+l), for 64 < k <= 128. Used only by the device-table selection.
constexpr int KMAX4 = 128;

struct WarpTopK4 {
    uint64_t r[4] = {0, 0, 0, 0};
    __device__ __forceinline__ uint64_t kth(int k) const {
        const int q = (k - 1) >> 5, l = (k - 1) & 31;
        const uint64_t x = q == 0 ? r[0] : (q == 1 ? r[1] : (q == 2 ? r[2] : r[3]));
        return __shfl_sync(0xffffffffu, x, l);
    }
    __device__ __forceinline__ void insert(uint64_t x) {
        const unsigned lane = threadIdx.x & 31;
        int pos = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) pos += __popc(__ballot_sync(0xffffffffu, r[j] > x));
        uint64_t up[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) up[j] = __shfl_up_sync(0xffffffffu, r[j], 1);
#pragma unroll
        for (int j = 3; j >= 1; --j) {
            const uint64_t carry = __shfl_sync(0xffffffffu, r[j - 1], 31);
            if (lane == 0) up[j] = carry;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int rank = 32 * j + (int)lane;
            r[j] = rank < pos ? r[j] : (rank == pos ? x : up[j]);
        }
    }
    // merge another descending 128-list in: the top 128 of the union (keys are
    // distinct or 0): reverse the other list, take elementwise maxima (a
    // bitonic sequence), then half-cleaners at distances 64, 32, 16 .. 1
    __device__ __forceinline__ void merge(const uint64_t (&x)[4]) {
        const unsigned lane = threadIdx.x & 31;
#pragma unroll
        for (int j = 0; j < 4; ++j) r[j] = umax64(r[j], __shfl_sync(0xffffffffu, x[3 - j], 31 - lane));
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const uint64_t hi = umax64(r[j], r[j + 2]), lo = umin64(r[j], r[j + 2]);
            r[j] = hi;
            r[j + 2] = lo;
        }
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
            const uint64_t hi = umax64(r[j], r[j + 1]), lo = umin64(r[j], r[j + 1]);
            r[j] = hi;
            r[j + 1] = lo;
        }
#pragma unroll
        for (int d = 16; d; d >>= 1) {
            const bool upper = lane & d;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t p = __shfl_xor_sync(0xffffffffu, r[j], d);
                r[j] = upper ? umin64(r[j], p) : umax64(r[j], p);
            }
        }
    }
    // offer one candidate per lane (0 = none)
    __device__ __forceinline__ void offer(uint64_t c, int k) {
        uint64_t thr = kth(k);
        unsigned m = __ballot_sync(0xffffffffu, c > thr);
        if (__popc(m) > 2) {
            const unsigned lane = threadIdx.x & 31;
#pragma unroll
            for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    const uint64_t pc = __shfl_xor_sync(0xffffffffu, c, j);
                    const bool desc = (lane & kk) == 0 || kk == 32;
                    const bool lower = (lane & j) == 0;
                    c = (lower == desc) ? umax64(c, pc) : umin64(c, pc);
                }
            }
            const uint64_t x[4] = {c, 0, 0, 0};
            merge(x);
            return;
        }
        while (m) {
            const int src = __ffs(m) - 1;
            insert(__shfl_sync(0xffffffffu, c, src));
            m &= m - 1;
            thr = kth(k);
            m &= __ballot_sync(0xffffffffu, c > thr);
        }
    }
};

// merge the 128-lists of all warps of the CTA into warp 0 (log-depth tree);
// `lists` holds 128 entries per warp; every thread of the CTA must call it
__device__ __forceinline__ void cta_merge4(WarpTopK4& t, unsigned long long* lists) {
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31;
    for (int s = 1; s < nw; s <<= 1) {
        if ((w & (2 * s - 1)) == s)
#pragma unroll
            for (int j = 0; j < 4; ++j) lists[w * KMAX4 + 32 * j + lane] = t.r[j];
        __syncthreads();
        if ((w & (2 * s - 1)) == 0 && w + s < nw) {
            uint64_t x[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = lists[(w + s) * KMAX4 + 32 * j + lane];
            t.merge(x);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void write_list4(const WarpTopK4& t, const OutRef& o, int64_t qi) {
    const unsigned lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int rk = (int)lane + 32 * j;
        const uint64_t sc = t.r[j];
        if (rk < o.k) {
            const int64_t at = qi * o.k + rk;
            if (o.ids) o.ids[at] = sc ? (int32_t)(0xffffffffu - (uint32_t)sc) : -1;
            o.cnt[at] = (uint32_t)(sc >> 32);
        }
    }
}

// ------------------------------------------------------ path insertion ---
struct PathsRef {
    const int32_t* rows;
    int64_t R;
    int L;
    const int64_t* off;
    const uint32_t* pid;
    int64_t n;
    const uint8_t* cls;   // path_code(|P_u|) per vertex
};

// insert the distinct vertices u != v of path r into the table (with thr > 0
// only the u with cls[u] >= thr)
template <int STRIDE, bool SHARED>
__device__ __forceinline__ bool insert_path(const PathsRef& P, uint32_t r, int32_t v, unsigned long long* tab,
                                            uint32_t nslots, uint32_t thr = 0) {
    if (r >= (uint64_t)P.R) return false;             // corrupt index entry: the caller flags it, nothing is read
    int32_t x[STRIDE];
    const int4* src = (const int4*)(P.rows + (uint64_t)r * STRIDE);
#pragma unroll
    for (int k = 0; k < STRIDE / 4; ++k) {
        int4 q = __ldg(src + k);
        x[4 * k] = q.x; x[4 * k + 1] = q.y; x[4 * k + 2] = q.z; x[4 * k + 3] = q.w;
    }
    bool ok = true;
#pragma unroll
    for (int j = 0; j < STRIDE; ++j) {
        if (j < P.L && x[j] != v) {
            bool dup = false;
#pragma unroll
            for (int i = 0; i < j; ++i) dup |= (x[i] == x[j]);
            if (!dup && (thr == 0 || __ldg(P.cls + x[j]) >= thr)) ok &= hash_add<SHARED>(tab, nslots, (uint32_t)x[j]);
        }
    }
    return ok;
}

// ----------------------------------------------------------- lane tier ---
// Queries touching at most LANE_NP paths (T <= 7): one thread per query. The
// rows sit in registers; every distinct u != v is counted at its first
// occurrence by comparing against the later rows, and the k best scores are
// kept in a register list sorted by insertion.
constexpr int LANE_NP = 6;
constexpr int LANE_K = 16;

// does one of the first LP entries of row r hold u?
template <int LP>
__device__ __forceinline__ bool row_has(const int32_t (&r)[8], int32_t u) {
    bool h = false;
#pragma unroll
    for (int j = 0; j < LP; ++j) h |= (r[j] == u);
    return h;
}

// Scores: count high, ascending id low. NARROW packs them in 32 bits (ids
// below 2^29: counts here are at most LANE_NP < 8), else in 64.
template <bool NARROW>
struct LaneScore {
    using T = typename std::conditional<NARROW, uint32_t, uint64_t>::type;
    static __device__ __forceinline__ T make(uint32_t c, int32_t u) {
        if (NARROW) return (T)((c << 29) | ((1u << 29) - 1u - (uint32_t)u));
        return (T)(((uint64_t)c << 32) | (uint64_t)(0xffffffffu - (uint32_t)u));
    }
    static __device__ __forceinline__ int32_t id(T s) {
        if (NARROW) return (int32_t)((1u << 29) - 1u - ((uint32_t)s & ((1u << 29) - 1u)));
        return (int32_t)(0xffffffffu - (uint32_t)s);
    }
    static __device__ __forceinline__ uint32_t count(T s) { return NARROW ? (uint32_t)s >> 29 : (uint32_t)((uint64_t)s >> 32); }
};

// LP: the row positions compared (T+1 = 6, the paper's T = 5, or all 8 with
// the positions past T+1 masked); KP: the length of the running list (k <= KP)
template <bool NARROW, int LP, int KP>
__global__ void __launch_bounds__(256, NARROW ? 3 : 2) lane_kernel(PathsRef P, const int32_t* __restrict__ queries,
                                                   const int32_t* __restrict__ list, const int* __restrict__ count,
                                                   int slot, OutRef o) {
    using LS = LaneScore<NARROW>;
    using T = typename LS::T;
    const int n = count[slot];
    const int stride = gridDim.x * blockDim.x;
    int it = blockIdx.x * blockDim.x + threadIdx.x;
    // the next query's vertex and path range are fetched one query ahead
    int32_t nv = 0;
    int64_t na = 0, nb = 0;
    if (it < n) {
        nv = queries ? queries[list[it]] : list[it];
        na = P.off[nv];
        nb = P.off[nv + 1];
    }
    for (; it < n; it += stride) {
        const int64_t qi = list[it];
        const int32_t v = nv;
        const int64_t a = na;
        const int np = (int)(nb - na);
        int32_t row[LANE_NP][8];
#pragma unroll
        for (int i = 0; i < LANE_NP; ++i) {
            const uint32_t r = i < np ? P.pid[a + i] : NO_PATH;
            if (r < (uint64_t)P.R) {
                const int4* src = (const int4*)(P.rows + (uint64_t)r * 8);
                int4 x = __ldg(src), y = __ldg(src + 1);
                row[i][0] = x.x; row[i][1] = x.y; row[i][2] = x.z; row[i][3] = x.w;
                row[i][4] = y.x; row[i][5] = y.y; row[i][6] = y.z; row[i][7] = y.w;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) row[i][j] = -1;
            }
            // positions past the path length never count (rows are padded with -1)
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j >= P.L) row[i][j] = -1;
        }
        if (it + stride < n) {
            nv = queries ? queries[list[it + stride]] : list[it + stride];
            na = P.off[nv];
            nb = P.off[nv + 1];
        }
        T best[KP];
#pragma unroll
        for (int t = 0; t < KP; ++t) best[t] = 0;
#pragma unroll
        for (int i = 0; i < LANE_NP; ++i) {
#pragma unroll
            for (int j = 0; j < LP; ++j) {
                const int32_t u = row[i][j];
                bool first = u >= 0 && u != v;
#pragma unroll
                for (int jj = 0; jj < j; ++jj) first &= row[i][jj] != u;
#pragma unroll
                for (int ii = 0; ii < i; ++ii) first &= !row_has<LP>(row[ii], u);
                if (first) {
                    uint32_t c = 1;
#pragma unroll
                    for (int ii = i + 1; ii < LANE_NP; ++ii) c += row_has<LP>(row[ii], u) ? 1u : 0u;
                    T sc = LS::make(c, u);
                    // sorted insertion (descending)
#pragma unroll
                    for (int t = 0; t < KP; ++t) {
                        T hi = best[t] > sc ? best[t] : sc;
                        T lo = best[t] > sc ? sc : best[t];
                        best[t] = hi;
                        sc = lo;
                    }
                }
            }
        }
#pragma unroll
        for (int t = 0; t < KP; ++t) {
            if (t < o.k) {
                const T sc = best[t];
                if (o.ids) o.ids[qi * o.k + t] = sc ? LS::id(sc) : -1;
                o.cnt[qi * o.k + t] = LS::count(sc);
            }
        }
    }
}

// Warp-convergent insertion: every lane of the warp calls these together
// (`active` marks the lanes with something to insert); the probe loop runs
// while any lane is still probing, so the warp never splits into nested
// divergent branches.
__device__ __forceinline__ bool hash_add_conv(unsigned long long* tab, uint32_t nslots, uint32_t key,
                                              uint32_t amount, bool active) {
    uint32_t s = active ? hslot(key, nslots) : 0;
    bool pending = active, ok = true;
    uint32_t probes = 0;
    while (__any_sync(0xffffffffu, pending)) {
        if (pending) {
            unsigned long long cur = tab[s];
            bool mine = cur != EMPTY && (uint32_t)(cur >> 32) == key;
            if (cur == EMPTY) {
                unsigned long long prev = atomicCAS(&tab[s], EMPTY, ((unsigned long long)key << 32) | amount);
                if (prev == EMPTY) pending = false;
                else mine = (uint32_t)(prev >> 32) == key;
            }
            if (mine) {
                atomicAdd(&tab[s], (unsigned long long)amount);
                pending = false;
            }
            if (pending) {
                s = (s + 1 == nslots) ? 0 : s + 1;
                if (++probes >= nslots) {
                    pending = false;
                    ok = false;
                }
            }
        }
    }
    return ok;
}

// Rows of 64 or 128 entries (T >= 32): the warp takes its lanes' paths one
// at a time. Lane l holds entries l, l+32, ... of the row (one coalesced
// 128-byte load per round); an entry is a candidate at its first occurrence
// in the row (no lower lane of its round, no lane of an earlier round holds
// it) and if it is not v; with thr > 0 only the u with cls[u] >= thr.
// Returns false if a table ran out of slots. Every lane must call it.
template <int STRIDE>
__device__ __forceinline__ bool insert_paths_warp(const PathsRef& P, uint32_t r, int32_t v, unsigned long long* tab,
                                                  uint32_t nslots, bool active, uint32_t thr) {
    constexpr int NR = STRIDE / 32;
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    active &= r < (uint64_t)P.R;
    unsigned pend = __ballot_sync(0xffffffffu, active);
    bool ok = true;
    while (pend) {                                        // warp-uniform
        const int src = __ffs(pend) - 1;
        pend &= pend - 1;
        const uint32_t rr = __shfl_sync(0xffffffffu, r, src);
        const int32_t* row = P.rows + (uint64_t)rr * STRIDE;
        int32_t y[NR];
#pragma unroll
        for (int m = 0; m < NR; ++m) y[m] = __ldg(row + m * 32 + lane);
#pragma unroll
        for (int m = 0; m < NR; ++m) {
            if (m * 32 >= P.L) break;                     // warp-uniform: the rest is padding
            bool take = m * 32 + (int)lane < P.L && y[m] != v;
            take &= (__match_any_sync(0xffffffffu, y[m]) & lt) == 0;
#pragma unroll
            for (int mm = 0; mm < m; ++mm)
#pragma unroll 8
                for (int sl = 0; sl < 32; ++sl) take &= __shfl_sync(0xffffffffu, y[mm], sl) != y[m];
            if (thr && take) take = __ldg(P.cls + y[m]) >= thr;
            if (__any_sync(0xffffffffu, take)) ok &= hash_add_conv(tab, nslots, (uint32_t)y[m], 1u, take);
        }
    }
    return ok;
}

// insert the distinct vertices u != v of path r (lanes with active == false pass NO_PATH);
// with thr > 0 only the u with cls[u] >= thr
template <int STRIDE>
__device__ __forceinline__ bool insert_path_conv(const PathsRef& P, uint32_t r, int32_t v, unsigned long long* tab,
                                                 uint32_t nslots, bool active, uint32_t thr = 0) {
    if constexpr (STRIDE > 32) return insert_paths_warp<STRIDE>(P, r, v, tab, nslots, active, thr);
    active &= r < (uint64_t)P.R;
    int32_t x[STRIDE];
    const int4* src = (const int4*)(P.rows + (uint64_t)(active ? r : 0u) * STRIDE);
#pragma unroll
    for (int k = 0; k < STRIDE / 4; ++k) {
        int4 q = active ? __ldg(src + k) : make_int4(-1, -1, -1, -1);
        x[4 * k] = q.x; x[4 * k + 1] = q.y; x[4 * k + 2] = q.z; x[4 * k + 3] = q.w;
    }
    bool ok = true;
#pragma unroll
    for (int j = 0; j < STRIDE; ++j) {
        bool take = active && j < P.L && x[j] != v;
#pragma unroll
        for (int i = 0; i < j; ++i) take &= (x[i] != x[j]);
        if (thr && take) take = __ldg(P.cls + x[j]) >= thr;
        if (__any_sync(0xffffffffu, take)) ok &= hash_add_conv(tab, nslots, (uint32_t)x[j], 1u, take);
    }
    return ok;
}


// --------------------------------------------------------- group tiers ---
// Queries with 7..32 paths (T <= 7, ids below 2^group_ub(G)): a group of
// G = 8, 16 or 32 lanes per query, lane j holding path j of P_v in 8
// registers, so a warp serves 32/G queries at once with no table. Each entry
// u != v becomes the key u << log2(G) | j; the G*8 keys are bitonic-sorted
// across the group, the number of distinct rows in each run of equal u is its
// count (a path that visits u twice gives two equal keys and counts once),
// and the run ends carry the scores count << group_ub(G) | reversed id,
// sorted again, descending.
__host__ __device__ constexpr int group_ub(int G) { return G == 32 ? 26 : 27; }   // count <= G fits above
__host__ __device__ constexpr int group_rb(int G) { return G == 8 ? 3 : (G == 16 ? 4 : 5); }

// bitonic sort of the 8*G keys of a group (element gl*8 + r is register r of
// group lane gl); ascending or descending
template <int G, bool ASC>
__device__ __forceinline__ void group_sort(uint32_t (&x)[8], unsigned gl) {
#pragma unroll
    for (int kk = 2; kk <= 8 * G; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j >= 8) {
                const unsigned lj = (unsigned)(j >> 3);
                const bool lower = (gl & lj) == 0;
                const bool up = kk == 8 * G || ((gl * 8) & (unsigned)kk) == 0;
                const bool take_min = (lower == up) == ASC;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const uint32_t p = __shfl_xor_sync(0xffffffffu, x[r], lj);
                    x[r] = take_min ? min(x[r], p) : max(x[r], p);
                }
            } else {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    if (r & j) continue;
                    const unsigned e = gl * 8 + (unsigned)r;
                    const bool up = kk == 8 * G || (e & (unsigned)kk) == 0;
                    const uint32_t lo = min(x[r], x[r + j]), hi = max(x[r], x[r + j]);
                    x[r] = (up == ASC) ? lo : hi;
                    x[r + j] = (up == ASC) ? hi : lo;
                }
            }
        }
    }
}

template <int G>
__global__ void __launch_bounds__(256) group_kernel(PathsRef P, const int32_t* __restrict__ queries,
                                                    const int32_t* __restrict__ list, const int* __restrict__ count,
                                                    int slot, OutRef o) {
    const int n = count[slot];
    const unsigned lane = threadIdx.x & 31, gl = lane & (G - 1);
    const int64_t ngroups = (int64_t)gridDim.x * blockDim.x / G;
    constexpr int UB = group_ub(G), RB = group_rb(G);
    constexpr uint32_t UMASK = (1u << UB) - 1u;
    // G >= 16: the scores above c* of each group (fewer than k <= 128),
    // gathered for ranking
    __shared__ uint32_t gbuf[G >= 16 ? 256 / G : 1][KMAX4];
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(unsigned)(G - 1)));
    for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;; it += ngroups) {
        const bool active = it < n;
        if (!__any_sync(0xffffffffu, active)) break;   // warp-uniform: the whole warp shuffles together
        int64_t qi = 0;
        int32_t v = -1;
        int np = 0;
        int64_t a = 0;
        if (active) {
            qi = list[it];
            v = queries ? queries[qi] : (int32_t)qi;
            a = P.off[v];
            np = (int)(P.off[v + 1] - a);
        }
        uint32_t x[8];
        {
            const uint32_t r = (int)gl < np ? P.pid[a + gl] : NO_PATH;
            int4 q0 = make_int4(-1, -1, -1, -1), q1 = q0;
            if (r < (uint64_t)P.R) {
                const int4* src = (const int4*)(P.rows + (uint64_t)r * 8);
                q0 = __ldg(src);
                q1 = __ldg(src + 1);
            }
            const int32_t y[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const bool ok = p < P.L && y[p] >= 0 && y[p] != v;
                x[p] = ok ? ((uint32_t)y[p] << RB) | gl : 0xffffffffu;
            }
        }
        group_sort<G, true>(x, gl);
        // run ends and the number of distinct rows per run of equal u
        const uint32_t prev7 = __shfl_up_sync(0xffffffffu, x[7], 1);
        const uint32_t next0 = __shfl_down_sync(0xffffffffu, x[0], 1);
        uint32_t c[8];
        unsigned lane_reset = 0;   // bit r: element r starts a new u
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint32_t pk = r ? x[r - 1] : (gl ? prev7 : 0xfffffffeu);
            const bool new_u = (x[r] >> RB) != (pk >> RB) || (r == 0 && gl == 0);
            const uint32_t d = (x[r] != pk || (r == 0 && gl == 0)) ? 1u : 0u;
            c[r] = (r == 0 || new_u) ? d : c[r - 1] + d;
            if (new_u) lane_reset |= 1u << r;
        }
        // carry the running count across lanes until a lane that starts a new u
        uint32_t carry = 0;   // distinct rows of the run that continues into this lane
        {
            // (total after the last reset, whether the lane resets) scanned over the group
            uint32_t t = c[7];
            bool f = lane_reset != 0;
#pragma unroll
            for (int d = 1; d < G; d <<= 1) {
                const uint32_t pt = __shfl_up_sync(0xffffffffu, t, d);
                const bool pf = __shfl_up_sync(0xffffffffu, f ? 1u : 0u, d) != 0;
                if (gl >= (unsigned)d && !f) {
                    t += pt;
                    f = pf;
                }
            }
            // exclusive: the inclusive value of the previous lane
            const uint32_t pt = __shfl_up_sync(0xffffffffu, t, 1);
            carry = gl ? pt : 0;
        }
        uint32_t sc[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const uint32_t cnt = ((lane_reset & ((2u << r) - 1u)) == 0) ? c[r] + carry : c[r];
            const uint32_t nk = r < 7 ? x[r + 1] : (gl + 1 < (unsigned)G ? next0 : 0xffffffffu);
            const bool last = (x[r] >> RB) != (nk >> RB) || (r == 7 && gl + 1 == (unsigned)G);
            const uint32_t u = x[r] >> RB;
            sc[r] = (last && x[r] != 0xffffffffu) ? (cnt << UB) | (UMASK - u) : 0u;
        }
        if constexpr (G >= 16) {
            // Ranks without a second sort. The run ends lie in ascending u,
            // the order that breaks ties. c* = the k-th largest count (1 when
            // fewer than k ends have a count of 2 or more); the g < k ends
            // above c* are gathered and ranked by comparison, the ends at c*
            // take ranks g, g+1, ... in their order.
            auto at_least = [&](uint32_t c) {
                int s = 0;
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    s += __popc(__ballot_sync(0xffffffffu, sc[r] != 0u && (sc[r] >> UB) >= c) & gmask);
                return s;
            };
            uint32_t cstar = 1;
            if (__any_sync(0xffffffffu, at_least(2) >= o.k)) {            // warp-uniform
                constexpr int CB = G == 32 ? 6 : 5;                         // counts <= G
                uint32_t cs = 0;
#pragma unroll
                for (int bit = CB - 1; bit >= 0; --bit)
                    if (at_least(cs | (1u << bit)) >= o.k) cs |= 1u << bit;
                cstar = cs > 1u ? cs : 1u;
            }
            // exclusive prefix over the group's lanes of a per-lane count
            auto group_excl = [&](uint32_t v) {
                uint32_t x = v;
#pragma unroll
                for (int d = 1; d < G; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d, G);
                    if ((int)gl >= d) x += y;
                }
                return x - v;
            };
            uint32_t ngt = 0, neq = 0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const uint32_t c = sc[r] >> UB;
                ngt += (sc[r] != 0u && c > cstar) ? 1u : 0u;
                neq += (sc[r] != 0u && c == cstar) ? 1u : 0u;
            }
            uint32_t pgt = group_excl(ngt), peq = group_excl(neq);
            const uint32_t g = __shfl_sync(0xffffffffu, pgt + ngt, G - 1, G);      // ends above c*
            const uint32_t tot = g + __shfl_sync(0xffffffffu, peq + neq, G - 1, G);
            uint32_t* buf = gbuf[(threadIdx.x & 255) / G];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const uint32_t c = sc[r] >> UB;
                if (sc[r] != 0u && c > cstar) buf[pgt++] = sc[r];          // g < k <= KMAX4 entries
                if (active && sc[r] != 0u && c == cstar) {
                    const uint32_t rank = g + peq++;
                    if ((int)rank < o.k) {
                        if (o.ids) o.ids[qi * o.k + rank] = (int32_t)(UMASK - (sc[r] & UMASK));
                        o.cnt[qi * o.k + rank] = c;
                    }
                }
            }
            __syncwarp();
            if (active) {
                for (uint32_t i = gl; i < g; i += G) {
                    const uint32_t s = buf[i];
                    uint32_t rank = 0;
                    for (uint32_t j = 0; j < g; ++j) rank += buf[j] > s ? 1u : 0u;
                    if (o.ids) o.ids[qi * o.k + rank] = (int32_t)(UMASK - (s & UMASK));
                    o.cnt[qi * o.k + rank] = s >> UB;
                }
                for (int e = (int)tot + (int)gl; e < o.k; e += G) {              // fewer than k ends: padding
                    if (o.ids) o.ids[qi * o.k + e] = -1;
                    o.cnt[qi * o.k + e] = 0;
                }
            }
            __syncwarp();
        } else {
            group_sort<G, false>(sc, gl);
            if (active) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int e = (int)gl * 8 + r;
                    if (e < o.k) {
                        if (o.ids) o.ids[qi * o.k + e] = sc[r] ? (int32_t)(UMASK - (sc[r] & UMASK)) : -1;
                        o.cnt[qi * o.k + e] = sc[r] >> UB;
                    }
                }
                for (int e = 8 * G + (int)gl; e < o.k; e += G) {   // k beyond the group's 8G ranks: padding
                    if (o.ids) o.ids[qi * o.k + e] = -1;
                    o.cnt[qi * o.k + e] = 0;
                }
            }
        }
    }
}

struct Tiers {
    int32_t* list[8];    // query indices per tier: warp, CTA, global, lane, groups of 8, 16, 32, big CTA
    int* count;          // [0..2] warp/CTA/global sizes, [3..4] fetch counters (warp, CTA), [5..8] lane,
                         // g8/16/32 sizes; [9..13] the same layout as [0..4] for the big-CTA pass
};

// classification: pads trivially empty queries and sorts the rest into tiers.
// A CTA classifies CL_PER queries per thread (strided by the block size, so
// loads and stores are coalesced) and reserves space in each tier list with
// one global atomic per tier, after counting in shared memory.
constexpr int CL_PER = 16;

__global__ void __launch_bounds__(256) classify_kernel(const int32_t* __restrict__ queries, int64_t q, PathsRef P,
                                                       int64_t ccap, int64_t ccap_big, bool lane_ok, int group_max,
                                                       bool all_hub,
                                                       Tiers tiers, OutRef o, uint32_t* status) {
    __shared__ unsigned tot[8];
    __shared__ int base[8];
    const int64_t c0 = (int64_t)blockIdx.x * blockDim.x * CL_PER;
    int8_t tier[CL_PER];
    if (threadIdx.x < 8) tot[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < CL_PER; ++j) {
        const int64_t i = c0 + (int64_t)j * blockDim.x + threadIdx.x;
        int t = -1;
        if (i < q) {
            const int64_t v = queries ? (int64_t)queries[i] : i;
            if (v < 0 || v >= P.n) {
                flag_status(status, ST_BAD_QUERY);
                atomicMin(status + 1, (uint32_t)i);
            } else {
                const int64_t np = P.off[v + 1] - P.off[v];
                int64_t cap = np * (P.L - 1);
                if (cap > P.n - 1) cap = P.n - 1;
                if (cap > 0) {
                    if (lane_ok && np <= LANE_NP) t = 3;
                    else if (np <= 8 && np <= group_max) t = 4;
                    else if (np <= 16 && np <= group_max) t = 5;
                    else if (np <= 32 && np <= group_max) t = 6;
                    else if (all_hub) t = 2;     // k > 64: the rest in device tables
                    else if (np > CTA_MAX_NP) t = 2;
                    else t = (cap <= WCAP && np <= WARP_MAX_NP) ? 0 : (cap <= ccap ? 1 : (cap <= ccap_big ? 7 : 2));
                }
            }
            if (t < 0) {
                for (int r = 0; r < o.k; ++r) {
                    if (o.ids) o.ids[i * o.k + r] = -1;
                    o.cnt[i * o.k + r] = 0;
                }
            }
        }
        tier[j] = (int8_t)t;
    }
    // this thread's entries per tier, its offset within the CTA's share
    unsigned mine[8], off[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) mine[t] = 0;
#pragma unroll
    for (int j = 0; j < CL_PER; ++j)
#pragma unroll
        for (int t = 0; t < 8; ++t) mine[t] += tier[j] == t ? 1u : 0u;
#pragma unroll
    for (int t = 0; t < 8; ++t) off[t] = mine[t] ? atomicAdd(&tot[t], mine[t]) : 0u;
    __syncthreads();
    if (threadIdx.x < 8) {
        const int t = threadIdx.x;
        base[t] = tot[t] ? atomicAdd(&tiers.count[t < 3 ? t : (t == 7 ? 10 : t + 2)], (int)tot[t]) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < CL_PER; ++j) {
        const int t = tier[j];
        if (t >= 0) {
            const int64_t i = c0 + (int64_t)j * blockDim.x + threadIdx.x;
            tiers.list[t][base[t] + off[t]++] = (int32_t)i;
        }
    }
}

// Top-k of a table of nslots slots, by a whole CTA (every thread calls it;
// ends with a barrier). The k-th largest count c* comes from a histogram of
// the counts (counts above 62 share bin 63), which also gives m = the slots
// with count >= c*. With m <= 64 only those slots are compacted and one warp
// sorts them; otherwise every slot is offered to per-warp lists, then merged.
// CLEAR empties each filled slot once read (tables that are reused). The
// list (ranks l and 32+l in lane l) goes to sink(t) in warp 0.
template <bool CLEAR, class Sink>
__device__ void cta_select(unsigned long long* tab, uint32_t nslots, unsigned long long* lists, int k, Sink sink) {
    __shared__ unsigned hist[64];
    __shared__ int s_cstar, s_m, s_at;
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x == 0) s_at = 0;
    __syncthreads();
    for (uint32_t base = (uint32_t)w * 32; base < nslots; base += (uint32_t)nw * 32) {   // warp-uniform
        const uint32_t s = base + lane;
        const unsigned long long x = s < nslots ? tab[s] : EMPTY;
        const uint32_t c = x == EMPTY ? 64u : min((uint32_t)x, 63u);
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        if (c < 64 && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&hist[c], (unsigned)__popc(peers));
    }
    __syncthreads();
    if (w == 0) {
        // S(c) = number of slots with count >= c, for c = lane and 32 + lane
        uint32_t hi = hist[32 + lane], lo = hist[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t yh = __shfl_down_sync(0xffffffffu, hi, d), yl = __shfl_down_sync(0xffffffffu, lo, d);
            if (lane + d < 32) {
                hi += yh;
                lo += yl;
            }
        }
        lo += __shfl_sync(0xffffffffu, hi, 0);
        const unsigned mh = __ballot_sync(0xffffffffu, hi >= (uint32_t)k);
        const unsigned ml = __ballot_sync(0xffffffffu, lo >= (uint32_t)k);
        int cstar = 1;   // fewer than k filled slots: take them all
        if (mh) cstar = 32 + 31 - __clz(mh);
        else if (ml) cstar = max(1, 31 - __clz(ml));
        const uint32_t m = cstar >= 32 ? __shfl_sync(0xffffffffu, hi, cstar - 32) : __shfl_sync(0xffffffffu, lo, cstar);
        if (lane == 0) {
            s_cstar = cstar;
            s_m = (int)m;
        }
    }
    __syncthreads();
    const uint32_t cstar = (uint32_t)s_cstar;
    const int m = s_m;
    if (m <= 64) {
        for (uint32_t base = (uint32_t)w * 32; base < nslots; base += (uint32_t)nw * 32) {   // warp-uniform
            const uint32_t s = base + lane;
            const unsigned long long x = s < nslots ? tab[s] : EMPTY;
            if (CLEAR && x != EMPTY) tab[s] = EMPTY;
            const bool pass = x != EMPTY && (uint32_t)x >= cstar;
            const unsigned mk = __ballot_sync(0xffffffffu, pass);
            if (!mk) continue;
            int at = 0;
            if (lane == 0) at = atomicAdd(&s_at, __popc(mk));
            at = __shfl_sync(0xffffffffu, at, 0) + __popc(mk & lt);
            if (pass) lists[at] = slot_score(x);
        }
        __syncthreads();
        if (w == 0) {
            WarpTopK t;
            t.a = lane < (unsigned)m ? lists[lane] : 0;
            t.b = 32 + lane < (unsigned)m ? lists[32 + lane] : 0;
            warp_sort64_desc(t.a, t.b);
            sink(t);
        }
        __syncthreads();
        return;
    }
    WarpTopK t;
    for (uint32_t base = (uint32_t)w * 32; base < nslots; base += (uint32_t)nw * 32) {
        const uint32_t s = base + lane;
        uint64_t sc = 0;
        if (s < nslots) {
            sc = slot_score(tab[s]);
            if (CLEAR && sc) tab[s] = EMPTY;
        }
        t.offer(sc, k);
    }
    cta_merge(t, lists);
    if (w == 0) sink(t);
    __syncthreads();
}

// CTA-wide: count one query into the shared table and write its top-k
template <int STRIDE>
__device__ void cta_query(const PathsRef& P, int32_t v, int64_t qi, unsigned long long* tab, uint32_t max_slots,
                          unsigned long long* lists, const OutRef& o, uint32_t* status) {
    int64_t a = P.off[v], b = P.off[v + 1];
    const uint32_t nslots = table_size((b - a) * (P.L - 1), 1024, max_slots);
    for (uint32_t s = threadIdx.x; s < nslots; s += blockDim.x) tab[s] = EMPTY;
    __syncthreads();
    bool ok = true;
    for (int64_t base = a + (threadIdx.x & ~31u); base < b; base += blockDim.x) {   // warp-uniform
        const int64_t e = base + (threadIdx.x & 31);
        const bool act = e < b;
        ok &= insert_path_conv<STRIDE>(P, act ? P.pid[e] : NO_PATH, v, tab, nslots, act);
    }
    if (!ok) flag_status(status, ST_HASH_FULL);
    __syncthreads();
    cta_select<false>(tab, nslots, lists, o.k, [&](const WarpTopK& t) { write_list(t, o, qi); });
}

template <int STRIDE>
__device__ void warp_query(const PathsRef& P, int32_t v, int64_t qi, unsigned long long* tab, const OutRef& o,
                           uint32_t* status) {
    unsigned lane = threadIdx.x & 31;
    int64_t a = P.off[v], b = P.off[v + 1];
    const uint32_t ns = table_size((b - a) * (P.L - 1), 64, WSLOTS);
    for (uint32_t s = lane; s < ns; s += 32) tab[s] = EMPTY;
    __syncwarp();
    bool ok = true;
    for (int64_t base = a; base < b; base += 32) {                   // warp-uniform trip count
        const int64_t e = base + lane;
        const bool act = e < b;
        ok &= insert_path_conv<STRIDE>(P, act ? P.pid[e] : NO_PATH, v, tab, ns, act);
    }
    if (!ok) flag_status(status, ST_HASH_FULL);
    __syncwarp();
    WarpTopK t = warp_table_topk(tab, ns, o.k);
    write_list(t, o, qi);
    __syncwarp();
}


// ------------------------------------------------- narrow warp tier ---
// When every vertex id fits in 32 - cb bits and every warp-tier count in cb
// bits, a slot is one 32-bit word key << cb | count: half the table, 32-bit
// atomics, and 32-bit keys to sort.
constexpr uint32_t EMPTY32 = 0xffffffffu;

__device__ __forceinline__ bool hash_add32_conv(uint32_t* tab, uint32_t nslots, uint32_t key, int cb, bool active) {
    uint32_t s = active ? hslot(key, nslots) : 0;
    bool pending = active, ok = true;
    uint32_t probes = 0;
    const uint32_t mine_word = (key << cb) | 1u;
    while (__any_sync(0xffffffffu, pending)) {
        if (pending) {
            uint32_t cur = tab[s];
            bool mine = cur != EMPTY32 && (cur >> cb) == key;
            if (cur == EMPTY32) {
                uint32_t prev = atomicCAS(&tab[s], EMPTY32, mine_word);
                if (prev == EMPTY32) pending = false;
                else mine = (prev >> cb) == key;
            }
            if (mine) {
                atomicAdd(&tab[s], 1u);
                pending = false;
            }
            if (pending) {
                s = (s + 1 == nslots) ? 0 : s + 1;
                if (++probes >= nslots) {
                    pending = false;
                    ok = false;
                }
            }
        }
    }
    return ok;
}

template <int STRIDE>
__device__ __forceinline__ bool insert_path32(const PathsRef& P, uint32_t r, int32_t v, uint32_t* tab, uint32_t nslots,
                                              int cb, bool active) {
    active &= r < (uint64_t)P.R;
    int32_t x[STRIDE];
    const int4* src = (const int4*)(P.rows + (uint64_t)(active ? r : 0u) * STRIDE);
#pragma unroll
    for (int k = 0; k < STRIDE / 4; ++k) {
        int4 q = active ? __ldg(src + k) : make_int4(-1, -1, -1, -1);
        x[4 * k] = q.x; x[4 * k + 1] = q.y; x[4 * k + 2] = q.z; x[4 * k + 3] = q.w;
    }
    bool ok = true;
#pragma unroll
    for (int j = 0; j < STRIDE; ++j) {
        bool take = active && j < P.L && x[j] != v;
#pragma unroll
        for (int i = 0; i < j; ++i) take &= (x[i] != x[j]);
        if (__any_sync(0xffffffffu, take)) ok &= hash_add32_conv(tab, nslots, (uint32_t)x[j], cb, take);
    }
    return ok;
}

// sort key of a narrow slot: count high, then ascending id (0 = empty)
__device__ __forceinline__ uint32_t slot_score32(uint32_t w, int cb) {
    if (w == EMPTY32) return 0;
    const uint32_t kb = 32 - cb, kmask = (1u << kb) - 1u;   // 1 <= cb <= 16
    return ((w & ((1u << cb) - 1u)) << kb) | (kmask - (w >> cb));
}

__device__ __forceinline__ uint64_t widen_score(uint32_t sc, int cb) {
    if (!sc) return 0;
    const uint32_t kb = 32 - cb, kmask = (1u << kb) - 1u;
    const uint32_t cnt = sc >> kb, id = kmask - (sc & kmask);
    return ((uint64_t)cnt << 32) | (uint64_t)(0xffffffffu - id);
}

// bitonic sort, descending, of the 64 32-bit keys (a: rank lane, b: rank 32 + lane)
__device__ __forceinline__ void warp_sort64_desc32(uint32_t& a, uint32_t& b) {
    const unsigned lane = threadIdx.x & 31;
#pragma unroll
    for (int kk = 2; kk <= 64; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            if (j == 32) {
                const bool desc = (lane & kk) == 0;
                const uint32_t hi = max(a, b), lo = min(a, b);
                a = desc ? hi : lo;
                b = desc ? lo : hi;
            } else {
                const uint32_t pa = __shfl_xor_sync(0xffffffffu, a, j);
                const uint32_t pb = __shfl_xor_sync(0xffffffffu, b, j);
                const bool lower = (lane & j) == 0;
                const bool da = kk == 64 || (lane & kk) == 0;
                const bool db = kk == 64 || ((32 + lane) & kk) == 0;
                a = (lower == da) ? max(a, pa) : min(a, pa);
                b = (lower == db) ? max(b, pb) : min(b, pb);
            }
        }
    }
}

__device__ __forceinline__ uint32_t warp_sort32_desc32(uint32_t a) {
    const unsigned lane = threadIdx.x & 31;
#pragma unroll
    for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
        for (int j = kk >> 1; j > 0; j >>= 1) {
            const uint32_t pa = __shfl_xor_sync(0xffffffffu, a, j);
            const bool lower = (lane & j) == 0;
            const bool da = kk == 32 || (lane & kk) == 0;
            a = (lower == da) ? max(a, pa) : min(a, pa);
        }
    }
    return a;
}

// returns false (and does nothing) when the query has 2^cb - 1 or more paths:
// its counts might not fit, or a slot might read as empty
template <int STRIDE>
__device__ bool warp_query32(const PathsRef& P, int32_t v, int64_t qi, uint32_t* tab, const OutRef& o, int cb,
                             uint32_t* status) {
    if constexpr (STRIDE > 32) return false;              // long rows: the wide form
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    const int64_t a = P.off[v], b = P.off[v + 1];
    if (b - a >= (int64_t(1) << cb) - 1) return false;
    const uint32_t ns = table_size((b - a) * (P.L - 1), 64, WSLOTS);
    for (uint32_t s = lane; s < ns; s += 32) tab[s] = EMPTY32;
    __syncwarp();
    bool ok = true;
    for (int64_t base = a; base < b; base += 32) {                   // warp-uniform trip count
        const int64_t e = base + lane;
        const bool act = e < b;
        ok &= insert_path32<STRIDE>(P, act ? P.pid[e] : NO_PATH, v, tab, ns, cb, act);
    }
    if (!ok) flag_status(status, ST_HASH_FULL);
    __syncwarp();
    // top-k: the slots with count >= c* are compacted in place and sorted
    // once. c* = 1 when at most 64 slots are filled; otherwise the k-th
    // largest count, found bit by bit (counts are below 2^cb) by counting the
    // slots at or above a threshold on a register copy of the table. More
    // than 64 slots at or above c* (many ties at c*): every slot is offered to
    // a running list instead.
    constexpr int NR = WSLOTS / 32;
    const uint32_t cmask = (1u << cb) - 1u;
    uint32_t wv[NR];
#pragma unroll
    for (int g = 0; g < NR; ++g) wv[g] = (uint32_t)g * 32u < ns ? tab[g * 32 + lane] : EMPTY32;
    auto at_least = [&](uint32_t c) {
        int s = 0;
#pragma unroll
        for (int g = 0; g < NR; ++g)
            s += __popc(__ballot_sync(0xffffffffu, wv[g] != EMPTY32 && (wv[g] & cmask) >= c));
        return s;
    };
    uint32_t cstar = 1;
    int filled = at_least(1);
    if (filled > 64) {
        cstar = 0;
        for (int bit = cb - 1; bit >= 0; --bit)                       // warp-uniform
            if (at_least(cstar | (1u << bit)) >= o.k) cstar |= 1u << bit;
        filled = at_least(cstar);
    }
    WarpTopK t;
    if (filled > 64) {
#pragma unroll
        for (int g = 0; g < NR; ++g)
            if ((uint32_t)g * 32u < ns) t.offer(widen_score(slot_score32(wv[g], cb), cb), o.k);
    } else {
        int pos = 0;
#pragma unroll
        for (int g = 0; g < NR; ++g) {
            const bool pass = wv[g] != EMPTY32 && (wv[g] & cmask) >= cstar;
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            if (pass) tab[pos + __popc(m & lt)] = slot_score32(wv[g], cb);   // the table is in registers
            pos += __popc(m);
        }
        __syncwarp();
        uint32_t ka = lane < (unsigned)filled ? tab[lane] : 0u;
        uint32_t kb2 = 32 + lane < (unsigned)filled ? tab[32 + lane] : 0u;
        if (filled <= 32) {
            ka = warp_sort32_desc32(ka);
            kb2 = 0;
        } else {
            warp_sort64_desc32(ka, kb2);
        }
        t.a = widen_score(ka, cb);
        t.b = widen_score(kb2, cb);
    }
    write_list(t, o, qi);
    __syncwarp();
    return true;
}

struct PersistArgs {
    PathsRef P;
    const int32_t* queries;
    Tiers tiers;
    OutRef o;
    uint32_t cta_slots;
    uint32_t* status;
    int narrow_cb;   // > 0: warp tier on 32-bit slots with this many count bits
};

template <int STRIDE>
__global__ void __launch_bounds__(1024, 1) persistent_kernel(PersistArgs A) {
    extern __shared__ unsigned long long smem[];
    unsigned long long* lists = smem + A.cta_slots;     // 64 entries per warp after the table
    __shared__ int s_item;
    const int nC = A.tiers.count[1], nW = A.tiers.count[0];
    // CTA tier first: the largest items, one query per fetch
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&A.tiers.count[4], 1);
        __syncthreads();
        int it = s_item;
        __syncthreads();
        if (it >= nC) break;
        int64_t qi = A.tiers.list[1][it];
        int32_t v = A.queries ? A.queries[qi] : (int32_t)qi;
        cta_query<STRIDE>(A.P, v, qi, smem, A.cta_slots, lists, A.o, A.status);
    }
    // warp tier, WCHUNK queries per fetch
    unsigned lane = threadIdx.x & 31;
    unsigned long long* wt = smem + (threadIdx.x >> 5) * WSLOTS;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&A.tiers.count[3], WCHUNK);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= nW) break;
        int end = it + WCHUNK < nW ? it + WCHUNK : nW;
        for (int j = it; j < end; ++j) {
            int64_t qi = A.tiers.list[0][j];
            int32_t v = A.queries ? A.queries[qi] : (int32_t)qi;
            if (!A.narrow_cb || !warp_query32<STRIDE>(A.P, v, qi, (uint32_t*)wt, A.o, A.narrow_cb, A.status))
                warp_query<STRIDE>(A.P, v, qi, wt, A.o, A.status);
        }
    }
}

// one query per launch (the comparison form): a CTA with the shared table, or
// the global table when the candidate bound exceeds it
template <int STRIDE>
__global__ void __launch_bounds__(1024, 1) single_kernel(PathsRef P, const int32_t* __restrict__ queries, int64_t qi, OutRef o,
                              uint32_t cta_slots, unsigned long long* gtab, uint32_t gslots, uint32_t* status) {
    extern __shared__ unsigned long long smem[];
    unsigned long long* lists = smem + cta_slots;       // 64 entries per warp after the table
    int64_t v = queries ? queries[qi] : qi;
    if (v < 0 || v >= P.n) {
        if (threadIdx.x == 0) flag_status(status, ST_BAD_QUERY);
        if (threadIdx.x < (unsigned)o.k) {
            if (o.ids) o.ids[qi * o.k + threadIdx.x] = -1;
            o.cnt[qi * o.k + threadIdx.x] = 0;
        }
        return;
    }
    int64_t np = P.off[v + 1] - P.off[v];
    int64_t cap = np * (P.L - 1);
    if (cap * 10 <= (int64_t)cta_slots * 7) {
        cta_query<STRIDE>(P, (int32_t)v, qi, smem, cta_slots, lists, o, status);
        return;
    }
    // global table: gtab is EMPTY on entry and left EMPTY on exit
    bool ok = true;
    if constexpr (STRIDE > 32) {
        for (int64_t base = P.off[v] + (threadIdx.x & ~31u); base < P.off[v + 1]; base += blockDim.x) {
            const int64_t e = base + (threadIdx.x & 31);
            const bool act = e < P.off[v + 1];
            ok &= insert_paths_warp<STRIDE>(P, act ? P.pid[e] : NO_PATH, (int32_t)v, gtab, gslots, act, 0);
        }
    } else {
        for (int64_t e = P.off[v] + threadIdx.x; e < P.off[v + 1]; e += blockDim.x)
            ok &= insert_path<STRIDE, false>(P, P.pid[e], (int32_t)v, gtab, gslots);
    }
    if (!ok) flag_status(status, ST_HASH_FULL);
    __syncthreads();
    __threadfence_block();
    WarpTopK t;
    int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    unsigned lane = threadIdx.x & 31;
    for (uint32_t base = (uint32_t)w * 32; base < gslots; base += (uint32_t)nw * 32) {
        uint32_t s = base + lane;
        uint64_t sc = 0;
        if (s < gslots) {
            sc = slot_score(gtab[s]);
            if (sc) gtab[s] = EMPTY;
        }
        t.offer(sc, o.k);
    }
    cta_merge(t, lists);
    if (w == 0) {
        write_list(t, o, qi);
    }
}

// ------------------------------------------------------- global tier ---
struct GPlan {
    const int32_t* qidx;      // [ng] query index of each global query in this round
    const int64_t* tab_off;   // [ng] first slot of its table in the arena
    const uint32_t* tab_n;    // [ng] slots
    const int64_t* item_off;  // [ng+1] prefix of count work items
    const int64_t* sel_off;   // [ng+1] prefix of select work items
    int ng;
    const uint32_t* thr;      // [ng] count only the u with cls[u] >= thr (0: every u), or null
};

constexpr int G_PATHS = 512;      // paths per count item (small: the tables of the queries in flight stay in L2)
constexpr int G_SLOTS = 16384;    // slots per select item

__device__ __forceinline__ int find_owner(const int64_t* pre, int ng, int64_t item) {
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int STRIDE>
__global__ void g_count_kernel(PathsRef P, const int32_t* __restrict__ queries, GPlan G,
                               unsigned long long* arena, uint32_t* status) {
    int64_t item = blockIdx.x;
    if (item >= G.item_off[G.ng]) return;
    int g = find_owner(G.item_off, G.ng, item);
    int64_t qi = G.qidx[g];
    int32_t v = queries ? queries[qi] : (int32_t)qi;
    int64_t a = P.off[v] + (item - G.item_off[g]) * G_PATHS;
    int64_t b = a + G_PATHS < P.off[v + 1] ? a + G_PATHS : P.off[v + 1];
    unsigned long long* tab = arena + G.tab_off[g];
    const uint32_t thr = G.thr ? G.thr[g] : 0;
    bool ok = true;
    if constexpr (STRIDE > 32) {
        for (int64_t base = a + (threadIdx.x & ~31u); base < b; base += blockDim.x) {   // warp-uniform
            const int64_t e = base + (threadIdx.x & 31);
            const bool act = e < b;
            ok &= insert_paths_warp<STRIDE>(P, act ? P.pid[e] : NO_PATH, v, tab, G.tab_n[g], act, thr);
        }
    } else {
        for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x)
            ok &= insert_path<STRIDE, false>(P, P.pid[e], v, tab, G.tab_n[g], thr);
    }
    if (!ok) flag_status(status, ST_HASH_FULL);
}

// 64 < k <= 128 sends every query of the batch to device tables; queries of
// at most WARP_NP paths are counted by one warp each instead of a CTA per
// 512 paths
constexpr int64_t WARP_NP = 2048;

template <int STRIDE>
__global__ void __launch_bounds__(256) g_count_warp_kernel(PathsRef P, const int32_t* __restrict__ queries, GPlan G,
                                                           unsigned long long* arena, uint32_t* status) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= G.ng) return;                           // warp-uniform
    const int g = (int)gw;
    const int64_t qi = G.qidx[g];
    const int32_t v = queries ? queries[qi] : (int32_t)qi;
    const int64_t a = P.off[v], b = P.off[v + 1];
    if (b - a > WARP_NP) return;                      // counted by g_count_kernel
    unsigned long long* tab = arena + G.tab_off[g];
    const uint32_t ns = G.tab_n[g];
    const uint32_t thr = G.thr ? G.thr[g] : 0;
    const unsigned lane = threadIdx.x & 31;
    bool ok = true;
    if constexpr (STRIDE > 32) {
        for (int64_t base = a; base < b; base += 32) {            // warp-uniform
            const int64_t e = base + lane;
            const bool act = e < b;
            ok &= insert_paths_warp<STRIDE>(P, act ? P.pid[e] : NO_PATH, v, tab, ns, act, thr);
        }
    } else {
        for (int64_t e = a + lane; e < b; e += 32) ok &= insert_path<STRIDE, false>(P, P.pid[e], v, tab, ns, thr);
    }
    if (!ok) flag_status(status, ST_HASH_FULL);
}

// partial top-k of one chunk of one table; empties the slots it read
__global__ void __launch_bounds__(512) g_select_kernel(GPlan G, unsigned long long* arena, int k,
                                                       unsigned long long* partial) {
    __shared__ unsigned long long lists[16 * KMAX];
    const int64_t item = blockIdx.x;
    const int g = find_owner(G.sel_off, G.ng, item);
    const int64_t c0 = (item - G.sel_off[g]) * G_SLOTS;
    const int64_t ns = G.tab_n[g];
    const uint32_t len = (uint32_t)(c0 + G_SLOTS < ns ? G_SLOTS : ns - c0);
    const unsigned lane = threadIdx.x & 31;
    cta_select<true>(arena + G.tab_off[g] + c0, len, lists, k, [&](const WarpTopK& t) {
        partial[item * KMAX + lane] = t.a;
        partial[item * KMAX + 32 + lane] = t.b;
    });
}

// merge the partial lists of one query with a whole CTA (warps take lists
// strided, then a tree merge)
__global__ void __launch_bounds__(256) g_merge_cta_kernel(GPlan G, const unsigned long long* __restrict__ partial,
                                                          OutRef o) {
    __shared__ unsigned long long lists[8 * KMAX];
    const int g = blockIdx.x;
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned lane = threadIdx.x & 31;
    WarpTopK t;
    for (int64_t it = G.sel_off[g] + w; it < G.sel_off[g + 1]; it += nw)
        t.merge(partial[it * KMAX + lane], partial[it * KMAX + 32 + lane]);
    cta_merge(t, lists);
    if (w == 0) write_list(t, o, G.qidx[g]);
}

__global__ void g_merge_kernel(GPlan G, const unsigned long long* __restrict__ partial, OutRef o) {
    int g = blockIdx.x;
    if (g >= G.ng || threadIdx.x >= 32) return;
    WarpTopK t;
    unsigned lane = threadIdx.x;
    for (int64_t it = G.sel_off[g]; it < G.sel_off[g + 1]; ++it) {
        t.offer(partial[it * KMAX + lane], o.k);
        if (o.k > 32) t.offer(partial[it * KMAX + 32 + lane], o.k);
    }
    write_list(t, o, G.qidx[g]);
}

// 64 < k <= 128: tables of at most SMALL4 slots are selected whole by one
// warp (most queries of a batch: their tables are sized to twice their
// candidate bound, from 64 slots); larger ones in chunks (partial 128-lists),
// then one merge per query
constexpr uint32_t SMALL4 = 2048;

__global__ void __launch_bounds__(256) g_small4_kernel(GPlan G, unsigned long long* arena, OutRef o) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= G.ng) return;                           // warp-uniform
    const int g = (int)gw;
    const uint32_t ns = G.tab_n[g];
    if (ns > SMALL4) return;
    unsigned long long* tab = arena + G.tab_off[g];
    const unsigned lane = threadIdx.x & 31;
    WarpTopK4 t;
    for (uint32_t base = 0; base < ns; base += 32) {  // ns is a power of two >= 64
        uint64_t sc = slot_score(tab[base + lane]);
        if (sc) tab[base + lane] = EMPTY;
        t.offer(sc, o.k);
    }
    write_list4(t, o, G.qidx[g]);
}

__global__ void __launch_bounds__(512) g_select4_kernel(GPlan G, unsigned long long* arena, int k,
                                                        unsigned long long* partial) {
    __shared__ unsigned long long lists[16 * KMAX4];
    const int64_t item = blockIdx.x;
    const int g = find_owner(G.sel_off, G.ng, item);
    const int64_t c0 = (item - G.sel_off[g]) * G_SLOTS;
    const int64_t ns = G.tab_n[g];
    const uint32_t len = (uint32_t)(c0 + G_SLOTS < ns ? G_SLOTS : ns - c0);
    unsigned long long* tab = arena + G.tab_off[g] + c0;
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31;
    WarpTopK4 t;
    for (uint32_t base = (uint32_t)w * 32; base < len; base += (uint32_t)nw * 32) {   // warp-uniform
        const uint32_t s = base + lane;
        uint64_t sc = 0;
        if (s < len) {
            sc = slot_score(tab[s]);
            if (sc) tab[s] = EMPTY;
        }
        t.offer(sc, k);
    }
    cta_merge4(t, lists);
    if (w == 0)
#pragma unroll
        for (int j = 0; j < 4; ++j) partial[item * KMAX4 + 32 * j + lane] = t.r[j];
}

__global__ void __launch_bounds__(256) g_merge4_kernel(GPlan G, const unsigned long long* __restrict__ partial,
                                                       OutRef o) {
    __shared__ unsigned long long lists[8 * KMAX4];
    const int g = blockIdx.x;
    if (G.tab_n[g] <= SMALL4) return;                 // answered by g_small4_kernel
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned lane = threadIdx.x & 31;
    WarpTopK4 t;
    for (int64_t it = G.sel_off[g] + w; it < G.sel_off[g + 1]; it += nw) {
        uint64_t x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = partial[it * KMAX4 + 32 * j + lane];
        t.merge(x);
    }
    cta_merge4(t, lists);
    if (w == 0) write_list4(t, o, G.qidx[g]);
}

// ---------------------------------------------- bucketed global tier ---
// A hub query is counted in two passes without device-wide atomics on
// counts: (1) a CTA counts one chunk of the hub's paths in shared memory and
// scatters its (vertex, partial count) pairs into nb buckets by a hash of the
// vertex; (2) one CTA per bucket sums the pairs of its bucket in shared
// memory and keeps that bucket's top-k. Partial lists merge per query. A
// bucket that fills up marks its query, which is then counted again by the
// global-table path.
constexpr int B_SLOTS1 = 8192;     // pass-1 table (one chunk, T <= 7)
constexpr int B_CAP = 4096;        // pairs per bucket
constexpr int B_SLOTS2 = 8192;     // pass-2 table
constexpr int B_TARGET = 2048;     // expected pairs per bucket when sizing nb
constexpr int B_T2 = 256;          // threads of a pass-2 CTA
constexpr double HUB_PRUNE = 0.03;   // first-round threshold = HUB_PRUNE * |P_v| / max(k, 10)
constexpr int64_t HUB_TABLE_BOUND = 1 << 19;   // filtered candidate bound counted in a device table

struct BPlan {
    int bpaths;                // paths per pass-1 chunk
    const int32_t* qidx;       // [ng] query index
    const uint32_t* thr;       // [ng] count only the u with cls[u] >= thr (0: every u)
    const int64_t* chunk_off;  // [ng+1] prefix of pass-1 chunks
    const int64_t* bucket_off; // [ng+1] prefix of buckets
    int ng;
    unsigned long long* pairs; // [total buckets][B_CAP]
    int* cursor;               // [total buckets]
    int* overflow;             // [ng]
};

__device__ __forceinline__ uint32_t bucket_of(uint32_t key, uint32_t nb) {
    uint32_t h = key * 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return __umulhi(h, nb);
}

template <int STRIDE>
__global__ void __launch_bounds__(512) b_scatter_kernel(PathsRef P, const int32_t* __restrict__ queries, BPlan B,
                                                        uint32_t* status) {
    extern __shared__ unsigned long long tab[];
    const int64_t item = blockIdx.x;
    const int g = find_owner(B.chunk_off, B.ng, item);
    const int64_t qi = B.qidx[g];
    const int32_t v = queries ? queries[qi] : (int32_t)qi;
    const int64_t a = P.off[v] + (item - B.chunk_off[g]) * B.bpaths;
    const int64_t b = a + B.bpaths < P.off[v + 1] ? a + B.bpaths : P.off[v + 1];
    const uint32_t nslots = B_SLOTS1, thr = B.thr[g];
    for (uint32_t s = threadIdx.x; s < nslots; s += blockDim.x) tab[s] = EMPTY;
    __syncthreads();
    bool ok = true;
    for (int64_t base = a + (threadIdx.x & ~31u); base < b; base += blockDim.x) {   // warp-uniform
        const int64_t e = base + (threadIdx.x & 31);
        const bool act = e < b;
        ok &= insert_path_conv<STRIDE>(P, act ? P.pid[e] : NO_PATH, v, tab, nslots, act, thr);
    }
    if (!ok) flag_status(status, ST_HASH_FULL);
    __syncthreads();
    const uint32_t nb = (uint32_t)(B.bucket_off[g + 1] - B.bucket_off[g]);
    const int64_t b0 = B.bucket_off[g];
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    for (uint32_t base = 0; base < nslots; base += blockDim.x) {      // warp-uniform trip count
        const uint32_t s = base + threadIdx.x;
        const unsigned long long x = s < nslots ? tab[s] : EMPTY;
        const bool valid = x != EMPTY;
        const uint32_t bkt = valid ? bucket_of((uint32_t)(x >> 32), nb) : 0xffffffffu;
        // one cursor atomic per (warp, bucket)
        const unsigned peers = __match_any_sync(0xffffffffu, bkt);
        const int leader = __ffs(peers) - 1;
        int first = 0;
        if (valid && (int)lane == leader) first = atomicAdd(&B.cursor[b0 + bkt], __popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (valid) {
            int pos = first + __popc(peers & lt);
            if (pos < B_CAP) B.pairs[(b0 + bkt) * B_CAP + pos] = x;
            else B.overflow[g] = 1;
        }
    }
}

__global__ void __launch_bounds__(B_T2) b_count_kernel(BPlan B, int k, unsigned long long* __restrict__ partial,
                                                       uint32_t* status) {
    extern __shared__ unsigned long long tab[];
    __shared__ unsigned long long lists[(B_T2 / 32) * KMAX];
    const int64_t bk = blockIdx.x;
    const int cnt = min(B.cursor[bk], B_CAP);
    const uint32_t nslots = table_size(cnt, 1024, B_SLOTS2);
    for (uint32_t s = threadIdx.x; s < nslots; s += blockDim.x) tab[s] = EMPTY;
    __syncthreads();
    bool ok = true;
    for (int base = threadIdx.x & ~31; base < cnt; base += blockDim.x) {              // warp-uniform
        const int i = base + (threadIdx.x & 31);
        const bool act = i < cnt;
        const unsigned long long x = act ? B.pairs[bk * B_CAP + i] : 0ull;
        ok &= hash_add_conv(tab, nslots, (uint32_t)(x >> 32), (uint32_t)x, act);
    }
    if (!ok) flag_status(status, ST_HASH_FULL);
    __syncthreads();
    WarpTopK t;
    int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    unsigned lane = threadIdx.x & 31;
    for (uint32_t base = (uint32_t)w * 32; base < nslots; base += (uint32_t)nw * 32) {
        uint32_t s = base + lane;
        t.offer(s < nslots ? slot_score(tab[s]) : 0, k);
    }
    cta_merge(t, lists);
    if (w == 0) {
        partial[bk * KMAX + lane] = t.a;
        partial[bk * KMAX + 32 + lane] = t.b;
    }
}

// after a filtered round: the k-th count c of the query over the u with
// cls[u] >= thr is a lower bound of its true k-th count, so every u of the true
// top-k has |P_u| >= c. Every dropped u has |P_u| < code_floor(thr): if
// c >= code_floor(thr) the filtered list is the answer (-1); otherwise the
// query is counted again with threshold path_code(c) (whose floor is <= c).
__global__ void hub_check_kernel(const int32_t* __restrict__ qidx, const uint32_t* __restrict__ thr, int ng, OutRef o,
                                 int32_t* __restrict__ redo) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    if (thr[i] == 0) {
        redo[i] = -1;
        return;
    }
    const uint32_t kth = o.cnt[(int64_t)qidx[i] * o.k + o.k - 1];
    redo[i] = (int64_t)kth >= code_floor(thr[i]) ? -1 : (int32_t)kth;
}

__global__ void g_info_kernel(const int32_t* __restrict__ list, int ng, const int32_t* __restrict__ queries,
                              const int64_t* __restrict__ off, int64_t* __restrict__ np) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ng) return;
    int64_t qi = list[i];
    int64_t v = queries ? (int64_t)queries[qi] : qi;
    np[i] = off[v + 1] - off[v];
}

__global__ void fill_empty_kernel(unsigned long long* p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t st = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += st) p[i] = EMPTY;
}

// slots of a hub device table: twice the candidate bound, rounded up to a
// multiple of lo (a multiple of 32: the selection reads whole warps of slots)
static uint32_t table_slots(int64_t bound, uint32_t lo) {
    const int64_t x = std::max<int64_t>(2 * bound, lo);
    return (uint32_t)((x + lo - 1) / lo * lo);
}

uint32_t pow2_at_least(int64_t x, uint32_t lo = 1024) {
    uint32_t p = lo;
    while ((int64_t)p < x && p < (1u << 31)) p <<= 1;
    return p;
}

}  // namespace

// the lane kernel instantiation for this batch: 32-bit scores when ids are
// below 2^29, exactly T+1 = 6 row positions at the paper's T = 5, a 12-entry
// list when k <= 12
static void launch_lane(bool narrow, bool l6, bool k12, unsigned blocks, cudaStream_t s, const PathsRef& P,
                        const int32_t* queries, const int32_t* list, const int* counts, const OutRef& o) {
#define PANTHER_LANE(NW, LPV, KPV) lane_kernel<NW, LPV, KPV><<<blocks, 256, 0, s>>>(P, queries, list, counts, 5, o)
    if (narrow) {
        if (l6) { if (k12) PANTHER_LANE(true, 6, 12); else PANTHER_LANE(true, 6, LANE_K); }
        else { if (k12) PANTHER_LANE(true, 8, 12); else PANTHER_LANE(true, 8, LANE_K); }
    } else {
        if (l6) { if (k12) PANTHER_LANE(false, 6, 12); else PANTHER_LANE(false, 6, LANE_K); }
        else { if (k12) PANTHER_LANE(false, 8, 12); else PANTHER_LANE(false, 8, LANE_K); }
    }
#undef PANTHER_LANE
}

// ------------------------------------------------------------ host side ---
constexpr int BIG_T = 512;
constexpr uint32_t BIG_SLOTS = 24576;
constexpr size_t BIG_SMEM = (size_t)BIG_SLOTS * 8 + (size_t)(BIG_T / 32) * KMAX * 8;

struct TopkShape {
    int threads;
    uint32_t cta_slots;
    int blocks_per_sm;
};

static TopkShape topk_shape(panther_ctx* ctx) {
    TopkShape s;
    s.threads = ctx->topk_threads ? ctx->topk_threads : 1024;
    s.cta_slots = ctx->topk_cta_slots ? (uint32_t)ctx->topk_cta_slots : 24576;
    s.blocks_per_sm = ctx->topk_blocks_per_sm ? ctx->topk_blocks_per_sm : 1;
    // warp tables must fit in the same dynamic area
    uint32_t need = (uint32_t)(s.threads / 32) * WSLOTS;
    if (s.cta_slots < need) s.cta_slots = need;
    return s;
}

template <int STRIDE>
static panther_status set_smem_attr(panther_ctx* ctx, size_t bytes) {
    PCK(ctx, cudaFuncSetAttribute(persistent_kernel<STRIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    PCK(ctx, cudaFuncSetAttribute(single_kernel<STRIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return PANTHER_OK;
}

struct HubQuery {
    int32_t qi;      // query index
    int64_t np;      // |P_v|
    uint32_t thr;    // count only the u with cls[u] >= thr (0: every u)
};

// bound of the distinct candidates of a hub query under its threshold
static int64_t hub_bound(const PathsRef& P, const HubQuery& h, const std::vector<int64_t>& above) {
    return std::min<int64_t>(std::min<int64_t>(h.np * (P.L - 1), P.n - 1), above[h.thr]);
}

// device copy of a small host plan (kept until the stream reaches it)
static panther_status upload(panther_ctx* ctx, const std::vector<char>& h, char** d) {
    panther_status st = dev_alloc(ctx, (void**)d, h.size());
    if (st) return st;
    PCK(ctx, cudaMemcpyAsync(*d, h.data(), h.size(), cudaMemcpyHostToDevice, ctx->stream));
    return PANTHER_OK;
}

template <class T>
static size_t put(std::vector<char>& h, const std::vector<T>& v) {
    size_t off = (h.size() + 15) & ~size_t(15);
    h.resize(off + sizeof(T) * v.size());
    memcpy(h.data() + off, v.data(), sizeof(T) * v.size());
    return off;
}

// Bucketed counting of hub queries (largest first, rounds under the scratch
// budget). Queries whose buckets overflowed are returned in `again`; filtered
// queries whose k-th count came out below their threshold are returned in
// `redo` with that count as the new threshold. `above[t]` = vertices with
// cls >= t (sizes the buckets of a filtered query).
static panther_status hub_buckets(panther_ctx* ctx, const PathsRef& P, const int32_t* queries, const OutRef& o, int k,
                                  std::vector<HubQuery> hubs, const std::vector<int64_t>& above,
                                  std::vector<HubQuery>& again, std::vector<HubQuery>& redo) {
    cudaStream_t s = ctx->stream;
    std::sort(hubs.begin(), hubs.end(),
              [](const HubQuery& a, const HubQuery& b) { return a.np != b.np ? a.np > b.np : a.qi < b.qi; });
    const int bpaths = std::max(32, B_SLOTS1 / (2 * std::max(1, P.L - 1)));
    const int64_t per_bucket = (int64_t)B_CAP * 8 + 4 + KMAX * 8;
    const int64_t budget = std::max<int64_t>(ctx->scratch_budget, per_bucket * 64);
    const int stride = path_stride(P.L);
    // The shared-memory attribute applies to the current device only: it is
    // set once per device (bit `device` of the mask). Contexts on several host
    // threads (the serving workers) may get here together; setting it twice
    // is harmless.
    static std::atomic<uint64_t> attr_set{0};
    const uint64_t dev_bit = ctx->device < 64 ? (uint64_t(1) << ctx->device) : 0;
    if (!dev_bit || !(attr_set.load(std::memory_order_acquire) & dev_bit)) {
        PCK(ctx, cudaFuncSetAttribute(b_scatter_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SLOTS1 * 8));
        PCK(ctx, cudaFuncSetAttribute(b_scatter_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SLOTS1 * 8));
        PCK(ctx, cudaFuncSetAttribute(b_scatter_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SLOTS1 * 8));
        PCK(ctx, cudaFuncSetAttribute(b_scatter_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SLOTS1 * 8));
        PCK(ctx, cudaFuncSetAttribute(b_scatter_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SLOTS1 * 8));
        PCK(ctx, cudaFuncSetAttribute(b_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SLOTS2 * 8));
        attr_set.fetch_or(dev_bit, std::memory_order_acq_rel);
    }
    size_t pos = 0;
    panther_status st;
    while (pos < hubs.size()) {
        std::vector<int32_t> rq;
        std::vector<uint32_t> rt;
        std::vector<int64_t> coff{0}, boff{0};
        std::vector<HubQuery> rh;
        int64_t used = 0;
        while (pos < hubs.size()) {
            const HubQuery& h = hubs[pos];
            int64_t nb = std::max<int64_t>(1, ceil_div(hub_bound(P, h, above), B_TARGET));
            if (!rq.empty() && used + nb * per_bucket > budget) break;
            rq.push_back(h.qi);
            rt.push_back(h.thr);
            rh.push_back(h);
            coff.push_back(coff.back() + ceil_div(h.np, bpaths));
            boff.push_back(boff.back() + nb);
            used += nb * per_bucket;
            ++pos;
        }
        const int rng = (int)rq.size();
        const int64_t nbt = boff.back();
        std::vector<char> hp;
        size_t o_q = put(hp, rq), o_t = put(hp, rt), o_c = put(hp, coff), o_b = put(hp, boff);
        char* dplan = nullptr;
        unsigned long long *pairs = nullptr, *partial = nullptr;
        int *cursor = nullptr, *ovf = nullptr;
        int32_t* dredo = nullptr;
        if ((st = upload(ctx, hp, &dplan)) || (st = dev_alloc(ctx, (void**)&pairs, 8ull * B_CAP * nbt)) ||
            (st = dev_alloc(ctx, (void**)&partial, 8ull * KMAX * nbt)) ||
            (st = dev_alloc(ctx, (void**)&cursor, sizeof(int) * nbt)) ||
            (st = dev_alloc(ctx, (void**)&ovf, sizeof(int) * rng)) ||
            (st = dev_alloc(ctx, (void**)&dredo, sizeof(int32_t) * rng))) {
            dev_free(ctx, dplan); dev_free(ctx, pairs); dev_free(ctx, partial); dev_free(ctx, cursor);
            dev_free(ctx, ovf);
            return st;
        }
        PCK(ctx, cudaMemsetAsync(cursor, 0, sizeof(int) * nbt, s));
        PCK(ctx, cudaMemsetAsync(ovf, 0, sizeof(int) * rng, s));
        BPlan B{bpaths, (const int32_t*)(dplan + o_q), (const uint32_t*)(dplan + o_t), (const int64_t*)(dplan + o_c),
                (const int64_t*)(dplan + o_b), rng, pairs, cursor, ovf};
        const unsigned g1 = (unsigned)coff.back();
        if (stride == 8) b_scatter_kernel<8><<<g1, 512, B_SLOTS1 * 8, s>>>(P, queries, B, ctx->d_status);
        else if (stride == 16) b_scatter_kernel<16><<<g1, 512, B_SLOTS1 * 8, s>>>(P, queries, B, ctx->d_status);
        else if (stride == 32) b_scatter_kernel<32><<<g1, 512, B_SLOTS1 * 8, s>>>(P, queries, B, ctx->d_status);
        else if (stride == 64) b_scatter_kernel<64><<<g1, 512, B_SLOTS1 * 8, s>>>(P, queries, B, ctx->d_status);
        else b_scatter_kernel<128><<<g1, 512, B_SLOTS1 * 8, s>>>(P, queries, B, ctx->d_status);
        b_count_kernel<<<(unsigned)nbt, B_T2, B_SLOTS2 * 8, s>>>(B, k, partial, ctx->d_status);
        GPlan G{B.qidx, nullptr, nullptr, nullptr, B.bucket_off, rng, nullptr};
        g_merge_cta_kernel<<<rng, 256, 0, s>>>(G, partial, o);
        hub_check_kernel<<<(unsigned)ceil_div(rng, 256), 256, 0, s>>>(B.qidx, B.thr, rng, o, dredo);
        ctx->launches += 4;
        PCK(ctx, cudaGetLastError());
        std::vector<int> hov(rng);
        std::vector<int32_t> hredo(rng);
        PCK(ctx, cudaMemcpyAsync(hov.data(), ovf, sizeof(int) * rng, cudaMemcpyDeviceToHost, s));
        PCK(ctx, cudaMemcpyAsync(hredo.data(), dredo, sizeof(int32_t) * rng, cudaMemcpyDeviceToHost, s));
        PCK(ctx, cudaStreamSynchronize(s));
        ctx->topk_stats[6] += rng;
        for (int i = 0; i < rng; ++i) {
            if (hov[i]) {
                ++ctx->topk_stats[8];
                HubQuery h = rh[i];
                h.thr = 0;
                again.push_back(h);
            } else if (hredo[i] >= 0) {
                HubQuery h = rh[i];
                h.thr = path_code(hredo[i]);
                redo.push_back(h);
            }
        }
        dev_free(ctx, dplan); dev_free(ctx, pairs); dev_free(ctx, partial); dev_free(ctx, cursor); dev_free(ctx, ovf);
        dev_free(ctx, dredo);
    }
    return PANTHER_OK;
}

// Hub queries counted in per-query device tables of twice their candidate
// bound (small filtered hubs, and the fallback of the bucketed path): rounds
// under the scratch budget. Filtered queries whose k-th count came out below
// their threshold are returned in `redo` (see hub_check_kernel).
static panther_status hub_tables(panther_ctx* ctx, const PathsRef& P, const int32_t* queries, const OutRef& o, int k,
                                 const std::vector<HubQuery>& hubs, const std::vector<int64_t>& above,
                                 std::vector<HubQuery>& redo) {
    cudaStream_t s = ctx->stream;
    const int64_t budget_slots = std::max<int64_t>(ctx->scratch_budget / 8 / 2, 1 << 20);
    const int stride = path_stride(P.L);
    size_t pos = 0;
    unsigned long long*& arena = ctx->hub_arena;
    int64_t& arena_slots = ctx->hub_arena_slots;
    panther_status st;
    while (pos < hubs.size()) {
        std::vector<int32_t> rq;
        std::vector<int64_t> roff, ioff{0}, soff{0};
        std::vector<uint32_t> rn, rt;
        std::vector<HubQuery> rh;
        int64_t used = 0;
        while (pos < hubs.size()) {
            const HubQuery& h = hubs[pos];
            // k > 64 sends every query here: small ones get small tables
            uint32_t slots = table_slots(hub_bound(P, h, above), k > KMAX ? 64u : 1024u);
            if (!rq.empty() && used + slots > budget_slots) break;
            rq.push_back(h.qi);
            rt.push_back(h.thr);
            rh.push_back(h);
            roff.push_back(used);
            rn.push_back(slots);
            used += slots;
            ioff.push_back(ioff.back() + ((k > KMAX && h.np <= WARP_NP) ? 0 : ceil_div(h.np, G_PATHS)));
            soff.push_back(soff.back() + ((k > KMAX && slots <= SMALL4) ? 0 : ceil_div(slots, G_SLOTS)));
            ++pos;
        }
        if (used > arena_slots) {
            dev_free(ctx, arena);
            arena = nullptr;
            arena_slots = 0;
            if ((st = dev_alloc(ctx, (void**)&arena, 8ull * used))) return st;
            arena_slots = used;
            ctx->hub_arena_clean = false;
        }
        if (!ctx->hub_arena_clean) {   // new, or left dirty by a call that failed midway
            fill_empty_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(arena, arena_slots);
            ctx->launches++;
            ctx->hub_arena_clean = true;
        }
        const int rng = (int)rq.size();
        std::vector<char> hp;
        size_t o_q = put(hp, rq), o_o = put(hp, roff), o_n = put(hp, rn), o_i = put(hp, ioff), o_s = put(hp, soff),
               o_t = put(hp, rt);
        char* dplan = nullptr;
        unsigned long long* partial = nullptr;
        int32_t* dredo = nullptr;
        const int kw = k > KMAX ? KMAX4 : KMAX;     // width of the partial lists
        if ((st = upload(ctx, hp, &dplan)) ||
            (st = dev_alloc(ctx, (void**)&partial, sizeof(unsigned long long) * kw * soff.back())) ||
            (st = dev_alloc(ctx, (void**)&dredo, sizeof(int32_t) * rng))) {
            dev_free(ctx, dplan);
            dev_free(ctx, partial);
            return st;
        }
        ctx->hub_arena_clean = false;   // until the select pass of this round has run
        GPlan G{(const int32_t*)(dplan + o_q), (const int64_t*)(dplan + o_o), (const uint32_t*)(dplan + o_n),
                (const int64_t*)(dplan + o_i), (const int64_t*)(dplan + o_s), rng, (const uint32_t*)(dplan + o_t)};
        if (k > KMAX) {
            const unsigned gwb = (unsigned)ceil_div((int64_t)rng * 32, 256);
            if (stride == 8) g_count_warp_kernel<8><<<gwb, 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else if (stride == 16) g_count_warp_kernel<16><<<gwb, 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else if (stride == 32) g_count_warp_kernel<32><<<gwb, 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else if (stride == 64) g_count_warp_kernel<64><<<gwb, 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else g_count_warp_kernel<128><<<gwb, 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            ctx->launches++;
        }
        if (ioff.back() > 0) {
            if (stride == 8) g_count_kernel<8><<<(unsigned)ioff.back(), 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else if (stride == 16) g_count_kernel<16><<<(unsigned)ioff.back(), 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else if (stride == 32) g_count_kernel<32><<<(unsigned)ioff.back(), 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else if (stride == 64) g_count_kernel<64><<<(unsigned)ioff.back(), 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else g_count_kernel<128><<<(unsigned)ioff.back(), 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
        }
        if (k > KMAX) {
            g_small4_kernel<<<(unsigned)ceil_div((int64_t)rng * 32, 256), 256, 0, s>>>(G, arena, o);
            if (soff.back() > 0) {
                g_select4_kernel<<<(unsigned)soff.back(), 512, 0, s>>>(G, arena, k, partial);
                g_merge4_kernel<<<rng, 256, 0, s>>>(G, partial, o);
            }
        } else {
            g_select_kernel<<<(unsigned)soff.back(), 512, 0, s>>>(G, arena, k, partial);
            g_merge_cta_kernel<<<rng, 256, 0, s>>>(G, partial, o);
        }
        hub_check_kernel<<<(unsigned)ceil_div(rng, 256), 256, 0, s>>>(G.qidx, G.thr, rng, o, dredo);
        ctx->launches += 4;
        PCK(ctx, cudaGetLastError());
        std::vector<int32_t> hredo(rng);
        PCK(ctx, cudaMemcpyAsync(hredo.data(), dredo, sizeof(int32_t) * rng, cudaMemcpyDeviceToHost, s));
        PCK(ctx, cudaStreamSynchronize(s));   // the host plan must outlive the copy
        ctx->hub_arena_clean = true;
        ctx->topk_stats[7] += rng;
        for (int i = 0; i < rng; ++i)
            if (hredo[i] >= 0) {
                HubQuery h = rh[i];
                h.thr = path_code(hredo[i]);
                redo.push_back(h);
            }
        dev_free(ctx, dplan);
        dev_free(ctx, partial);
        dev_free(ctx, dredo);
    }
    return PANTHER_OK;
}

// Internal entry shared by panther_topk and pantherpp_vectors: queries may be
// NULL (meaning 0..q-1); ids may be NULL (counts only, e.g. theta rows).
panther_status topk_run(panther_ctx* ctx, const panther_index* ix, const panther_paths* p, const int32_t* queries,
                        int64_t q, int k, int32_t* ids, uint32_t* cnt, bool plain) {
    cudaStream_t s = ctx->stream;
    TopkShape sh = topk_shape(ctx);
    const size_t smem = (size_t)sh.cta_slots * 8 + (size_t)(sh.threads / 32) * KMAX * 8;
    // the attribute is process-wide (contexts of several threads share it):
    // always the larger of this shape and the big-table pass
    const size_t attr = std::max(smem, BIG_SMEM);
    panther_status st;
    if (p->stride == 8) st = set_smem_attr<8>(ctx, attr);
    else if (p->stride == 16) st = set_smem_attr<16>(ctx, attr);
    else if (p->stride == 32) st = set_smem_attr<32>(ctx, attr);
    else if (p->stride == 64) st = set_smem_attr<64>(ctx, attr);
    else st = set_smem_attr<128>(ctx, attr);
    if (st) return st;
    PathsRef P{p->rows, p->R, p->L, ix->off, ix->pid, ix->n, ix->cls};
    OutRef o{ids, cnt, k};
    int64_t ccap = (int64_t)sh.cta_slots * 7 / 10;
    // queries above the tuned shape's table but within a 24,576-slot one take a
    // second persistent pass with one 1,024-thread CTA per SM
    int64_t ccap_big = sh.cta_slots < BIG_SLOTS ? (int64_t)BIG_SLOTS * 7 / 10 : ccap;
    if (ctx->dbg_hub_min_cap > 0) {   // test routing: a lower hub-tier bound
        ccap = std::min(ccap, std::max<int64_t>(ctx->dbg_hub_min_cap, WCAP));
        ccap_big = std::min(ccap_big, ccap);
    }
    for (int i = 0; i < 10; ++i) ctx->topk_stats[i] = 0;
    ctx->topk_stats[0] = q;

    if (plain && k > KMAX) {
        // one query at a time through the device-table path (the 128-entry lists)
        for (int64_t i = 0; i < q; ++i) {
            const int32_t* qi = queries ? queries + i : nullptr;
            if (!qi) return set_err(ctx, PANTHER_EINVAL, "the plain form with k > 64 needs a query array");
            panther_status r = topk_run(ctx, ix, p, qi, 1, k, ids ? ids + i * k : nullptr, cnt + i * k, false);
            if (r) return r;
        }
        ctx->topk_stats[0] = q;
        return PANTHER_OK;
    }
    if (plain) {
        for (int i = 0; i < 10; ++i) ctx->topk_stats[i] = 0;
        ctx->topk_stats[0] = q;
        uint32_t gslots = pow2_at_least(2 * ix->n);
        unsigned long long* gtab = nullptr;
        if ((st = dev_alloc(ctx, (void**)&gtab, 8ull * gslots))) return st;
        fill_empty_kernel<<<ctx->num_sms * 4, 256, 0, s>>>(gtab, gslots);
        ctx->launches++;
        for (int64_t i = 0; i < q; ++i) {
            if (p->stride == 8)
                single_kernel<8><<<1, sh.threads, smem, s>>>(P, queries, i, o, sh.cta_slots, gtab, gslots, ctx->d_status);
            else if (p->stride == 16)
                single_kernel<16><<<1, sh.threads, smem, s>>>(P, queries, i, o, sh.cta_slots, gtab, gslots, ctx->d_status);
            else if (p->stride == 32)
                single_kernel<32><<<1, sh.threads, smem, s>>>(P, queries, i, o, sh.cta_slots, gtab, gslots, ctx->d_status);
            else if (p->stride == 64)
                single_kernel<64><<<1, sh.threads, smem, s>>>(P, queries, i, o, sh.cta_slots, gtab, gslots, ctx->d_status);
            else
                single_kernel<128><<<1, sh.threads, smem, s>>>(P, queries, i, o, sh.cta_slots, gtab, gslots,
                                                              ctx->d_status);
            ctx->launches++;
        }
        dev_free(ctx, gtab);
        PCK(ctx, cudaGetLastError());
        return PANTHER_OK;
    }

    int32_t* lists = nullptr;
    int* counts = nullptr;
    if ((st = dev_alloc(ctx, (void**)&lists, sizeof(int32_t) * 8 * (size_t)q)) ||
        (st = dev_alloc(ctx, (void**)&counts, sizeof(int) * 16))) {
        dev_free(ctx, lists);
        return st;
    }
    Tiers tiers{{lists, lists + q, lists + 2 * q, lists + 3 * q, lists + 4 * q, lists + 5 * q, lists + 6 * q, lists + 7 * q},
                counts};
    const bool all_hub = k > KMAX;                      // 64 < k <= 128: device tables only
    // largest |P_v| the group tiers take: ids must fit below 2^group_ub(G)
    // (any k: G = 8 ranks at most 56 candidates, larger groups rank directly)
    const int group_max = p->stride != 8 ? 0
                          : ix->n <= (int64_t(1) << group_ub(32)) ? 32
                          : ix->n <= (int64_t(1) << group_ub(16)) ? 16 : 0;
    const bool lane_ok = p->stride == 8 && k <= LANE_K;
    PCK(ctx, cudaMemsetAsync(counts, 0, sizeof(int) * 16, s));
    classify_kernel<<<(unsigned)ceil_div(q, 256 * CL_PER), 256, 0, s>>>(queries, q, P, ccap, ccap_big, lane_ok,
                                                                         group_max, all_hub, tiers, o, ctx->d_status);
    ctx->launches++;
    // the lane and group tiers are independent of the persistent passes: they
    // run on the side streams (joined back into `s` below)
    const bool side = ctx->side[0] != nullptr;
    cudaStream_t s0 = side ? ctx->side[0] : s, s1 = side ? ctx->side[1] : s;
    if (side) {
        PCK(ctx, cudaEventRecord(ctx->fork, s));
        PCK(ctx, cudaStreamWaitEvent(s0, ctx->fork, 0));
        PCK(ctx, cudaStreamWaitEvent(s1, ctx->fork, 0));
    }
    if (lane_ok) {
        launch_lane(ix->n <= (int64_t(1) << 29), P.L == 6, k <= 12, (unsigned)(ctx->num_sms * 8), s0, P, queries,
                    lists + 3 * q, counts, o);
        ctx->launches++;
    }
    if (group_max >= 16) {
        group_kernel<8><<<(unsigned)(ctx->num_sms * 8), 256, 0, s0>>>(P, queries, lists + 4 * q, counts, 6, o);
        group_kernel<16><<<(unsigned)(ctx->num_sms * 8), 256, 0, s1>>>(P, queries, lists + 5 * q, counts, 7, o);
        ctx->launches += 2;
    }
    if (group_max >= 32) {
        group_kernel<32><<<(unsigned)(ctx->num_sms * 8), 256, 0, s1>>>(P, queries, lists + 6 * q, counts, 8, o);
        ctx->launches++;
    }
    if (side) {
        PCK(ctx, cudaEventRecord(ctx->join[0], s0));
        PCK(ctx, cudaEventRecord(ctx->join[1], s1));
    }
    // narrow warp tier: ids below 2^(32 - cb) with cb bits for the largest
    // warp-tier count (a count never exceeds the query's number of paths)
    int cb = 1;
    while ((1 << cb) <= WCAP / std::max(1, P.L - 1)) ++cb;
    const int narrow_cb = (cb <= 16 && ix->n <= (int64_t(1) << (32 - cb))) ? cb : 0;   // ids < 2^(32-cb)
    PersistArgs A{P, queries, tiers, o, sh.cta_slots, ctx->d_status, narrow_cb};
    unsigned blocks = (unsigned)(ctx->num_sms * sh.blocks_per_sm);
    if (!all_hub) {
    if (p->stride == 8) persistent_kernel<8><<<blocks, sh.threads, smem, s>>>(A);
    else if (p->stride == 16) persistent_kernel<16><<<blocks, sh.threads, smem, s>>>(A);
    else if (p->stride == 32) persistent_kernel<32><<<blocks, sh.threads, smem, s>>>(A);
    else if (p->stride == 64) persistent_kernel<64><<<blocks, sh.threads, smem, s>>>(A);
    else persistent_kernel<128><<<blocks, sh.threads, smem, s>>>(A);
    ctx->launches++;
    if (ccap_big > ccap) {
        // CTA tier only: its list is tier 7's, its counters start at [9]
        Tiers big{{lists, lists + 7 * q, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr}, counts + 9};
        PersistArgs B{P, queries, big, o, BIG_SLOTS, ctx->d_status, 0};
        const unsigned bb = (unsigned)ctx->num_sms;
        if (p->stride == 8) persistent_kernel<8><<<bb, BIG_T, BIG_SMEM, s>>>(B);
        else if (p->stride == 16) persistent_kernel<16><<<bb, BIG_T, BIG_SMEM, s>>>(B);
        else if (p->stride == 32) persistent_kernel<32><<<bb, BIG_T, BIG_SMEM, s>>>(B);
        else if (p->stride == 64) persistent_kernel<64><<<bb, BIG_T, BIG_SMEM, s>>>(B);
        else persistent_kernel<128><<<bb, BIG_T, BIG_SMEM, s>>>(B);
        ctx->launches++;
    }
    }   // !all_hub
    if (side) {
        PCK(ctx, cudaStreamWaitEvent(s, ctx->join[0], 0));
        PCK(ctx, cudaStreamWaitEvent(s, ctx->join[1], 0));
    }
    PCK(ctx, cudaGetLastError());

    // global tier: read its size (one synchronisation), then run in rounds
    int h_counts[16];
    PCK(ctx, cudaMemcpyAsync(h_counts, counts, sizeof(int) * 16, cudaMemcpyDeviceToHost, s));
    PCK(ctx, cudaStreamSynchronize(s));
    const int ng = h_counts[2];
    ctx->topk_stats[1] = lane_ok ? h_counts[5] : 0;
    ctx->topk_stats[2] = (int64_t)h_counts[6] + h_counts[7] + h_counts[8];
    ctx->topk_stats[3] = h_counts[0];
    ctx->topk_stats[4] = (int64_t)h_counts[1] + (ccap_big > ccap ? h_counts[10] : 0);
    ctx->topk_stats[5] = ng;
    if (ng > 0) {
        std::vector<int32_t> gq(ng);
        std::vector<int64_t> npv(ng);
        int64_t* d_np = nullptr;
        if ((st = dev_alloc(ctx, (void**)&d_np, sizeof(int64_t) * ng))) {
            dev_free(ctx, lists);
            dev_free(ctx, counts);
            return st;
        }
        g_info_kernel<<<(unsigned)ceil_div(ng, 256), 256, 0, s>>>(lists + 2 * q, ng, queries, ix->off, d_np);
        ctx->launches++;
        std::vector<int64_t> hist(256), above(257, 0);
        PCK(ctx, cudaMemcpyAsync(gq.data(), lists + 2 * q, sizeof(int32_t) * ng, cudaMemcpyDeviceToHost, s));
        PCK(ctx, cudaMemcpyAsync(npv.data(), d_np, sizeof(int64_t) * ng, cudaMemcpyDeviceToHost, s));
        PCK(ctx, cudaMemcpyAsync(hist.data(), ix->cls_hist, sizeof(int64_t) * 256, cudaMemcpyDeviceToHost, s));
        PCK(ctx, cudaStreamSynchronize(s));
        dev_free(ctx, d_np);
        for (int t = 255; t >= 0; --t) above[t] = above[t + 1] + hist[t];
        // First round: count only candidates u with path_code(|P_u|) >=
        // path_code(t), t = HUB_PRUNE * |P_v| / max(k, 10), which keeps every u
        // with |P_u| >= t (the k-th count of a hub tends to lie well above t);
        // a query whose k-th count comes out below the code's floor is counted
        // again with that count's code, which is then exact (hub_check_kernel).
        std::vector<HubQuery> hubs(ng);
        for (int i = 0; i < ng; ++i) {
            int64_t t = (int64_t)((double)npv[i] * HUB_PRUNE / std::max(k, 10));
            hubs[i] = HubQuery{gq[i], npv[i], (t < 2 || all_hub) ? 0u : path_code(t)};
        }
        // queries with a small filtered candidate bound count straight into a
        // device table (it stays in L2); the others go through the buckets
        auto run = [&](const std::vector<HubQuery>& list, std::vector<HubQuery>& again,
                       std::vector<HubQuery>& redo) -> panther_status {
            std::vector<HubQuery> tq, bq;
            for (const HubQuery& h : list) {
                bool table = h.thr > 0 && hub_bound(P, h, above) <= HUB_TABLE_BOUND;
                if (ctx->dbg_hub_route == 1) table = false;
                if (ctx->dbg_hub_route == 2) table = true;
                if (all_hub) table = true;                 // the buckets keep 64-entry lists
                (table ? tq : bq).push_back(h);
            }
            panther_status r = PANTHER_OK;
            if (!tq.empty()) r = hub_tables(ctx, P, queries, o, k, tq, above, redo);
            if (!r && !bq.empty()) r = hub_buckets(ctx, P, queries, o, k, bq, above, again, redo);
            return r;
        };
        std::vector<HubQuery> again, redo, redo2;
        st = run(hubs, again, redo);
        ctx->topk_stats[9] = (int64_t)redo.size();
        if (!st && !redo.empty()) st = run(redo, again, redo2);
        // a threshold equal to a lower bound of the k-th count always holds
        if (!st && !redo2.empty()) st = set_err(ctx, PANTHER_ECUDA, "hub threshold check failed twice");
        std::vector<HubQuery> none;
        if (!st && !again.empty()) st = hub_tables(ctx, P, queries, o, k, again, above, none);
        if (st) {
            dev_free(ctx, lists);
            dev_free(ctx, counts);
            return st;
        }
    }
    dev_free(ctx, lists);
    dev_free(ctx, counts);
    return PANTHER_OK;
}

extern "C" panther_status panther_topk(panther_ctx* ctx, const panther_index* ix, const panther_paths* p,
                                       const int32_t* queries, int64_t q, int k, int32_t* out_ids,
                                       uint32_t* out_counts, int flags) {
    if (!ctx || !ix || !p) return PANTHER_EINVAL;
    if (q < 0 || q > 0x7fffffffLL) return set_err(ctx, PANTHER_EINVAL, "q must be in [0, 2^31)");
    if (k < 1 || k > KMAX4) return set_err(ctx, PANTHER_EINVAL, "k must be in [1, 128]");
    if (ix->n != p->n || ix->R != p->R)
        return set_err(ctx, PANTHER_EINVAL, "index and paths do not belong together");
    if (q == 0) return PANTHER_OK;
    if (!queries || !out_ids || !out_counts) return set_err(ctx, PANTHER_EINVAL, "null query or output array");
    int mode = flags & 0xff;
    if (mode != PANTHER_TOPK_BATCHED && mode != PANTHER_TOPK_PLAIN) return set_err(ctx, PANTHER_EINVAL, "bad flags");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    bool host = (flags & PANTHER_IO_HOST) != 0;
    const int32_t* dq = queries;
    int32_t* di = out_ids;
    uint32_t* dc = out_counts;
    panther_status st;
    if (host) {
        int32_t* buf = nullptr;
        size_t qb = sizeof(int32_t) * q, ob = sizeof(int32_t) * q * k;
        if ((st = dev_alloc(ctx, (void**)&buf, qb + 2 * ob))) return st;
        PCK(ctx, cudaMemcpyAsync(buf, queries, qb, cudaMemcpyHostToDevice, s));
        dq = buf;
        di = buf + q;
        dc = (uint32_t*)(buf + q + (size_t)q * k);
        // Large batches run in chunks; the rows of a finished chunk travel to
        // the host on the copy stream while the next chunk computes.
        const int64_t chunk = (q >= (int64_t(1) << 22) && ctx->copy) ? ceil_div(q, 4) : q;
        cudaStream_t cs = ctx->copy ? ctx->copy : s;
        int64_t stats[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t c0 = 0; c0 < q && !st; c0 += chunk) {
            const int64_t qc = std::min(chunk, q - c0);
            st = topk_run(ctx, ix, p, dq + c0, qc, k, di + c0 * k, dc + c0 * k, mode == PANTHER_TOPK_PLAIN);
            if (st) break;
            for (int i = 0; i < 10; ++i) stats[i] += ctx->topk_stats[i];
            cudaError_t e = cs == s ? cudaSuccess : cudaEventRecord(ctx->copy_ev, s);
            if (!e && cs != s) e = cudaStreamWaitEvent(cs, ctx->copy_ev, 0);
            if (!e) e = cudaMemcpyAsync(out_ids + c0 * k, di + c0 * k, sizeof(int32_t) * qc * k,
                                        cudaMemcpyDeviceToHost, cs);
            if (!e) e = cudaMemcpyAsync(out_counts + c0 * k, dc + c0 * k, sizeof(uint32_t) * qc * k,
                                        cudaMemcpyDeviceToHost, cs);
            if (e) st = cuda_err(ctx, e, "top-k result copy");
        }
        for (int i = 0; i < 10; ++i) ctx->topk_stats[i] = stats[i];
        // the copies must finish before the buffer goes back to the pool
        cudaError_t e = cudaStreamSynchronize(cs);
        dev_free(ctx, buf);
        if (!st && e) st = cuda_err(ctx, e, "top-k result copy");
        if (!st) PCK(ctx, cudaStreamSynchronize(s));
        return st;
    }
    return topk_run(ctx, ix, p, dq, q, k, di, dc, mode == PANTHER_TOPK_PLAIN);
}

// pantherpp_vectors needs the counts-only form over all vertices
panther_status topk_counts_all(panther_ctx* ctx, const panther_index* ix, const panther_paths* p, int D,
                               uint32_t* theta) {
    return topk_run(ctx, ix, p, nullptr, ix->n, D, nullptr, theta, false);
}

// Autotuner: time the candidate launch shapes of the persistent kernel on the
// caller's own batch (CUDA events on the context stream, best of 3 after one
// warm-up run each) and keep the fastest in the context. Every shape returns
// identical results; only the split between tiers and the occupancy change.
extern "C" panther_status panther_tune_topk(panther_ctx* ctx, const panther_index* ix, const panther_paths* p,
                                            const int32_t* queries, int64_t q, int k, int32_t* out_ids,
                                            uint32_t* out_counts, int* chosen) {
    if (!ctx || !ix || !p || !queries || !out_ids || !out_counts || q < 1 || k < 1 || k > KMAX4)
        return set_err(ctx, PANTHER_EINVAL, "bad tuner arguments");
    if (ix->n != p->n || ix->R != p->R) return set_err(ctx, PANTHER_EINVAL, "index and paths do not belong together");
    cudaSetDevice(ctx->device);
    struct Shape { int threads, slots, bps; };
    const Shape cand[] = {{1024, 24576, 1}, {512, 12288, 2}, {256, 6144, 4}, {256, 4096, 6},
                          {512, 24576, 1}, {256, 8192, 3}, {128, 3072, 8}, {128, 4096, 6}};
    cudaEvent_t a, b;
    PCK(ctx, cudaEventCreate(&a));
    PCK(ctx, cudaEventCreate(&b));
    float best = 1e30f;
    int bi = 0;
    for (int i = 0; i < (int)(sizeof(cand) / sizeof(cand[0])); ++i) {
        ctx->topk_threads = cand[i].threads;
        ctx->topk_cta_slots = cand[i].slots;
        ctx->topk_blocks_per_sm = cand[i].bps;
        panther_status st = topk_run(ctx, ix, p, queries, q, k, out_ids, out_counts, false);
        if (st) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return st;
        }
        float t = 1e30f;
        for (int r = 0; r < 3; ++r) {
            PCK(ctx, cudaEventRecord(a, ctx->stream));
            if ((st = topk_run(ctx, ix, p, queries, q, k, out_ids, out_counts, false))) return st;
            PCK(ctx, cudaEventRecord(b, ctx->stream));
            PCK(ctx, cudaEventSynchronize(b));
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            t = ms < t ? ms : t;
        }
        if (t < best) {
            best = t;
            bi = i;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->topk_threads = cand[bi].threads;
    ctx->topk_cta_slots = cand[bi].slots;
    ctx->topk_blocks_per_sm = cand[bi].bps;
    if (chosen) {
        chosen[0] = cand[bi].threads;
        chosen[1] = cand[bi].slots;
        chosen[2] = cand[bi].bps;
    }
    return PANTHER_OK;
}

extern "C" panther_status panther_set_topk_shape(panther_ctx* ctx, int threads, int table_slots, int ctas_per_sm) {
    if (!ctx) return PANTHER_EINVAL;
    if ((threads != 128 && threads != 256 && threads != 512 && threads != 1024) || table_slots % 32 != 0 ||
        table_slots < threads / 32 * WSLOTS || table_slots > 24576 || ctas_per_sm < 1 || ctas_per_sm > 8)
        return set_err(ctx, PANTHER_EINVAL, "unsupported top-k launch shape");
    ctx->topk_threads = threads;
    ctx->topk_cta_slots = table_slots;
    ctx->topk_blocks_per_sm = ctas_per_sm;
    return PANTHER_OK;
}

extern "C" panther_status panther_topk_stats(panther_ctx* ctx, int64_t stats[10]) {
    if (!ctx || !stats) return PANTHER_EINVAL;
    for (int i = 0; i < 10; ++i) stats[i] = ctx->topk_stats[i];
    return PANTHER_OK;
}

extern "C" panther_status panther_debug_topk_route(panther_ctx* ctx, int64_t hub_min_cap, int route) {
    if (!ctx) return PANTHER_EINVAL;
    if (hub_min_cap < 0 || route < 0 || route > 2) return set_err(ctx, PANTHER_EINVAL, "bad test routing");
    ctx->dbg_hub_min_cap = hub_min_cap;
    ctx->dbg_hub_route = route;
    return PANTHER_OK;
}
