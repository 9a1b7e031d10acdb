// Graph upload, validation and the transition tables of Eq. (3).
//
// Per-vertex record vrec[v] = {start, deg, S_lo, S_hi} (16 B, one sector),
// S = sum of the row's weights.
//
// PREFIX table: entry j of row v = {inclusive cumulative weight, neighbour}
//   (uint2 when every S < 2^32, else uint4 {cum_lo, cum_hi, col, 0}).
// ALIAS table: entry c of row v = {thr_lo, thr_hi, col[c], col[alias[c]]}.
//   It is the integer Vose table with LIFO worklists (q_j = w_j * deg against
//   capacity S). A column popped as "small" gets the large that is current at
//   that moment; that large is determined by prefix sums of the deficits of
//   the smalls (S - q) and the excesses of the larges (q - S) taken in pop
//   order (descending column index), so every row is built in parallel and
//   the result equals the sequential construction:
//     small s_j (pop order j):  alias = L_i, i = min{ i : E_i >= D_(j-1) }
//     large L_i: if D_total > E_i, thr = S - (D_j* - E_i) with
//                j* = min{ j : D_j > E_i } and alias = L_(i+1);
//                otherwise thr = S and alias = itself.
//   D = inclusive prefix of deficits, E = inclusive prefix of excesses.
//
// Rows of degree <= 16 take one thread (the sequential construction), rows up
// to BIG_DEG one warp, and longer rows are cut into segments of SEG entries
// spread over CTAs, with a per-row scan of the segment sums in between.
//
// UNWEIGHTED: no table. The graph keeps its own copy of col, and a step picks
// col[start + Uniform[0, deg)] (t_ij = 1/deg, Eq. (3) with equal weights).
// The validation kernels read a NULL weight array as all ones.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int64_t BIG_DEG = 2048;   // rows above this are split into segments
constexpr int BLK = 512;            // threads of the CTA-per-row kernels

// ------------------------------------------------------------ groups ---
struct WarpG {
    static constexpr int size = 32;
    static constexpr int IPT = 1;
    __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ uint64_t incl_scan(uint64_t v, uint64_t* total) const {
        int l = rank();
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (l >= o) v += y;
        }
        *total = __shfl_sync(0xffffffffu, v, 31);
        return v;
    }
    __device__ __forceinline__ uint64_t sum(uint64_t v) const {
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
    __device__ __forceinline__ bool any(bool p) const { return __any_sync(0xffffffffu, p); }
    // inclusive scan of the chunk (thread r holds item r); returns the chunk total
    __device__ __forceinline__ uint64_t chunk_scan(uint64_t (&v)[IPT]) const {
        uint64_t tot;
        v[0] = incl_scan(v[0], &tot);
        return tot;
    }
};

struct BlockG {
    static constexpr int size = BLK;
    static constexpr int IPT = 16;
    uint64_t* sh;   // >= BLK/32 + 1 entries
    __device__ __forceinline__ int rank() const { return threadIdx.x; }
    __device__ __forceinline__ void sync() const { __syncthreads(); }
    __device__ uint64_t incl_scan(uint64_t v, uint64_t* total) const {
        int l = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (l >= o) v += y;
        }
        if (l == 31) sh[wi] = v;
        __syncthreads();
        if (wi == 0) {
            uint64_t s = l < BLK / 32 ? sh[l] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (l >= o) s += y;
            }
            if (l < BLK / 32) sh[l] = s;
        }
        __syncthreads();
        uint64_t r = v + (wi ? sh[wi - 1] : 0);
        *total = sh[BLK / 32 - 1];
        __syncthreads();
        return r;
    }
    __device__ uint64_t sum(uint64_t v) const {
        uint64_t t;
        incl_scan(v, &t);
        return t;
    }
    __device__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
    // inclusive scan of the chunk in blocked order (thread r holds items
    // r*IPT .. r*IPT+IPT-1): a sequential scan per thread, one block scan of
    // the thread totals; returns the chunk total
    template <int N>
    __device__ uint64_t chunk_scan(uint64_t (&v)[N]) const {
        uint64_t run = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            run += v[j];
            v[j] = run;
        }
        uint64_t tot;
        uint64_t before = incl_scan(run, &tot) - run;
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] += before;
        return tot;
    }
};


// G lanes of a warp per row (G divides 32), IPT items per lane in blocked
// order. Every lane of the warp must make the same calls (the shuffles span
// the warp, each group of G lanes scanning its own row).
template <int G, int IPT_>
struct SubG {
    static constexpr int size = G;
    static constexpr int IPT = IPT_;
    __device__ __forceinline__ int rank() const { return threadIdx.x & (G - 1); }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ uint64_t incl_scan(uint64_t v, uint64_t* total) const {
        const int l = rank();
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, v, o, G);
            if (l >= o) v += y;
        }
        *total = __shfl_sync(0xffffffffu, v, G - 1, G);
        return v;
    }
    __device__ __forceinline__ uint64_t sum(uint64_t v) const {
#pragma unroll
        for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
        return v;
    }
    __device__ __forceinline__ bool any(bool p) const {
        const unsigned m = __ballot_sync(0xffffffffu, p);
        const unsigned gbase = (threadIdx.x & 31) & ~(unsigned)(G - 1);
        return ((G == 32 ? m : (m >> gbase) & ((1u << G) - 1u))) != 0;
    }
    // inclusive scan of the group's G*IPT items; returns the total
    template <int N>
    __device__ __forceinline__ uint64_t chunk_scan(uint64_t (&v)[N]) const {
        uint64_t run = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            run += v[j];
            v[j] = run;
        }
        uint64_t tot;
        const uint64_t before = incl_scan(run, &tot) - run;
#pragma unroll
        for (int j = 0; j < N; ++j) v[j] += before;
        return tot;
    }
};

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdULL;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ULL;
    z ^= z >> 33;
    return z;
}
// hash of a directed entry; the graph is symmetric iff the sum over entries of
// H(v,u,w) equals the sum of H(u,v,w) (as multisets, with high probability)
__device__ __forceinline__ uint64_t edge_hash(uint64_t a, uint64_t b, uint64_t w) {
    return mix64((a << 32 | b) ^ mix64(w + 0x9E3779B97F4A7C15ULL));
}

// -------------------------------------------------------- row stats ---
struct StatsOut {
    uint4* vrec;
    uint32_t* status;
    unsigned long long* acc;   // [0] max S, [1] hash(v,u,w), [2] hash(u,v,w)
};

template <class G>
__device__ void row_stats(const G& g, int64_t v, int64_t start, int64_t deg, int64_t n, const int32_t* col,
                          const uint32_t* w, const StatsOut& o, uint64_t& h1, uint64_t& h2, uint64_t& mx) {
    uint64_t s = 0, a1 = 0, a2 = 0;
    bool bad = false;
    for (int64_t i = g.rank(); i < deg; i += G::size) {
        int32_t u = col[start + i];
        uint32_t ww = w ? w[start + i] : 1u;
        bad |= (u < 0) || ((int64_t)u >= n) || ((int64_t)u == v) || (ww == 0) ||
               (i > 0 && col[start + i - 1] >= u);
        s += ww;
        if (u >= 0) {
            a1 += edge_hash((uint64_t)v, (uint64_t)u, ww);
            a2 += edge_hash((uint64_t)u, (uint64_t)v, ww);
        }
    }
    s = g.sum(s);
    a1 = g.sum(a1);
    a2 = g.sum(a2);
    bad = g.any(bad);
    if (g.rank() == 0) {
        o.vrec[v] = make_uint4((uint32_t)start, (uint32_t)deg, (uint32_t)s, (uint32_t)(s >> 32));
        // q = w * deg must stay below 2^63 for the alias construction
        if (deg > 0 && (__umul64hi(s, (uint64_t)deg) != 0 || s * (uint64_t)deg >= (1ull << 63)))
            flag_status(o.status, ST_OVERFLOW);
        if (bad) {
            flag_status(o.status, ST_GRAPH_BAD);
            atomicMin(o.status + 1, (uint32_t)v);
        }
    }
    h1 += a1;
    h2 += a2;
    mx = s > mx ? s : mx;
}

// Rows of 17..4G entries are built by G lanes each (G = 8, 16, 32; four
// entries per lane, one chunk per pass), longer ones up to BIG_DEG by a warp
// in chunks of 32.
constexpr int64_t SHORT_LO = 17, SHORT_HI = 128;

// Row-pointer checks, and the lists of rows by length. counts: [0] rows above
// BIG_DEG (`big`), [1] 17..32 entries (front of `mid`), [2] 129..BIG_DEG
// (back of `mid`), [3] 33..64 (front of `mid2`), [4] 65..128 (back of `mid2`).
__global__ void rows_check_kernel(const int64_t* __restrict__ row_ptr, int64_t n, int64_t m,
                                  int32_t* __restrict__ big, int32_t* __restrict__ mid, int32_t* __restrict__ mid2,
                                  int* __restrict__ counts, uint32_t* status) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
    int cls = -1;
    if (v <= n) {
        const int64_t a = row_ptr[v];
        if (v == 0 && a != 0) flag_status(status, ST_GRAPH_BAD);
        if (v == n) {
            if (a != m) flag_status(status, ST_GRAPH_BAD);
        } else {
            const int64_t b = row_ptr[v + 1], d = b - a;
            if (b < a || a < 0 || b > m) flag_status(status, ST_GRAPH_BAD);
            else if (d > BIG_DEG) cls = 0;
            else if (d > SHORT_HI) cls = 2;
            else if (d > 64) cls = 4;
            else if (d > 32) cls = 3;
            else if (d >= SHORT_LO) cls = 1;
        }
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {   // one atomic per warp and list
        const unsigned mk = __ballot_sync(0xffffffffu, cls == c);
        if (!mk) continue;
        const int leader = __ffs(mk) - 1;
        int at = 0;
        if ((int)lane == leader) at = atomicAdd(&counts[c], __popc(mk));
        at = __shfl_sync(0xffffffffu, at, leader) + __popc(mk & lt);
        if (cls == c) {
            if (c == 0) big[at] = (int32_t)v;
            else if (c == 1) mid[at] = (int32_t)v;
            else if (c == 2) mid[n - 1 - at] = (int32_t)v;
            else if (c == 3) mid2[at] = (int32_t)v;
            else mid2[n - 1 - at] = (int32_t)v;
        }
    }
}

// list i of a short class: `rows[i]` (front) or `rows[n - 1 - i]` (back)
__device__ __forceinline__ int64_t list_at(const int32_t* rows, int64_t n, bool back, int64_t i) {
    return rows[back ? n - 1 - i : i];
}

// rows of degree <= SMALL_STATS: one thread per row
constexpr int64_t SMALL_STATS = 16;

__global__ void __launch_bounds__(256) stats_thread_kernel(const int64_t* __restrict__ row_ptr, int64_t n,
                                                           const int32_t* __restrict__ col,
                                                           const uint32_t* __restrict__ w, StatsOut o) {
    uint64_t h1 = 0, h2 = 0, mx = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = row_ptr[v], b = row_ptr[v + 1];
        if (b < a || b - a > SMALL_STATS) continue;
        uint64_t s = 0;
        bool bad = false;
        int32_t prev = -1;
        for (int64_t i = a; i < b; ++i) {
            int32_t u = col[i];
            uint32_t ww = w ? w[i] : 1u;
            bad |= (u < 0) || ((int64_t)u >= n) || ((int64_t)u == v) || (ww == 0) || (i > a && prev >= u);
            prev = u;
            s += ww;
            if (u >= 0) {
                h1 += edge_hash((uint64_t)v, (uint64_t)u, ww);
                h2 += edge_hash((uint64_t)u, (uint64_t)v, ww);
            }
        }
        const uint64_t deg = (uint64_t)(b - a);
        o.vrec[v] = make_uint4((uint32_t)a, (uint32_t)deg, (uint32_t)s, (uint32_t)(s >> 32));
        if (deg > 0 && (__umul64hi(s, deg) != 0 || s * deg >= (1ull << 63))) flag_status(o.status, ST_OVERFLOW);
        if (bad) {
            flag_status(o.status, ST_GRAPH_BAD);
            atomicMin(o.status + 1, (uint32_t)v);
        }
        mx = s > mx ? s : mx;
    }
    // one atomic per warp
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        h1 += __shfl_xor_sync(0xffffffffu, h1, d);
        h2 += __shfl_xor_sync(0xffffffffu, h2, d);
        uint64_t m2 = __shfl_xor_sync(0xffffffffu, mx, d);
        mx = m2 > mx ? m2 : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(o.acc + 0, (unsigned long long)mx);
        atomicAdd(o.acc + 1, (unsigned long long)h1);
        atomicAdd(o.acc + 2, (unsigned long long)h2);
    }
}

// ------------------------------------------------ rows above BIG_DEG ---
// Their work is split into segments of SEG entries (one CTA of BLK threads,
// SEG_IPT consecutive entries per thread): the plan seg_off[i] ..
// seg_off[i+1] holds the segments of big row i.
constexpr int SEG_IPT = 8;
constexpr int64_t SEG = (int64_t)BLK * SEG_IPT;

__device__ __forceinline__ int64_t seg_owner(const int64_t* seg_off, int64_t nbig, int64_t item) {
    int64_t lo = 0, hi = nbig - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void big_deg_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ big, int64_t nbig,
                               int64_t* __restrict__ deg) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nbig) deg[i] = row_ptr[big[i] + 1] - row_ptr[big[i]];
}

__global__ void stats_seg_kernel(const int64_t* __restrict__ row_ptr, int64_t n, const int32_t* __restrict__ col,
                                 const uint32_t* __restrict__ w, const int32_t* __restrict__ big,
                                 const int64_t* __restrict__ seg_off, int64_t nbig,
                                 unsigned long long* __restrict__ bigS, StatsOut o) {
    __shared__ uint64_t sh[BLK / 32 + 1];
    BlockG g{sh};
    const int64_t i = seg_owner(seg_off, nbig, blockIdx.x);
    const int64_t v = big[i];
    const int64_t start = row_ptr[v], end = row_ptr[v + 1];
    const int64_t a = start + (blockIdx.x - seg_off[i]) * SEG;
    const int64_t b = a + SEG < end ? a + SEG : end;
    uint64_t sum = 0, a1 = 0, a2 = 0;
    bool bad = false;
    for (int64_t e = a + threadIdx.x; e < b; e += BLK) {
        int32_t u = col[e];
        uint32_t ww = (w ? w[e] : 1u);
        bad |= (u < 0) || ((int64_t)u >= n) || ((int64_t)u == v) || (ww == 0) || (e > start && col[e - 1] >= u);
        sum += ww;
        if (u >= 0) {
            a1 += edge_hash((uint64_t)v, (uint64_t)u, ww);
            a2 += edge_hash((uint64_t)u, (uint64_t)v, ww);
        }
    }
    sum = g.sum(sum);
    a1 = g.sum(a1);
    a2 = g.sum(a2);
    bad = g.any(bad);
    if (threadIdx.x == 0) {
        atomicAdd(bigS + i, (unsigned long long)sum);
        atomicAdd(o.acc + 1, (unsigned long long)a1);
        atomicAdd(o.acc + 2, (unsigned long long)a2);
        if (bad) {
            flag_status(o.status, ST_GRAPH_BAD);
            atomicMin(o.status + 1, (uint32_t)v);
        }
    }
}

__global__ void big_finalize_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ big, int64_t nbig,
                                    const unsigned long long* __restrict__ bigS, StatsOut o) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbig) return;
    const int64_t v = big[i];
    const uint64_t start = (uint64_t)row_ptr[v], deg = (uint64_t)(row_ptr[v + 1] - row_ptr[v]);
    const uint64_t S = bigS[i];
    o.vrec[v] = make_uint4((uint32_t)start, (uint32_t)deg, (uint32_t)S, (uint32_t)(S >> 32));
    if (__umul64hi(S, deg) != 0 || S * deg >= (1ull << 63)) flag_status(o.status, ST_OVERFLOW);
    atomicMax(o.acc + 0, (unsigned long long)S);
}

// short rows (at most 4G entries): G lanes per row, 32/G rows per warp; the
// loop is warp-uniform (idle groups take a row of length 0 and write nothing)
template <int G>
__global__ void stats_short_kernel(const int64_t* __restrict__ row_ptr, int64_t n, const int32_t* __restrict__ col,
                                   const uint32_t* __restrict__ w, const int32_t* __restrict__ rows, bool back,
                                   int64_t nrows, StatsOut o) {
    SubG<G, 4> g;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / G;
    uint64_t h1 = 0, h2 = 0, mx = 0;
    for (int64_t it = gid;; it += ng) {
        const bool act = it < nrows;
        if (!__any_sync(0xffffffffu, act)) break;
        const int64_t v = act ? list_at(rows, n, back, it) : 0;
        const int64_t a = act ? row_ptr[v] : 0, deg = act ? row_ptr[v + 1] - a : 0;
        uint64_t sum = 0, a1 = 0, a2 = 0;
        bool bad = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = (int64_t)g.rank() * 4 + j;
            if (i < deg) {
                const int32_t u = col[a + i];
                const uint32_t ww = (w ? w[a + i] : 1u);
                bad |= (u < 0) || ((int64_t)u >= n) || ((int64_t)u == v) || (ww == 0) ||
                       (i > 0 && col[a + i - 1] >= u);
                sum += ww;
                if (u >= 0) {
                    a1 += edge_hash((uint64_t)v, (uint64_t)u, ww);
                    a2 += edge_hash((uint64_t)u, (uint64_t)v, ww);
                }
            }
        }
        h1 += a1;
        h2 += a2;
        sum = g.sum(sum);
        bad = g.any(bad);
        if (act && g.rank() == 0) {
            o.vrec[v] = make_uint4((uint32_t)a, (uint32_t)deg, (uint32_t)sum, (uint32_t)(sum >> 32));
            if (__umul64hi(sum, (uint64_t)deg) != 0 || sum * (uint64_t)deg >= (1ull << 63))
                flag_status(o.status, ST_OVERFLOW);
            if (bad) {
                flag_status(o.status, ST_GRAPH_BAD);
                atomicMin(o.status + 1, (uint32_t)v);
            }
        }
        mx = sum > mx ? sum : mx;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        h1 += __shfl_xor_sync(0xffffffffu, h1, d);
        h2 += __shfl_xor_sync(0xffffffffu, h2, d);
        const uint64_t m2 = __shfl_xor_sync(0xffffffffu, mx, d);
        mx = m2 > mx ? m2 : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(o.acc + 0, (unsigned long long)mx);
        atomicAdd(o.acc + 1, (unsigned long long)h1);
        atomicAdd(o.acc + 2, (unsigned long long)h2);
    }
}

// medium rows (listed from the back of `mid`): one warp per row
__global__ void stats_warp_kernel(const int64_t* __restrict__ row_ptr, int64_t n, const int32_t* __restrict__ col,
                                  const uint32_t* __restrict__ w, const int32_t* __restrict__ mid, int64_t nmed,
                                  StatsOut o) {
    WarpG g;
    int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t h1 = 0, h2 = 0, mx = 0;
    for (int64_t i = wid; i < nmed; i += nw) {
        const int64_t v = mid[n - 1 - i];
        const int64_t a = row_ptr[v], b = row_ptr[v + 1];
        row_stats(g, v, a, b - a, n, col, w, o, h1, h2, mx);
    }
    if (g.rank() == 0) {
        atomicMax(o.acc + 0, (unsigned long long)mx);
        atomicAdd(o.acc + 1, (unsigned long long)h1);
        atomicAdd(o.acc + 2, (unsigned long long)h2);
    }
}

// ---------------------------------------------------------- prefix ---
template <class G, bool WIDE>
__device__ void row_prefix(const G& g, int64_t start, int64_t deg, const int32_t* col, const uint32_t* w,
                           void* tab) {
    constexpr int IPT = G::IPT;
    uint64_t carry = 0;
    for (int64_t base = 0; base < deg; base += (int64_t)G::size * IPT) {
        uint64_t v[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            int64_t i = base + (int64_t)g.rank() * IPT + j;
            v[j] = i < deg ? w[start + i] : 0;
        }
        uint64_t tot = g.chunk_scan(v);
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            int64_t i = base + (int64_t)g.rank() * IPT + j;
            if (i < deg) {
                uint64_t inc = carry + v[j];
                if (WIDE)
                    ((uint4*)tab)[start + i] =
                        make_uint4((uint32_t)inc, (uint32_t)(inc >> 32), (uint32_t)col[start + i], 0u);
                else
                    ((uint2*)tab)[start + i] = make_uint2((uint32_t)inc, (uint32_t)col[start + i]);
            }
        }
        carry += tot;
    }
}

template <bool WIDE>
__global__ void prefix_warp_kernel(const int64_t* __restrict__ row_ptr, int64_t n, const int32_t* __restrict__ col,
                                   const uint32_t* __restrict__ w, void* tab) {
    WarpG g;
    int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = wid; v < n; v += nw) {
        int64_t a = row_ptr[v], d = row_ptr[v + 1] - a;
        if (d > BIG_DEG) continue;
        row_prefix<WarpG, WIDE>(g, a, d, col, w, tab);
    }
}

template <bool WIDE>
__global__ void prefix_block_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                    const uint32_t* __restrict__ w, const int32_t* __restrict__ big, void* tab) {
    __shared__ uint64_t sh[BLK / 32 + 1];
    BlockG g{sh};
    int64_t v = big[blockIdx.x];
    row_prefix<BlockG, WIDE>(g, row_ptr[v], row_ptr[v + 1] - row_ptr[v], col, w, tab);
}

// ----------------------------------------------------------- alias ---
// first index in [0,cnt) with a[i] >= x (cnt if none)
__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* a, int64_t cnt, uint64_t x) {
    int64_t lo = 0, hi = cnt;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}
// first index in [0,cnt) with a[i] > x (cnt if none)
__device__ __forceinline__ int64_t upper_bound_u64(const uint64_t* a, int64_t cnt, uint64_t x) {
    int64_t lo = 0, hi = cnt;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <class G>
__device__ int64_t row_alias_prep(const G& g, int64_t start, int64_t deg, uint64_t S, const uint32_t* w,
                                  int32_t* sidx, uint64_t* scum) {
    if (deg == 0) return 0;
    const uint64_t d = (uint64_t)deg;
    // A: number of small columns (q < S)
    uint64_t ns = 0;
    for (int64_t i = g.rank(); i < deg; i += G::size) ns += ((uint64_t)w[start + i] * d < S);
    ns = g.sum(ns);
    const int64_t nsm = (int64_t)ns, nl = deg - nsm;
    // B: columns in pop order (descending index) - smalls at [0,ns), larges at [ns,deg)
    constexpr int IPT = G::IPT;
    constexpr int64_t CH = (int64_t)G::size * IPT;
    uint64_t cs = 0;
    for (int64_t base = 0; base < deg; base += CH) {
        uint64_t f[IPT];
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            int64_t i = base + (int64_t)g.rank() * IPT + j;
            f[j] = (i < deg && (uint64_t)w[start + i] * d < S) ? 1 : 0;
        }
        uint64_t ts = g.chunk_scan(f);   // f = smalls up to and including each item within the chunk
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            int64_t i = base + (int64_t)g.rank() * IPT + j;
            if (i < deg) {
                bool sm = (uint64_t)w[start + i] * d < S;
                int64_t rs = (int64_t)(cs + f[j]) - (sm ? 1 : 0);   // smalls before i
                int64_t rl = i - rs;                     // larges before i
                if (sm) sidx[start + nsm - 1 - rs] = (int32_t)i;
                else sidx[start + nsm + nl - 1 - rl] = (int32_t)i;
            }
        }
        cs += ts;
    }
    g.sync();
    // C: D = prefix of deficits S - q over smalls, E = prefix of excesses q - S over larges
    for (int part = 0; part < 2; ++part) {
        const int64_t cnt = part == 0 ? nsm : nl;
        const int64_t o0 = part == 0 ? 0 : nsm;
        uint64_t carry = 0;
        for (int64_t base = 0; base < cnt; base += CH) {
            uint64_t x[IPT];
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                int64_t p = base + (int64_t)g.rank() * IPT + j;
                uint64_t q = p < cnt ? (uint64_t)w[start + sidx[start + o0 + p]] * d : 0;
                x[j] = p < cnt ? (part == 0 ? S - q : q - S) : 0;
            }
            uint64_t tot = g.chunk_scan(x);   // inclusive
#pragma unroll
            for (int j = 0; j < IPT; ++j) {
                int64_t p = base + (int64_t)g.rank() * IPT + j;
                if (p < cnt) scum[start + o0 + p] = carry + x[j];
            }
            carry += tot;
        }
    }
    g.sync();
    return nsm;
}

// Pass D of the alias construction: thread `tid` of `nthreads` takes a
// contiguous run of the smalls and of the larges (in pop order) and walks the
// other sorted sequence forward from one binary search.
constexpr int ASSIGN_WAYS = 4;

__device__ void alias_assign(int64_t start, int64_t deg, uint64_t S, int64_t nsm, const int32_t* __restrict__ col,
                             const uint32_t* __restrict__ w, uint4* __restrict__ tab,
                             const int32_t* __restrict__ sidx, const uint64_t* __restrict__ scum, int64_t tid,
                             int64_t nthreads) {
    const uint64_t d = (uint64_t)deg;
    const int64_t nl = deg - nsm;
    const uint64_t* __restrict__ D = scum + start;
    const uint64_t* __restrict__ E = scum + start + nsm;
    const int32_t* __restrict__ SI = sidx + start;
    const int32_t* __restrict__ LI = sidx + start + nsm;
    const uint64_t Dtot = nsm ? D[nsm - 1] : 0;
    // D: table entries. Each thread takes a contiguous run and walks the
    // other sorted sequence forward from one binary search; the run is split
    // in ASSIGN_WAYS parts walked in lockstep, so as many independent chains
    // of loads are in flight.
    {
        const int64_t per = (nsm + nthreads - 1) / nthreads;
        const int64_t p0 = tid * per, p1 = p0 + per < nsm ? p0 + per : nsm;
        if (p0 < p1) {
            constexpr int W = ASSIGN_WAYS;
            const int64_t len = (p1 - p0 + W - 1) / W;
            int64_t pp[W], pe[W], ii[W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                pp[u] = p0 + u * len < p1 ? p0 + u * len : p1;
                pe[u] = pp[u] + len < p1 ? pp[u] + len : p1;
                ii[u] = (nl && pp[u] < pe[u]) ? lower_bound_u64(E, nl, pp[u] ? D[pp[u] - 1] : 0) : 0;
            }
            auto small_step = [&](int64_t p, int64_t& i) {
                const int32_t j = SI[p];
                const uint64_t dprev = p ? D[p - 1] : 0;
                const uint32_t wj = w[start + j];
                const int32_t self = col[start + j];
                while (i < nl && E[i] < dprev) ++i;
                const uint64_t q = (uint64_t)wj * d;
                if (nl == 0 || i >= nl)   // cannot happen for consistent integer weights
                    tab[start + j] = make_uint4((uint32_t)S, (uint32_t)(S >> 32), (uint32_t)self, (uint32_t)self);
                else
                    tab[start + j] = make_uint4((uint32_t)q, (uint32_t)(q >> 32), (uint32_t)self,
                                                (uint32_t)col[start + LI[i]]);
            };
            for (int64_t s2 = 0; s2 < len; ++s2)
#pragma unroll
                for (int u = 0; u < W; ++u)
                    if (pp[u] + s2 < pe[u]) small_step(pp[u] + s2, ii[u]);
        }
    }
    {
        const int64_t per = (nl + nthreads - 1) / nthreads;
        const int64_t i0 = tid * per, i1 = i0 + per < nl ? i0 + per : nl;
        if (i0 < i1) {
            constexpr int W = ASSIGN_WAYS;
            const int64_t len = (i1 - i0 + W - 1) / W;
            int64_t xx[W], xe[W], jj[W];
#pragma unroll
            for (int u = 0; u < W; ++u) {
                xx[u] = i0 + u * len < i1 ? i0 + u * len : i1;
                xe[u] = xx[u] + len < i1 ? xx[u] + len : i1;
                jj[u] = xx[u] < xe[u] ? upper_bound_u64(D, nsm, E[xx[u]]) : 0;
            }
            auto large_step = [&](int64_t i, int64_t& js) {
                const uint64_t Ei = E[i];
                const int32_t j = LI[i];
                const int32_t jnext = i + 1 < nl ? LI[i + 1] : -1;
                const int32_t self = col[start + j];
                while (js < nsm && D[js] <= Ei) ++js;
                if (Dtot > Ei && i + 1 < nl) {
                    uint64_t thr = S - (D[js] - Ei);
                    tab[start + j] = make_uint4((uint32_t)thr, (uint32_t)(thr >> 32), (uint32_t)self,
                                                (uint32_t)col[start + jnext]);
                } else {
                    tab[start + j] = make_uint4((uint32_t)S, (uint32_t)(S >> 32), (uint32_t)self, (uint32_t)self);
                }
            };
            for (int64_t s2 = 0; s2 < len; ++s2)
#pragma unroll
                for (int u = 0; u < W; ++u)
                    if (xx[u] + s2 < xe[u]) large_step(xx[u] + s2, jj[u]);
        }
    }
}


template <class G>
__device__ void row_alias(const G& g, int64_t start, int64_t deg, uint64_t S, const int32_t* col,
                          const uint32_t* w, uint4* tab, int32_t* sidx, uint64_t* scum) {
    if (deg == 0) return;
    int64_t nsm = row_alias_prep(g, start, deg, S, w, sidx, scum);
    alias_assign(start, deg, S, nsm, col, w, tab, sidx, scum, g.rank(), G::size);
}

// rows of degree <= SMALL_DEG: one thread per row runs the sequential LIFO
// construction (worklists in registers/local memory), writing each entry
// when it is final
constexpr int SMALL_DEG = 16;

__global__ void __launch_bounds__(256) alias_thread_kernel(const uint4* __restrict__ vrec, int64_t n,
                                                           const int32_t* __restrict__ col,
                                                           const uint32_t* __restrict__ w, uint4* tab) {
    // the worklists and the row's columns live in shared memory, one column
    // per thread (no local memory, no bank conflicts)
    __shared__ uint64_t qs[SMALL_DEG][256];
    __shared__ int32_t cs[SMALL_DEG][256];
    __shared__ int8_t sms[SMALL_DEG][256], lgs[SMALL_DEG][256];
    const int t = threadIdx.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        uint4 r = vrec[v];
        const int d = (int)r.y;
        if (d == 0 || d > SMALL_DEG) continue;
        const int64_t start = r.x;
        const uint64_t S = (uint64_t)r.z | ((uint64_t)r.w << 32);
        auto q = [&](int j) -> uint64_t& { return qs[j][t]; };
        auto c = [&](int j) -> int32_t& { return cs[j][t]; };
        auto sm = [&](int j) -> int8_t& { return sms[j][t]; };
        auto lg = [&](int j) -> int8_t& { return lgs[j][t]; };
        // the row's weights and columns: every load issued before the first use
        uint32_t wr[SMALL_DEG];
        int32_t cr[SMALL_DEG];
#pragma unroll
        for (int j = 0; j < SMALL_DEG; ++j)
            if (j < d) {
                wr[j] = w[start + j];
                cr[j] = col[start + j];
            }
        int ns = 0, nl = 0;
#pragma unroll
        for (int j = 0; j < SMALL_DEG; ++j)
            if (j < d) {
                const uint64_t qj = (uint64_t)wr[j] * (uint64_t)d;
                q(j) = qj;
                c(j) = cr[j];
                if (qj < S) sm(ns++) = (int8_t)j; else lg(nl++) = (int8_t)j;
            }
        while (ns > 0 && nl > 0) {
            const int a = sm(--ns), b = lg(--nl);
            const uint64_t qa = q(a);
            tab[start + a] = make_uint4((uint32_t)qa, (uint32_t)(qa >> 32), (uint32_t)c(a), (uint32_t)c(b));
            const uint64_t qb = q(b) - (S - qa);
            q(b) = qb;
            if (qb < S) sm(ns++) = (int8_t)b; else lg(nl++) = (int8_t)b;
        }
        while (nl > 0) {
            const int b = lg(--nl);
            tab[start + b] = make_uint4((uint32_t)S, (uint32_t)(S >> 32), (uint32_t)c(b), (uint32_t)c(b));
        }
        while (ns > 0) {
            const int a = sm(--ns);
            tab[start + a] = make_uint4((uint32_t)S, (uint32_t)(S >> 32), (uint32_t)c(a), (uint32_t)c(a));
        }
    }
}

__global__ void alias_warp_kernel(const uint4* __restrict__ vrec, int64_t n, const int32_t* __restrict__ col,
                                  const uint32_t* __restrict__ w, const int32_t* __restrict__ mid, int64_t nmed,
                                  uint4* tab, int32_t* sidx, uint64_t* scum) {
    WarpG g;
    int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = wid; i < nmed; i += nw) {
        const uint4 r = vrec[mid[n - 1 - i]];
        row_alias(g, (int64_t)r.x, (int64_t)r.y, (uint64_t)r.z | ((uint64_t)r.w << 32), col, w, tab, sidx, scum);
    }
}

// Short rows: G lanes per row, 4 entries per lane, so every pass is one
// chunk and every group of the warp makes the same shuffles (idle groups run
// on a row of length 0).
template <int G>
__global__ void alias_short_kernel(const uint4* __restrict__ vrec, int64_t n, const int32_t* __restrict__ col,
                                   const uint32_t* __restrict__ w, const int32_t* __restrict__ rows, bool back,
                                   int64_t nrows, uint4* tab, int32_t* sidx, uint64_t* scum) {
    SubG<G, 4> g;
    const int64_t gid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int64_t ng = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t it = gid;; it += ng) {
        const bool act = it < nrows;
        if (!__any_sync(0xffffffffu, act)) break;
        uint4 r = make_uint4(0, 0, 0, 0);
        if (act) r = vrec[list_at(rows, n, back, it)];
        const int64_t start = (int64_t)r.x, deg = (int64_t)r.y;
        const uint64_t S = (uint64_t)r.z | ((uint64_t)r.w << 32), d = (uint64_t)deg;
        const int rk = g.rank();
        // A+B: smalls (q < S) and their pop positions
        uint64_t f[4];
        uint32_t wv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = (int64_t)rk * 4 + j;
            wv[j] = i < deg ? w[start + i] : 0u;
            f[j] = (i < deg && (uint64_t)wv[j] * d < S) ? 1 : 0;
        }
        const int64_t nsm = (int64_t)g.chunk_scan(f), nl = deg - nsm;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = (int64_t)rk * 4 + j;
            if (i < deg) {
                const bool sm = (uint64_t)wv[j] * d < S;
                const int64_t rs = (int64_t)f[j] - (sm ? 1 : 0);   // smalls before i
                sidx[start + (sm ? nsm - 1 - rs : deg - 1 - (i - rs))] = (int32_t)i;
            }
        }
        g.sync();
        // C: inclusive prefixes of deficits (smalls) and excesses (larges) in pop order
        uint64_t x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t p = (int64_t)rk * 4 + j;
            x[j] = p < nsm ? S - (uint64_t)w[start + sidx[start + p]] * d : 0;
        }
        g.chunk_scan(x);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t p = (int64_t)rk * 4 + j;
            if (p < nsm) scum[start + p] = x[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t p = (int64_t)rk * 4 + j;
            x[j] = p < nl ? (uint64_t)w[start + sidx[start + nsm + p]] * d - S : 0;
        }
        g.chunk_scan(x);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t p = (int64_t)rk * 4 + j;
            if (p < nl) scum[start + nsm + p] = x[j];
        }
        g.sync();
        if (deg > 0) alias_assign(start, deg, S, nsm, col, w, tab, sidx, scum, rk, G);
        g.sync();
    }
}

// Passes A-C for the rows above BIG_DEG, split over segments. In pop order
// (descending index) the smalls come first, so the small at index i has pop
// position nsm-1-rs(i) (rs = smalls before i) and its inclusive prefix of
// deficits D is the sum over the smalls at index >= i: a suffix sum in index
// order. Likewise for the larges and E. Each segment therefore needs only the
// smalls before it and the deficit / excess sums after it within its row.
struct SegRow {
    int64_t row, start, deg, a, b;   // entries a .. b-1 of the row's deg
    uint64_t S;
};

__device__ __forceinline__ SegRow seg_row(const uint4* vrec, const int32_t* big, const int64_t* seg_off,
                                          int64_t nbig) {
    SegRow r;
    r.row = seg_owner(seg_off, nbig, blockIdx.x);
    const uint4 v = vrec[big[r.row]];
    r.start = (int64_t)v.x;
    r.deg = (int64_t)v.y;
    r.S = (uint64_t)v.z | ((uint64_t)v.w << 32);
    r.a = (blockIdx.x - seg_off[r.row]) * SEG;
    r.b = r.a + SEG < r.deg ? r.a + SEG : r.deg;
    return r;
}

// per segment: smalls, sum of deficits S - q, sum of excesses q - S
__global__ void __launch_bounds__(BLK) big_count_kernel(const uint4* __restrict__ vrec, const uint32_t* __restrict__ w,
                                                        const int32_t* __restrict__ big,
                                                        const int64_t* __restrict__ seg_off, int64_t nbig,
                                                        uint64_t* __restrict__ segsum) {
    __shared__ uint64_t sh[BLK / 32 + 1];
    BlockG g{sh};
    const SegRow r = seg_row(vrec, big, seg_off, nbig);
    const uint64_t d = (uint64_t)r.deg;
    uint64_t ns = 0, df = 0, ex = 0;
    for (int64_t i = r.a + threadIdx.x; i < r.b; i += BLK) {
        const uint64_t q = (uint64_t)w[r.start + i] * d;
        if (q < r.S) {
            ++ns;
            df += r.S - q;
        } else {
            ex += q - r.S;
        }
    }
    ns = g.sum(ns);
    df = g.sum(df);
    ex = g.sum(ex);
    if (threadIdx.x == 0) {
        segsum[3 * blockIdx.x + 0] = ns;
        segsum[3 * blockIdx.x + 1] = df;
        segsum[3 * blockIdx.x + 2] = ex;
    }
}

// one warp per big row: smalls before each segment, deficit and excess sums
// after it (in place over segsum), and the row's small count
__global__ void big_rowscan_kernel(const int64_t* __restrict__ seg_off, int64_t nbig, uint64_t* __restrict__ segsum,
                                   int64_t* __restrict__ bign) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= nbig) return;
    WarpG g;
    const int64_t s0 = seg_off[row], s1 = seg_off[row + 1];
    uint64_t tdf = 0, tex = 0;
    for (int64_t sg = s0 + lane; sg < s1; sg += 32) {
        tdf += segsum[3 * sg + 1];
        tex += segsum[3 * sg + 2];
    }
    tdf = g.sum(tdf);
    tex = g.sum(tex);
    uint64_t cns = 0, cdf = 0, cex = 0;
    for (int64_t base = s0; base < s1; base += 32) {
        const int64_t sg = base + lane;
        const bool ok = sg < s1;
        const uint64_t ns = ok ? segsum[3 * sg + 0] : 0, df = ok ? segsum[3 * sg + 1] : 0,
                       ex = ok ? segsum[3 * sg + 2] : 0;
        uint64_t t_ns, t_df, t_ex;
        const uint64_t i_ns = g.incl_scan(ns, &t_ns), i_df = g.incl_scan(df, &t_df), i_ex = g.incl_scan(ex, &t_ex);
        if (ok) {
            segsum[3 * sg + 0] = cns + i_ns - ns;
            segsum[3 * sg + 1] = tdf - (cdf + i_df);
            segsum[3 * sg + 2] = tex - (cex + i_ex);
        }
        cns += t_ns;
        cdf += t_df;
        cex += t_ex;
    }
    if (lane == 0) bign[row] = (int64_t)cns;
}

// pop-order positions (sidx) and inclusive prefixes D / E (scum) of a segment
__global__ void __launch_bounds__(BLK) big_place_kernel(const uint4* __restrict__ vrec, const uint32_t* __restrict__ w,
                                                        const int32_t* __restrict__ big,
                                                        const int64_t* __restrict__ seg_off, int64_t nbig,
                                                        const uint64_t* __restrict__ segsum,
                                                        const int64_t* __restrict__ bign, int32_t* __restrict__ sidx,
                                                        uint64_t* __restrict__ scum) {
    __shared__ uint64_t sh[BLK / 32 + 1];
    BlockG g{sh};
    const SegRow r = seg_row(vrec, big, seg_off, nbig);
    const uint64_t d = (uint64_t)r.deg;
    const uint64_t ns_before = segsum[3 * blockIdx.x + 0], df_after = segsum[3 * blockIdx.x + 1],
                   ex_after = segsum[3 * blockIdx.x + 2];
    const int64_t nsm = bign[r.row];
    const int64_t i0 = r.a + (int64_t)threadIdx.x * SEG_IPT;
    uint64_t q[SEG_IPT], x[SEG_IPT];   // q = S marks an entry past the segment (in neither class)
    int32_t pos[SEG_IPT];
#pragma unroll
    for (int j = 0; j < SEG_IPT; ++j) {
        q[j] = i0 + j < r.b ? (uint64_t)w[r.start + i0 + j] * d : r.S;
        x[j] = q[j] < r.S ? 1 : 0;
    }
    g.chunk_scan(x);   // smalls up to and including each entry within the segment
#pragma unroll
    for (int j = 0; j < SEG_IPT; ++j) {
        const int64_t i = i0 + j;
        const int64_t rs = (int64_t)(ns_before + x[j]) - (q[j] < r.S ? 1 : 0);   // smalls before i
        pos[j] = q[j] < r.S ? (int32_t)(nsm - 1 - rs) : (int32_t)(r.deg - 1 - (i - rs));
    }
    // deficits, then excesses: suffix within the segment = total - inclusive prefix + own
#pragma unroll
    for (int j = 0; j < SEG_IPT; ++j) x[j] = q[j] < r.S ? r.S - q[j] : 0;
    uint64_t tot = g.chunk_scan(x);
#pragma unroll
    for (int j = 0; j < SEG_IPT; ++j)
        if (q[j] < r.S) {
            sidx[r.start + pos[j]] = (int32_t)(i0 + j);
            scum[r.start + pos[j]] = df_after + (tot - x[j]) + (r.S - q[j]);
        }
#pragma unroll
    for (int j = 0; j < SEG_IPT; ++j) x[j] = (q[j] >= r.S && i0 + j < r.b) ? q[j] - r.S : 0;
    tot = g.chunk_scan(x);
#pragma unroll
    for (int j = 0; j < SEG_IPT; ++j)
        if (q[j] >= r.S && i0 + j < r.b) {
            sidx[r.start + pos[j]] = (int32_t)(i0 + j);
            scum[r.start + pos[j]] = ex_after + (tot - x[j]) + (q[j] - r.S);
        }
}

// pass D for the rows above BIG_DEG: one CTA per segment of the row
__global__ void alias_assign_kernel(const uint4* __restrict__ vrec, const int32_t* __restrict__ col,
                                    const uint32_t* __restrict__ w, const int32_t* __restrict__ big,
                                    const int64_t* __restrict__ bign, const int64_t* __restrict__ seg_off,
                                    int64_t nbig, uint4* tab, const int32_t* __restrict__ sidx,
                                    const uint64_t* __restrict__ scum) {
    const int64_t row = seg_owner(seg_off, nbig, blockIdx.x);
    const int64_t parts = seg_off[row + 1] - seg_off[row], part = blockIdx.x - seg_off[row];
    uint4 r = vrec[big[row]];
    alias_assign((int64_t)r.x, (int64_t)r.y, (uint64_t)r.z | ((uint64_t)r.w << 32), bign[row], col, w, tab, sidx,
                 scum, part * blockDim.x + threadIdx.x, parts * blockDim.x);
}

unsigned grid_for(panther_ctx* ctx, int64_t items_per_block_unit, int64_t n, int threads) {
    int64_t blocks = ceil_div(n, items_per_block_unit);
    int64_t cap = (int64_t)ctx->num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    (void)threads;
    return (unsigned)blocks;
}

}  // namespace

extern "C" panther_status panther_build_graph(panther_ctx* ctx, int64_t n, int64_t m, const int64_t* row_ptr,
                                              const int32_t* col, const uint32_t* w, int mem, int modes,
                                              panther_graph** out) {
    if (!ctx || !out) return PANTHER_EINVAL;
    *out = nullptr;
    if (n < 1 || n >= (int64_t(1) << 31)) return set_err(ctx, PANTHER_EINVAL, "n must be in [1, 2^31)");
    if (m < 0) return set_err(ctx, PANTHER_EINVAL, "m must be >= 0");
    if (m >= (int64_t(1) << 32)) return set_err(ctx, PANTHER_EOVERFLOW, "m must be < 2^32");
    if (modes < 1 || modes > 7)
        return set_err(ctx, PANTHER_EINVAL, "modes must combine PREFIX, ALIAS and UNWEIGHTED");
    if (!row_ptr || (m > 0 && (!col || (!w && modes != PANTHER_MODE_UNWEIGHTED))))
        return set_err(ctx, PANTHER_EINVAL, "null graph array (w may be NULL only for UNWEIGHTED alone)");
    if (mem != PANTHER_MEM_HOST && mem != PANTHER_MEM_DEVICE) return set_err(ctx, PANTHER_EINVAL, "bad mem");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    cudaMemcpyKind kind = mem == PANTHER_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;

    panther_graph* g = new panther_graph();
    g->ctx = ctx;
    g->n = n;
    g->m = m;
    g->modes = modes;
    // Host inputs are staged in temporary device buffers; device inputs are
    // read in place (the call returns only after the tables are built, and the
    // tables carry the neighbour ids, so nothing of the CSR is kept).
    int64_t* t_rp = nullptr;
    int32_t* t_col = nullptr;
    uint32_t* t_w = nullptr;
    int32_t* big = nullptr;
    int32_t* mid = nullptr;
    int32_t* mid2 = nullptr;
    int* nbig = nullptr;
    unsigned long long* acc = nullptr;
    panther_status st = PANTHER_OK;
    auto fail = [&](panther_status e) {
        dev_free(ctx, t_rp);
        dev_free(ctx, t_col);
        dev_free(ctx, t_w);
        dev_free(ctx, big);
        dev_free(ctx, mid);
        dev_free(ctx, mid2);
        dev_free(ctx, nbig);
        dev_free(ctx, acc);
        cudaStreamSynchronize(s);
        panther_free_graph(g);
        return e;
    };
    if ((st = dev_alloc(ctx, (void**)&g->vrec, sizeof(uint4) * n)) ||
        (st = dev_alloc(ctx, (void**)&big, sizeof(int32_t) * (n + 1))) ||
        (st = dev_alloc(ctx, (void**)&mid, sizeof(int32_t) * n)) ||
        (st = dev_alloc(ctx, (void**)&mid2, sizeof(int32_t) * n)) ||
        (st = dev_alloc(ctx, (void**)&nbig, sizeof(int) * 8)) ||
        (st = dev_alloc(ctx, (void**)&acc, sizeof(unsigned long long) * 4)))
        return fail(st);
    cudaError_t e;
    if (mem == PANTHER_MEM_HOST) {
        if ((st = dev_alloc(ctx, (void**)&t_rp, sizeof(int64_t) * (n + 1))) ||
            (st = dev_alloc(ctx, (void**)&t_col, sizeof(int32_t) * m)) ||
            (w && (st = dev_alloc(ctx, (void**)&t_w, sizeof(uint32_t) * m))))
            return fail(st);
        if ((e = cudaMemcpyAsync(t_rp, row_ptr, sizeof(int64_t) * (n + 1), kind, s)) ||
            (m && (e = cudaMemcpyAsync(t_col, col, sizeof(int32_t) * m, kind, s))) ||
            (m && w && (e = cudaMemcpyAsync(t_w, w, sizeof(uint32_t) * m, kind, s))))
            return fail(cuda_err(ctx, e, "graph upload"));
    }
    const int64_t* d_rp = mem == PANTHER_MEM_HOST ? t_rp : row_ptr;
    const int32_t* d_col = mem == PANTHER_MEM_HOST ? t_col : col;
    const uint32_t* d_w = w ? (mem == PANTHER_MEM_HOST ? t_w : w) : nullptr;
    if ((e = cudaMemsetAsync(nbig, 0, sizeof(int) * 8, s)) ||
        (e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * 4, s)) ||
        (e = cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), s)) ||
        (e = cudaMemsetAsync(ctx->d_status + 1, 0xff, sizeof(uint32_t), s)))
        return fail(cuda_err(ctx, e, "graph upload"));

    rows_check_kernel<<<(unsigned)ceil_div(n + 1, 256), 256, 0, s>>>(d_rp, n, m, big, mid, mid2, nbig,
                                                                     ctx->d_status);
    ctx->launches++;
    int h_lists[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint32_t h_st[2];
    if ((e = cudaMemcpyAsync(h_lists, nbig, sizeof(int) * 8, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(h_st, ctx->d_status, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return fail(cuda_err(ctx, e, "row check"));
    if (h_st[0]) return fail(set_err(ctx, PANTHER_EINVAL, "row_ptr is not a valid CSR offset array"));
    const int h_nbig = h_lists[0];
    const int64_t nshort = h_lists[1], nmed = h_lists[2], n16 = h_lists[3], n32 = h_lists[4];
    auto rows_grid = [&](int64_t rows, int lanes_per_row) {
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(rows * lanes_per_row, 256),
                                                                (int64_t)ctx->num_sms * 16));
    };

    // segment plan of the rows above BIG_DEG
    int64_t* bdeg = nullptr;
    int64_t* seg_off = nullptr;
    unsigned long long* bigS = nullptr;
    int64_t nseg = 0;
    std::vector<int64_t> hseg(1, 0);
    if (h_nbig) {
        std::vector<int64_t> hdeg(h_nbig);
        if ((st = dev_alloc(ctx, (void**)&bdeg, sizeof(int64_t) * h_nbig)) ||
            (st = dev_alloc(ctx, (void**)&seg_off, sizeof(int64_t) * (h_nbig + 1))) ||
            (st = dev_alloc(ctx, (void**)&bigS, sizeof(unsigned long long) * h_nbig)))
            return fail(st);
        big_deg_kernel<<<(unsigned)ceil_div(h_nbig, 256), 256, 0, s>>>(d_rp, big, h_nbig, bdeg);
        ctx->launches++;
        if ((e = cudaMemcpyAsync(hdeg.data(), bdeg, sizeof(int64_t) * h_nbig, cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s)))
            return fail(cuda_err(ctx, e, "big-row plan"));
        hseg.resize(h_nbig + 1);
        for (int i = 0; i < h_nbig; ++i) hseg[i + 1] = hseg[i] + ceil_div(hdeg[i], SEG);
        nseg = hseg[h_nbig];
        if ((e = cudaMemcpyAsync(seg_off, hseg.data(), sizeof(int64_t) * (h_nbig + 1), cudaMemcpyHostToDevice, s)) ||
            (e = cudaMemsetAsync(bigS, 0, sizeof(unsigned long long) * h_nbig, s)))
            return fail(cuda_err(ctx, e, "big-row plan"));
    }
    auto free_plan = [&]() {
        dev_free(ctx, bdeg);
        dev_free(ctx, seg_off);
        dev_free(ctx, bigS);
        bdeg = nullptr;
        seg_off = nullptr;
        bigS = nullptr;
    };
    StatsOut so{g->vrec, ctx->d_status, acc};
    unsigned gw = grid_for(ctx, 64, n, 256);
    stats_thread_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->num_sms * 16), 256, 0, s>>>(
        d_rp, n, d_col, d_w, so);
    ctx->launches++;
    if (nshort) {
        stats_short_kernel<8><<<rows_grid(nshort, 8), 256, 0, s>>>(d_rp, n, d_col, d_w, mid, false, nshort, so);
        ctx->launches++;
    }
    if (n16) {
        stats_short_kernel<16><<<rows_grid(n16, 16), 256, 0, s>>>(d_rp, n, d_col, d_w, mid2, false, n16, so);
        ctx->launches++;
    }
    if (n32) {
        stats_short_kernel<32><<<rows_grid(n32, 32), 256, 0, s>>>(d_rp, n, d_col, d_w, mid2, true, n32, so);
        ctx->launches++;
    }
    if (nmed) {
        stats_warp_kernel<<<rows_grid(nmed, 32), 256, 0, s>>>(d_rp, n, d_col, d_w, mid, nmed, so);
        ctx->launches++;
    }
    if (h_nbig) {
        stats_seg_kernel<<<(unsigned)nseg, BLK, 0, s>>>(d_rp, n, d_col, d_w, big, seg_off, h_nbig, bigS, so);
        big_finalize_kernel<<<(unsigned)ceil_div(h_nbig, 256), 256, 0, s>>>(d_rp, big, h_nbig, bigS, so);
        ctx->launches += 2;
    }
    unsigned long long h_acc[3];
    if ((e = cudaMemcpyAsync(h_acc, acc, sizeof(h_acc), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(h_st, ctx->d_status, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return free_plan(), fail(cuda_err(ctx, e, "graph validation"));
    if (h_st[0] & ST_OVERFLOW) {
        cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), s);
        return free_plan(), fail(set_err(ctx, PANTHER_EOVERFLOW, "a row's weight sum times its degree reaches 2^63"));
    }
    if (h_st[0]) {
        cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), s);
        return free_plan(), fail(set_err(ctx, PANTHER_EINVAL,
                            "malformed graph at row %u (column range, order, self-loop or zero weight)", h_st[1]));
    }
    if (h_acc[1] != h_acc[2])
        return free_plan(), fail(set_err(ctx, PANTHER_EINVAL, "graph is not symmetric with equal weights"));
    g->max_row_sum = h_acc[0];
    g->prefix_wide = h_acc[0] >= (1ull << 32) ? 1 : 0;

    if (modes & PANTHER_MODE_PREFIX) {
        size_t esz = g->prefix_wide ? sizeof(uint4) : sizeof(uint2);
        if ((st = dev_alloc(ctx, &g->prefix, esz * (size_t)m))) return free_plan(), fail(st);
        if (g->prefix_wide) {
            prefix_warp_kernel<true><<<gw, 256, 0, s>>>(d_rp, n, d_col, d_w, g->prefix);
            if (h_nbig) prefix_block_kernel<true><<<h_nbig, BLK, 0, s>>>(d_rp, d_col, d_w, big, g->prefix);
        } else {
            prefix_warp_kernel<false><<<gw, 256, 0, s>>>(d_rp, n, d_col, d_w, g->prefix);
            if (h_nbig) prefix_block_kernel<false><<<h_nbig, BLK, 0, s>>>(d_rp, d_col, d_w, big, g->prefix);
        }
        ctx->launches += h_nbig ? 2 : 1;
        if ((e = cudaGetLastError())) return free_plan(), fail(cuda_err(ctx, e, "prefix table"));
    }
    if (modes & PANTHER_MODE_ALIAS) {
        int32_t* sidx = nullptr;
        uint64_t* scum = nullptr;
        if ((st = dev_alloc(ctx, (void**)&g->alias, sizeof(uint4) * m)) ||
            (st = dev_alloc(ctx, (void**)&sidx, sizeof(int32_t) * m)) ||
            (st = dev_alloc(ctx, (void**)&scum, sizeof(uint64_t) * m))) {
            dev_free(ctx, sidx);
            return free_plan(), fail(st);
        }
        alias_thread_kernel<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->num_sms * 16), 256, 0, s>>>(
            g->vrec, n, d_col, d_w, g->alias);
        ctx->launches++;
        if (nshort) {
            alias_short_kernel<8><<<rows_grid(nshort, 8), 256, 0, s>>>(g->vrec, n, d_col, d_w, mid, false, nshort,
                                                                       g->alias, sidx, scum);
            ctx->launches++;
        }
        if (n16) {
            alias_short_kernel<16><<<rows_grid(n16, 16), 256, 0, s>>>(g->vrec, n, d_col, d_w, mid2, false, n16,
                                                                      g->alias, sidx, scum);
            ctx->launches++;
        }
        if (n32) {
            alias_short_kernel<32><<<rows_grid(n32, 32), 256, 0, s>>>(g->vrec, n, d_col, d_w, mid2, true, n32,
                                                                      g->alias, sidx, scum);
            ctx->launches++;
        }
        if (nmed) {
            alias_warp_kernel<<<rows_grid(nmed, 32), 256, 0, s>>>(g->vrec, n, d_col, d_w, mid, nmed, g->alias, sidx,
                                                                  scum);
            ctx->launches++;
        }
        if (h_nbig) {
            int64_t* bign = nullptr;
            if ((st = dev_alloc(ctx, (void**)&bign, sizeof(int64_t) * h_nbig))) {
                dev_free(ctx, sidx);
                dev_free(ctx, scum);
                return free_plan(), fail(st);
            }
            uint64_t* segsum = nullptr;
            if ((st = dev_alloc(ctx, (void**)&segsum, sizeof(uint64_t) * 3 * nseg))) {
                dev_free(ctx, bign);
                dev_free(ctx, sidx);
                dev_free(ctx, scum);
                return free_plan(), fail(st);
            }
            big_count_kernel<<<(unsigned)nseg, BLK, 0, s>>>(g->vrec, d_w, big, seg_off, h_nbig, segsum);
            big_rowscan_kernel<<<(unsigned)ceil_div(h_nbig * 32, 256), 256, 0, s>>>(seg_off, h_nbig, segsum, bign);
            big_place_kernel<<<(unsigned)nseg, BLK, 0, s>>>(g->vrec, d_w, big, seg_off, h_nbig, segsum, bign, sidx,
                                                            scum);
            alias_assign_kernel<<<(unsigned)nseg, 256, 0, s>>>(g->vrec, d_col, d_w, big, bign, seg_off, h_nbig,
                                                               g->alias, sidx, scum);
            ctx->launches += 4;
            dev_free(ctx, segsum);
            dev_free(ctx, bign);
        }
        e = cudaGetLastError();
        dev_free(ctx, sidx);
        dev_free(ctx, scum);
        if (e) return free_plan(), fail(cuda_err(ctx, e, "alias table"));
    }
    if ((modes & PANTHER_MODE_UNWEIGHTED) && m > 0) {
        if (mem == PANTHER_MEM_HOST) {         // the staged copy becomes the graph's own
            g->col = t_col;
            t_col = nullptr;
        } else {
            if ((st = dev_alloc(ctx, (void**)&g->col, sizeof(int32_t) * m))) return free_plan(), fail(st);
            if ((e = cudaMemcpyAsync(g->col, col, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s)))
                return free_plan(), fail(cuda_err(ctx, e, "column copy"));
        }
    }
    free_plan();
    dev_free(ctx, t_rp);
    dev_free(ctx, t_col);
    dev_free(ctx, t_w);
    dev_free(ctx, big);
    dev_free(ctx, mid);
    dev_free(ctx, mid2);
    dev_free(ctx, nbig);
    dev_free(ctx, acc);
    if ((e = cudaStreamSynchronize(s))) {
        t_rp = nullptr; t_col = nullptr; t_w = nullptr; big = nullptr; mid = nullptr; mid2 = nullptr; nbig = nullptr;
        acc = nullptr;
        return fail(cuda_err(ctx, e, "graph tables"));
    }
    *out = g;
    return PANTHER_OK;
}

extern "C" {
// Debug/test access: copy the alias table (thr, col_self, col_alias) or the
// prefix table entries of the graph to caller device memory.
panther_status panther_debug_graph_tables(const panther_graph* g, void* dev_alias16, void* dev_prefix,
                                                     int* prefix_wide) {
    if (!g) return PANTHER_EINVAL;
    panther_ctx* ctx = g->ctx;
    if (prefix_wide) *prefix_wide = g->prefix_wide;
    if (dev_alias16 && g->alias)
        PCK(ctx, cudaMemcpyAsync(dev_alias16, g->alias, sizeof(uint4) * g->m, cudaMemcpyDeviceToDevice, ctx->stream));
    if (dev_prefix && g->prefix)
        PCK(ctx, cudaMemcpyAsync(dev_prefix, g->prefix, (g->prefix_wide ? 16 : 8) * g->m, cudaMemcpyDeviceToDevice,
                                 ctx->stream));
    PCK(ctx, cudaStreamSynchronize(ctx->stream));
    return PANTHER_OK;
}
}  // extern "C"
