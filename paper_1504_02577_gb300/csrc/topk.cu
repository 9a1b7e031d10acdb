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
#include <vector>

#include "internal.cuh"

namespace {

constexpr uint64_t EMPTY = ~0ull;
constexpr int WSLOTS = 512;      // warp-tier table slots
constexpr int WCAP = 256;        // warp-tier candidate bound
constexpr int KMAX = 64;
constexpr int WCHUNK = 16;       // warp-tier queries fetched per atomic

__device__ __forceinline__ uint32_t hslot(uint32_t key, uint32_t nslots) {
    return __umulhi(key * 0x9E3779B1u ^ (key >> 15), nslots);
}

// add 1 to the count of `key`; returns false if the table is full
template <bool SHARED>
__device__ __forceinline__ bool hash_add(unsigned long long* tab, uint32_t nslots, uint32_t key) {
    uint32_t s = hslot(key, nslots);
    for (uint32_t probe = 0; probe < nslots; ++probe) {
        unsigned long long cur = tab[s];
        if ((uint32_t)(cur >> 32) == key && cur != EMPTY) {
            atomicAdd(&tab[s], 1ull);
            return true;
        }
        if (cur == EMPTY) {
            unsigned long long prev = atomicCAS(&tab[s], EMPTY, ((unsigned long long)key << 32) | 1ull);
            if (prev == EMPTY) return true;
            if ((uint32_t)(prev >> 32) == key) {
                atomicAdd(&tab[s], 1ull);
                return true;
            }
        }
        s = (s + 1 == nslots) ? 0 : s + 1;
    }
    return false;
}

// ------------------------------------------------------ warp top-k list ---
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
    // offer one candidate per lane (0 = none)
    __device__ __forceinline__ void offer(uint64_t c, int k) {
        uint64_t thr = kth(k);
        unsigned m = __ballot_sync(0xffffffffu, c > thr);
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

__device__ __forceinline__ uint64_t slot_score(unsigned long long s) {
    if (s == EMPTY) return 0;
    uint32_t key = (uint32_t)(s >> 32), cnt = (uint32_t)s;
    return ((uint64_t)cnt << 32) | (uint64_t)(0xffffffffu - key);
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

// ------------------------------------------------------ path insertion ---
struct PathsRef {
    const int32_t* rows;
    int64_t R;
    int L;
    const int64_t* off;
    const int32_t* pid;
    int64_t n;
};

// insert the distinct vertices u != v of path r into the table
template <int STRIDE, bool SHARED>
__device__ __forceinline__ bool insert_path(const PathsRef& P, int32_t r, int32_t v, unsigned long long* tab,
                                            uint32_t nslots) {
    if ((uint32_t)r >= (uint64_t)P.R) return false;   // corrupt index entry: the caller flags it, nothing is read
    int32_t x[STRIDE];
    const int4* src = (const int4*)(P.rows + (int64_t)r * STRIDE);
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
            if (!dup) ok &= hash_add<SHARED>(tab, nslots, (uint32_t)x[j]);
        }
    }
    return ok;
}

struct Tiers {
    int32_t* list[3];    // query indices per tier: warp, CTA, global
    int* count;          // [3] tier sizes, [3..4] fetch counters (warp, CTA)
};

// classification: pads trivially empty queries and sorts the rest into tiers
__global__ void classify_kernel(const int32_t* __restrict__ queries, int64_t q, PathsRef P, int64_t ccap,
                                Tiers tiers, OutRef o, uint32_t* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned lane = threadIdx.x & 31;
    int tier = -1;
    if (i < q) {
        int64_t v = queries ? (int64_t)queries[i] : i;
        if (v < 0 || v >= P.n) {
            flag_status(status, ST_BAD_QUERY);
            atomicMin(status + 1, (uint32_t)i);
        } else {
            int64_t np = P.off[v + 1] - P.off[v];
            int64_t cap = np * (P.L - 1);
            if (cap > P.n - 1) cap = P.n - 1;
            if (cap > 0) tier = cap <= WCAP ? 0 : (cap <= ccap ? 1 : 2);
        }
        if (tier < 0) {
            for (int r = 0; r < o.k; ++r) {
                if (o.ids) o.ids[i * o.k + r] = -1;
                o.cnt[i * o.k + r] = 0;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        unsigned m = __ballot_sync(0xffffffffu, tier == t);
        if (!m) continue;
        int leader = __ffs(m) - 1;
        int base = 0;
        if ((int)lane == leader) base = atomicAdd(&tiers.count[t], __popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (tier == t) tiers.list[t][base + __popc(m & ((1u << lane) - 1u))] = (int32_t)i;
    }
}

// CTA-wide: count one query into the shared table and write its top-k
template <int STRIDE>
__device__ void cta_query(const PathsRef& P, int32_t v, int64_t qi, unsigned long long* tab, uint32_t nslots,
                          unsigned long long* lists, const OutRef& o, uint32_t* status) {
    for (uint32_t s = threadIdx.x; s < nslots; s += blockDim.x) tab[s] = EMPTY;
    __syncthreads();
    int64_t a = P.off[v], b = P.off[v + 1];
    bool ok = true;
    for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) ok &= insert_path<STRIDE, true>(P, P.pid[e], v, tab, nslots);
    if (!ok) flag_status(status, ST_HASH_FULL);
    __syncthreads();
    WarpTopK t;
    int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    unsigned lane = threadIdx.x & 31;
    for (uint32_t base = (uint32_t)w * 32; base < nslots; base += (uint32_t)nw * 32) {
        uint32_t s = base + lane;
        t.offer(s < nslots ? slot_score(tab[s]) : 0, o.k);
    }
    // merge warp lists through shared memory (reuses the list area)
    lists[w * KMAX + lane] = t.a;
    lists[w * KMAX + 32 + lane] = t.b;
    __syncthreads();
    if (w == 0) {
        for (int ww = 1; ww < nw; ++ww) {
            t.offer(lists[ww * KMAX + lane], o.k);
            if (o.k > 32) t.offer(lists[ww * KMAX + 32 + lane], o.k);
        }
        write_list(t, o, qi);
    }
    __syncthreads();
}

template <int STRIDE>
__device__ void warp_query(const PathsRef& P, int32_t v, int64_t qi, unsigned long long* tab, const OutRef& o,
                           uint32_t* status) {
    unsigned lane = threadIdx.x & 31;
    for (int s = lane; s < WSLOTS; s += 32) tab[s] = EMPTY;
    __syncwarp();
    int64_t a = P.off[v], b = P.off[v + 1];
    bool ok = true;
    for (int64_t e = a + lane; e < b; e += 32) ok &= insert_path<STRIDE, true>(P, P.pid[e], v, tab, WSLOTS);
    if (!ok) flag_status(status, ST_HASH_FULL);
    __syncwarp();
    WarpTopK t;
    for (int base = 0; base < WSLOTS; base += 32) t.offer(slot_score(tab[base + lane]), o.k);
    write_list(t, o, qi);
    __syncwarp();
}

struct PersistArgs {
    PathsRef P;
    const int32_t* queries;
    Tiers tiers;
    OutRef o;
    uint32_t cta_slots;
    uint32_t* status;
};

template <int STRIDE>
__global__ void __launch_bounds__(1024, 1) persistent_kernel(PersistArgs A) {
    extern __shared__ unsigned long long smem[];
    __shared__ unsigned long long lists[32 * KMAX];
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
    __shared__ unsigned long long lists[32 * KMAX];
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
    for (int64_t e = P.off[v] + threadIdx.x; e < P.off[v + 1]; e += blockDim.x)
        ok &= insert_path<STRIDE, false>(P, P.pid[e], (int32_t)v, gtab, gslots);
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
    lists[w * KMAX + lane] = t.a;
    lists[w * KMAX + 32 + lane] = t.b;
    __syncthreads();
    if (w == 0) {
        for (int ww = 1; ww < nw; ++ww) {
            t.offer(lists[ww * KMAX + lane], o.k);
            if (o.k > 32) t.offer(lists[ww * KMAX + 32 + lane], o.k);
        }
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
};

constexpr int G_PATHS = 2048;     // paths per count item
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
    bool ok = true;
    for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x)
        ok &= insert_path<STRIDE, false>(P, P.pid[e], v, tab, G.tab_n[g]);
    if (!ok) flag_status(status, ST_HASH_FULL);
}

// partial top-k of one chunk of one table; empties the slots it read
__global__ void g_select_kernel(GPlan G, unsigned long long* arena, int k, unsigned long long* partial) {
    __shared__ unsigned long long lists[32 * KMAX];
    int64_t item = blockIdx.x;
    int g = find_owner(G.sel_off, G.ng, item);
    int64_t c0 = (item - G.sel_off[g]) * G_SLOTS;
    uint32_t ns = G.tab_n[g];
    unsigned long long* tab = arena + G.tab_off[g];
    int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
    unsigned lane = threadIdx.x & 31;
    WarpTopK t;
    int64_t end = c0 + G_SLOTS < (int64_t)ns ? c0 + G_SLOTS : (int64_t)ns;
    for (int64_t base = c0 + w * 32; base < end; base += nw * 32) {
        int64_t s = base + lane;
        uint64_t sc = 0;
        if (s < end) {
            sc = slot_score(tab[s]);
            if (sc) tab[s] = EMPTY;
        }
        t.offer(sc, k);
    }
    lists[w * KMAX + lane] = t.a;
    lists[w * KMAX + 32 + lane] = t.b;
    __syncthreads();
    if (w == 0) {
        for (int ww = 1; ww < nw; ++ww) {
            t.offer(lists[ww * KMAX + lane], k);
            if (k > 32) t.offer(lists[ww * KMAX + 32 + lane], k);
        }
        partial[item * KMAX + lane] = t.a;
        partial[item * KMAX + 32 + lane] = t.b;
    }
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

uint32_t pow2_at_least(int64_t x) {
    uint32_t p = 1024;
    while ((int64_t)p < x && p < (1u << 31)) p <<= 1;
    return p;
}

}  // namespace

// ------------------------------------------------------------ host side ---
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

// Internal entry shared by panther_topk and pantherpp_vectors: queries may be
// NULL (meaning 0..q-1); ids may be NULL (counts only, e.g. theta rows).
panther_status topk_run(panther_ctx* ctx, const panther_index* ix, const panther_paths* p, const int32_t* queries,
                        int64_t q, int k, int32_t* ids, uint32_t* cnt, bool plain) {
    cudaStream_t s = ctx->stream;
    TopkShape sh = topk_shape(ctx);
    const size_t smem = (size_t)sh.cta_slots * 8;
    panther_status st;
    if (p->stride == 8) st = set_smem_attr<8>(ctx, smem);
    else if (p->stride == 16) st = set_smem_attr<16>(ctx, smem);
    else st = set_smem_attr<32>(ctx, smem);
    if (st) return st;
    PathsRef P{p->rows, p->R, p->L, ix->off, ix->pid, ix->n};
    OutRef o{ids, cnt, k};
    const int64_t ccap = (int64_t)sh.cta_slots * 7 / 10;

    if (plain) {
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
            else
                single_kernel<32><<<1, sh.threads, smem, s>>>(P, queries, i, o, sh.cta_slots, gtab, gslots, ctx->d_status);
            ctx->launches++;
        }
        dev_free(ctx, gtab);
        PCK(ctx, cudaGetLastError());
        return PANTHER_OK;
    }

    int32_t* lists = nullptr;
    int* counts = nullptr;
    if ((st = dev_alloc(ctx, (void**)&lists, sizeof(int32_t) * 3 * (size_t)q)) ||
        (st = dev_alloc(ctx, (void**)&counts, sizeof(int) * 8))) {
        dev_free(ctx, lists);
        return st;
    }
    Tiers tiers{{lists, lists + q, lists + 2 * q}, counts};
    PCK(ctx, cudaMemsetAsync(counts, 0, sizeof(int) * 8, s));
    classify_kernel<<<(unsigned)ceil_div(q, 256), 256, 0, s>>>(queries, q, P, ccap, tiers, o, ctx->d_status);
    ctx->launches++;
    PersistArgs A{P, queries, tiers, o, sh.cta_slots, ctx->d_status};
    unsigned blocks = (unsigned)(ctx->num_sms * sh.blocks_per_sm);
    if (p->stride == 8) persistent_kernel<8><<<blocks, sh.threads, smem, s>>>(A);
    else if (p->stride == 16) persistent_kernel<16><<<blocks, sh.threads, smem, s>>>(A);
    else persistent_kernel<32><<<blocks, sh.threads, smem, s>>>(A);
    ctx->launches++;
    PCK(ctx, cudaGetLastError());

    // global tier: read its size (one synchronisation), then run in rounds
    int h_counts[3];
    PCK(ctx, cudaMemcpyAsync(h_counts, counts, sizeof(int) * 3, cudaMemcpyDeviceToHost, s));
    PCK(ctx, cudaStreamSynchronize(s));
    const int ng = h_counts[2];
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
        PCK(ctx, cudaMemcpyAsync(gq.data(), lists + 2 * q, sizeof(int32_t) * ng, cudaMemcpyDeviceToHost, s));
        PCK(ctx, cudaMemcpyAsync(npv.data(), d_np, sizeof(int64_t) * ng, cudaMemcpyDeviceToHost, s));
        PCK(ctx, cudaStreamSynchronize(s));
        dev_free(ctx, d_np);
        // largest first, then pack rounds under the scratch budget
        std::vector<int> order(ng);
        for (int i = 0; i < ng; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int x, int y) {
            return npv[x] != npv[y] ? npv[x] > npv[y] : x < y;
        });
        const int64_t budget_slots = std::max<int64_t>(ctx->scratch_budget / 8 / 2, 1 << 20);
        size_t pos = 0;
        unsigned long long* arena = nullptr;
        int64_t arena_slots = 0;
        while (pos < order.size()) {
            std::vector<int32_t> rq;
            std::vector<int64_t> roff, ioff{0}, soff{0};
            std::vector<uint32_t> rn;
            int64_t used = 0;
            while (pos < order.size()) {
                int i = order[pos];
                int64_t np = npv[i];
                int64_t cap = std::min<int64_t>(np * (p->L - 1), ix->n - 1);
                uint32_t slots = pow2_at_least(cap * 2);
                if (!rq.empty() && used + slots > budget_slots) break;
                rq.push_back(gq[i]);
                roff.push_back(used);
                rn.push_back(slots);
                used += slots;
                ioff.push_back(ioff.back() + ceil_div(np, G_PATHS));
                soff.push_back(soff.back() + ceil_div(slots, G_SLOTS));
                ++pos;
            }
            if (used > arena_slots) {
                dev_free(ctx, arena);
                arena = nullptr;
                if ((st = dev_alloc(ctx, (void**)&arena, 8ull * used))) {
                    dev_free(ctx, lists);
                    dev_free(ctx, counts);
                    return st;
                }
                arena_slots = used;
                fill_empty_kernel<<<ctx->num_sms * 8, 256, 0, s>>>(arena, used);
                ctx->launches++;
            }
            int rng = (int)rq.size();
            // plan arrays in one device buffer
            size_t bytes = sizeof(int32_t) * rng + sizeof(int64_t) * rng + sizeof(uint32_t) * rng +
                           sizeof(int64_t) * (rng + 1) * 2 + 64;
            std::vector<char> hbuf(bytes);
            char* hp = hbuf.data();
            size_t o0 = 0, o1 = o0 + sizeof(int32_t) * rng;
            o1 = (o1 + 7) & ~size_t(7);
            size_t o2 = o1 + sizeof(int64_t) * rng;
            size_t o3 = o2 + sizeof(uint32_t) * rng;
            o3 = (o3 + 7) & ~size_t(7);
            size_t o4 = o3 + sizeof(int64_t) * (rng + 1);
            memcpy(hp + o0, rq.data(), sizeof(int32_t) * rng);
            memcpy(hp + o1, roff.data(), sizeof(int64_t) * rng);
            memcpy(hp + o2, rn.data(), sizeof(uint32_t) * rng);
            memcpy(hp + o3, ioff.data(), sizeof(int64_t) * (rng + 1));
            memcpy(hp + o4, soff.data(), sizeof(int64_t) * (rng + 1));
            char* dplan = nullptr;
            unsigned long long* partial = nullptr;
            if ((st = dev_alloc(ctx, (void**)&dplan, bytes)) ||
                (st = dev_alloc(ctx, (void**)&partial, sizeof(unsigned long long) * KMAX * soff.back()))) {
                dev_free(ctx, dplan);
                dev_free(ctx, arena);
                dev_free(ctx, lists);
                dev_free(ctx, counts);
                return st;
            }
            PCK(ctx, cudaMemcpyAsync(dplan, hp, bytes, cudaMemcpyHostToDevice, s));
            GPlan G{(const int32_t*)(dplan + o0), (const int64_t*)(dplan + o1), (const uint32_t*)(dplan + o2),
                    (const int64_t*)(dplan + o3), (const int64_t*)(dplan + o4), rng};
            if (p->stride == 8) g_count_kernel<8><<<(unsigned)ioff.back(), 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else if (p->stride == 16) g_count_kernel<16><<<(unsigned)ioff.back(), 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            else g_count_kernel<32><<<(unsigned)ioff.back(), 256, 0, s>>>(P, queries, G, arena, ctx->d_status);
            g_select_kernel<<<(unsigned)soff.back(), 512, 0, s>>>(G, arena, k, partial);
            g_merge_kernel<<<rng, 32, 0, s>>>(G, partial, o);
            ctx->launches += 3;
            PCK(ctx, cudaGetLastError());
            // the host plan buffer must outlive the async copy
            PCK(ctx, cudaStreamSynchronize(s));
            dev_free(ctx, dplan);
            dev_free(ctx, partial);
        }
        dev_free(ctx, arena);
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
    if (k < 1 || k > KMAX) return set_err(ctx, PANTHER_EINVAL, "k must be in [1, 64]");
    if (ix->n != p->n) return set_err(ctx, PANTHER_EINVAL, "index and paths belong to different graphs");
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
        st = topk_run(ctx, ix, p, dq, q, k, di, dc, mode == PANTHER_TOPK_PLAIN);
        if (!st) {
            PCK(ctx, cudaMemcpyAsync(out_ids, di, ob, cudaMemcpyDeviceToHost, s));
            PCK(ctx, cudaMemcpyAsync(out_counts, dc, ob, cudaMemcpyDeviceToHost, s));
        }
        dev_free(ctx, buf);
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
    if (!ctx || !ix || !p || !queries || !out_ids || !out_counts || q < 1 || k < 1 || k > KMAX)
        return set_err(ctx, PANTHER_EINVAL, "bad tuner arguments");
    cudaSetDevice(ctx->device);
    struct Shape { int threads, slots, bps; };
    const Shape cand[] = {{1024, 24576, 1}, {512, 24576, 1}, {512, 11264, 2}, {256, 8192, 3}, {1024, 16384, 1}};
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
