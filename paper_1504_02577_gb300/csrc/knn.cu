// Panther++ (Sec. 3.3, Algorithm 2): feature vectors theta(v) and exact
// k-nearest neighbours under Euclidean distance.
//
// theta(v) = the D largest counts cnt(v,u), u != v (the counting kernels of
// topk.cu with k = D, counts only).
//
// Nearest neighbours. For query a and candidate b (integer vectors) the
// squared distance is d = |a|^2 + y with y = |b|^2 - 2 a.b; ranking by d is
// ranking by y. y is screened on the tensor cores:
//   A row (query)      = [bf16(a_0..a_{D-1}), 1 x 8, 0 ...]         (64 columns)
//   B row (candidate)  = [-2 bf16(b_0..b_{D-1}), p_0 .. p_7, 0 ...]
// where p_i = ((|b|^2 >> 8i) & 255) << 8i are the eight 8-bit pieces of the
// exact squared norm (each exactly representable in BF16). One tcgen05.mma
// chain (M=128 queries, N=256 candidates, K=64, FP32 accumulation in TMEM)
// produces y_hat = |b|^2 - 2 a_hat.b_hat directly.
//
// Error bound. With u = 2^-8 (BF16 round to nearest), gamma = 2^-16 (64
// additions at a conservative 2^-22 each) and s = a.b <= |a||b|:
//   |y_hat - y| <= [2(2u+u^2) + 2 gamma (1+u)^2] |a||b| + gamma |b|^2
// If every entry of a and of b is <= 256, the BF16 inputs are exact and every
// partial sum is an integer of magnitude < 2^24, so y_hat = y exactly.
//
// Selection (one thread per query row of the tile) keeps the k best keys in
// shared memory: exact pairs insert (y, id); other pairs are kept while their
// lower bound y_hat - E does not exceed the k-th key, insert (y_hat + E, id)
// and are appended to a per-query shortlist. Afterwards every kept candidate
// is re-ranked with exact uint64 arithmetic on the integer vectors, so the
// answer is exact. Candidates (and queries) are stored exact rows first, so
// whole 256-candidate tiles take the one-compare fast path.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

panther_status topk_counts_all(panther_ctx* ctx, const panther_index* ix, const panther_paths* p, int D,
                               uint32_t* theta);

namespace {

constexpr int KN_M = 128;          // queries per tile
constexpr int KN_N = 256;          // candidates per tile
constexpr int KN_K = 64;           // padded vector length (bf16)
constexpr int KN_STAGES = 4;
constexpr int KN_KMAX = 32;
constexpr int KN_SCAP = 256;       // shortlist capacity per query
constexpr int KN_SPLIT = 2;        // selection warps per TMEM lane quarter (each takes one column slice)
constexpr int KN_THREADS = 64 + 128 * KN_SPLIT;   // warp 0 TMA, warp 1 MMA, then the selection warps
constexpr float KN_ALPHA = 0.0157f;    // >= 2(2u+u^2) + 2 gamma (1+u)^2
constexpr float KN_BETA = 1.6e-5f;     // >= gamma = 2^-16
constexpr uint32_t MAX_EXACT = 256;

struct VecMeta {
    int64_t n, npad;                 // vertices, padded to a multiple of 256
    int64_t nexact;                  // number of exact rows (they come first)
    int D;
};

// round a uint32 to 8 significant bits, nearest, ties to even (bf16 of an integer)
__device__ __forceinline__ uint32_t round8(uint32_t x) {
    if (x < 256) return x;
    int p = 31 - __clz(x);           // leading bit
    int sh = p - 7;
    uint32_t q = x >> sh, rem = x & ((1u << sh) - 1), half = 1u << (sh - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
    return q << sh;                  // may carry to 2^(p+1): still 8 significant bits
}

// minimum of three floats in one instruction (the values are finite here)
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ uint16_t bf16_bits_of(float f) {   // f exactly representable
    return (uint16_t)(__float_as_uint(f) >> 16);
}

// per-vertex statistics and the exact-row flag
__global__ void vec_stats_kernel(const uint32_t* __restrict__ theta, int64_t n, int D, uint64_t* __restrict__ norm2,
                                 float* __restrict__ nrm, uint8_t* __restrict__ exact, int64_t* __restrict__ flag,
                                 unsigned* __restrict__ maxv) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    uint64_t s = 0;
    uint32_t mx = 0;
    for (int d = 0; d < D; ++d) {
        uint32_t x = theta[v * D + d];
        s += (uint64_t)x * x;
        mx = x > mx ? x : mx;
    }
    norm2[v] = s;
    float r = sqrtf(__ull2float_ru(s));
    nrm[v] = r * (1.0f + 1.0f / (1 << 21));
    uint8_t e = mx <= MAX_EXACT;
    exact[v] = e;
    flag[v] = e;
    atomicMax(maxv, mx);
}

// position of every vertex: exact rows first (id ascending), then the rest
__global__ void vec_perm_kernel(const uint8_t* __restrict__ exact, const int64_t* __restrict__ exscan, int64_t n,
                                int64_t nexact, int32_t* __restrict__ perm, int64_t* __restrict__ pos) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int64_t p = exact[v] ? exscan[v] : nexact + (v - exscan[v]);
    perm[p] = (int32_t)v;
    pos[v] = p;
}

// B rows (candidate role) in permuted order + SoA candidate info
__global__ void vec_brow_kernel(const uint32_t* __restrict__ theta, const uint64_t* __restrict__ norm2,
                                const float* __restrict__ nrm, const int32_t* __restrict__ perm, VecMeta M,
                                uint16_t* __restrict__ B, int32_t* __restrict__ cid, float* __restrict__ cnrm,
                                float* __restrict__ cncf) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M.npad) return;
    uint16_t* row = B ? B + p * KN_K : nullptr;      // no BF16 rows when D > 56 (FP32 form only)
    if (p >= M.n) {
        // padding: y = 2^40 for every query, id -1 (never selected)
        if (row) {
            for (int d = 0; d < KN_K; ++d) row[d] = 0;
            row[M.D] = bf16_bits_of(1099511627776.0f);
        }
        cid[p] = -1;
        cnrm[p] = 0.f;
        cncf[p] = 1099511627776.0f;
        return;
    }
    int32_t v = perm[p];
    for (int d = 0; row && d < KN_K; ++d) {
        float f = 0.f;
        if (d < M.D) f = -2.0f * (float)round8(theta[(int64_t)v * M.D + d]);
        else if (d < M.D + 8) {
            int i = d - M.D;
            uint64_t piece = (norm2[v] >> (8 * i)) & 255ull;
            f = ldexpf((float)piece, 8 * i);
        }
        row[d] = bf16_bits_of(f);
    }
    cid[p] = v;
    cnrm[p] = nrm[v];
    cncf[p] = __ull2float_ru(norm2[v]);
}

// A rows (query role) for a list of query slots
__global__ void vec_arow_kernel(const uint32_t* __restrict__ theta, const int32_t* __restrict__ qv, int64_t qpad,
                                int D, uint16_t* __restrict__ A) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= qpad) return;
    uint16_t* row = A + s * KN_K;
    int32_t v = qv[s];
    for (int d = 0; d < KN_K; ++d) {
        float f = 0.f;
        if (v >= 0) {
            if (d < D) f = (float)round8(theta[(int64_t)v * D + d]);
            else if (d < D + 8) f = 1.0f;
        }
        row[d] = bf16_bits_of(f);
    }
}

__global__ void tile_flags_kernel(const uint8_t* __restrict__ exact, const int32_t* __restrict__ ids, int64_t count,
                                  int tile, uint8_t* __restrict__ out, int64_t ntiles) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    uint8_t all = 1;
    for (int64_t i = t * tile; i < (t + 1) * tile && i < count; ++i) {
        int32_t v = ids[i];
        if (v >= 0 && !exact[v]) all = 0;
    }
    out[t] = all;
}

// ----------------------------------------------------------- PTX helpers ---
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for a phase that is certain to complete (copies or MMAs already in
// flight), bounded all the same; used only to drain after an abort
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try(bar, parity) && clock64() - t0 < (1ll << 31)) {
    }
}
// bounded wait: about one second of SM clocks, then report and give up
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* status, volatile int* abort_flag) {
    if (mbar_try(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > (1ll << 31)) {
            flag_status(status, ST_TIMEOUT);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// tcgen05 shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)(16 >> 4) << 16;                    // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // SWIZZLE_128B
    return d;
}

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, N = 256, M = 128
constexpr uint32_t KN_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(KN_N >> 3) << 17) |
                              ((uint32_t)(KN_M >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(KN_IDESC), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 columns of this thread's TMEM lane into r (asynchronous: wait before use)
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// ties the registers to a point after the wait, so no use is scheduled before it
__device__ __forceinline__ void reg_fence(uint32_t (&r)[32]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

// ---------------------------------------------------------- selection ---
// Per query row: the k best keys live in shared memory (ascending by
// (key, id)); only the k-th key and id stay in registers for the fast test.
struct Row {
    float thr;       // key of the k-th entry (+inf until k entries)
    int thr_id;
    int n;           // entries held
    int scount;      // shortlist entries appended
};

struct RowConst {
    int qid;         // query vertex (-1: padding row)
    int self;        // candidate id excluded from the answer (the query itself; -2 across graphs)
    bool exact;
    float anrm;      // KN_ALPHA * |a| (BF16) or 2 eps |a| (FP32)
    float2* list;    // k entries {key, id bits}
    int32_t* sl;     // shortlist
    int* overflow;
    int k;
};

// insert (key, id) (caller checked it beats the k-th entry); out of line: rare
__device__ __noinline__ Row row_insert(Row r, const RowConst& c, float key, int id) {
    int i = r.n < c.k ? r.n : c.k - 1;
    if (r.n < c.k) ++r.n;
    while (i > 0) {
        float2 e = c.list[i - 1];
        int eid = __float_as_int(e.y);
        if (e.x < key || (e.x == key && eid < id)) break;
        c.list[i] = e;
        --i;
    }
    c.list[i] = make_float2(key, __int_as_float(id));
    if (r.n == c.k) {
        float2 last = c.list[c.k - 1];
        r.thr = last.x;
        r.thr_id = __float_as_int(last.y);
    }
    return r;
}

__device__ __forceinline__ Row take_exact(Row r, const RowConst& c, float y, int cid) {
    if (cid < 0 || cid == c.self) return r;
    if (y < r.thr || (y == r.thr && cid < r.thr_id)) r = row_insert(r, c, y, cid);
    return r;
}

// a pair whose screened value carries an error bound E
__device__ __noinline__ Row take_bounded(Row r, const RowConst& c, float y, float E, int cid, bool cexact) {
    if (cid < 0 || cid == c.self) return r;
    if (c.exact && cexact) return take_exact(r, c, y, cid);
    if (__fsub_rd(y, E) > r.thr) return r;
    if (r.scount < KN_SCAP) c.sl[r.scount] = cid; else *c.overflow = 1;
    ++r.scount;
    float ub = __fadd_ru(y, E);
    if (ub < r.thr || (ub == r.thr && cid < r.thr_id)) r = row_insert(r, c, ub, cid);
    return r;
}

// one group of 32 screened values y (columns pos0 .. pos0+31)
__device__ __forceinline__ Row select_group(Row r, const RowConst& c, const float (&y)[32], bool fast,
                                            const int32_t* cid, const float* cnrm, const float* cncf, int64_t pos0,
                                            int64_t nexact) {
    if (c.qid < 0) return r;
    if (fast) {
        // exact tiles hold exact rows in ascending id order, after every row
        // already in the list, so a candidate tied with the k-th key never
        // wins its tie: only y < thr can enter. The minimum of the 32 values
        // decides whether any can: three-input minima, 16 instructions.
        float t11[11];
#pragma unroll
        for (int j = 0; j < 10; ++j) t11[j] = fmin3(y[3 * j], y[3 * j + 1], y[3 * j + 2]);
        t11[10] = fminf(y[30], y[31]);
        const float m = fminf(fmin3(fmin3(t11[0], t11[1], t11[2]), fmin3(t11[3], t11[4], t11[5]),
                                    fmin3(t11[6], t11[7], t11[8])),
                              fminf(t11[9], t11[10]));
        if (m < r.thr) {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (y[j] < r.thr) r = take_exact(r, c, y[j], cid[j]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float E = fmaf(c.anrm, cnrm[j], fmaf(KN_BETA, cncf[j], 1.0f)) * 1.0001f;
            if (__fsub_rd(y[j], E) <= r.thr) r = take_bounded(r, c, y[j], E, cid[j], pos0 + j < nexact);
        }
    }
    return r;
}

struct ScreenArgs {
    const int32_t* cid;      // [npad] candidate vertex per position
    const float* cnrm;       // [npad]
    const float* cncf;       // [npad]
    const uint8_t* ctile;    // [npad/256] all-exact flags
    int64_t nct;             // candidate tiles
    int64_t nexact;          // exact candidate positions
    const int32_t* qv;       // [qpad] query vertex per slot (-1 pad)
    const float* qnrm;       // [qpad]
    const uint8_t* qexact;   // [qpad]
    const uint8_t* qtile;    // [qpad/128] all-exact flags
    int64_t nqt;
    int64_t nchunk;          // candidate ranges per query tile (work item = tile x range)
    int k;
    float2* lists;           // [qpad][nchunk][KN_SPLIT][k]
    int32_t* shortlist;      // [qpad][nchunk][KN_SPLIT][KN_SCAP]
    int32_t* scount;         // [qpad][nchunk][KN_SPLIT]
    int* overflow;           // [qpad]
    uint32_t* status;
    bool exclude_self;       // queries and candidates are the same vertices
    float* dump;             // DUMP form only: y_hat of every pair, [q][npad] by query index
    const int32_t* qidx;     // DUMP form only: query index of each slot
    int64_t npad;
};

// shared memory map (offsets from a 1024-aligned base)
constexpr uint32_t SM_A = 0;                                   // 16 KB
constexpr uint32_t SM_B = SM_A + KN_M * KN_K * 2;              // KN_STAGES x 32 KB
constexpr uint32_t SM_INFO = SM_B + KN_STAGES * KN_N * KN_K * 2;  // KN_STAGES x 3 KB
constexpr uint32_t SM_LIST = SM_INFO + KN_STAGES * KN_N * 12;  // 128 x SPLIT x KMAX x 8 B
constexpr uint32_t SM_BAR = SM_LIST + KN_M * KN_SPLIT * KN_KMAX * 8;   // barriers
constexpr uint32_t SM_TOTAL = SM_BAR + 256;
constexpr uint32_t KN_SMEM_BYTES = SM_TOTAL + 1024;

// DUMP = true is the measurement form (pantherpp_debug_screen): it also
// writes every screened value y_hat to S.dump; DUMP = false is the k-NN path.
template <bool DUMP>
__global__ void __launch_bounds__(KN_THREADS, 1)
    screen_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, ScreenArgs S) {
    extern __shared__ uint8_t smraw[];
    const uint32_t raw = smem_u32(smraw);
    const uint32_t base = (raw + 1023) & ~1023u;
    uint8_t* gbase = smraw + (base - raw);
    // barriers: full[4], empty[4], tfull[2], tempty[2], afull, aempty
    const uint32_t bar0 = base + SM_BAR;
    auto FULL = [&](int s) { return bar0 + 8 * s; };
    auto EMPTY = [&](int s) { return bar0 + 8 * (KN_STAGES + s); };
    auto TFULL = [&](int b) { return bar0 + 8 * (2 * KN_STAGES + b); };
    auto TEMPTY = [&](int b) { return bar0 + 8 * (2 * KN_STAGES + 2 + b); };
    const uint32_t AFULL = bar0 + 8 * (2 * KN_STAGES + 4), AEMPTY = AFULL + 8;
    const uint32_t DRAIN = bar0 + 8 * (2 * KN_STAGES + 8);   // completion of this CTA's MMAs after an abort
    volatile int* abort_flag = (volatile int*)(gbase + SM_BAR + 8 * (2 * KN_STAGES + 6));
    uint32_t* tmem_slot = (uint32_t*)(gbase + SM_BAR + 8 * (2 * KN_STAGES + 7));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < KN_STAGES; ++s) {
            mbar_init(FULL(s), 1);
            mbar_init(EMPTY(s), 1 + 4 * KN_SPLIT);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(TFULL(b), 1);
            mbar_init(TEMPTY(b), 4 * KN_SPLIT);
        }
        mbar_init(AFULL, 1);
        mbar_init(AEMPTY, 1);
        mbar_init(DRAIN, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // what was issued, for the drain after an abort: the parity of the last A
    // load and of the last B load per stage (-1: none), and whether MMAs ran
    int last_a = -1;
    int last_b[KN_STAGES];
    for (int st = 0; st < KN_STAGES; ++st) last_b[st] = -1;
    bool mma_issued = false;
    if (warp == 0) {
        // ------------------------------------------------ TMA producer ---
        if (lane == 0) {
            int64_t it = 0;
            int j = 0;
            bool ok = true;
            for (int64_t wi = blockIdx.x; wi < S.nqt * S.nchunk && ok; wi += gridDim.x, ++j) {
                const int64_t qt = wi / S.nchunk, ch = wi % S.nchunk;
                const int64_t ct0 = ch * S.nct / S.nchunk, ct1 = (ch + 1) * S.nct / S.nchunk;
                if (!mbar_wait(AEMPTY, (j & 1) ^ 1, S.status, abort_flag)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(AFULL, KN_M * KN_K * 2);
                tma_load_2d(base + SM_A, &tmA, 0, (int)(qt * KN_M), AFULL);
                last_a = j & 1;
                for (int64_t ct = ct0; ct < ct1; ++ct, ++it) {
                    int s = (int)(it % KN_STAGES);
                    uint32_t ph = (uint32_t)((it / KN_STAGES) & 1);
                    if (!mbar_wait(EMPTY(s), ph ^ 1, S.status, abort_flag)) { ok = false; break; }
                    mbar_expect_tx(FULL(s), KN_N * KN_K * 2 + 3 * KN_N * 4);
                    tma_load_2d(base + SM_B + s * (KN_N * KN_K * 2), &tmB, 0, (int)(ct * KN_N), FULL(s));
                    uint32_t info = base + SM_INFO + s * (KN_N * 12);
                    bulk_load(info, S.cid + ct * KN_N, KN_N * 4, FULL(s));
                    bulk_load(info + KN_N * 4, S.cnrm + ct * KN_N, KN_N * 4, FULL(s));
                    bulk_load(info + KN_N * 8, S.cncf + ct * KN_N, KN_N * 4, FULL(s));
                    last_b[s] = (int)ph;
                }
            }
        }
    } else if (warp == 1) {
        // --------------------------------------------------- MMA issuer ---
        if (lane == 0) {
            int64_t it = 0;
            int j = 0;
            for (int64_t wi = blockIdx.x; wi < S.nqt * S.nchunk; wi += gridDim.x, ++j) {
                const int64_t ch = wi % S.nchunk;
                const int64_t ct0 = ch * S.nct / S.nchunk, ct1 = (ch + 1) * S.nct / S.nchunk;
                if (!mbar_wait(AFULL, j & 1, S.status, abort_flag)) break;
                bool ok = true;
                for (int64_t ct = ct0; ct < ct1; ++ct, ++it) {
                    int s = (int)(it % KN_STAGES);
                    uint32_t ph = (uint32_t)((it / KN_STAGES) & 1);
                    int b = (int)(it & 1);
                    uint32_t pb = (uint32_t)((it >> 1) & 1);
                    if (!mbar_wait(FULL(s), ph, S.status, abort_flag) ||
                        !mbar_wait(TEMPTY(b), pb ^ 1, S.status, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    uint32_t a0 = base + SM_A, b0 = base + SM_B + s * (KN_N * KN_K * 2);
#pragma unroll
                    for (int kk = 0; kk < KN_K / 16; ++kk)
                        umma_bf16(tmem + b * KN_N, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), kk > 0);
                    umma_commit(EMPTY(s));
                    umma_commit(TFULL(b));
                    mma_issued = true;
                }
                umma_commit(AEMPTY);
                if (!ok) break;
            }
        }
    } else {
        // --------------------------------------------------- selection ---
        const int quarter = warp & 3;             // TMEM lanes 32*quarter .. +31
        const int half = (warp - 2) >> 2;         // column slice of every tile this warp screens
        const int row = quarter * 32 + lane;
        float2* mylist = (float2*)(gbase + SM_LIST) + (row * KN_SPLIT + half) * KN_KMAX;
        int64_t it = 0;
        for (int64_t wi = blockIdx.x; wi < S.nqt * S.nchunk; wi += gridDim.x) {
            const int64_t qt = wi / S.nchunk, ch = wi % S.nchunk;
            const int64_t ct0 = ch * S.nct / S.nchunk, ct1 = (ch + 1) * S.nct / S.nchunk;
            const int64_t slot = qt * KN_M + row;
            Row r{__int_as_float(0x7f800000), 0x7fffffff, 0, 0};
            const int64_t state = (slot * S.nchunk + ch) * KN_SPLIT + half;
            const RowConst rc{S.qv[slot], S.exclude_self ? S.qv[slot] : -2, S.qexact[slot] != 0,
                              KN_ALPHA * S.qnrm[slot], mylist, S.shortlist + state * KN_SCAP, S.overflow + slot, S.k};
            const bool qtile_exact = S.qtile[qt] != 0;
            bool ok = true;
            for (int64_t ct = ct0; ct < ct1; ++ct, ++it) {
                int s = (int)(it % KN_STAGES);
                uint32_t ph = (uint32_t)((it / KN_STAGES) & 1);
                int b = (int)(it & 1);
                uint32_t pb = (uint32_t)((it >> 1) & 1);
                if (!mbar_wait(FULL(s), ph, S.status, abort_flag) || !mbar_wait(TFULL(b), pb, S.status, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint8_t* info = gbase + SM_INFO + s * (KN_N * 12);
                const int32_t* cid = (const int32_t*)info;
                const float* cnrm = (const float*)(info + KN_N * 4);
                const float* cncf = (const float*)(info + KN_N * 8);
                const bool fast = qtile_exact && S.ctile[ct];
                const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + b * KN_N;
                {
                    const int h = half;                   // 128 columns per selection warp
                    uint32_t u0[32], u1[32], u2[32], u3[32];
                    __syncwarp();
                    tmem_ld32_async(tbase + h * 128 + 0, u0);
                    tmem_ld32_async(tbase + h * 128 + 32, u1);
                    tmem_ld32_async(tbase + h * 128 + 64, u2);
                    tmem_ld32_async(tbase + h * 128 + 96, u3);
                    tmem_wait_ld();
                    reg_fence(u0);
                    reg_fence(u1);
                    reg_fence(u2);
                    reg_fence(u3);
                    float y[32];
#define KN_GROUP(U, G)                                                                                   \
    {                                                                                                    \
        _Pragma("unroll") for (int j = 0; j < 32; ++j) y[j] = __uint_as_float(U[j]);                     \
        const int c0 = h * 128 + (G) * 32;                                                               \
        if (DUMP && rc.qid >= 0) {                                                                       \
            float* dst = S.dump + (int64_t)S.qidx[slot] * S.npad + ct * KN_N + c0;                       \
            _Pragma("unroll") for (int j = 0; j < 32; ++j) dst[j] = y[j];                                \
        }                                                                                                \
        r = select_group(r, rc, y, fast, cid + c0, cnrm + c0, cncf + c0, ct * KN_N + c0, S.nexact);      \
    }
                    KN_GROUP(u0, 0)
                    KN_GROUP(u1, 1)
                    KN_GROUP(u2, 2)
                    KN_GROUP(u3, 3)
#undef KN_GROUP
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(TEMPTY(b));
                    mbar_arrive(EMPTY(s));
                }
            }
            if (!ok) break;
            for (int i = 0; i < S.k; ++i)
                S.lists[state * S.k + i] = i < r.n ? mylist[i] : make_float2(0.f, __int_as_float(-1));
            S.scount[state] = r.scount;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag) {
        // a wait ran out somewhere in the CTA: the copies issued into shared
        // memory land and the MMAs issued complete before the CTA releases
        // TMEM and exits (each drain is bounded too)
        if (warp == 0 && lane == 0) {
            if (last_a >= 0) mbar_drain(AFULL, (uint32_t)last_a);
            for (int st = 0; st < KN_STAGES; ++st)
                if (last_b[st] >= 0) mbar_drain(FULL(st), (uint32_t)last_b[st]);
        }
        if (warp == 1 && lane == 0 && mma_issued) {
            umma_commit(DRAIN);
            mbar_drain(DRAIN, 0);
        }
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// ------------------------------------------------ FP32 comparison form ---
// One thread per query row, candidates streamed through shared memory in
// tiles of 256; y = |b|^2 - 2 a.b with the dot product in FP32 FMAs. Bound:
// |y_hat - y| <= (D+3) 2^-23 (2|a||b| + |b|^2) + 1.
constexpr int F_T = 128, F_TILE = 32;

// KK: padded vector length, 64 (D <= 64) or 128 (D <= 128)
template <int KK>
__global__ void __launch_bounds__(F_T) fp32_kernel(const uint32_t* __restrict__ theta_q,
                                                   const uint32_t* __restrict__ theta_c, bool exclude_self, int D,
                                                   const int32_t* __restrict__ qv,
                                                   const uint8_t* __restrict__ qexact, const float* __restrict__ qnrm,
                                                   int64_t qpad, int64_t nexact,
                                                   const int32_t* __restrict__ cidv, const float* __restrict__ cnrmv,
                                                   const float* __restrict__ cncfv, int64_t npad, int k,
                                                   float2* __restrict__ lists, int32_t* __restrict__ shortlist,
                                                   int32_t* __restrict__ scount, int* __restrict__ overflow) {
    __shared__ float cb[F_TILE][KK];
    __shared__ float cn2[F_TILE], cnr[F_TILE];
    __shared__ int cidx[F_TILE];
    __shared__ float2 lst[F_T * KN_KMAX];
    const int64_t slot = (int64_t)blockIdx.x * F_T + threadIdx.x;
    // candidate range blockIdx.y of gridDim.y (whole 256-candidate tiles)
    const int64_t nch = gridDim.y, ch = blockIdx.y, nct = npad / 256;
    const int64_t cbeg = ch * nct / nch * 256, cend = (ch + 1) * nct / nch * 256;
    const int64_t state = slot * nch + ch;
    const float epsD = (float)(D + 3) * (1.0f / 8388608.0f);
    const int qid = slot < qpad ? qv[slot] : -1;
    // rows with every entry <= 256 give exact FP32 products and partial sums
    // (all integers below 2^24); other pairs carry the bound
    const bool qex = slot < qpad && qexact[slot] != 0;
    const RowConst rc{qid, exclude_self ? qid : -2, qex, 2.0f * epsD * (slot < qpad ? qnrm[slot] : 0.f),
                      lst + threadIdx.x * KN_KMAX, shortlist + (slot < qpad ? state : 0) * KN_SPLIT * KN_SCAP,
                      overflow + (slot < qpad ? slot : 0), k};
    Row r{__int_as_float(0x7f800000), 0x7fffffff, 0, 0};
    float a[KK];
#pragma unroll
    for (int d = 0; d < KK; ++d) a[d] = (qid >= 0 && d < D) ? (float)theta_q[(int64_t)qid * D + d] : 0.f;
    for (int64_t c0 = cbeg; c0 < cend; c0 += F_TILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < F_TILE * KK; i += F_T) {
            int c = i / KK, d = i % KK;
            int32_t v = cidv[c0 + c];
            cb[c][d] = (v >= 0 && d < D) ? (float)theta_c[(int64_t)v * D + d] : 0.f;
        }
        if (threadIdx.x < F_TILE) {
            cidx[threadIdx.x] = cidv[c0 + threadIdx.x];
            cn2[threadIdx.x] = cncfv[c0 + threadIdx.x];
            cnr[threadIdx.x] = cnrmv[c0 + threadIdx.x];
        }
        __syncthreads();
        if (qid < 0) continue;
        for (int c = 0; c < F_TILE; ++c) {
            float s = 0.f;
#pragma unroll
            for (int d = 0; d < KK; ++d) s = fmaf(a[d], cb[c][d], s);
            float y = fmaf(-2.0f, s, cn2[c]);
            float E = (fmaf(rc.anrm, cnr[c], epsD * cn2[c]) + 1.0f) * 1.0001f;
            if (__fsub_rd(y, E) <= r.thr) r = take_bounded(r, rc, y, E, cidx[c], c0 + c < nexact);
        }
    }
    if (slot < qpad) {
        for (int i = 0; i < k; ++i) {
            lists[(state * KN_SPLIT) * k + i] = i < r.n ? rc.list[i] : make_float2(0.f, __int_as_float(-1));
            for (int h = 1; h < KN_SPLIT; ++h) lists[(state * KN_SPLIT + h) * k + i] = make_float2(0.f, __int_as_float(-1));
        }
        scount[state * KN_SPLIT] = r.scount;
        for (int h = 1; h < KN_SPLIT; ++h) scount[state * KN_SPLIT + h] = 0;
    }
}

// ------------------------------------------------------------- rerank ---
// exact squared distance between row a of theta_q and row b of theta_c
__device__ __forceinline__ uint64_t exact_d2(const uint32_t* __restrict__ theta_q, const uint32_t* __restrict__ theta_c,
                                             int D, int32_t a, int32_t b) {
    uint64_t s = 0;
    const uint32_t* x = theta_q + (int64_t)a * D;
    const uint32_t* y = theta_c + (int64_t)b * D;
    for (int d = 0; d < D; ++d) {
        int64_t t = (int64_t)x[d] - (int64_t)y[d];
        s += (uint64_t)(t * t);
    }
    return s;
}

__device__ __forceinline__ bool pair_less(uint64_t d1, int i1, uint64_t d2, int i2) {
    return d1 < d2 || (d1 == d2 && i1 < i2);
}

// One warp per (query slot, candidate range): exact distances of every kept
// candidate, top-k of the range. With one range per query the rows go to the
// output; otherwise to part_d2 / part_id ([qpad][nchunk][k]) for chunk_merge.
__global__ void rerank_kernel(const uint32_t* __restrict__ theta_q, const uint32_t* __restrict__ theta_c, int D,
                              const int32_t* __restrict__ qv,
                              const int32_t* __restrict__ qidx, int64_t qpad, int64_t nchunk, int k,
                              const float2* __restrict__ lists, const int32_t* __restrict__ shortlist,
                              const int32_t* __restrict__ scount, const int* __restrict__ overflow,
                              int32_t* __restrict__ out_ids, uint64_t* __restrict__ out_d2,
                              int32_t* __restrict__ part_id, uint64_t* __restrict__ part_d2) {
    const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (grp >= qpad * nchunk) return;
    const int64_t slot = grp / nchunk;
    const int32_t v = qv[slot];
    if (v < 0 || overflow[slot]) return;   // padding, or handled by the brute-force fallback
    int32_t* oid = nchunk == 1 ? out_ids + (int64_t)qidx[slot] * k : part_id + grp * k;
    uint64_t* od = nchunk == 1 ? out_d2 + (int64_t)qidx[slot] * k : part_d2 + grp * k;
    // candidates: the lists of the column slices, then their shortlists
    int ns[KN_SPLIT];
    int nst = 0;
#pragma unroll
    for (int h = 0; h < KN_SPLIT; ++h) {
        ns[h] = min(scount[grp * KN_SPLIT + h], KN_SCAP);
        nst += ns[h];
    }
    const int nl = KN_SPLIT * k;
    const int total = nl + nst;
    // each lane holds up to ceil(total/32) candidates
    constexpr int PER = (KN_SPLIT * (KN_KMAX + KN_SCAP) + 31) / 32;
    uint64_t dd[PER];
    int id[PER];
#pragma unroll
    for (int t = 0; t < PER; ++t) {
        int i = lane + 32 * t;
        id[t] = -1;
        dd[t] = ~0ull;
        if (i < total) {
            int c;
            if (i < nl) {
                c = __float_as_int(lists[grp * nl + i].y);
            } else {
                int j = i - nl, h = 0;
                while (h < KN_SPLIT - 1 && j >= ns[h]) j -= ns[h++];
                c = shortlist[(grp * KN_SPLIT + h) * KN_SCAP + j];
            }
            if (c >= 0) {
                id[t] = c;
                dd[t] = exact_d2(theta_q, theta_c, D, v, c);
            }
        }
    }
    uint64_t lastd = 0;
    int lasti = -1;
    bool first = true;
    for (int r = 0; r < k; ++r) {
        uint64_t bd = ~0ull;
        int bi = 0x7fffffff;
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            if (id[t] < 0) continue;
            bool after = first || pair_less(lastd, lasti, dd[t], id[t]);
            if (after && pair_less(dd[t], id[t], bd, bi)) {
                bd = dd[t];
                bi = id[t];
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            uint64_t od = __shfl_xor_sync(0xffffffffu, bd, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (pair_less(od, oi, bd, bi)) {
                bd = od;
                bi = oi;
            }
        }
        if (lane == 0) {
            oid[r] = bi == 0x7fffffff ? -1 : bi;
            od[r] = bi == 0x7fffffff ? ~0ull : bd;
        }
        if (bi == 0x7fffffff) {
            for (int rr = r + 1; rr < k && lane == 0; ++rr) {
                oid[rr] = -1;
                od[rr] = ~0ull;
            }
            break;
        }
        lastd = bd;
        lasti = bi;
        first = false;
    }
}

// one CTA per query slot: top-k of the nchunk exact top-k lists of its ranges
// (the ranges are disjoint, so no candidate appears twice)
// With `slots` given, entry i of the lists belongs to query slot slots[i]
// (the brute-force fallback); otherwise to slot i, skipping overflowed slots.
__global__ void __launch_bounds__(256) chunk_merge_kernel(const int32_t* __restrict__ qv,
                                                          const int32_t* __restrict__ qidx,
                                                          const int* __restrict__ overflow,
                                                          const int32_t* __restrict__ slots, int64_t count,
                                                          int64_t nchunk, int k, const int32_t* __restrict__ part_id,
                                                          const uint64_t* __restrict__ part_d2,
                                                          int32_t* __restrict__ out_ids,
                                                          uint64_t* __restrict__ out_d2) {
    __shared__ uint64_t sd[8];
    __shared__ int si[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t total = nchunk * k;
    for (int64_t e = blockIdx.x; e < count; e += gridDim.x) {
        const int64_t slot = slots ? slots[e] : e;
        if (qv[slot] < 0 || (!slots && overflow[slot])) continue;
        const int64_t qi = qidx[slot], base = e * total;
        uint64_t lastd = 0;
        int lasti = -1;
        for (int r = 0; r < k; ++r) {
            uint64_t bd = ~0ull;
            int bi = 0x7fffffff;
            for (int64_t t = threadIdx.x; t < total; t += 256) {
                const int id = part_id[base + t];
                if (id < 0) continue;
                const uint64_t d = part_d2[base + t];
                if ((r == 0 || pair_less(lastd, lasti, d, id)) && pair_less(d, id, bd, bi)) {
                    bd = d;
                    bi = id;
                }
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                uint64_t od = __shfl_xor_sync(0xffffffffu, bd, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (pair_less(od, oi, bd, bi)) {
                    bd = od;
                    bi = oi;
                }
            }
            if (lane == 0) {
                sd[warp] = bd;
                si[warp] = bi;
            }
            __syncthreads();
            bd = sd[0];
            bi = si[0];
#pragma unroll
            for (int w = 1; w < 8; ++w)
                if (pair_less(sd[w], si[w], bd, bi)) {
                    bd = sd[w];
                    bi = si[w];
                }
            __syncthreads();
            if (threadIdx.x == 0) {
                out_ids[qi * k + r] = bi == 0x7fffffff ? -1 : bi;
                out_d2[qi * k + r] = bi == 0x7fffffff ? ~0ull : bd;
            }
            lastd = bd;
            lasti = bi;
        }
    }
}

// Exact brute force for the (rare) queries whose shortlist overflowed: the
// vertex range of each such query is cut into nparts pieces, one warp each.
// A warp keeps its k best (d2, id) sorted across its lanes (lane l holds rank
// l); a batch of 32 candidates costs one compare and a ballot unless one of
// them beats the k-th entry. The nparts lists go through chunk_merge_kernel.
__global__ void __launch_bounds__(256) brute_warp_kernel(const uint32_t* __restrict__ theta_q,
                                                         const uint32_t* __restrict__ theta_c, bool exclude_self,
                                                         int D, int64_t n,
                                                         const int32_t* __restrict__ qv,
                                                         const int32_t* __restrict__ ovslots, int64_t nov,
                                                         int64_t nparts, int k, int32_t* __restrict__ part_id,
                                                         uint64_t* __restrict__ part_d2) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= nov * nparts) return;
    const int64_t oi = gw / nparts, part = gw % nparts;
    const int32_t v = qv[ovslots[oi]];
    const int64_t u0 = part * n / nparts, u1 = (part + 1) * n / nparts;
    uint64_t ld = ~0ull;   // this lane's rank of the list
    int li = 0x7fffffff;
    for (int64_t base = u0; base < u1; base += 32) {
        const int64_t u = base + lane;
        uint64_t d = ~0ull;
        const bool cand = u < u1 && (!exclude_self || u != v);
        if (cand) d = exact_d2(theta_q, theta_c, D, v, (int32_t)u);
        const uint64_t td = __shfl_sync(0xffffffffu, ld, k - 1);
        const int ti = __shfl_sync(0xffffffffu, li, k - 1);
        unsigned pass = __ballot_sync(0xffffffffu, cand && pair_less(d, (int)u, td, ti));
        while (pass) {
            const int src = __ffs(pass) - 1;
            pass &= pass - 1;
            const uint64_t nd = __shfl_sync(0xffffffffu, d, src);
            const int ni = (int)__shfl_sync(0xffffffffu, (int)u, src);
            // entries at or after the insertion point move up one lane
            const bool after = pair_less(nd, ni, ld, li);
            const unsigned am = __ballot_sync(0xffffffffu, after);
            const uint64_t upd = __shfl_up_sync(0xffffffffu, ld, 1);
            const int upi = __shfl_up_sync(0xffffffffu, li, 1);
            if (am) {
                const int pos = __ffs(am) - 1;
                if (lane == pos) {
                    ld = nd;
                    li = ni;
                } else if (lane > pos) {
                    ld = upd;
                    li = upi;
                }
            }
            // candidates of this batch that no longer beat the k-th entry drop out
            const uint64_t td2 = __shfl_sync(0xffffffffu, ld, k - 1);
            const int ti2 = __shfl_sync(0xffffffffu, li, k - 1);
            pass &= __ballot_sync(0xffffffffu, pair_less(d, (int)u, td2, ti2));
        }
    }
    if (lane < k) {
        part_id[gw * k + lane] = li == 0x7fffffff ? -1 : li;
        part_d2[gw * k + lane] = ld;
    }
}

// query slots: exact queries first (stable), padded to a multiple of 128
__global__ void query_slots_kernel(const int32_t* __restrict__ queries, int64_t q, const uint8_t* __restrict__ exact,
                                   int64_t n, const int64_t* __restrict__ exscan, int64_t nexq,
                                   int32_t* __restrict__ qv, int32_t* __restrict__ qidx, uint32_t* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    int32_t v = queries ? queries[i] : (int32_t)i;
    bool bad = v < 0 || v >= n;
    if (bad) flag_status(status, ST_BAD_QUERY);
    bool e = bad ? true : exact[v] != 0;
    int64_t p = e ? exscan[i] : nexq + (i - exscan[i]);
    qv[p] = bad ? -1 : v;
    qidx[p] = (int32_t)i;
}

__global__ void query_info_kernel(const int32_t* __restrict__ qv, int64_t qpad, const uint8_t* __restrict__ exact,
                                  const float* __restrict__ nrm, uint8_t* __restrict__ qexact, float* __restrict__ qnrm) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= qpad) return;
    int32_t v = qv[s];
    qexact[s] = v < 0 ? 1 : exact[v];
    qnrm[s] = v < 0 ? 0.f : nrm[v];
}

__global__ void exact_flags_of_queries(const int32_t* __restrict__ queries, int64_t q, const uint8_t* __restrict__ exact,
                                       int64_t n, int64_t* __restrict__ f) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    int32_t v = queries ? queries[i] : (int32_t)i;
    f[i] = (v < 0 || v >= n) ? 1 : exact[v];
}

__global__ void fill_i32(int32_t* p, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

// ---------------------------------------------------------------- host ---
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn(panther_ctx* ctx) {
    // looked up once (thread-safe static initialisation: serving workers race here)
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)p;
        return nullptr;
    }();
    if (!fn) set_err(ctx, PANTHER_ECUDA, "cuTensorMapEncodeTiled is not available");
    return fn;
}

static bool make_map(panther_ctx* ctx, CUtensorMap* m, const void* base, int64_t rows, int box_rows) {
    auto fn = encode_fn(ctx);
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)KN_K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)KN_K * 2};
    cuuint32_t box[2] = {(cuuint32_t)KN_K, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_err(ctx, PANTHER_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return false;
    }
    return true;
}

extern "C" panther_status pantherpp_vectors(panther_ctx* ctx, const panther_index* ix, const panther_paths* p, int D,
                                            pantherpp_vecs** out) {
    if (!ctx || !ix || !p || !out) return PANTHER_EINVAL;
    *out = nullptr;
    if (D < 1 || D > 128) return set_err(ctx, PANTHER_EINVAL, "D must be in [1, 128]");
    if (ix->n != p->n || ix->R != p->R)
        return set_err(ctx, PANTHER_EINVAL, "index and paths do not belong together");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    const int64_t n = ix->n;
    pantherpp_vecs* v = new pantherpp_vecs();
    v->ctx = ctx;
    v->n = n;
    v->D = D;
    panther_status st;
    int64_t* flag = nullptr;
    int64_t* pos = nullptr;
    unsigned* maxv = nullptr;
    auto fail = [&](panther_status x) {
        dev_free(ctx, flag);
        dev_free(ctx, pos);
        dev_free(ctx, maxv);
        pantherpp_free_vecs(v);
        return x;
    };
    if ((st = dev_alloc(ctx, (void**)&v->theta, sizeof(uint32_t) * n * D))) return fail(st);
    if ((st = topk_counts_all(ctx, ix, p, D, v->theta))) return fail(st);
    if ((st = dev_alloc(ctx, (void**)&v->norm2, sizeof(uint64_t) * n)) ||
        (st = dev_alloc(ctx, (void**)&v->nrm, sizeof(float) * n)) ||
        (st = dev_alloc(ctx, (void**)&v->exact, n)) || (st = dev_alloc(ctx, (void**)&flag, sizeof(int64_t) * n)) ||
        (st = dev_alloc(ctx, (void**)&pos, sizeof(int64_t) * n)) || (st = dev_alloc(ctx, (void**)&maxv, 4)))
        return fail(st);
    PCK(ctx, cudaMemsetAsync(maxv, 0, 4, s));
    unsigned gb = (unsigned)ceil_div(n, 256);
    vec_stats_kernel<<<gb, 256, 0, s>>>(v->theta, n, D, v->norm2, v->nrm, v->exact, flag, maxv);
    ctx->launches++;
    // number of exact rows = sum of flags (read before the scan overwrites them)
    if ((st = scan_exclusive_i64(ctx, flag, n))) return fail(st);
    int64_t last_scan = 0;
    uint8_t last_flag = 0;
    unsigned hmax = 0;
    PCK(ctx, cudaMemcpyAsync(&last_scan, flag + n - 1, 8, cudaMemcpyDeviceToHost, s));
    PCK(ctx, cudaMemcpyAsync(&last_flag, v->exact + n - 1, 1, cudaMemcpyDeviceToHost, s));
    PCK(ctx, cudaMemcpyAsync(&hmax, maxv, 4, cudaMemcpyDeviceToHost, s));
    PCK(ctx, cudaStreamSynchronize(s));
    v->max_val = hmax;
    if ((unsigned __int128)hmax * hmax * (unsigned)D >= ((unsigned __int128)1 << 64))
        return fail(set_err(ctx, PANTHER_EOVERFLOW, "max count^2 * D reaches 2^64: squared distances could overflow"));
    pantherpp_vecs& x = *v;
    x.nexact = last_scan + last_flag;
    x.npad = ceil_div(n, KN_N) * KN_N;
    int32_t* perm = nullptr;
    if ((st = dev_alloc(ctx, (void**)&perm, sizeof(int32_t) * x.npad)) ||
        (D <= KN_K - 8 && (st = dev_alloc(ctx, (void**)&x.B, (size_t)x.npad * KN_K * 2))) ||
        (st = dev_alloc(ctx, (void**)&x.cid, sizeof(int32_t) * x.npad)) ||
        (st = dev_alloc(ctx, (void**)&x.cnrm, sizeof(float) * x.npad)) ||
        (st = dev_alloc(ctx, (void**)&x.cncf, sizeof(float) * x.npad)) ||
        (st = dev_alloc(ctx, (void**)&x.ctile, x.npad / KN_N))) {
        dev_free(ctx, perm);
        return fail(st);
    }
    vec_perm_kernel<<<gb, 256, 0, s>>>(v->exact, flag, n, x.nexact, perm, pos);
    vec_brow_kernel<<<(unsigned)ceil_div(x.npad, 256), 256, 0, s>>>(v->theta, v->norm2, v->nrm, perm,
                                                                    VecMeta{n, x.npad, x.nexact, D}, x.B, x.cid,
                                                                    x.cnrm, x.cncf);
    tile_flags_kernel<<<(unsigned)ceil_div(x.npad / KN_N, 256), 256, 0, s>>>(v->exact, x.cid, x.npad, KN_N, x.ctile,
                                                                             x.npad / KN_N);
    ctx->launches += 3;
    dev_free(ctx, perm);
    dev_free(ctx, flag);
    dev_free(ctx, pos);
    dev_free(ctx, maxv);
    flag = nullptr;
    pos = nullptr;
    maxv = nullptr;
    cudaError_t ce = cudaStreamSynchronize(s);
    if (ce) return fail(cuda_err(ctx, ce, "vector preparation"));
    *out = v;
    return PANTHER_OK;
}

// Candidate ranges per query tile: with fewer query tiles than SMs, the
// candidate tiles are cut into ranges so that tiles x ranges work items fill
// the GPU; the choice minimises waves x range length, at least KN_STAGES
// candidate tiles per range (both forms).
static int64_t knn_ranges(int64_t nqt, int64_t nct, int num_sms, bool fp32) {
    (void)fp32;   // both forms cut the candidates the same way
    if (nqt >= num_sms) return 1;
    const int64_t pmax = std::max<int64_t>(1, std::min<int64_t>(nct / KN_STAGES, 256));
    int64_t best = 1;
    double best_cost = (double)ceil_div(nqt, num_sms);
    for (int64_t p = 2; p <= pmax; ++p) {
        double cost = (double)ceil_div(nqt * p, num_sms) / (double)p;
        if (cost < best_cost * 0.999) {
            best = p;
            best_cost = cost;
        }
    }
    return best;
}

// queries are vertices of vq, candidates every vertex of vc; `same` excludes
// the candidate with the query's id (one graph: the query itself)
static panther_status knn_run(panther_ctx* ctx, const pantherpp_vecs* vq, const pantherpp_vecs* vc, bool same,
                              const int32_t* queries, int64_t q, int k, int32_t* ids, uint64_t* d2, bool fp32,
                              float* dump = nullptr) {
    const pantherpp_vecs& x = *vc;
    const pantherpp_vecs* v = vq;
    cudaStream_t s = ctx->stream;
    const int64_t n = vq->n;
    const int64_t qpad = ceil_div(q, KN_M) * KN_M;
    const int64_t nch = knn_ranges(qpad / KN_M, x.npad / KN_N, ctx->num_sms, fp32);
    panther_status st;
    int64_t* qf = nullptr;
    int32_t *qv = nullptr, *qidx = nullptr, *sl = nullptr, *sc = nullptr, *pid = nullptr;
    int* ovf = nullptr;
    uint8_t *qex = nullptr, *qtile = nullptr;
    float* qn = nullptr;
    float2* lists = nullptr;
    uint16_t* A = nullptr;
    uint64_t* pd = nullptr;
    auto cleanup = [&]() {
        dev_free(ctx, qf); dev_free(ctx, qv); dev_free(ctx, qidx); dev_free(ctx, sl); dev_free(ctx, sc);
        dev_free(ctx, ovf); dev_free(ctx, qex); dev_free(ctx, qtile); dev_free(ctx, qn); dev_free(ctx, lists);
        dev_free(ctx, A); dev_free(ctx, pid); dev_free(ctx, pd);
    };
    const int64_t nstate = qpad * nch * KN_SPLIT;
    if ((st = dev_alloc(ctx, (void**)&qf, sizeof(int64_t) * q)) ||
        (st = dev_alloc(ctx, (void**)&qv, sizeof(int32_t) * qpad)) ||
        (st = dev_alloc(ctx, (void**)&qidx, sizeof(int32_t) * qpad)) ||
        (st = dev_alloc(ctx, (void**)&sl, sizeof(int32_t) * nstate * KN_SCAP)) ||
        (st = dev_alloc(ctx, (void**)&sc, sizeof(int32_t) * nstate)) ||
        (st = dev_alloc(ctx, (void**)&ovf, sizeof(int) * qpad)) || (st = dev_alloc(ctx, (void**)&qex, qpad)) ||
        (st = dev_alloc(ctx, (void**)&qtile, qpad / KN_M)) || (st = dev_alloc(ctx, (void**)&qn, sizeof(float) * qpad)) ||
        (st = dev_alloc(ctx, (void**)&lists, sizeof(float2) * nstate * k)) ||
        (nch > 1 && ((st = dev_alloc(ctx, (void**)&pid, sizeof(int32_t) * qpad * nch * k)) ||
                     (st = dev_alloc(ctx, (void**)&pd, sizeof(uint64_t) * qpad * nch * k)))) ||
        (!fp32 && (st = dev_alloc(ctx, (void**)&A, (size_t)qpad * KN_K * 2)))) {
        cleanup();
        return st;
    }
    unsigned gq = (unsigned)ceil_div(q, 256), gp = (unsigned)ceil_div(qpad, 256);
    exact_flags_of_queries<<<gq, 256, 0, s>>>(queries, q, v->exact, n, qf);
    if ((st = scan_exclusive_i64(ctx, qf, q))) { cleanup(); return st; }
    // number of exact queries: recompute the last flag on the host side of the scan
    int64_t last = 0;
    int32_t lastq = 0;
    PCK(ctx, cudaMemcpyAsync(&last, qf + q - 1, 8, cudaMemcpyDeviceToHost, s));
    if (queries) PCK(ctx, cudaMemcpyAsync(&lastq, queries + q - 1, 4, cudaMemcpyDeviceToHost, s));
    else lastq = (int32_t)(q - 1);
    PCK(ctx, cudaStreamSynchronize(s));
    uint8_t lastex = 1;
    if (lastq >= 0 && lastq < n) {
        PCK(ctx, cudaMemcpyAsync(&lastex, v->exact + lastq, 1, cudaMemcpyDeviceToHost, s));
        PCK(ctx, cudaStreamSynchronize(s));
    }
    const int64_t nexq = last + lastex;
    fill_i32<<<gp, 256, 0, s>>>(qv, qpad, -1);
    fill_i32<<<gp, 256, 0, s>>>(qidx, qpad, 0);
    PCK(ctx, cudaMemsetAsync(ovf, 0, sizeof(int) * qpad, s));
    query_slots_kernel<<<gq, 256, 0, s>>>(queries, q, v->exact, n, qf, nexq, qv, qidx, ctx->d_status);
    query_info_kernel<<<gp, 256, 0, s>>>(qv, qpad, v->exact, v->nrm, qex, qn);
    tile_flags_kernel<<<(unsigned)ceil_div(qpad / KN_M, 256), 256, 0, s>>>(v->exact, qv, qpad, KN_M, qtile,
                                                                           qpad / KN_M);
    ctx->launches += 6;
    if (!fp32) {
        vec_arow_kernel<<<gp, 256, 0, s>>>(v->theta, qv, qpad, v->D, A);
        ctx->launches++;
        CUtensorMap tmA, tmB;
        if (!make_map(ctx, &tmA, A, qpad, KN_M) || !make_map(ctx, &tmB, x.B, x.npad, KN_N)) {
            cleanup();
            return PANTHER_ECUDA;
        }
        ScreenArgs S{x.cid, x.cnrm, x.cncf, x.ctile, x.npad / KN_N, x.nexact, qv, qn, qex, qtile, qpad / KN_M,
                     nch, k, lists, sl, sc, ovf, ctx->d_status, same, dump, qidx, x.npad};
        int64_t grid = std::min<int64_t>(qpad / KN_M * nch, ctx->num_sms);
        if (dump) {
            PCK(ctx, cudaFuncSetAttribute(screen_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)KN_SMEM_BYTES));
            screen_kernel<true><<<(unsigned)grid, KN_THREADS, KN_SMEM_BYTES, s>>>(tmA, tmB, S);
        } else {
            PCK(ctx, cudaFuncSetAttribute(screen_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)KN_SMEM_BYTES));
            screen_kernel<false><<<(unsigned)grid, KN_THREADS, KN_SMEM_BYTES, s>>>(tmA, tmB, S);
        }
        ctx->launches++;
    } else {
        if (v->D <= KN_K)
            fp32_kernel<64><<<dim3((unsigned)(qpad / F_T), (unsigned)nch), F_T, 0, s>>>(vq->theta, vc->theta, same, v->D, qv, qex, qn, qpad,
                                                            x.nexact, x.cid,
                                                            x.cnrm, x.cncf, x.npad, k, lists, sl, sc, ovf);
        else
            fp32_kernel<128><<<dim3((unsigned)(qpad / F_T), (unsigned)nch), F_T, 0, s>>>(vq->theta, vc->theta, same, v->D, qv, qex, qn, qpad,
                                                            x.nexact, x.cid,
                                                            x.cnrm, x.cncf, x.npad, k, lists, sl, sc, ovf);
        ctx->launches++;
    }
    PCK(ctx, cudaGetLastError());
    rerank_kernel<<<(unsigned)ceil_div(qpad * nch * 32, 256), 256, 0, s>>>(vq->theta, vc->theta, v->D, qv, qidx,
                                                                            qpad, nch, k,
                                                                            lists, sl, sc, ovf, ids, d2, pid, pd);
    ctx->launches++;
    if (nch > 1) {
        chunk_merge_kernel<<<(unsigned)std::min<int64_t>(qpad, 8 * ctx->num_sms), 256, 0, s>>>(
            qv, qidx, ovf, nullptr, qpad, nch, k, pid, pd, ids, d2);
        ctx->launches++;
    }
    PCK(ctx, cudaGetLastError());
    // screening statistics (pairs screened, kept for rerank, overflowed queries)
    std::vector<int32_t> hsc(nstate);
    std::vector<int> hov(qpad);
    PCK(ctx, cudaMemcpyAsync(hsc.data(), sc, sizeof(int32_t) * nstate, cudaMemcpyDeviceToHost, s));
    PCK(ctx, cudaMemcpyAsync(hov.data(), ovf, sizeof(int) * qpad, cudaMemcpyDeviceToHost, s));
    PCK(ctx, cudaStreamSynchronize(s));
    int64_t kept = 0, over = 0;
    std::vector<int32_t> hslots;
    for (int64_t i = 0; i < nstate; ++i) kept += hsc[i];
    for (int64_t i = 0; i < qpad; ++i)
        if (hov[i]) hslots.push_back((int32_t)i);
    over = (int64_t)hslots.size();
    if (over) {
        // the overflowed queries: exact brute force over all vertices, spread over the GPU
        const int64_t nparts = std::max<int64_t>(1, std::min<int64_t>(1024, ceil_div(vc->n, 4096)));
        int32_t* dsl = nullptr;
        int32_t* bid = nullptr;
        uint64_t* bd = nullptr;
        auto bfree = [&]() { dev_free(ctx, dsl); dev_free(ctx, bid); dev_free(ctx, bd); };
        if ((st = dev_alloc(ctx, (void**)&dsl, sizeof(int32_t) * over)) ||
            (st = dev_alloc(ctx, (void**)&bid, sizeof(int32_t) * over * nparts * k)) ||
            (st = dev_alloc(ctx, (void**)&bd, sizeof(uint64_t) * over * nparts * k))) {
            bfree();
            cleanup();
            return st;
        }
        cudaError_t ce = cudaMemcpyAsync(dsl, hslots.data(), sizeof(int32_t) * over, cudaMemcpyHostToDevice, s);
        if (!ce) {
            brute_warp_kernel<<<(unsigned)ceil_div(over * nparts * 32, 256), 256, 0, s>>>(
                vq->theta, vc->theta, same, v->D, vc->n, qv, dsl, over, nparts, k, bid, bd);
            chunk_merge_kernel<<<(unsigned)std::min<int64_t>(over, 8 * ctx->num_sms), 256, 0, s>>>(
                qv, qidx, ovf, dsl, over, nparts, k, bid, bd, ids, d2);
            ctx->launches += 2;
            ce = cudaGetLastError();
        }
        if (!ce) ce = cudaStreamSynchronize(s);   // the host slot list must outlive the copy
        bfree();
        if (ce) {
            cleanup();
            return cuda_err(ctx, ce, "k-NN brute-force fallback");
        }
    }
    ctx->knn_stats[0] = q * vc->n;
    ctx->knn_stats[1] = kept;
    ctx->knn_stats[2] = over;
    ctx->knn_stats[3] = x.nexact;
    cleanup();
    return PANTHER_OK;
}

static panther_status knn_entry(panther_ctx* ctx, const pantherpp_vecs* v, const pantherpp_vecs* vc, bool same,
                                const int32_t* queries, int64_t q, int k, int32_t* out_ids, uint64_t* out_dist2,
                                int flags) {
    if (!ctx || !v || !vc) return PANTHER_EINVAL;
    if (vc->D != v->D) return set_err(ctx, PANTHER_EINVAL, "query and candidate vectors differ in D");
    if (q < 0 || q > 0x7fffffffLL) return set_err(ctx, PANTHER_EINVAL, "q must be in [0, 2^31)");
    if (k < 1 || k > KN_KMAX) return set_err(ctx, PANTHER_EINVAL, "k must be in [1, 32]");
    int mode = flags & 0xff;
    if (mode != PANTHER_KNN_BF16_SCREEN && mode != PANTHER_KNN_FP32) return set_err(ctx, PANTHER_EINVAL, "bad flags");
    // vectors wider than the BF16 screen's 56 columns take the FP32 screen
    // (64 or 128 columns), with the same exact rerank
    const bool fp32 = mode == PANTHER_KNN_FP32 || v->D > KN_K - 8;
    auto run = [&](const int32_t* qs, int32_t* oi, uint64_t* od) {
        return knn_run(ctx, v, vc, same, qs, q, k, oi, od, fp32);
    };
    if (q == 0) return PANTHER_OK;
    if (!queries || !out_ids || !out_dist2) return set_err(ctx, PANTHER_EINVAL, "null query or output array");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    if (flags & PANTHER_IO_HOST) {
        int32_t* buf = nullptr;
        size_t qb = ((sizeof(int32_t) * q + 15) / 16) * 16, ib = sizeof(int32_t) * q * k, db = sizeof(uint64_t) * q * k;
        panther_status st = dev_alloc(ctx, (void**)&buf, qb + ib + db + 16);
        if (st) return st;
        uint64_t* dd = (uint64_t*)((char*)buf + qb + ((ib + 15) / 16) * 16);
        int32_t* di = (int32_t*)((char*)buf + qb);
        PCK(ctx, cudaMemcpyAsync(buf, queries, sizeof(int32_t) * q, cudaMemcpyHostToDevice, s));
        st = run(buf, di, dd);
        if (!st) {
            PCK(ctx, cudaMemcpyAsync(out_ids, di, ib, cudaMemcpyDeviceToHost, s));
            PCK(ctx, cudaMemcpyAsync(out_dist2, dd, db, cudaMemcpyDeviceToHost, s));
            PCK(ctx, cudaStreamSynchronize(s));
        }
        dev_free(ctx, buf);
        return st;
    }
    return run(queries, out_ids, out_dist2);
}

extern "C" panther_status pantherpp_knn(panther_ctx* ctx, const pantherpp_vecs* v, const int32_t* queries, int64_t q,
                                        int k, int32_t* out_ids, uint64_t* out_dist2, int flags) {
    return knn_entry(ctx, v, v, true, queries, q, k, out_ids, out_dist2, flags);
}

extern "C" panther_status pantherpp_knn_cross(panther_ctx* ctx, const pantherpp_vecs* vq, const pantherpp_vecs* vc,
                                              const int32_t* queries, int64_t q, int k, int32_t* out_ids,
                                              uint64_t* out_dist2, int flags) {
    return knn_entry(ctx, vq, vc, false, queries, q, k, out_ids, out_dist2, flags);
}

extern "C" panther_status pantherpp_knn_stats(panther_ctx* ctx, int64_t stats[4]) {
    if (!ctx || !stats) return PANTHER_EINVAL;
    for (int i = 0; i < 4; ++i) stats[i] = ctx->knn_stats[i];
    return PANTHER_OK;
}

// Measurement of the BF16 screening error (no counterpart in the paper): the
// tensor-core screen of up to 128 queries against every candidate, keeping
// every screened value. out_y[i][p] = y_hat = |b|^2 - 2 a_hat.b_hat for query
// i and the candidate at position p (out_cid[p], -1 for padding); the exact
// value is |b|^2 - 2 a.b, so d_hat = |a|^2 + y_hat.
extern "C" panther_status pantherpp_debug_screen(panther_ctx* ctx, const pantherpp_vecs* v, const int32_t* queries,
                                                 int64_t q, float* out_y, int32_t* out_cid, int64_t* npad) {
    if (!ctx || !v || !npad) return PANTHER_EINVAL;
    *npad = v->npad;
    if (!out_y && !out_cid) return PANTHER_OK;
    if (!queries || !out_y || !out_cid || q < 1 || q > KN_M)
        return set_err(ctx, PANTHER_EINVAL, "1 <= q <= 128 queries and both outputs are needed");
    if (v->D > KN_K - 8) return set_err(ctx, PANTHER_EINVAL, "BF16 screening needs D <= 56");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    int32_t* ids = nullptr;
    uint64_t* d2 = nullptr;
    panther_status st;
    if ((st = dev_alloc(ctx, (void**)&ids, sizeof(int32_t) * q)) || (st = dev_alloc(ctx, (void**)&d2, 8 * q))) {
        dev_free(ctx, ids);
        return st;
    }
    PCK(ctx, cudaMemsetAsync(out_y, 0xff, sizeof(float) * q * v->npad, s));   // NaN where nothing is screened
    st = knn_run(ctx, v, v, true, queries, q, 1, ids, d2, false, out_y);
    if (!st) {
        cudaError_t e = cudaMemcpyAsync(out_cid, v->cid, sizeof(int32_t) * v->npad, cudaMemcpyDeviceToDevice, s);
        if (!e) e = cudaStreamSynchronize(s);
        if (e) st = cuda_err(ctx, e, "screen dump");
    }
    dev_free(ctx, ids);
    dev_free(ctx, d2);
    return st;
}
