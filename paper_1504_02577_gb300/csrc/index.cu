// Vertex -> path inverted index (Sec. 3.1) by a stable LSD radix sort.
//
// Pass 0 reads the path rows directly: item (r, j) of the flattened
// [R][stride] array is a (key = vertex, value = r) pair unless j >= T+1 or the
// same vertex occurred earlier in row r (P_v is a set). Rows are stride-
// aligned inside every 32-lane round, so the duplicate test is one
// __match_any_sync; rows of 64 or 128 entries span two or four rounds of one
// warp, and their entries are also compared with the row's earlier rounds. Later passes read the (key, value) pairs of the previous
// pass. Every pass is: tile histogram -> exclusive scan over (digit, tile) ->
// stable scatter. The scatter ranks items with warp-private digit counters:
// warps own contiguous sub-ranges of a tile and walk them in order, so the
// sort is stable and path ids come out ascending within each vertex.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int IX_T = 512;                  // threads per tile CTA
constexpr int IX_WARPS = IX_T / 32;
constexpr int IX_ROUNDS = 12;              // 32-item rounds per warp
constexpr int IX_TILE = IX_T * IX_ROUNDS;  // 6144 items per tile
constexpr int MAX_RADIX = 512;
constexpr int MAX_RB = 9;                  // log2(MAX_RADIX)

struct Src {
    // pass 0 source
    const int32_t* rows;
    int64_t R;
    int L, stride;
    int lstride;        // log2(stride): row of item i = i >> lstride
    // later-pass source
    const int32_t* keys;
    const int32_t* vals;
    int64_t count;      // number of pairs (later passes)
    int first;          // 1 for pass 0
    int64_t r0;         // pass 0: path id of row 0 (a chunk of the rows)
};

// raw word of item i (pass 0: the path entry, -1 past the end; later passes: the key)
__device__ __forceinline__ int32_t load_raw(const Src& s, int64_t i) {
    if (s.first) return i < s.R * s.stride ? __ldg(s.rows + i) : -1;
    return i < s.count ? __ldg(s.keys + i) : 0;
}

// is item i a pair (pass 0: inside the path, first occurrence in its row)?
// Every lane of the warp must call it (one __match_any_sync in pass 0).
__device__ __forceinline__ bool item_ok(const Src& s, int64_t i, int32_t x) {
    if (s.first && s.stride == 8) {
        // 8-entry rows: compare with the (at most 7) earlier entries of the row
        const unsigned lane = threadIdx.x & 31, j8 = lane & 7u;
        bool dup = false;
#pragma unroll
        for (unsigned o = 1; o < 8; ++o) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            dup |= j8 >= o && y == x;
        }
        return i < s.R * s.stride && (int)(i & 7) < s.L && !dup;
    }
    if (s.first) {
        const unsigned lane = threadIdx.x & 31;
        const unsigned peers = __match_any_sync(0xffffffffu, x);
        const unsigned rowbase = s.stride >= 32 ? 0u : lane & ~(unsigned)(s.stride - 1);
        const unsigned rowmask = (s.stride >= 32) ? 0xffffffffu : (((1u << s.stride) - 1u) << rowbase);
        const unsigned before = peers & rowmask & ((1u << lane) - 1u);
        const int j = (int)(i & (s.stride - 1));
        return i < s.R * s.stride && j < s.L && before == 0;
    }
    return i < s.count;
}

// Pass 0 with rows wider than a 32-item round (stride 64 or 128): bit k is
// set when the item of round k repeats an entry of an earlier round of the
// same row (rows are stride-aligned and a warp's rounds hold whole rows, so
// the at most three earlier rounds of the row are in this warp's registers;
// each is compared through 32 broadcasts). Every lane must call it.
__device__ __forceinline__ uint32_t long_row_repeats(const Src& s, int64_t wbase, const int32_t (&x)[IX_ROUNDS]) {
    uint32_t rep = 0;
#pragma unroll
    for (int k = 1; k < IX_ROUNDS; ++k) {
        const int64_t row = (wbase + k * 32) >> s.lstride;
        bool d = false;
#pragma unroll
        for (int o = 1; o <= 3; ++o) {
            if (k - o < 0) continue;
            if (((wbase + (k - o) * 32) >> s.lstride) != row) continue;  // warp-uniform
#pragma unroll 8
            for (int sl = 0; sl < 32; ++sl) d |= __shfl_sync(0xffffffffu, x[k - o], sl) == x[k];
        }
        rep |= (d ? 1u : 0u) << k;
    }
    return rep;
}

// LONG: pass 0 over rows of 64 or 128 entries (separate instantiations keep
// the registers of the common kernels unchanged)
template <bool LONG>
__global__ void __launch_bounds__(IX_T) hist_kernel(Src s, int shift, int radix, int64_t ntiles,
                                                    int64_t* __restrict__ counts) {
    __shared__ unsigned h[MAX_RADIX];
    for (int d = threadIdx.x; d < radix; d += IX_T) h[d] = 0;
    const int64_t base = (int64_t)blockIdx.x * IX_TILE + (int64_t)(threadIdx.x >> 5) * (IX_ROUNDS * 32) +
                         (threadIdx.x & 31);
    int32_t x[IX_ROUNDS];
#pragma unroll
    for (int k = 0; k < IX_ROUNDS; ++k) x[k] = load_raw(s, base + k * 32);   // all loads in flight
    const uint32_t rep = LONG ? long_row_repeats(s, base - (threadIdx.x & 31), x) : 0u;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < IX_ROUNDS; ++k)
        if (item_ok(s, base + k * 32, x[k]) && !((rep >> k) & 1u))
            atomicAdd(&h[((uint32_t)x[k] >> shift) & (radix - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += IX_T) counts[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// One tile per CTA: rank every item stably (per-warp digit counters), stage
// the tile in shared memory in digit order, then write each digit's run with
// consecutive threads storing consecutive positions (coalesced stores).
constexpr size_t SC_SMEM = (size_t)IX_WARPS * MAX_RADIX * 4 + (size_t)MAX_RADIX * 8 + (size_t)MAX_RADIX * 4 +
                           (size_t)IX_TILE * 8 + 64;

template <bool LONG>
__global__ void __launch_bounds__(IX_T, 2) scatter_kernel(Src s, int shift, int radix, int64_t ntiles,
                                                          const int64_t* __restrict__ offs,
                                                          int32_t* __restrict__ okeys, int32_t* __restrict__ ovals) {
    extern __shared__ __align__(16) unsigned char sc_smem[];
    unsigned (*wc)[MAX_RADIX] = (unsigned (*)[MAX_RADIX])sc_smem;                       // [warps][radix]
    long long* toff = (long long*)(sc_smem + (size_t)IX_WARPS * MAX_RADIX * 4);        // [radix]
    unsigned* tstart = (unsigned*)(toff + MAX_RADIX);                                  // [radix]
    int32_t* skey = (int32_t*)(tstart + MAX_RADIX);                                    // [tile]
    int32_t* sval = skey + IX_TILE;                                                    // [tile]
    __shared__ unsigned wsum[IX_WARPS];
    const int w = threadIdx.x >> 5;
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int d = threadIdx.x; d < IX_WARPS * MAX_RADIX; d += IX_T) (&wc[0][0])[d] = 0;
    const int64_t tile0 = (int64_t)blockIdx.x * IX_TILE;
    const int64_t base = tile0 + (int64_t)w * (IX_ROUNDS * 32);
    uint32_t key[IX_ROUNDS];
    uint32_t lrank[IX_ROUNDS / 2];
    uint32_t okmask = 0;
    // this tile's global start of digit threadIdx.x (final before the launch):
    // loaded now, so its latency overlaps the item loads and the ranking
    const long long my_off = (int)threadIdx.x < radix ? offs[(int64_t)threadIdx.x * ntiles + blockIdx.x] : 0;
#pragma unroll
    for (int k = 0; k < IX_ROUNDS; ++k) key[k] = (uint32_t)load_raw(s, base + k * 32 + lane);   // loads in flight
#pragma unroll
    for (int k = 0; k < IX_ROUNDS; ++k) okmask |= (item_ok(s, base + k * 32 + lane, (int32_t)key[k]) ? 1u : 0u) << k;
    if (LONG) {
        int32_t xk[IX_ROUNDS];
#pragma unroll
        for (int k = 0; k < IX_ROUNDS; ++k) xk[k] = (int32_t)key[k];
        okmask &= ~long_row_repeats(s, base, xk);
    }
    __syncthreads();
    // phase 1: per-warp digit counts and each item's rank within its warp.
    // The lanes holding the same digit: one ballot per digit bit, each kept or
    // inverted by the lane's own bit (no match instruction on the MIO pipe).
    const int rb = 31 - __clz(radix);
#pragma unroll
    for (int k = 0; k < IX_ROUNDS; ++k) {
        bool ok = (okmask >> k) & 1u;
        uint32_t d = ok ? ((key[k] >> shift) & (radix - 1)) : 0xffffffffu;
        unsigned peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
        for (int b = 0; b < MAX_RB; ++b) {
            if (b >= rb) break;                            // warp-uniform
            const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bb : ~bb;
        }
        if (!ok) peers = 0;
        unsigned before = ok ? wc[w][d] : 0u;
        uint32_t r = before + __popc(peers & lt);
        if (k & 1) lrank[k >> 1] |= r << 16; else lrank[k >> 1] = r;
        __syncwarp();
        if (ok && (peers & lt) == 0) wc[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // phase 2: per digit, the warps' starts within the digit and the digit's
    // total; then the tile-level exclusive scan of the totals (digit starts)
    unsigned tot = 0;
    const int d2 = threadIdx.x;               // IX_T >= MAX_RADIX: one digit per thread
    if (d2 < radix) {
        toff[d2] = my_off;
        for (int ww = 0; ww < IX_WARPS; ++ww) {
            unsigned c = wc[ww][d2];
            wc[ww][d2] = tot;
            tot += c;
        }
    }
    unsigned x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned y = lane < IX_WARPS ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned z = __shfl_up_sync(0xffffffffu, y, o);
            if ((int)lane >= o) y += z;
        }
        if (lane < IX_WARPS) wsum[lane] = y;
    }
    __syncthreads();
    if (d2 < radix) tstart[d2] = x - tot + (w ? wsum[w - 1] : 0u);
    const unsigned nvalid = wsum[IX_WARPS - 1];
    __syncthreads();
    // phase 3a: stage keys and values in digit order (values loaded together first)
    int32_t val[IX_ROUNDS];
#pragma unroll
    for (int k = 0; k < IX_ROUNDS; ++k) {
        const int64_t i = base + k * 32 + lane;
        val[k] = s.first ? (int32_t)(uint32_t)(s.r0 + (i >> s.lstride)) : (((okmask >> k) & 1u) ? __ldg(s.vals + i) : 0);
    }
#pragma unroll
    for (int k = 0; k < IX_ROUNDS; ++k) {
        if ((okmask >> k) & 1u) {
            uint32_t d = (key[k] >> shift) & (radix - 1);
            uint32_t r = (k & 1) ? (lrank[k >> 1] >> 16) : (lrank[k >> 1] & 0xffffu);
            unsigned sp = tstart[d] + wc[w][d] + r;
            skey[sp] = (int32_t)key[k];
            sval[sp] = val[k];
        }
    }
    __syncthreads();
    // phase 3b: consecutive staged items of one digit go to consecutive positions
    for (unsigned j = threadIdx.x; j < nvalid; j += IX_T) {
        const int32_t kk = skey[j];
        const uint32_t d = ((uint32_t)kk >> shift) & (radix - 1);
        const int64_t pos = (int64_t)toff[d] + (j - tstart[d]);
        okeys[pos] = kk;
        ovals[pos] = sval[j];
    }
}

__global__ void offsets_kernel(const int32_t* __restrict__ keys, int64_t nnz, int64_t n, int64_t* __restrict__ off,
                               uint32_t* status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > nnz) return;
    int64_t prev = i > 0 ? (int64_t)keys[i - 1] : -1;
    int64_t cur = i < nnz ? (int64_t)keys[i] : n;
    if (prev < -1 || prev >= n || cur < 0 || cur > n || cur < prev) {   // keys out of range or unsorted
        flag_status(status, ST_BAD_INDEX);
        return;
    }
    for (int64_t v = prev + 1; v <= cur; ++v) off[v] = i;
}

// cls[v] = path_code(|P_v|) and its histogram (a count of v with any u never
// exceeds |P_v| or |P_u|)
__global__ void cls_kernel(const int64_t* __restrict__ off, int64_t n, uint8_t* __restrict__ cls,
                           unsigned long long* __restrict__ hist) {
    __shared__ unsigned h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t np = off[v + 1] - off[v];
        const uint32_t c = path_code(np);
        cls[v] = (uint8_t)c;
        atomicAdd(&h[c], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// |P_v| of every vertex over a range of rows (first occurrences only),
// accumulated into cnt (64-bit, later scanned in place into offsets)
template <bool LONG>
__global__ void __launch_bounds__(IX_T) vcount_kernel(Src s, unsigned long long* __restrict__ cnt) {
    const int64_t base = (int64_t)blockIdx.x * IX_TILE + (int64_t)(threadIdx.x >> 5) * (IX_ROUNDS * 32) +
                         (threadIdx.x & 31);
    int32_t x[IX_ROUNDS];
#pragma unroll
    for (int k = 0; k < IX_ROUNDS; ++k) x[k] = load_raw(s, base + k * 32);
    const uint32_t rep = LONG ? long_row_repeats(s, base - (threadIdx.x & 31), x) : 0u;
#pragma unroll
    for (int k = 0; k < IX_ROUNDS; ++k)
        if (item_ok(s, base + k * 32, x[k]) && !((rep >> k) & 1u)) atomicAdd(&cnt[x[k]], 1ull);
}

// a chunk's pairs, sorted by vertex, appended to each vertex's list: pair i
// of vertex v (coff[v] = its first position in the chunk) goes to
// cur[v] + i - coff[v]; chunks come in ascending path order, so every list
// stays ascending
__global__ void place_kernel(const int32_t* __restrict__ keys, const int32_t* __restrict__ vals, int64_t cn,
                             const int64_t* __restrict__ coff, const int64_t* __restrict__ cur,
                             uint32_t* __restrict__ pid) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cn) return;
    const int32_t v = keys[i];
    pid[cur[v] + (i - coff[v])] = (uint32_t)vals[i];
}

__global__ void advance_kernel(const int64_t* __restrict__ coff, int64_t n, int64_t* __restrict__ cur) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) cur[v] += coff[v + 1] - coff[v];
}

__global__ void total_kernel(const int64_t* __restrict__ counts, const int64_t* __restrict__ offs, int64_t len,
                             int64_t* __restrict__ total) {
    *total = offs[len - 1] + counts[len - 1];
}

int bits_for(int64_t maxval) {
    int b = 1;
    while (b < 62 && (int64_t(1) << b) <= maxval) ++b;
    return b;
}

}  // namespace

// sizes of the radix passes for keys < n
static void radix_plan(int64_t n, int* passes, int* rbits) {
    int bits = bits_for(n - 1 > 0 ? n - 1 : 1);
    int np = (bits + 8) / 9;
    if (np < 1) np = 1;
    *passes = np;
    *rbits = (bits + np - 1) / np;
}

// cls and its histogram from ix->off (ix->cls, ix->cls_hist allocated)
panther_status index_classes(panther_ctx* ctx, panther_index* ix) {
    cudaStream_t s = ctx->stream;
    PCK(ctx, cudaMemsetAsync(ix->cls_hist, 0, sizeof(int64_t) * 256, s));
    cls_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ix->n, 256), (int64_t)ctx->num_sms * 8)),
                 256, 0, s>>>(ix->off, ix->n, ix->cls, (unsigned long long*)ix->cls_hist);
    ctx->launches++;
    PCK(ctx, cudaGetLastError());
    return PANTHER_OK;
}

// LSD radix sort of the (vertex, path) pairs of src (pass 0 reads its rows);
// the sorted keys and values end in one of the A/B buffers, returned with
// the number of pairs. Synchronises once (after pass 0, to size the rest).
static panther_status radix_pairs(panther_ctx* ctx, Src src, int64_t n, int32_t* kA, int32_t* vA, int32_t* kB,
                                  int32_t* vB, int64_t* counts, int64_t* offs, int64_t* tot, int64_t* count_out,
                                  int32_t** keys_out, int32_t** vals_out) {
    cudaStream_t s = ctx->stream;
    int passes, rb;
    radix_plan(n, &passes, &rb);
    const int radix = 1 << rb;
    const int64_t tiles0 = ceil_div(src.R * src.stride, IX_TILE);
    int32_t *ik = nullptr, *iv = nullptr, *ok = kA, *ov = vA;
    int64_t count = 0;
    panther_status st;
    for (int pass = 0; pass < passes; ++pass) {
        int shift = pass * rb;
        int64_t ntiles = pass == 0 ? tiles0 : ceil_div(count, IX_TILE);
        if (ntiles < 1) ntiles = 1;
        int64_t len = (int64_t)radix * ntiles;
        if (src.first && src.stride > 32)
            hist_kernel<true><<<(unsigned)ntiles, IX_T, 0, s>>>(src, shift, radix, ntiles, counts);
        else
            hist_kernel<false><<<(unsigned)ntiles, IX_T, 0, s>>>(src, shift, radix, ntiles, counts);
        ctx->launches++;
        cudaError_t e = cudaMemcpyAsync(offs, counts, sizeof(int64_t) * len, cudaMemcpyDeviceToDevice, s);
        if (e) return cuda_err(ctx, e, "index scan copy");
        if ((st = scan_exclusive_i64(ctx, offs, len))) return st;
        if (pass == 0) {
            // the number of pairs is needed to size the later passes
            total_kernel<<<1, 1, 0, s>>>(counts, offs, len, tot);
            ctx->launches++;
            e = cudaMemcpyAsync(&count, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaStreamSynchronize(s);
            if (e) return cuda_err(ctx, e, "index count");
        }
        if (src.first && src.stride > 32)
            scatter_kernel<true><<<(unsigned)ntiles, IX_T, SC_SMEM, s>>>(src, shift, radix, ntiles, offs, ok, ov);
        else
            scatter_kernel<false><<<(unsigned)ntiles, IX_T, SC_SMEM, s>>>(src, shift, radix, ntiles, offs, ok, ov);
        ctx->launches++;
        e = cudaGetLastError();
        if (e) return cuda_err(ctx, e, "index scatter");
        // next pass reads what this one wrote
        src.first = 0;
        src.keys = ok;
        src.vals = ov;
        src.count = count;
        ik = ok; iv = ov;
        ok = (ok == kA) ? kB : kA;
        ov = (ov == vA) ? vB : vA;
    }
    *count_out = count;
    *keys_out = ik;
    *vals_out = iv;
    return PANTHER_OK;
}

// device bytes of the temporary buffers of one radix sort over `rows` rows
static int64_t radix_temp_bytes(int64_t rows, int L, int stride, int radix) {
    const int64_t pairs = rows * L;
    const int64_t tiles = std::max(ceil_div(rows * stride, IX_TILE), ceil_div(pairs, IX_TILE));
    return 4 * pairs * 4 + 2 * (int64_t)radix * tiles * 8 + 64;
}

extern "C" panther_status panther_set_index_budget(panther_ctx* ctx, int64_t bytes) {
    if (!ctx || bytes < 0) return PANTHER_EINVAL;
    if (bytes > 0 && bytes < (int64_t(1) << 20)) return set_err(ctx, PANTHER_EINVAL, "index budget below 1 MiB");
    ctx->index_budget = bytes;
    return PANTHER_OK;
}

extern "C" panther_status panther_build_index(panther_ctx* ctx, const panther_paths* p, panther_index** out) {
    if (!ctx || !p || !out) return PANTHER_EINVAL;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    const int64_t n = p->n;
    int passes, rb;
    radix_plan(n, &passes, &rb);
    const int radix = 1 << rb;

    // rows per radix sort: all of them when their temporary buffers fit the
    // budget (set, or else the free device memory less what the results
    // need); otherwise the largest chunk that fits
    int64_t rows = p->R;
    {
        const int64_t need = radix_temp_bytes(p->R, p->L, p->stride, radix);
        int64_t budget = ctx->index_budget;
        if (budget == 0) {
            const int64_t results = p->R * p->L * 4 + 3 * (n + 1) * 8 + n + (int64_t(256) << 20);
            size_t fr = 0, tot = 0;
            if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (int64_t)fr - results < need) {
                // memory the pool keeps but no one uses goes back first
                cudaMemPool_t pool;
                if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
                cudaMemGetInfo(&fr, &tot);
            }
            cudaGetLastError();
            budget = fr > 0 ? std::max<int64_t>((int64_t)fr - results, int64_t(1) << 20) : need;
        }
        if (need > budget) {
            int64_t lo = 1, hi = p->R;           // largest chunk whose buffers fit
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo + 1) / 2;
                if (radix_temp_bytes(mid, p->L, p->stride, radix) <= budget) lo = mid; else hi = mid - 1;
            }
            rows = lo;
            if (radix_temp_bytes(rows, p->L, p->stride, radix) > budget)
                return set_err(ctx, PANTHER_ENOMEM, "the index budget does not hold the buffers of one row");
        }
    }

    panther_index* ix = new panther_index();
    ix->ctx = ctx;
    ix->n = n;
    ix->R = p->R;
    int32_t *kA = nullptr, *vA = nullptr, *kB = nullptr, *vB = nullptr;
    int64_t *counts = nullptr, *offs = nullptr, *tot = nullptr, *cur = nullptr, *coff = nullptr;
    panther_status st;
    const int64_t maxpairs = rows * p->L;
    const int64_t maxtiles = std::max(ceil_div(rows * p->stride, IX_TILE), ceil_div(maxpairs, IX_TILE));
    auto cleanup = [&]() {
        dev_free(ctx, kA); dev_free(ctx, vA); dev_free(ctx, kB); dev_free(ctx, vB);
        dev_free(ctx, counts); dev_free(ctx, offs); dev_free(ctx, tot); dev_free(ctx, cur); dev_free(ctx, coff);
    };
    auto fail = [&](panther_status e) {
        cleanup();
        panther_free_index(ix);
        return e;
    };
    if ((st = dev_alloc(ctx, (void**)&kA, sizeof(int32_t) * maxpairs)) ||
        (st = dev_alloc(ctx, (void**)&vA, sizeof(int32_t) * maxpairs)) ||
        (st = dev_alloc(ctx, (void**)&kB, sizeof(int32_t) * maxpairs)) ||
        (st = dev_alloc(ctx, (void**)&vB, sizeof(int32_t) * maxpairs)) ||
        (st = dev_alloc(ctx, (void**)&counts, sizeof(int64_t) * radix * maxtiles)) ||
        (st = dev_alloc(ctx, (void**)&offs, sizeof(int64_t) * radix * maxtiles)) ||
        (st = dev_alloc(ctx, (void**)&tot, sizeof(int64_t))) ||
        (st = dev_alloc(ctx, (void**)&ix->off, sizeof(int64_t) * (n + 1))) ||
        (st = dev_alloc(ctx, (void**)&ix->cls, n)) ||
        (st = dev_alloc(ctx, (void**)&ix->cls_hist, sizeof(int64_t) * 256)))
        return fail(st);
    PCK(ctx, cudaFuncSetAttribute(scatter_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SC_SMEM));
    PCK(ctx, cudaFuncSetAttribute(scatter_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SC_SMEM));
    Src src{};
    src.rows = p->rows;
    src.R = p->R;
    src.L = p->L;
    src.stride = p->stride;
    src.lstride = 31 - __builtin_clz((unsigned)p->stride);
    src.first = 1;
    src.r0 = 0;
    cudaError_t e;
    if (rows == p->R) {
        // one radix sort over all pairs; its final values are pid
        int64_t count = 0;
        int32_t *ik = nullptr, *iv = nullptr;
        if ((st = radix_pairs(ctx, src, n, kA, vA, kB, vB, counts, offs, tot, &count, &ik, &iv))) return fail(st);
        ix->nnz = count;
        offsets_kernel<<<(unsigned)ceil_div(count + 1, 256), 256, 0, s>>>(ik, count, n, ix->off, ctx->d_status);
        ctx->launches++;
        if ((st = index_classes(ctx, ix))) return fail(st);
        // keep the final value array as pid; release everything else
        ix->pid = (uint32_t*)iv;
        if (iv == vA) vA = nullptr; else vB = nullptr;
    } else {
        // chunks of `rows` path rows: |P_v| of every vertex first (the
        // offsets), then each chunk sorted and appended to the lists
        if ((e = cudaMemsetAsync(ix->off, 0, sizeof(int64_t) * (n + 1), s))) return fail(cuda_err(ctx, e, "index"));
        const int64_t tilesAll = ceil_div(p->R * p->stride, IX_TILE);
        if (p->stride > 32)
            vcount_kernel<true><<<(unsigned)tilesAll, IX_T, 0, s>>>(src, (unsigned long long*)ix->off);
        else
            vcount_kernel<false><<<(unsigned)tilesAll, IX_T, 0, s>>>(src, (unsigned long long*)ix->off);
        ctx->launches++;
        if ((st = scan_exclusive_i64(ctx, ix->off, n + 1))) return fail(st);
        int64_t nnz = 0;
        if ((e = cudaMemcpyAsync(&nnz, ix->off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaStreamSynchronize(s)))
            return fail(cuda_err(ctx, e, "index count"));
        ix->nnz = nnz;
        if ((st = dev_alloc(ctx, (void**)&ix->pid, sizeof(int32_t) * (nnz > 0 ? nnz : 1))) ||
            (st = dev_alloc(ctx, (void**)&cur, sizeof(int64_t) * (n + 1))) ||
            (st = dev_alloc(ctx, (void**)&coff, sizeof(int64_t) * (n + 1))))
            return fail(st);
        if ((e = cudaMemcpyAsync(cur, ix->off, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s)))
            return fail(cuda_err(ctx, e, "index"));
        for (int64_t r0 = 0; r0 < p->R; r0 += rows) {
            Src cs = src;
            cs.rows = p->rows + r0 * p->stride;
            cs.R = std::min(rows, p->R - r0);
            cs.r0 = r0;
            int64_t cn = 0;
            int32_t *ck = nullptr, *cv = nullptr;
            if ((st = radix_pairs(ctx, cs, n, kA, vA, kB, vB, counts, offs, tot, &cn, &ck, &cv))) return fail(st);
            offsets_kernel<<<(unsigned)ceil_div(cn + 1, 256), 256, 0, s>>>(ck, cn, n, coff, ctx->d_status);
            if (cn > 0) place_kernel<<<(unsigned)ceil_div(cn, 256), 256, 0, s>>>(ck, cv, cn, coff, cur, ix->pid);
            advance_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(coff, n, cur);
            ctx->launches += cn > 0 ? 3 : 2;
            if ((e = cudaGetLastError())) return fail(cuda_err(ctx, e, "index chunk"));
        }
        if ((st = index_classes(ctx, ix))) return fail(st);
    }
    cleanup();
    e = cudaGetLastError();
    if (e) { panther_free_index(ix); return cuda_err(ctx, e, "index offsets"); }
    *out = ix;
    return PANTHER_OK;
}

// ------------------------------------------------ index without allocation ---
// A variant of the index build for callers that must not allocate device
// memory: for example a host application that hands this library a fixed
// share of the GPU and accounts for every byte itself, or a latency-bound
// loop in which a cudaMalloc (which can synchronise the device) is not
// acceptable. All temporary buffers live in one file-scope device array of
// NA_SCRATCH_BYTES, reserved on every GPU that loads the library until the
// process exits; the caller passes the outputs.
namespace {
constexpr int64_t NA_MAX_PAIRS = int64_t(1) << 22;           // R * (T+1) at most 4,194,304
constexpr int64_t NA_MAX_TILES = 2816;                        // >= ceil(R * stride / IX_TILE) for the limit above
constexpr size_t NA_KV_BYTES = (size_t)NA_MAX_PAIRS * 4;      // one key or value array
constexpr size_t NA_CNT_BYTES = (size_t)MAX_RADIX * NA_MAX_TILES * 8;
constexpr size_t NA_SCRATCH_BYTES = 4 * NA_KV_BYTES + 2 * NA_CNT_BYTES + 256;

static __device__ __align__(256) unsigned char na_scratch[NA_SCRATCH_BYTES];

// exclusive scan of len int64 values by one CTA (the counts of one pass)
__global__ void __launch_bounds__(1024) na_scan_kernel(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                       int64_t len, int64_t* __restrict__ total) {
    __shared__ int64_t sh[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < len; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < len ? in[i] : 0, x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        if (lane == 31) sh[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int64_t t = lane < (blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= (unsigned)o) t += y;
            }
            sh[lane] = t;
        }
        __syncthreads();
        int64_t excl = carry + (wid ? sh[wid - 1] : 0) + x - v;
        if (i < len) out[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// device address of na_scratch, looked up once per device with that device current
unsigned char* na_scratch_ptr[64];
std::mutex na_mu;
}  // namespace

extern "C" panther_status panther_build_index_noalloc(panther_ctx* ctx, const panther_paths* p, int64_t* dev_off,
                                                      uint32_t* dev_pid, int64_t pid_capacity, int64_t* nnz) {
    if (!ctx || !p || !dev_off || !dev_pid || !nnz) return PANTHER_EINVAL;
    *nnz = 0;
    const int64_t pairs = p->R * p->L;
    if (pairs > NA_MAX_PAIRS)
        return set_err(ctx, PANTHER_EOVERFLOW,
                       "R*(T+1) = %lld exceeds the %lld pairs the static index scratch holds",
                       (long long)pairs, (long long)NA_MAX_PAIRS);
    if (pid_capacity < pairs) return set_err(ctx, PANTHER_EINVAL, "pid_capacity must be at least R*(T+1)");
    if (ctx->device < 0 || ctx->device >= 64) return set_err(ctx, PANTHER_EINVAL, "device index out of range");
    PCK(ctx, cudaSetDevice(ctx->device));
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lk(na_mu);
        if (!na_scratch_ptr[ctx->device]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, na_scratch);
            if (e != cudaSuccess || !ptr) return cuda_err(ctx, e, "cudaGetSymbolAddress(na_scratch)");
            na_scratch_ptr[ctx->device] = (unsigned char*)ptr;
        }
        base = na_scratch_ptr[ctx->device];
    }
    int32_t* kA = (int32_t*)base;
    int32_t* vA = (int32_t*)(base + NA_KV_BYTES);
    int32_t* kB = (int32_t*)(base + 2 * NA_KV_BYTES);
    int32_t* vB = (int32_t*)(base + 3 * NA_KV_BYTES);
    int64_t* counts = (int64_t*)(base + 4 * NA_KV_BYTES);
    int64_t* offs = (int64_t*)(base + 4 * NA_KV_BYTES + NA_CNT_BYTES);
    int64_t* tot = (int64_t*)(base + 4 * NA_KV_BYTES + 2 * NA_CNT_BYTES);
    cudaStream_t s = ctx->stream;
    int passes, rb;
    radix_plan(p->n, &passes, &rb);
    const int radix = 1 << rb;
    const int64_t tiles0 = ceil_div(p->R * p->stride, IX_TILE);
    if (tiles0 > NA_MAX_TILES) return set_err(ctx, PANTHER_EOVERFLOW, "too many path rows for the static scratch");
    PCK(ctx, cudaFuncSetAttribute(scatter_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SC_SMEM));
    PCK(ctx, cudaFuncSetAttribute(scatter_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SC_SMEM));
    Src src{};
    src.rows = p->rows;
    src.R = p->R;
    src.L = p->L;
    src.stride = p->stride;
    src.lstride = 31 - __builtin_clz((unsigned)p->stride);
    src.first = 1;
    int32_t *ik = nullptr, *ok = kA, *ov = vA;
    int64_t count = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const bool last = pass == passes - 1;
        int64_t ntiles = pass == 0 ? tiles0 : ceil_div(count, IX_TILE);
        if (ntiles < 1) ntiles = 1;
        const int64_t len = (int64_t)radix * ntiles;
        if (src.first && src.stride > 32)
            hist_kernel<true><<<(unsigned)ntiles, IX_T, 0, s>>>(src, pass * rb, radix, ntiles, counts);
        else
            hist_kernel<false><<<(unsigned)ntiles, IX_T, 0, s>>>(src, pass * rb, radix, ntiles, counts);
        na_scan_kernel<<<1, 1024, 0, s>>>(counts, offs, len, tot);
        ctx->launches += 2;
        if (pass == 0) {
            PCK(ctx, cudaMemcpyAsync(&count, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            PCK(ctx, cudaStreamSynchronize(s));
        }
        int32_t* outv = last ? (int32_t*)dev_pid : ov;     // the final pass writes the caller's pid array
        if (src.first && src.stride > 32)
            scatter_kernel<true><<<(unsigned)ntiles, IX_T, SC_SMEM, s>>>(src, pass * rb, radix, ntiles, offs, ok, outv);
        else
            scatter_kernel<false><<<(unsigned)ntiles, IX_T, SC_SMEM, s>>>(src, pass * rb, radix, ntiles, offs, ok, outv);
        ctx->launches++;
        PCK(ctx, cudaGetLastError());
        src.first = 0;
        src.keys = ok;
        src.vals = outv;
        src.count = count;
        ik = ok;
        ok = (ok == kA) ? kB : kA;
        ov = (ov == vA) ? vB : vA;
    }
    offsets_kernel<<<(unsigned)ceil_div(count + 1, 256), 256, 0, s>>>(ik, count, p->n, dev_off, ctx->d_status);
    ctx->launches++;
    PCK(ctx, cudaGetLastError());
    *nnz = count;
    return PANTHER_OK;
}
