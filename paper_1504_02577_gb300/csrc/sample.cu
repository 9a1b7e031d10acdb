// Random path sampling (Algorithm 3).
//
// One thread walks one path at a time (grid-stride over path ids). Each step
// is a dependent chain: the 16-byte vertex record (start, deg, S), then either
// a binary search over the prefix table ending in a short unrolled scan whose
// final sector also carries the neighbour id, or a single 16-byte alias entry
// that already carries both candidate neighbour ids. The row is kept in
// registers and stored as 32-byte vectors (stride 8/16/32 int32).
#include "internal.cuh"

namespace {

// smallest j in [0,deg) with cum[j] > x; returns the neighbour stored there
__device__ __forceinline__ uint32_t pick_prefix32(const uint2* __restrict__ e, uint32_t deg, uint32_t x) {
    uint32_t lo = 0, hi = deg - 1;
    while (hi - lo > 7) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&e[mid].x) > x) hi = mid; else lo = mid + 1;
    }
    uint2 c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = (lo + k <= hi) ? __ldg(&e[lo + k]) : make_uint2(0xffffffffu, 0u);
    uint32_t v = c[7].y;
#pragma unroll
    for (int k = 7; k >= 0; --k)
        if (lo + k <= hi && c[k].x > x) v = c[k].y;
    return v;
}

__device__ __forceinline__ uint32_t pick_prefix64(const uint4* __restrict__ e, uint32_t deg, uint64_t x) {
    uint32_t lo = 0, hi = deg - 1;
    while (hi - lo > 3) {
        uint32_t mid = (lo + hi) >> 1;
        uint4 t = __ldg(&e[mid]);
        uint64_t cm = (uint64_t)t.x | ((uint64_t)t.y << 32);
        if (cm > x) hi = mid; else lo = mid + 1;
    }
    uint4 c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = (lo + k <= hi) ? __ldg(&e[lo + k]) : make_uint4(0xffffffffu, 0xffffffffu, 0, 0);
    uint32_t v = c[3].z;
#pragma unroll
    for (int k = 3; k >= 0; --k) {
        uint64_t cm = (uint64_t)c[k].x | ((uint64_t)c[k].y << 32);
        if (lo + k <= hi && cm > x) v = c[k].z;
    }
    return v;
}

// MODE 1 = prefix, 2 = alias, 4 = unweighted (tab = the column array)
template <int MODE, bool WIDE, int STRIDE>
__global__ void __launch_bounds__(256, 5) sample_kernel(const uint4* __restrict__ vrec, const void* __restrict__ tab,
                                                     int64_t n, uint64_t seed, int64_t r0, int64_t R, int T,
                                                     int32_t* __restrict__ rows, uint32_t* status) {
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += nthreads) {
        int32_t p[STRIDE];
        uint64_t v = 0;
        for (uint32_t att = 0;; ++att) {
            pword4 x = path_draw(seed, (uint64_t)(r0 + r), 0, att);
            if (lemire64((uint64_t)x.x | ((uint64_t)x.y << 32), (uint64_t)n, &v)) break;
        }
        p[0] = (int32_t)v;
#pragma unroll
        for (int t = 1; t < STRIDE; ++t) {
            if (t <= T) {
                uint4 rec = __ldg(&vrec[v]);
                if (rec.y != 0) {
                    uint64_t S = (uint64_t)rec.z | ((uint64_t)rec.w << 32);
                    if (MODE == 4) {
                        // t_ij = 1/deg: Uniform[0, deg) from the same words as
                        // the prefix draw, so the walk equals prefix selection
                        // with every weight 1
                        uint64_t c = 0;
                        for (uint32_t att = 0;; ++att) {
                            pword4 w = path_draw(seed, (uint64_t)(r0 + r), (uint32_t)t, att);
                            if (lemire64((uint64_t)w.x | ((uint64_t)w.y << 32), (uint64_t)rec.y, &c)) break;
                        }
                        v = (uint64_t)(uint32_t)__ldg((const int32_t*)tab + rec.x + c);
                    } else if (MODE == 1) {
                        uint64_t x = 0;
                        for (uint32_t att = 0;; ++att) {
                            pword4 w = path_draw(seed, (uint64_t)(r0 + r), (uint32_t)t, att);
                            if (lemire64((uint64_t)w.x | ((uint64_t)w.y << 32), S, &x)) break;
                        }
                        if (WIDE)
                            v = pick_prefix64((const uint4*)tab + rec.x, rec.y, x);
                        else
                            v = pick_prefix32((const uint2*)tab + rec.x, rec.y, (uint32_t)x);
                    } else {
                        uint64_t c = 0, u = 0;
                        for (uint32_t att = 0;; ++att) {
                            pword4 w = path_draw(seed, (uint64_t)(r0 + r), (uint32_t)t, att);
                            bool ok0 = lemire64((uint64_t)w.x | ((uint64_t)w.y << 32), (uint64_t)rec.y, &c);
                            bool ok1 = lemire64((uint64_t)w.z | ((uint64_t)w.w << 32), S, &u);
                            if (ok0 && ok1) break;
                        }
                        uint4 e = __ldg((const uint4*)tab + rec.x + c);
                        uint64_t thr = (uint64_t)e.x | ((uint64_t)e.y << 32);
                        v = u < thr ? e.z : e.w;
                    }
                    if (v >= (uint64_t)n) {   // a corrupt table entry: report, never index with it
                        flag_status(status, ST_BAD_INDEX);
                        v = 0;
                    }
                }
                p[t] = (int32_t)v;
            } else {
                p[t] = -1;
            }
        }
        int4* dst = (int4*)(rows + r * STRIDE);
#pragma unroll
        for (int k = 0; k < STRIDE / 4; ++k) dst[k] = make_int4(p[4 * k], p[4 * k + 1], p[4 * k + 2], p[4 * k + 3]);
    }
}

// Rows of 64 or 128 entries (T >= 32): the same walk, but the row is not
// held in registers; every 8 entries go out as two 16-byte stores.
template <int MODE, bool WIDE>
__global__ void __launch_bounds__(256) sample_long_kernel(const uint4* __restrict__ vrec, const void* __restrict__ tab,
                                                          int64_t n, uint64_t seed, int64_t r0, int64_t R, int T,
                                                          int stride, int32_t* __restrict__ rows, uint32_t* status) {
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += nthreads) {
        int32_t buf[8];
        int4* dst = (int4*)(rows + r * stride);
        uint64_t v = 0;
        for (uint32_t att = 0;; ++att) {
            pword4 x = path_draw(seed, (uint64_t)(r0 + r), 0, att);
            if (lemire64((uint64_t)x.x | ((uint64_t)x.y << 32), (uint64_t)n, &v)) break;
        }
        buf[0] = (int32_t)v;
        for (int t8 = 0; t8 < stride; t8 += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = t8 + u;
                if (t == 0) continue;
                if (t > T) {
                    buf[u] = -1;
                    continue;
                }
                const uint4 rec = __ldg(&vrec[v]);
                if (rec.y != 0) {
                    const uint64_t S = (uint64_t)rec.z | ((uint64_t)rec.w << 32);
                    if (MODE == 4) {
                        uint64_t c = 0;
                        for (uint32_t att = 0;; ++att) {
                            pword4 w = path_draw(seed, (uint64_t)(r0 + r), (uint32_t)t, att);
                            if (lemire64((uint64_t)w.x | ((uint64_t)w.y << 32), (uint64_t)rec.y, &c)) break;
                        }
                        v = (uint64_t)(uint32_t)__ldg((const int32_t*)tab + rec.x + c);
                    } else if (MODE == 1) {
                        uint64_t x = 0;
                        for (uint32_t att = 0;; ++att) {
                            pword4 w = path_draw(seed, (uint64_t)(r0 + r), (uint32_t)t, att);
                            if (lemire64((uint64_t)w.x | ((uint64_t)w.y << 32), S, &x)) break;
                        }
                        if (WIDE)
                            v = pick_prefix64((const uint4*)tab + rec.x, rec.y, x);
                        else
                            v = pick_prefix32((const uint2*)tab + rec.x, rec.y, (uint32_t)x);
                    } else {
                        uint64_t c = 0, uu = 0;
                        for (uint32_t att = 0;; ++att) {
                            pword4 w = path_draw(seed, (uint64_t)(r0 + r), (uint32_t)t, att);
                            bool ok0 = lemire64((uint64_t)w.x | ((uint64_t)w.y << 32), (uint64_t)rec.y, &c);
                            bool ok1 = lemire64((uint64_t)w.z | ((uint64_t)w.w << 32), S, &uu);
                            if (ok0 && ok1) break;
                        }
                        const uint4 e = __ldg((const uint4*)tab + rec.x + c);
                        const uint64_t thr = (uint64_t)e.x | ((uint64_t)e.y << 32);
                        v = uu < thr ? e.z : e.w;
                    }
                    if (v >= (uint64_t)n) {
                        flag_status(status, ST_BAD_INDEX);
                        v = 0;
                    }
                }
                buf[u] = (int32_t)v;
            }
            dst[t8 / 4] = make_int4(buf[0], buf[1], buf[2], buf[3]);
            dst[t8 / 4 + 1] = make_int4(buf[4], buf[5], buf[6], buf[7]);
        }
    }
}

template <int MODE, bool WIDE>
void launch_sample(panther_ctx* ctx, const panther_graph* g, const void* tab, uint64_t seed, int64_t r0, int64_t R,
                   int T, int stride, int32_t* rows, unsigned blocks) {
    cudaStream_t s = ctx->stream;
    if (stride == 8)
        sample_kernel<MODE, WIDE, 8><<<blocks, 256, 0, s>>>(g->vrec, tab, g->n, seed, r0, R, T, rows, ctx->d_status);
    else if (stride == 16)
        sample_kernel<MODE, WIDE, 16><<<blocks, 256, 0, s>>>(g->vrec, tab, g->n, seed, r0, R, T, rows, ctx->d_status);
    else if (stride == 32)
        sample_kernel<MODE, WIDE, 32><<<blocks, 256, 0, s>>>(g->vrec, tab, g->n, seed, r0, R, T, rows, ctx->d_status);
    else
        sample_long_kernel<MODE, WIDE><<<blocks, 256, 0, s>>>(g->vrec, tab, g->n, seed, r0, R, T, stride, rows,
                                                              ctx->d_status);
}

}  // namespace

extern "C" panther_status panther_sample_paths_range(panther_ctx* ctx, const panther_graph* g, uint64_t seed,
                                                     int64_t r0, int64_t R, int T, int mode, panther_paths** out) {
    if (!ctx || !g || !out) return PANTHER_EINVAL;
    *out = nullptr;
    if (R < 1) return set_err(ctx, PANTHER_EINVAL, "R must be at least 1");
    if (R > 0xffffffffLL) return set_err(ctx, PANTHER_EOVERFLOW, "R exceeds the 32-bit path ids (at most 2^32-1 paths)");
    if (r0 < 0 || r0 > INT64_MAX - R) return set_err(ctx, PANTHER_EINVAL, "r0 must be >= 0 and r0 + R < 2^63");
    if (T < 1 || T > MAX_T) return set_err(ctx, PANTHER_EINVAL, "T must be in [1, 127]");
    if (mode != PANTHER_MODE_PREFIX && mode != PANTHER_MODE_ALIAS && mode != PANTHER_MODE_UNWEIGHTED)
        return set_err(ctx, PANTHER_EINVAL, "mode must be PREFIX, ALIAS or UNWEIGHTED");
    if (!(g->modes & mode)) return set_err(ctx, PANTHER_EINVAL, "the graph has no table for this mode");
    cudaSetDevice(ctx->device);
    panther_paths* p = new panther_paths();
    p->ctx = ctx;
    p->n = g->n;
    p->R = R;
    p->T = T;
    p->L = T + 1;
    p->stride = path_stride(p->L);
    p->mode = mode;
    p->seed = seed;
    p->r0 = r0;
    panther_status st = dev_alloc(ctx, (void**)&p->rows, sizeof(int32_t) * (size_t)R * p->stride);
    if (st) {
        delete p;
        return st;
    }
    int64_t want = ceil_div(R, 256);
    int64_t cap = (int64_t)ctx->num_sms * 8;
    unsigned blocks = (unsigned)(want < cap ? want : cap);
    if (mode == PANTHER_MODE_PREFIX) {
        if (g->prefix_wide)
            launch_sample<1, true>(ctx, g, g->prefix, seed, r0, R, T, p->stride, p->rows, blocks);
        else
            launch_sample<1, false>(ctx, g, g->prefix, seed, r0, R, T, p->stride, p->rows, blocks);
    } else if (mode == PANTHER_MODE_ALIAS) {
        launch_sample<2, false>(ctx, g, g->alias, seed, r0, R, T, p->stride, p->rows, blocks);
    } else {
        launch_sample<4, false>(ctx, g, g->col, seed, r0, R, T, p->stride, p->rows, blocks);
    }
    ctx->launches++;
    cudaError_t e = cudaGetLastError();
    if (e) {
        panther_free_paths(p);
        return cuda_err(ctx, e, "sample kernel");
    }
    *out = p;
    return PANTHER_OK;
}

extern "C" panther_status panther_sample_paths(panther_ctx* ctx, const panther_graph* g, uint64_t seed, int64_t R,
                                               int T, int mode, panther_paths** out) {
    return panther_sample_paths_range(ctx, g, seed, 0, R, T, mode, out);
}
