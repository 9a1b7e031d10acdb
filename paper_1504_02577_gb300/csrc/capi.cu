// Context, errors, allocation, sample size and handle views of libpanther.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "internal.cuh"

panther_status set_err(panther_ctx* ctx, panther_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

panther_status cuda_err(panther_ctx* ctx, cudaError_t e, const char* what) {
    cudaGetLastError();   // clear a non-sticky error
    return set_err(ctx, e == cudaErrorMemoryAllocation ? PANTHER_ENOMEM : PANTHER_ECUDA,
                   "%s: %s", what, cudaGetErrorString(e));
}

panther_status dev_alloc(panther_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (ctx->fail_alloc_at >= 0 && ctx->alloc_seen++ == ctx->fail_alloc_at) {
        ctx->fail_alloc_at = -1;
        return set_err(ctx, PANTHER_ENOMEM, "injected allocation failure (%zu bytes)", bytes);
    }
    cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_err(ctx, PANTHER_ENOMEM, "device allocation of %zu bytes failed: %s", bytes,
                       cudaGetErrorString(e));
    }
    return PANTHER_OK;
}

void dev_free(panther_ctx* ctx, void* p) {
    if (p) cudaFreeAsync(p, ctx->stream);
}

extern "C" {

panther_status panther_create(panther_ctx** out, int device, void* cuda_stream) {
    if (!out) return PANTHER_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return PANTHER_EINVAL;
    }
    panther_ctx* ctx = new panther_ctx();
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return PANTHER_ECUDA; }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return PANTHER_ECUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaMalloc(&ctx->d_status, 4 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_status, 4 * sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, 4 * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_status) cudaFree(ctx->d_status);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return PANTHER_ECUDA;
    }
    // side streams and their events (optional: without them everything runs on `stream`)
    bool side_ok = cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < 2 && side_ok; ++i)
        side_ok = cudaStreamCreateWithFlags(&ctx->side[i], cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&ctx->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!side_ok) {
        cudaGetLastError();
        for (int i = 0; i < 2; ++i) {
            if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
            if (ctx->join[i]) cudaEventDestroy(ctx->join[i]);
            ctx->side[i] = nullptr;
            ctx->join[i] = nullptr;
        }
        if (ctx->fork) cudaEventDestroy(ctx->fork);
        ctx->fork = nullptr;
    }
    // a stream for result copies (optional: without it they go on `stream`)
    if (cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->copy_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->copy) cudaStreamDestroy(ctx->copy);
        ctx->copy = nullptr;
        ctx->copy_ev = nullptr;
    }
    // keep freed stream-ordered memory in the pool between calls
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = ctx;
    return PANTHER_OK;
}

void panther_destroy(panther_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->hub_arena) cudaFreeAsync(ctx->hub_arena, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    // the device pool keeps freed blocks for reuse between calls; what no one
    // uses any more goes back to the device when a context ends
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    cudaGetLastError();
    for (int i = 0; i < 2; ++i) {
        if (ctx->side[i]) cudaStreamDestroy(ctx->side[i]);
        if (ctx->join[i]) cudaEventDestroy(ctx->join[i]);
    }
    if (ctx->fork) cudaEventDestroy(ctx->fork);
    if (ctx->copy) {
        cudaStreamSynchronize(ctx->copy);
        cudaStreamDestroy(ctx->copy);
    }
    if (ctx->copy_ev) cudaEventDestroy(ctx->copy_ev);
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_status);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* panther_last_error(const panther_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

panther_status panther_sync(panther_ctx* ctx) {
    if (!ctx) return PANTHER_EINVAL;
    PCK(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                             ctx->stream));
    PCK(ctx, cudaStreamSynchronize(ctx->stream));
    uint32_t f = ctx->h_status[0];
    if (f) {
        PCK(ctx, cudaMemsetAsync(ctx->d_status, 0, 4 * sizeof(uint32_t), ctx->stream));
        PCK(ctx, cudaStreamSynchronize(ctx->stream));
        if (f & ST_TIMEOUT) return set_err(ctx, PANTHER_ETIMEOUT, "device wait ran out (status 0x%x)", f);
        if (f & (ST_HASH_FULL | ST_OVERFLOW))
            return set_err(ctx, PANTHER_EOVERFLOW, "device overflow (status 0x%x)", f);
        return set_err(ctx, PANTHER_EINVAL, "device detected invalid data (status 0x%x, detail %u)", f,
                       ctx->h_status[1]);
    }
    return PANTHER_OK;
}

panther_status panther_set_scratch_budget(panther_ctx* ctx, int64_t bytes) {
    if (!ctx || bytes < (int64_t(1) << 20)) return PANTHER_EINVAL;
    ctx->scratch_budget = bytes;
    return PANTHER_OK;
}

int64_t panther_launch_count(const panther_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

panther_status panther_sample_size(double eps, double delta, double c, int T, int64_t* R) {
    if (!R) return PANTHER_EINVAL;
    *R = 0;
    if (!(eps > 0 && eps < 1) || !(delta > 0 && delta < 1) || !(c > 0) || T < 2) return PANTHER_EINVAL;
    // Lemma 1: VC dimension <= log2 C(T,2) + 1; Theorem 1: c/eps^2 (d + ln 1/delta)
    double d = log2((double)T * (double)(T - 1) * 0.5) + 1.0;
    double r = ceil(c / (eps * eps) * (d + log(1.0 / delta)));
    if (!(r < 9.2e18)) return PANTHER_EOVERFLOW;
    *R = (int64_t)r;
    return PANTHER_OK;
}

panther_status panther_paths_view(const panther_paths* p, const int32_t** dev_rows, int64_t* R, int* L,
                                  int* stride) {
    if (!p) return PANTHER_EINVAL;
    if (dev_rows) *dev_rows = p->rows;
    if (R) *R = p->R;
    if (L) *L = p->L;
    if (stride) *stride = p->stride;
    return PANTHER_OK;
}

panther_status panther_paths_info(const panther_paths* p, int64_t* n, int64_t* R, int* T, int64_t* r0) {
    if (!p) return PANTHER_EINVAL;
    if (n) *n = p->n;
    if (R) *R = p->R;
    if (T) *T = p->T;
    if (r0) *r0 = p->r0;
    return PANTHER_OK;
}

panther_status panther_index_view(const panther_index* ix, const int64_t** dev_off, const uint32_t** dev_pid,
                                  int64_t* n, int64_t* nnz) {
    if (!ix) return PANTHER_EINVAL;
    if (dev_off) *dev_off = ix->off;
    if (dev_pid) *dev_pid = ix->pid;
    if (n) *n = ix->n;
    if (nnz) *nnz = ix->nnz;
    return PANTHER_OK;
}

panther_status pantherpp_vecs_view(const pantherpp_vecs* v, const uint32_t** dev_theta, int64_t* n, int* D) {
    if (!v) return PANTHER_EINVAL;
    if (dev_theta) *dev_theta = v->theta;
    if (n) *n = v->n;
    if (D) *D = v->D;
    return PANTHER_OK;
}

void panther_free_graph(panther_graph* g) {
    if (!g) return;
    panther_ctx* c = g->ctx;
    dev_free(c, g->vrec);
    dev_free(c, g->prefix);
    dev_free(c, g->alias);
    dev_free(c, g->col);
    cudaStreamSynchronize(c->stream);
    delete g;
}

void panther_free_paths(panther_paths* p) {
    if (!p) return;
    dev_free(p->ctx, p->rows);
    cudaStreamSynchronize(p->ctx->stream);
    delete p;
}

void panther_free_index(panther_index* ix) {
    if (!ix) return;
    dev_free(ix->ctx, ix->off);
    dev_free(ix->ctx, ix->pid);
    dev_free(ix->ctx, ix->cls);
    dev_free(ix->ctx, ix->cls_hist);
    cudaStreamSynchronize(ix->ctx->stream);
    delete ix;
}

void pantherpp_free_vecs(pantherpp_vecs* v) {
    if (!v) return;
    panther_ctx* c = v->ctx;
    dev_free(c, v->theta);
    dev_free(c, v->B);
    dev_free(c, v->cid);
    dev_free(c, v->cnrm);
    dev_free(c, v->cncf);
    dev_free(c, v->ctile);
    dev_free(c, v->norm2);
    dev_free(c, v->nrm);
    dev_free(c, v->exact);
    cudaStreamSynchronize(c->stream);
    delete v;
}

}  // extern "C"

// ------------------------------------------------------------------ scan ---
// Device-wide exclusive scan of int64 (reduce, scan of block sums, downsweep).
namespace {
constexpr int SCAN_T = 512;
constexpr int SCAN_PER = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_PER;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total) {
    // warp inclusive scan
    unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int64_t s = lane < (unsigned)nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= (unsigned)o) s += y;
        }
        if (lane < (unsigned)nw) sh[lane] = s;
    }
    __syncthreads();
    int64_t before = (wid ? sh[wid - 1] : 0) + x - v;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void scan_reduce_kernel(const int64_t* __restrict__ d, int64_t n, int64_t* __restrict__ sums) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int i = 0; i < SCAN_PER; ++i) {
        int64_t j = base + (int64_t)i * SCAN_T + threadIdx.x;
        if (j < n) s += d[j];
    }
    int64_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void scan_single_kernel(int64_t* __restrict__ sums, int64_t nb) {
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += SCAN_T) {
        int64_t j = base + threadIdx.x;
        int64_t v = j < nb ? sums[j] : 0;
        int64_t tot;
        int64_t ex = block_excl_scan(v, sh, &tot);
        if (j < nb) sums[j] = carry + ex;
        carry += tot;
    }
}

__global__ void scan_down_kernel(int64_t* __restrict__ d, int64_t n, const int64_t* __restrict__ sums) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    // each thread owns SCAN_PER consecutive elements
    int64_t v[SCAN_PER];
    int64_t s = 0;
    int64_t my = base + (int64_t)threadIdx.x * SCAN_PER;
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        v[i] = (my + i < n) ? d[my + i] : 0;
        s += v[i];
    }
    int64_t ex = block_excl_scan(s, sh, nullptr) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_PER; ++i) {
        if (my + i < n) d[my + i] = ex;
        ex += v[i];
    }
}
}  // namespace

panther_status scan_exclusive_i64(panther_ctx* ctx, int64_t* data, int64_t n) {
    if (n <= 0) return PANTHER_OK;
    int64_t nb = ceil_div(n, SCAN_TILE);
    int64_t* sums = nullptr;
    panther_status st = dev_alloc(ctx, (void**)&sums, sizeof(int64_t) * nb);
    if (st) return st;
    scan_reduce_kernel<<<(unsigned)nb, SCAN_T, 0, ctx->stream>>>(data, n, sums);
    PLAUNCH(ctx);
    scan_single_kernel<<<1, SCAN_T, 0, ctx->stream>>>(sums, nb);
    PLAUNCH(ctx);
    scan_down_kernel<<<(unsigned)nb, SCAN_T, 0, ctx->stream>>>(data, n, sums);
    PLAUNCH(ctx);
    dev_free(ctx, sums);
    return PANTHER_OK;
}
