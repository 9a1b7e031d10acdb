// Test support: Philox words from this library's generator next to curand's
// Philox4_32_10 for the same key and counter, so that both the device
// generator and the CPU oracle's generator can be checked against an
// independent implementation of the published algorithm.
#include <curand_kernel.h>

#include "internal.cuh"

namespace {
__global__ void philox_check_kernel(uint32_t k0, uint32_t k1, uint64_t r0, uint32_t c2, uint32_t c3, int64_t count,
                                    uint4* out, uint4* ref) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint64_t r = r0 + (uint64_t)i;
    pword4 w = philox10((uint32_t)r, (uint32_t)(r >> 32), c2, c3, k0, k1);
    out[i] = make_uint4(w.x, w.y, w.z, w.w);
    // curand: counter = (offset/4 as 64 bits, subsequence as 64 bits), key = seed
    curandStatePhilox4_32_10_t st;
    curand_init(((unsigned long long)k1 << 32) | k0, ((unsigned long long)c3 << 32) | c2, 4ull * r, &st);
    ref[i] = curand4(&st);
}
}  // namespace

extern "C" panther_status panther_debug_philox(panther_ctx* ctx, uint32_t k0, uint32_t k1, uint64_t r0, uint32_t c2,
                                               uint32_t c3, int64_t count, uint32_t* dev_out, uint32_t* dev_ref) {
    if (!ctx || count < 0 || (count && (!dev_out || !dev_ref))) return PANTHER_EINVAL;
    if (count == 0) return PANTHER_OK;
    cudaSetDevice(ctx->device);
    philox_check_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, ctx->stream>>>(k0, k1, r0, c2, c3, count,
                                                                                 (uint4*)dev_out, (uint4*)dev_ref);
    ctx->launches++;
    PCK(ctx, cudaGetLastError());
    PCK(ctx, cudaStreamSynchronize(ctx->stream));
    return PANTHER_OK;
}

namespace {
// waits for *flag (never set) at most limit cycles, then records a timeout
__global__ void wait_flag_kernel(const volatile uint32_t* flag, long long limit, uint32_t* status) {
    const long long t0 = clock64();
    while (*flag == 0) {
        if (clock64() - t0 > limit) {
            if (threadIdx.x == 0) flag_status(status, ST_TIMEOUT);
            return;
        }
    }
}
}  // namespace

extern "C" panther_status panther_debug_fail_alloc(panther_ctx* ctx, int64_t nth) {
    if (!ctx) return PANTHER_EINVAL;
    ctx->fail_alloc_at = nth < 0 ? -1 : nth;
    ctx->alloc_seen = 0;
    return PANTHER_OK;
}

extern "C" panther_status panther_debug_wait_timeout(panther_ctx* ctx, int64_t limit_cycles) {
    if (!ctx) return PANTHER_EINVAL;
    if (limit_cycles < 1 || limit_cycles > (int64_t(1) << 31))
        return set_err(ctx, PANTHER_EINVAL, "limit_cycles must be in [1, 2^31]");
    cudaSetDevice(ctx->device);
    uint32_t* flag = nullptr;
    panther_status st = dev_alloc(ctx, (void**)&flag, sizeof(uint32_t));
    if (st) return st;
    PCK(ctx, cudaMemsetAsync(flag, 0, sizeof(uint32_t), ctx->stream));
    wait_flag_kernel<<<1, 32, 0, ctx->stream>>>(flag, (long long)limit_cycles, ctx->d_status);
    ctx->launches++;
    dev_free(ctx, flag);
    PCK(ctx, cudaGetLastError());
    return panther_sync(ctx);
}
