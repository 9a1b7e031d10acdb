// Checkpoint files for sampled paths and the inverted index (no counterpart
// in the paper, whose processing and query phases run in one process).
//
// A file is a 64-byte little-endian header followed by the raw device
// arrays:
//   0  char[8]  magic "PNTHPATH" or "PNTHINDX"
//   8  u32      version (1)
//   12 u32      T          16 u32 L        20 u32 stride      24 u32 mode
//   28 u32      reserved (0)
//   32 i64      n          40 i64 R
//   48 i64      r0 (paths) or nnz (index)
//   56 u64      seed (paths) or 0
// paths: int32[R][stride]; index: int64 off[n+1], uint32 pid[nnz].
// Arrays move through a pinned staging buffer in chunks. A loaded index is
// validated on the device (offsets monotone from 0 to nnz, path ids below R)
// before it is handed out, so a damaged file is refused rather than read out
// of bounds later.
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "internal.cuh"

namespace {

struct FileHeader {
    char magic[8];
    uint32_t version, T, L, stride, mode, reserved;
    int64_t n, R, x;   // x: r0 or nnz
    uint64_t seed;
};
static_assert(sizeof(FileHeader) == 64, "header layout");

constexpr size_t CHUNK = size_t(64) << 20;

struct File {
    FILE* f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

// device <-> file through one pinned buffer
panther_status copy_out(panther_ctx* ctx, FILE* f, const void* dev, size_t bytes) {
    void* h = nullptr;
    if (cudaMallocHost(&h, std::min(bytes, CHUNK) + 1) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, PANTHER_ENOMEM, "pinned staging buffer");
    }
    panther_status st = PANTHER_OK;
    for (size_t done = 0; done < bytes && !st;) {
        const size_t n = std::min(CHUNK, bytes - done);
        cudaError_t e = cudaMemcpyAsync(h, (const char*)dev + done, n, cudaMemcpyDeviceToHost, ctx->stream);
        if (!e) e = cudaStreamSynchronize(ctx->stream);
        if (e) st = cuda_err(ctx, e, "checkpoint copy");
        else if (fwrite(h, 1, n, f) != n) st = set_err(ctx, PANTHER_EINVAL, "checkpoint write failed");
        done += n;
    }
    cudaFreeHost(h);
    return st;
}

panther_status copy_in(panther_ctx* ctx, FILE* f, void* dev, size_t bytes) {
    void* h = nullptr;
    if (cudaMallocHost(&h, std::min(bytes, CHUNK) + 1) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, PANTHER_ENOMEM, "pinned staging buffer");
    }
    panther_status st = PANTHER_OK;
    for (size_t done = 0; done < bytes && !st;) {
        const size_t n = std::min(CHUNK, bytes - done);
        if (fread(h, 1, n, f) != n) {
            st = set_err(ctx, PANTHER_EINVAL, "checkpoint file is shorter than its header says");
            break;
        }
        cudaError_t e = cudaMemcpyAsync((char*)dev + done, h, n, cudaMemcpyHostToDevice, ctx->stream);
        if (!e) e = cudaStreamSynchronize(ctx->stream);
        if (e) st = cuda_err(ctx, e, "checkpoint copy");
        done += n;
    }
    cudaFreeHost(h);
    return st;
}

panther_status read_header(panther_ctx* ctx, FILE* f, const char* magic, FileHeader* hd) {
    if (fread(hd, 1, sizeof(*hd), f) != sizeof(*hd)) return set_err(ctx, PANTHER_EINVAL, "checkpoint header missing");
    if (memcmp(hd->magic, magic, 8) != 0) return set_err(ctx, PANTHER_EINVAL, "not a %.8s checkpoint", magic);
    if (hd->version != 1) return set_err(ctx, PANTHER_EINVAL, "checkpoint version %u", hd->version);
    return PANTHER_OK;
}

// offsets start at 0, never decrease, end at nnz; path ids in [0, R)
__global__ void check_index_kernel(const int64_t* __restrict__ off, int64_t n, const uint32_t* __restrict__ pid,
                                   int64_t nnz, int64_t R, uint32_t* status) {
    const int64_t st = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += st) {
        const int64_t a = off[v];
        const bool bad = (v == 0 && a != 0) || (v == n && a != nnz) || a < 0 || a > nnz ||
                         (v < n && off[v + 1] < a);
        if (bad) flag_status(status, ST_BAD_INDEX);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += st)
        if ((int64_t)pid[i] >= R) flag_status(status, ST_BAD_INDEX);
}

}  // namespace

extern "C" {

panther_status panther_save_paths(const panther_paths* p, const char* path) {
    if (!p || !path) return PANTHER_EINVAL;
    panther_ctx* ctx = p->ctx;
    cudaSetDevice(ctx->device);
    File fl;
    if (!(fl.f = fopen(path, "wb"))) return set_err(ctx, PANTHER_EINVAL, "cannot open %s for writing", path);
    FileHeader hd{};
    memcpy(hd.magic, "PNTHPATH", 8);
    hd.version = 1;
    hd.T = (uint32_t)p->T;
    hd.L = (uint32_t)p->L;
    hd.stride = (uint32_t)p->stride;
    hd.mode = (uint32_t)p->mode;
    hd.n = p->n;
    hd.R = p->R;
    hd.x = p->r0;
    hd.seed = p->seed;
    if (fwrite(&hd, 1, sizeof(hd), fl.f) != sizeof(hd)) return set_err(ctx, PANTHER_EINVAL, "checkpoint write failed");
    return copy_out(ctx, fl.f, p->rows, sizeof(int32_t) * (size_t)p->R * p->stride);
}

panther_status panther_load_paths(panther_ctx* ctx, const char* path, panther_paths** out) {
    if (!ctx || !path || !out) return PANTHER_EINVAL;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    File fl;
    if (!(fl.f = fopen(path, "rb"))) return set_err(ctx, PANTHER_EINVAL, "cannot open %s", path);
    FileHeader hd;
    panther_status st = read_header(ctx, fl.f, "PNTHPATH", &hd);
    if (st) return st;
    if (hd.T < 1 || hd.T > (uint32_t)MAX_T || hd.L != hd.T + 1 || hd.stride != (uint32_t)path_stride((int)hd.L) || hd.n < 1 ||
        hd.n >= (int64_t(1) << 31) || hd.R < 1 || hd.R > 0xffffffffLL || hd.x < 0 ||
        (hd.mode != PANTHER_MODE_PREFIX && hd.mode != PANTHER_MODE_ALIAS && hd.mode != PANTHER_MODE_UNWEIGHTED))
        return set_err(ctx, PANTHER_EINVAL, "inconsistent paths checkpoint header");
    panther_paths* p = new panther_paths();
    p->ctx = ctx;
    p->n = hd.n;
    p->R = hd.R;
    p->T = (int)hd.T;
    p->L = (int)hd.L;
    p->stride = (int)hd.stride;
    p->mode = (int)hd.mode;
    p->seed = hd.seed;
    p->r0 = hd.x;
    if ((st = dev_alloc(ctx, (void**)&p->rows, sizeof(int32_t) * (size_t)p->R * p->stride)) ||
        (st = copy_in(ctx, fl.f, p->rows, sizeof(int32_t) * (size_t)p->R * p->stride))) {
        panther_free_paths(p);
        return st;
    }
    *out = p;
    return PANTHER_OK;
}

panther_status panther_save_index(const panther_index* ix, const char* path) {
    if (!ix || !path) return PANTHER_EINVAL;
    panther_ctx* ctx = ix->ctx;
    cudaSetDevice(ctx->device);
    File fl;
    if (!(fl.f = fopen(path, "wb"))) return set_err(ctx, PANTHER_EINVAL, "cannot open %s for writing", path);
    FileHeader hd{};
    memcpy(hd.magic, "PNTHINDX", 8);
    hd.version = 1;
    hd.n = ix->n;
    hd.R = ix->R;
    hd.x = ix->nnz;
    if (fwrite(&hd, 1, sizeof(hd), fl.f) != sizeof(hd)) return set_err(ctx, PANTHER_EINVAL, "checkpoint write failed");
    panther_status st = copy_out(ctx, fl.f, ix->off, sizeof(int64_t) * (size_t)(ix->n + 1));
    if (!st && ix->nnz) st = copy_out(ctx, fl.f, ix->pid, sizeof(int32_t) * (size_t)ix->nnz);
    return st;
}

panther_status panther_load_index(panther_ctx* ctx, const char* path, panther_index** out) {
    if (!ctx || !path || !out) return PANTHER_EINVAL;
    *out = nullptr;
    cudaSetDevice(ctx->device);
    File fl;
    if (!(fl.f = fopen(path, "rb"))) return set_err(ctx, PANTHER_EINVAL, "cannot open %s", path);
    FileHeader hd;
    panther_status st = read_header(ctx, fl.f, "PNTHINDX", &hd);
    if (st) return st;
    if (hd.n < 1 || hd.n >= (int64_t(1) << 31) || hd.R < 1 || hd.R > 0xffffffffLL || hd.x < 0 ||
        hd.x > hd.R * (MAX_T + 1))
        return set_err(ctx, PANTHER_EINVAL, "inconsistent index checkpoint header");
    panther_index* ix = new panther_index();
    ix->ctx = ctx;
    ix->n = hd.n;
    ix->R = hd.R;
    ix->nnz = hd.x;
    auto fail = [&](panther_status e) {
        panther_free_index(ix);
        return e;
    };
    if ((st = dev_alloc(ctx, (void**)&ix->off, sizeof(int64_t) * (size_t)(ix->n + 1))) ||
        (st = dev_alloc(ctx, (void**)&ix->pid, sizeof(int32_t) * (size_t)std::max<int64_t>(ix->nnz, 1))) ||
        (st = dev_alloc(ctx, (void**)&ix->cls, ix->n)) ||
        (st = dev_alloc(ctx, (void**)&ix->cls_hist, sizeof(int64_t) * 256)) ||
        (st = copy_in(ctx, fl.f, ix->off, sizeof(int64_t) * (size_t)(ix->n + 1))) ||
        (ix->nnz && (st = copy_in(ctx, fl.f, ix->pid, sizeof(int32_t) * (size_t)ix->nnz))))
        return fail(st);
    PCK(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), ctx->stream));
    check_index_kernel<<<(unsigned)(ctx->num_sms * 8), 256, 0, ctx->stream>>>(ix->off, ix->n, ix->pid, ix->nnz, ix->R,
                                                                             ctx->d_status);
    ctx->launches++;
    if ((st = panther_sync(ctx))) return fail(set_err(ctx, PANTHER_EINVAL, "index checkpoint fails validation"));
    if ((st = index_classes(ctx, ix)) || (st = panther_sync(ctx))) return fail(st);
    *out = ix;
    return PANTHER_OK;
}

}  // extern "C"
