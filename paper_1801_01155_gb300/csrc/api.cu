// Context, memory staging, error reporting and export entry points.
#include <stdarg.h>

#include <atomic>
#include <stdio.h>

#include "lvr_internal.cuh"

// ------------------------------------------------------------------ errors
lvr_status set_err(lvr_ctx *ctx, lvr_status st, const char *fmt, ...) {
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

lvr_status cuda_err(lvr_ctx *ctx, cudaError_t e, const char *what) {
    lvr_status st = e == cudaErrorMemoryAllocation ? LVR_ENOMEM : LVR_ECUDA;
    return set_err(ctx, st, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ memory
bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Test hooks: a one-shot allocation failure after n more allocations, and
// the count of device allocations held (every device allocation of the
// library goes through dev_alloc / dev_free).
static std::atomic<int64_t> g_fail_after{-1};
static std::atomic<int64_t> g_live{0};
void alloc_fail_after(int64_t n) { g_fail_after.store(n < 0 ? -1 : n); }
int64_t alloc_live() { return g_live.load(); }

lvr_status dev_alloc(lvr_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    int64_t f = g_fail_after.load();
    while (f >= 0 && !g_fail_after.compare_exchange_weak(f, f - 1)) {
    }
    if (f == 0) return set_err(ctx, LVR_ENOMEM, "device allocation of %zu bytes refused (test hook)", bytes);
    cudaError_t e = cudaMallocAsync(p, bytes, ctx->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_err(ctx, e, "device allocation");
    }
    g_live.fetch_add(1);
    return LVR_OK;
}

void dev_free(lvr_ctx *ctx, void *p) {
    if (p) {
        cudaFreeAsync(p, ctx->stream);
        g_live.fetch_sub(1);
    }
}

static lvr_status grow(lvr_ctx *ctx, void **buf, size_t *have, size_t want) {
    if (*have >= want && *buf) return LVR_OK;
    size_t n = want + want / 4 + 256;
    dev_free(ctx, *buf);
    *buf = nullptr;
    *have = 0;
    lvr_status st = dev_alloc(ctx, buf, n);
    if (st == LVR_OK) *have = n;
    return st;
}

lvr_status ensure_scratch(lvr_ctx *ctx, size_t bytes) {
    return grow(ctx, &ctx->scratch, &ctx->scratch_bytes, bytes);
}
lvr_status ensure_stage_in(lvr_ctx *ctx, size_t bytes) {
    return grow(ctx, &ctx->stage_in, &ctx->stage_in_bytes, bytes);
}
lvr_status ensure_stage_out(lvr_ctx *ctx, size_t bytes) {
    return grow(ctx, &ctx->stage_out, &ctx->stage_out_bytes, bytes);
}

lvr_status stage_input(lvr_ctx *ctx, const void *p, size_t bytes, size_t slot_offset,
                       const void **dev) {
    if (!p || is_device_ptr(p)) {
        *dev = p;
        return LVR_OK;
    }
    char *dst = (char *)ctx->stage_in + slot_offset;
    LVR_CUDA(ctx, cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *dev = dst;
    return LVR_OK;
}

lvr_status copy_out(lvr_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (!dst || bytes == 0) return LVR_OK;
    if (is_device_ptr(dst)) {
        LVR_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        return LVR_OK;
    }
    LVR_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LVR_OK;
}

// ------------------------------------------------------------------ context
extern "C" int lvr_version(void) { return LVR_API_VERSION; }

extern "C" lvr_status lvr_create(int device, void *cuda_stream, lvr_ctx **out) {
    if (!out) return LVR_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return LVR_EDEVICE;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess || prop.major < 10) return LVR_EDEVICE;
    if (cudaSetDevice(device) != cudaSuccess) return LVR_EDEVICE;
    // keep freed stream-ordered allocations in this process's pool instead of
    // returning them to the driver at every synchronisation: line sets and
    // LoDs are allocated and freed once per frame
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    lvr_ctx *ctx = new lvr_ctx();
    ctx->device = device;
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return LVR_ECUDA;
        }
        ctx->own_stream = true;
    }
    if (cudaMalloc(&ctx->d_status, 64) != cudaSuccess ||
        cudaMalloc(&ctx->d_u64, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_pinned, 256) != cudaSuccess) {
        lvr_destroy(ctx);
        return LVR_ENOMEM;
    }
    *out = ctx;
    return LVR_OK;
}

extern "C" void lvr_destroy(lvr_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, ctx->scratch);
    dev_free(ctx, ctx->d_tf);
    dev_free(ctx, ctx->stage_in);
    dev_free(ctx, ctx->stage_out);
    dev_free(ctx, ctx->vox_pair);
    dev_free(ctx, ctx->frag_t);
    dev_free(ctx, ctx->frag_id);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_u64) cudaFree(ctx->d_u64);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

extern "C" const char *lvr_last_error(const lvr_ctx *ctx) {
    return ctx ? ctx->err.c_str() : "no context";
}

extern "C" lvr_status lvr_sync(lvr_ctx *ctx) {
    if (!ctx) return LVR_EINVAL;
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LVR_OK;
}

// ------------------------------------------------------------------ line set info / export
extern "C" lvr_status lvr_lineset_info_get(const lvr_lineset *ls, lvr_lineset_info *info) {
    if (!ls || !info) return LVR_EINVAL;
    for (int a = 0; a < 3; a++) {
        info->res[a] = ls->res[a];
        info->origin[a] = ls->origin[a];
    }
    info->bins = ls->bins;
    info->scale = ls->scale;
    info->n_voxels = ls->nvox;
    info->n_segments = ls->nseg;
    info->bytes = (int64_t)((ls->nvox + 1) * 4 + ls->nseg * 16);
    return LVR_OK;
}

__global__ void export_fields_kernel(const uint64_t *__restrict__ rec, const uint64_t *__restrict__ key,
                                     int64_t n, uint8_t *fields, uint32_t *curve, uint32_t *ordinal) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t r = rec[i];
        if (fields) {
            uint8_t *f = fields + 8 * i;
            f[0] = (uint8_t)rec_face_in(r);
            f[1] = (uint8_t)rec_u_in(r);
            f[2] = (uint8_t)rec_v_in(r);
            f[3] = (uint8_t)rec_face_out(r);
            f[4] = (uint8_t)rec_u_out(r);
            f[5] = (uint8_t)rec_v_out(r);
            f[6] = (uint8_t)rec_attr(r);
            f[7] = (uint8_t)rec_cont(r);
        }
        uint64_t k = key[i];
        if (curve) curve[i] = (uint32_t)(k >> 32);
        if (ordinal) ordinal[i] = (uint32_t)(k & 0xffffffffu);
    }
}

extern "C" lvr_status lvr_export_lineset(lvr_ctx *ctx, const lvr_lineset *ls, uint32_t *offset,
                                         uint8_t *fields, uint32_t *curve, uint32_t *ordinal) {
    if (!ctx || !ls) return LVR_EINVAL;
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    lvr_status st = copy_out(ctx, offset, ls->offset, (size_t)(ls->nvox + 1) * 4);
    if (st != LVR_OK) return st;
    const int64_t n = ls->nseg;
    if (n == 0 || (!fields && !curve && !ordinal)) return LVR_OK;
    // device destinations directly, host destinations via staging
    uint8_t *df = fields;
    uint32_t *dc = curve, *dor = ordinal;
    bool hf = fields && !is_device_ptr(fields), hc = curve && !is_device_ptr(curve),
         ho = ordinal && !is_device_ptr(ordinal);
    size_t need = (hf ? n * 8 : 0) + (hc ? n * 4 : 0) + (ho ? n * 4 : 0);
    if (need) {
        st = ensure_stage_out(ctx, need);
        if (st != LVR_OK) return st;
        char *p = (char *)ctx->stage_out;
        if (hf) { df = (uint8_t *)p; p += n * 8; }
        if (hc) { dc = (uint32_t *)p; p += n * 4; }
        if (ho) { dor = (uint32_t *)p; }
    }
    export_fields_kernel<<<grid1d(n, 256) > 4096 ? 4096 : grid1d(n, 256), 256, 0, ctx->stream>>>(
        ls->rec, ls->key, n, df, dc, dor);
    LVR_CUDA(ctx, cudaGetLastError());
    if (hf) LVR_CUDA(ctx, cudaMemcpyAsync(fields, df, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (hc) LVR_CUDA(ctx, cudaMemcpyAsync(curve, dc, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (ho) LVR_CUDA(ctx, cudaMemcpyAsync(ordinal, dor, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LVR_OK;
}

extern "C" void lvr_free_lineset(lvr_lineset *ls) {
    if (!ls) return;
    lvr_ctx *ctx = ls->ctx;
    cudaSetDevice(ctx->device);
    dev_free(ctx, ls->offset);
    dev_free(ctx, ls->rec);
    dev_free(ctx, ls->key);
    dev_free(ctx, ls->rec16);
    dev_free(ctx, ls->halo_off);
    dev_free(ctx, ls->halo);
    delete ls;
}
