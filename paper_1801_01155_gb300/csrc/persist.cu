// Import of saved voxel models and LoDs, and the learned-AO trainer's
// checkpoint (model state): the inverse of the export calls, so that a line
// set, its density LoD and a model in training can be written out by the
// caller and resumed later without re-running the voxeliser or the trainer.
#include <math.h>
#include <string.h>

#include "ao_mlp.cuh"
#include "lvr_internal.cuh"

namespace {

constexpr uint32_t IMP_BAD_OFFSETS = 1u, IMP_BAD_FIELDS = 2u, IMP_BAD_ORDER = 4u, IMP_BAD_LOD = 8u;

// One thread per voxel: offsets non-decreasing and within the segment count,
// each segment's fields in range (faces < 6, bins < N, flag 0 / 1), and the
// segments of a voxel in strictly increasing (curve, position) order, the
// voxeliser's canonical order (Sec. 3.3).
__global__ void import_check_kernel(const uint32_t *__restrict__ off, int64_t nvox, int64_t nseg,
                                    const uint8_t *__restrict__ f, const uint32_t *__restrict__ curve,
                                    const uint32_t *__restrict__ ord, int bins, uint32_t *status) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v == 0 && (off[0] != 0u || (int64_t)off[nvox] != nseg)) atomicOr(status, IMP_BAD_OFFSETS);
    if (v >= nvox) return;
    const uint32_t b = off[v], e = off[v + 1];
    if (b > e || (int64_t)e > nseg) {
        atomicOr(status, IMP_BAD_OFFSETS);
        return;
    }
    uint64_t prev = 0;
    for (uint32_t i = b; i < e; i++) {
        const uint8_t *s = f + 8 * (int64_t)i;
        if (s[0] >= 6 || s[3] >= 6 || s[1] >= bins || s[2] >= bins || s[4] >= bins || s[5] >= bins || s[7] > 1)
            atomicOr(status, IMP_BAD_FIELDS);
        const uint64_t k = (uint64_t)curve[i] << 32 | ord[i];
        if (i > b && k <= prev) atomicOr(status, IMP_BAD_ORDER);
        prev = k;
    }
}

__global__ void import_pack_kernel(const uint8_t *__restrict__ f, const uint32_t *__restrict__ curve,
                                   const uint32_t *__restrict__ ord, int64_t n, uint64_t *rec, uint64_t *key) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t *s = f + 8 * i;
        rec[i] = rec_pack(s[0], s[1], s[2], s[3], s[4], s[5], s[6], s[7], curve[i]);
        key[i] = (uint64_t)curve[i] << 32 | ord[i];
    }
}

// LoD level values: counts any, lengths and densities finite and >= 0.
__global__ void lod_check_kernel(const float *__restrict__ len, const float *__restrict__ dens, int64_t n,
                                 uint32_t *status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!(len[i] >= 0.0f && len[i] < INFINITY && dens[i] >= 0.0f && dens[i] < INFINITY))
            atomicOr(status, IMP_BAD_LOD);
}

// Copy `bytes` from host or device memory into a device buffer.
lvr_status copy_in(lvr_ctx *ctx, void *dst, const void *src, size_t bytes) {
    if (bytes == 0) return LVR_OK;
    LVR_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
    return LVR_OK;
}

lvr_status read_status(lvr_ctx *ctx, uint32_t *status, uint32_t *out) {
    uint32_t *h = (uint32_t *)ctx->h_pinned;
    LVR_CUDA(ctx, cudaMemcpyAsync(h, status, 4, cudaMemcpyDeviceToHost, ctx->stream));
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *out = h[0];
    return LVR_OK;
}

}  // namespace

extern "C" lvr_status lvr_import_lineset(lvr_ctx *ctx, const lvr_lineset_info *info, const uint32_t *offset,
                                         const uint8_t *fields, const uint32_t *curve, const uint32_t *ordinal,
                                         lvr_lineset **out) {
    if (!ctx) return LVR_EINVAL;
    if (!info || !offset || !out) return set_err(ctx, LVR_EINVAL, "lvr_import_lineset: null argument");
    *out = nullptr;
    int64_t nvox = 1;
    for (int a = 0; a < 3; a++) {
        if (info->res[a] < 1 || info->res[a] > 4096) return set_err(ctx, LVR_EINVAL, "res must be in [1,4096]");
        nvox *= info->res[a];
    }
    if (nvox >= (int64_t)1 << 32) return set_err(ctx, LVR_EINVAL, "grid has 2^32 or more voxels");
    if (info->bins < 2 || info->bins > 128 || (info->bins & (info->bins - 1)))
        return set_err(ctx, LVR_EINVAL, "bins must be a power of two in [2,128]");
    if (!(info->scale > 0.0f) || !isfinite(info->scale)) return set_err(ctx, LVR_EINVAL, "scale must be > 0");
    const int64_t nseg = info->n_segments;
    if (nseg < 0 || nseg > 0xffffffffLL) return set_err(ctx, LVR_EINVAL, "n_segments out of range");
    if (nseg > 0 && (!fields || !curve || !ordinal))
        return set_err(ctx, LVR_EINVAL, "lvr_import_lineset: fields, curve and ordinal are needed");
    if (info->n_voxels != nvox) return set_err(ctx, LVR_EINVAL, "n_voxels does not match res");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    lvr_lineset *ls = new lvr_lineset();
    ls->ctx = ctx;
    for (int a = 0; a < 3; a++) {
        ls->res[a] = info->res[a];
        ls->origin[a] = info->origin[a];
    }
    ls->bins = info->bins;
    ls->scale = info->scale;
    ls->nvox = nvox;
    ls->nseg = nseg;
    lvr_status st;
    if ((st = dev_alloc(ctx, (void **)&ls->offset, (size_t)(nvox + 1) * 4)) != LVR_OK ||
        (st = dev_alloc(ctx, (void **)&ls->rec, (size_t)nseg * 8)) != LVR_OK ||
        (st = dev_alloc(ctx, (void **)&ls->key, (size_t)nseg * 8)) != LVR_OK) {
        lvr_free_lineset(ls);
        return st;
    }
    // the fields, curves and ordinals go through the context's staging buffer
    const size_t fb = ((size_t)nseg * 8 + 255) & ~(size_t)255, cb = ((size_t)nseg * 4 + 255) & ~(size_t)255;
    if ((st = ensure_stage_in(ctx, fb + 2 * cb + 256)) != LVR_OK) {
        lvr_free_lineset(ls);
        return st;
    }
    uint8_t *df = (uint8_t *)ctx->stage_in;
    uint32_t *dc = (uint32_t *)((char *)ctx->stage_in + fb), *dor = (uint32_t *)((char *)ctx->stage_in + fb + cb);
    uint32_t *status = ctx->d_status + 4;
    uint32_t flags = 0;
    if ((st = copy_in(ctx, ls->offset, offset, (size_t)(nvox + 1) * 4)) != LVR_OK ||
        (st = copy_in(ctx, df, fields, (size_t)nseg * 8)) != LVR_OK ||
        (st = copy_in(ctx, dc, curve, (size_t)nseg * 4)) != LVR_OK ||
        (st = copy_in(ctx, dor, ordinal, (size_t)nseg * 4)) != LVR_OK) {
        lvr_free_lineset(ls);
        return st;
    }
    cudaError_t e = cudaMemsetAsync(status, 0, 4, s);
    if (e == cudaSuccess) {
        import_check_kernel<<<grid1d(nvox, 256), 256, 0, s>>>(ls->offset, nvox, nseg, df, dc, dor, ls->bins, status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess || (st = read_status(ctx, status, &flags)) != LVR_OK) {
        lvr_free_lineset(ls);
        return e != cudaSuccess ? cuda_err(ctx, e, "lvr_import_lineset") : st;
    }
    if (flags) {
        lvr_free_lineset(ls);
        return set_err(ctx, LVR_EINVAL, "lvr_import_lineset: %s", (flags & IMP_BAD_OFFSETS) ? "offsets out of order or range"
                                                                : (flags & IMP_BAD_FIELDS) ? "a segment field out of range"
                                                                                           : "segments of a voxel not in (curve, position) order");
    }
    if (nseg > 0) {
        import_pack_kernel<<<grid1d(nseg, 256) > 4096 ? 4096 : grid1d(nseg, 256), 256, 0, s>>>(df, dc, dor, nseg, ls->rec,
                                                                                            ls->key);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            lvr_free_lineset(ls);
            return cuda_err(ctx, e, "lvr_import_lineset");
        }
    }
    *out = ls;
    return LVR_OK;
}

extern "C" lvr_status lvr_import_lod(lvr_ctx *ctx, int levels, const int32_t dims0[3], const uint32_t *const *cnt,
                                     const float *const *len, const float *const *dens, lvr_lod **out) {
    if (!ctx) return LVR_EINVAL;
    if (!dims0 || !cnt || !len || !dens || !out) return set_err(ctx, LVR_EINVAL, "lvr_import_lod: null argument");
    *out = nullptr;
    if (levels < 1 || levels > 4) return set_err(ctx, LVR_EINVAL, "levels must be in [1,4]");
    int64_t nvox = 1;
    for (int a = 0; a < 3; a++) {
        if (dims0[a] < 1 || dims0[a] > 4096) return set_err(ctx, LVR_EINVAL, "dims must be in [1,4096]");
        nvox *= dims0[a];
    }
    if (nvox >= (int64_t)1 << 32) return set_err(ctx, LVR_EINVAL, "grid has 2^32 or more voxels");
    for (int l = 0; l < levels; l++)
        if (!cnt[l] || !len[l] || !dens[l]) return set_err(ctx, LVR_EINVAL, "lvr_import_lod: null level array");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    lvr_lod *L = nullptr;
    lvr_status st = lod_alloc(ctx, levels, dims0, &L);
    if (st != LVR_OK) return st;
    uint32_t *status = ctx->d_status + 4;
    LVR_CUDA(ctx, cudaMemsetAsync(status, 0, 4, ctx->stream));
    for (int l = 0; l < levels && st == LVR_OK; l++) {
        const int64_t n = (int64_t)L->dims[l][0] * L->dims[l][1] * L->dims[l][2];
        if ((st = copy_in(ctx, L->cnt[l], cnt[l], (size_t)n * 4)) != LVR_OK ||
            (st = copy_in(ctx, L->len[l], len[l], (size_t)n * 4)) != LVR_OK ||
            (st = copy_in(ctx, L->dens[l], dens[l], (size_t)n * 4)) != LVR_OK)
            break;
        lod_check_kernel<<<grid1d(n, 256) > 4096 ? 4096 : grid1d(n, 256), 256, 0, ctx->stream>>>(L->len[l], L->dens[l], n,
                                                                                              status);
    }
    uint32_t flags = 0;
    if (st == LVR_OK) st = read_status(ctx, status, &flags);
    if (st == LVR_OK && flags) st = set_err(ctx, LVR_EINVAL, "lvr_import_lod: lengths and densities must be finite and >= 0");
    if (st == LVR_OK) st = lod_pack(ctx, L);
    if (st != LVR_OK) {
        lvr_free_lod(L);
        return st;
    }
    *out = L;
    return LVR_OK;
}

// ------------------------------------------------------------------ learned-AO trainer checkpoint
extern "C" lvr_status lvr_ao_model_state(lvr_ctx *ctx, const lvr_ao_model *m, float *params, float *adam_m,
                                         float *adam_v, int64_t *step) {
    if (!ctx) return LVR_EINVAL;
    if (!m || !params || !adam_m || !adam_v || !step) return set_err(ctx, LVR_EINVAL, "lvr_ao_model_state: null argument");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t b = (size_t)aomlp::NPARAM * 4;
    lvr_status st = copy_out(ctx, params, m->params, b);
    if (st != LVR_OK) return st;
    if (m->adam_m && m->adam_v) {
        if ((st = copy_out(ctx, adam_m, m->adam_m, b)) != LVR_OK || (st = copy_out(ctx, adam_v, m->adam_v, b)) != LVR_OK)
            return st;
        *step = m->adam_t;
        return LVR_OK;
    }
    // no Adam step taken yet: zero moments, step 0
    if ((st = ensure_stage_out(ctx, b)) != LVR_OK) return st;
    LVR_CUDA(ctx, cudaMemsetAsync(ctx->stage_out, 0, b, ctx->stream));
    if ((st = copy_out(ctx, adam_m, ctx->stage_out, b)) != LVR_OK || (st = copy_out(ctx, adam_v, ctx->stage_out, b)) != LVR_OK)
        return st;
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *step = 0;
    return LVR_OK;
}

extern "C" lvr_status lvr_ao_model_set_state(lvr_ctx *ctx, lvr_ao_model *m, const float *params, const float *adam_m,
                                             const float *adam_v, int64_t step) {
    if (!ctx) return LVR_EINVAL;
    if (!m || !params || !adam_m || !adam_v) return set_err(ctx, LVR_EINVAL, "lvr_ao_model_set_state: null argument");
    if (step < 0) return set_err(ctx, LVR_EINVAL, "step must be >= 0");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    return ao_set_state(ctx, m, params, adam_m, adam_v, step);
}

// ------------------------------------------------------------------ test hooks
extern "C" void lvr_test_fail_allocation(int64_t n) { alloc_fail_after(n); }
extern "C" int64_t lvr_test_live_allocations(void) { return alloc_live(); }
