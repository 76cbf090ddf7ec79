// Internal types and helpers of the lvr CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/lvr.h"

// ------------------------------------------------------------------ status words
// Bits a kernel may raise in the context's device status word.
enum : uint32_t {
    ST_BAD_VERTEX = 1u << 0,    // vertex not finite or outside +-2^14 voxels
    ST_BAD_ATTR = 1u << 1,      // attribute not finite
    ST_BAD_OFFSETS = 1u << 2,   // curve offsets not monotone / out of range
    ST_OVERFLOW = 1u << 3,      // more than 2^32 - 1 segments
    ST_INTERNAL = 1u << 4,      // internal consistency check failed
};

// ------------------------------------------------------------------ handles
struct lvr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    uint32_t *d_status = nullptr;          // device status word
    unsigned long long *d_u64 = nullptr;   // small device counters [8]
    void *h_pinned = nullptr;              // pinned readback area (256 B)
    float *d_tf = nullptr;                 // single-view render: the transfer function (1024 floats)
    // grow-only device scratch, reused across calls
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    // grow-only device staging for host inputs / outputs
    void *stage_in = nullptr;
    size_t stage_in_bytes = 0;
    void *stage_out = nullptr;
    size_t stage_out_bytes = 0;
    int render_blocks[32] = {};            // persistent render grid per kernel variant (SMs x resident blocks):
                                           // [mode * 2 + layout], batched [16 + mode * 2 + layout]
    // voxeliser: grow-only scatter target of (record, key) pairs
    void *vox_pair = nullptr;
    size_t vox_pair_bytes = 0;
    // rasterised comparison system: grow-only fragment store (depths, capsule ids)
    uint64_t *frag_t = nullptr;
    uint32_t *frag_id = nullptr;
    size_t frag_cap = 0;
};

struct lvr_lineset {
    lvr_ctx *ctx = nullptr;
    int32_t res[3] = {0, 0, 0};
    int32_t bins = 0;
    float origin[3] = {0, 0, 0};
    float scale = 0;
    int64_t nvox = 0;
    int64_t nseg = 0;
    uint32_t *offset = nullptr;   // [nvox + 1]
    uint64_t *rec = nullptr;      // [nseg] packed segment records
    uint64_t *key = nullptr;      // [nseg] (curve << 32) | ordinal
    void *rec16 = nullptr;        // [nseg] 16-byte records (lvr_lineset_layout), or null
    // camera at rest (lvr_lineset_neighbours): per voxel, the records of its
    // 3x3x3 neighbourhood that come within the radius of it, as
    // (neighbour index 0..26 << 32) | record; built for radius^2 <= halo_r2
    uint32_t *halo_off = nullptr; // [nvox + 1], or null
    uint64_t *halo = nullptr;     // [halo_n]
    int64_t halo_n = 0;
    float halo_r2 = 0.0f;
};

struct lvr_lod {
    lvr_ctx *ctx = nullptr;
    uint64_t gen = 0;             // unique per LoD built in this process
    int levels = 0;
    int32_t dims[4][3] = {};
    uint32_t *cnt[4] = {};
    float *len[4] = {};
    float *dens[4] = {};
    // sampling copy of dens: per cell (i, j, k) of the padded grid 32 bytes,
    // two float4 for z-slices k and k + 1, each holding the x/y corners as
    // (v(i, j), v(i+1, j) - v(i, j), v(i, j+1), v(i+1, j+1) - v(i, j+1))
    // (zero outside the grid): one aligned 32-byte load per trilinear
    // sample, its x differences already taken. Level l is padded by
    // pad_lo[l] cells below and pad_hi[l][a] above on each axis, enough that
    // every sample point of the density field's support (the grid enlarged
    // by half a coarsest-level cell) has its eight corners inside the copy,
    // so a sampler that checks the support needs no per-corner range check.
    // pk[l] is the padded cell (0, 0, 0), pk0[l] the grid's cell (0, 0, 0);
    // strides pstride[l] = {row, slice} in cells; fewer than 2^32 padded
    // cells per level, so cell indices are 32-bit. pbias[l] folds the
    // padding and the float-to-integer offset of the sampler's floor
    // (bit pattern 0x4B400000 + n for the integer n) into one constant:
    // cell index = bx + row * by + slice * bz - pbias (mod 2^32). One more
    // cell, all zeros, follows the last (index pzero[l]).
    float4 *pk[4] = {};
    const float4 *pk0[4] = {};
    int32_t pad_lo[4] = {};
    int32_t pad_hi[4][3] = {};
    int64_t pstride[4][2] = {};
    uint32_t pbias[4] = {};
    uint32_t pzero[4] = {};
    // spherical per-voxel AO (lvr_lod_ao_field), or null
    float *aof = nullptr;
    // representative lines per level (lvr_lod_rep_lines), or null: per cell one
    // word, bytes 0 valid, 1-3 face/u/v of the start point, 4-6 of the end point
    uint64_t *rep[4] = {};
    int rep_bins = 0;
};

struct lvr_ao_model {
    lvr_ctx *ctx = nullptr;
    float *params = nullptr;      // float32 masters, layout of ao_mlp.cuh
    float *grads = nullptr;       // training: gradient of the last step
    float *adam_m = nullptr, *adam_v = nullptr;
    int64_t adam_t = 0;
    void *w1b = nullptr, *w2b = nullptr, *w3b = nullptr;   // bf16 copies
    float *w4b = nullptr;
    // the renderer's B operands of the mma tiles in fragment order: per
    // n-tile and lane, layer 1's per-hit k-step (8 bytes), then layers 2 and
    // 3 (32 bytes each: the four k-steps), refreshed with the bf16 copies
    void *wfrag = nullptr;
    void *logd = nullptr;         // scratch: bf16 per cell of levels 0..2, log1p(8 dens_l / 8^l)
    size_t logd_bytes = 0;
    float *vcoarse = nullptr;     // scratch: fp32 voxel-term parts of the level-1 and level-2 cells
    size_t vcoarse_bytes = 0;
    // voxel terms of the last LoDs the model was bound to (least recently used replaced)
    static constexpr int kBound = 8;
    struct Bound {
        uint64_t gen = 0;         // LoD generation, 0: empty
        void *vterm = nullptr;    // bf16 [voxels][64]
        size_t bytes = 0;
        uint64_t used = 0;
    } bound[kBound];
    uint64_t clock = 0;
};

// Bind `m` to `lod`: the layer-1 voxel term of every voxel of `lod`, from
// the cache or computed (ao_mlp.cu). *vterm stays valid until kBound other
// LoDs have been bound or the weights change.
lvr_status ao_bind(lvr_ctx *ctx, lvr_ao_model *m, const lvr_lod *lod, const void **vterm);
// The learned-AO voxel term of every level-0 voxel on the tensor cores
// (ao_vterm.cu); ao_vterm_tc_status synchronises and reports a pipeline wait
// that ran out (LVR_ETIMEOUT).
lvr_status ao_vterm_tc(lvr_ctx *ctx, const void *const logd[3], const int pitch[3], const int dims[3][3],
                       float *coarse, const void *w1b, void *vterm);
lvr_status ao_vterm_tc_status(lvr_ctx *ctx);
// LoD handle allocation and the packed sampling copies (lod.cu), shared by
// lvr_build_lod and lvr_import_lod.
lvr_status lod_alloc(lvr_ctx *ctx, int levels, const int32_t dims0[3], lvr_lod **out);
lvr_status lod_pack(lvr_ctx *ctx, lvr_lod *L);
// Restore a learned-AO model's training state (ao_mlp.cu).
lvr_status ao_set_state(lvr_ctx *ctx, lvr_ao_model *m, const float *params, const float *adam_m, const float *adam_v,
                        int64_t step);
// Device-allocation test hooks (api.cu): the n-th next allocation (0: the
// next one) fails once with LVR_ENOMEM, n < 0 switches that off; and the
// number of the library's device allocations currently held.
void alloc_fail_after(int64_t n);
int64_t alloc_live();

// The cached voxel term of `lod` in `m`, or null (no side effects).
inline const void *ao_cached(const lvr_ao_model *m, const lvr_lod *lod) {
    for (const auto &b : m->bound)
        if (b.gen == lod->gen && b.vterm) return b.vterm;
    return nullptr;
}

// ------------------------------------------------------------------ packed record
// 64-bit segment record (Sec. 3.2 / Sec. 6.2 encoding, widened to one word):
//   bits  0- 2 face_in   3- 9 u_in   10-16 v_in
//   bits 17-19 face_out 20-26 u_out  27-33 v_out
//   bits 34-41 attribute byte, bit 42 continues-previous, bits 43-47 local id
//   (curve index mod 32, the paper's 5-bit local line id); 48-63 zero.
__host__ __device__ inline uint64_t rec_pack(uint32_t fi, uint32_t ui, uint32_t vi, uint32_t fo,
                                             uint32_t uo, uint32_t vo, uint32_t attr,
                                             uint32_t cont, uint32_t lid) {
    return (uint64_t)fi | ((uint64_t)ui << 3) | ((uint64_t)vi << 10) | ((uint64_t)fo << 17) |
           ((uint64_t)uo << 20) | ((uint64_t)vo << 27) | ((uint64_t)attr << 34) |
           ((uint64_t)cont << 42) | ((uint64_t)(lid & 31u) << 43);
}
__host__ __device__ inline uint32_t rec_face_in(uint64_t r) { return (uint32_t)(r & 7u); }
__host__ __device__ inline uint32_t rec_u_in(uint64_t r) { return (uint32_t)((r >> 3) & 127u); }
__host__ __device__ inline uint32_t rec_v_in(uint64_t r) { return (uint32_t)((r >> 10) & 127u); }
__host__ __device__ inline uint32_t rec_face_out(uint64_t r) { return (uint32_t)((r >> 17) & 7u); }
__host__ __device__ inline uint32_t rec_u_out(uint64_t r) { return (uint32_t)((r >> 20) & 127u); }
__host__ __device__ inline uint32_t rec_v_out(uint64_t r) { return (uint32_t)((r >> 27) & 127u); }
__host__ __device__ inline uint32_t rec_attr(uint64_t r) { return (uint32_t)((r >> 34) & 255u); }
__host__ __device__ inline uint32_t rec_cont(uint64_t r) { return (uint32_t)((r >> 42) & 1u); }
__host__ __device__ inline uint32_t rec_line_id(uint64_t r) { return (uint32_t)((r >> 43) & 31u); }

// ------------------------------------------------------------------ host helpers
lvr_status set_err(lvr_ctx *ctx, lvr_status st, const char *fmt, ...);
lvr_status cuda_err(lvr_ctx *ctx, cudaError_t e, const char *what);
#define LVR_CUDA(ctx, call)                                  \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call); \
    } while (0)

bool is_device_ptr(const void *p);
// Device copy of a host-or-device input (host data staged into ctx buffers).
lvr_status stage_input(lvr_ctx *ctx, const void *p, size_t bytes, size_t slot_offset,
                       const void **dev);
lvr_status ensure_scratch(lvr_ctx *ctx, size_t bytes);
lvr_status ensure_stage_in(lvr_ctx *ctx, size_t bytes);
lvr_status ensure_stage_out(lvr_ctx *ctx, size_t bytes);
lvr_status dev_alloc(lvr_ctx *ctx, void **p, size_t bytes);
void dev_free(lvr_ctx *ctx, void *p);
// Copy `bytes` from device `src` into host-or-device `dst` (sync if host).
lvr_status copy_out(lvr_ctx *ctx, void *dst, const void *src, size_t bytes);

// Exclusive scan of n uint32 counts into offset[0..n] (offset[n] = total;
// more than 2^32 - 1 sets ST_OVERFLOW in *status); tiles: scan_tile_count(n)
// 64-bit words of scratch.
int64_t scan_tile_count(int64_t n);
void scan_counts(cudaStream_t s, const uint32_t *cnt, int64_t n, unsigned long long *tiles, uint32_t *offset,
                 uint32_t *status);
// Camera basis of a view (float64, rounded to float32); false if degenerate.
// Build (or keep) the camera-at-rest neighbour lists of `ls` for radius^2 r2.
lvr_status ensure_neighbours(lvr_ctx *ctx, lvr_lineset *ls, float r2);
bool camera_basis(const lvr_view *view, float F[3], float R[3], float U[3], float *th, float *tw, float Lt[3]);

inline unsigned grid1d(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 0x7fffffff) g = 0x7fffffff;
    return (unsigned)g;
}
