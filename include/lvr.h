/*
 * lvr — voxel-based ray casting of large 3D line sets on one GB300 GPU.
 *
 * C ABI of the CUDA library (liblvr.so). Method: Kanzler, Rautenhaus,
 * Westermann, "A Voxel-based Rendering Pipeline for Large 3D Line Sets"
 * (arXiv 1801.01155). Section numbers below refer to that paper.
 *
 * Conventions
 *  - Every entry point returns an lvr_status; on failure lvr_last_error()
 *    gives a message owned by the context, valid until its next call.
 *  - Pointer arguments marked "host or device" may point to either; the
 *    library detects which (cudaPointerGetAttributes) and stages host data
 *    through its own device buffers. Everything else is host memory.
 *  - Inputs are owned by the caller and are only read, and only until the
 *    call returns (device inputs: until the work queued on the context's
 *    stream has consumed them). Handles (lvr_lineset, lvr_lod,
 *    lvr_ao_model) are owned by the library and released by their
 *    lvr_free_* call, which must come before lvr_destroy of their context.
 *    Output buffers are owned by the caller.
 *  - Work is queued on the context's CUDA stream in call order. Calls that
 *    return host-visible results (sizes, exports into host memory)
 *    synchronise that stream. Arguments are validated before any work is
 *    queued; conditions found on the device (a bad vertex, a count
 *    overflow) make the call that finds them fail.
 *  - A context is not thread-safe; use one per host thread.
 */
#ifndef LVR_H
#define LVR_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LVR_API_VERSION 1

typedef enum lvr_status {
    LVR_OK = 0,
    LVR_EINVAL = 1,     /* bad argument or input data */
    LVR_ENOMEM = 2,     /* device or host allocation failed */
    LVR_ECUDA = 3,      /* CUDA runtime error */
    LVR_EOVERFLOW = 4,  /* a count beyond 2^32 - 1 (segments, neighbour-list entries,
                           fragments) or beyond a caller-owned capacity */
    LVR_ETIMEOUT = 5,   /* a bounded device-side wait gave up (the learned-AO voxel term's
                           tensor-core pipeline: lvr_render, lvr_ao_infer, lvr_batch_create) */
    LVR_EDEVICE = 6     /* no usable sm_103 device */
} lvr_status;

typedef struct lvr_ctx lvr_ctx;
typedef struct lvr_lineset lvr_lineset;
typedef struct lvr_lod lvr_lod;
typedef struct lvr_ao_model lvr_ao_model;

/* Library version (LVR_API_VERSION). */
int lvr_version(void);

/* Create a context on CUDA device `device`, queuing work on `cuda_stream`
 * (a cudaStream_t; NULL: the context creates and owns a stream). */
lvr_status lvr_create(int device, void *cuda_stream, lvr_ctx **out);
void lvr_destroy(lvr_ctx *ctx);
const char *lvr_last_error(const lvr_ctx *ctx);
/* Wait for all work queued on the context's stream. */
lvr_status lvr_sync(lvr_ctx *ctx);

/* ------------------------------------------------------------------ voxelisation
 * Sec. 3.1-3.3. Input curves are polylines with optional per-vertex
 * attributes. Each edge is clipped at the voxel faces in order of
 * occurrence; each pair of consecutive face points forms one linear segment
 * in the voxel between them, and the pieces before a curve's first and after
 * its last face point are dropped (Sec. 3.1). Face points are quantised to
 * the centres of an N x N subdivision of their face and encoded by a 3-bit
 * face id and the bin indices (Sec. 3.2). Segments are stored per voxel,
 * contiguously, behind an offset table (Sec. 3.3); within a voxel they are
 * ordered by (curve index, position along the curve).
 *
 * Grid transform: p = fl32(fl32(v - origin) * scale) per component; every
 * decision after that is exact integer arithmetic on round(p * 2^16).
 * Vertices must map to |p| < 2^14 voxels and be finite (else LVR_EINVAL).
 */
typedef struct lvr_grid_desc {
    int32_t res[3];      /* voxels per axis (each 1..4096, product < 2^32) */
    int32_t bins;        /* N, sub-squares per face edge: power of two, 2..128 */
    int32_t fit;         /* 1: fit the grid to the vertices' bounding box,
                            keeping its aspect ratio (Sec. 3.1): res[0] voxels
                            along the longest extent; origin, scale and the
                            other res[] are outputs written back here */
    float   origin[3];   /* world point mapped to grid coordinate 0 */
    float   scale;       /* grid units (voxels) per world unit, > 0 */
    float   attr_min;    /* attribute range mapped to 0..65535 (16-bit codes, */
    float   attr_max;    /*   one byte kept per segment); max <= min: all 0 */
} lvr_grid_desc;

/* xyz: host or device float32 [n_vertices * 3]; attr: host or device float32
 * [n_vertices] or NULL; curve_offsets: host or device int64 [n_curves + 1],
 * curve c = vertices [curve_offsets[c], curve_offsets[c+1]), starting at 0,
 * non-decreasing, ending at n_vertices. `grid` is read (and, in fit mode,
 * written). On success *out owns the voxel model. */
lvr_status lvr_voxelize(lvr_ctx *ctx, const float *xyz, const float *attr,
                        const int64_t *curve_offsets, int64_t n_curves, int64_t n_vertices,
                        lvr_grid_desc *grid, lvr_lineset **out);

typedef struct lvr_lineset_info {
    int32_t res[3];
    int32_t bins;
    float   origin[3];
    float   scale;
    int64_t n_voxels;
    int64_t n_segments;
    int64_t bytes;        /* device bytes held by the handle */
} lvr_lineset_info;
lvr_status lvr_lineset_info_get(const lvr_lineset *ls, lvr_lineset_info *info);

/* Decoded copy of the voxel model (for tests and tools). Any pointer may be
 * NULL. offset: uint32 [n_voxels + 1]; fields: uint8 [n_segments * 8] =
 * face_in, u_in, v_in, face_out, u_out, v_out, attribute byte, continues-
 * previous flag; curve, ordinal: uint32 [n_segments]. Host or device. */
lvr_status lvr_export_lineset(lvr_ctx *ctx, const lvr_lineset *ls, uint32_t *offset,
                              uint8_t *fields, uint32_t *curve, uint32_t *ordinal);
void lvr_free_lineset(lvr_lineset *ls);

/* ------------------------------------------------------------------ allocation-free voxelisation
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: code that runs where cudaMalloc is not
 * allowed or not wanted (a real-time loop with a fixed memory budget, a
 * host application whose allocator owns all device memory, a plug-in that
 * receives its buffers from the host program). It computes what
 * lvr_voxelize computes, into buffers the caller owns, and allocates
 * nothing: its temporary storage is one static device array of 16 MiB
 * plus 4 KiB, reserved on every GPU that loads the library until the
 * process exits, which limits grids to LVR_STATIC_MAX_VOXELS voxels
 * (128^3).
 *
 * All pointers are device pointers of the current device (host pointers or
 * another device's memory: LVR_EINVAL; nothing is staged). grid->fit must
 * be 0. offset: uint32 [voxels + 1]; records and
 * keys: uint64 [capacity] receive the segments, voxel-major and by (curve,
 * position along the curve) within a voxel. Record bits: 0-2 entry face
 * (0=-x,1=+x,2=-y,3=+y,4=-z,5=+z), 3-9 / 10-16 entry bins on the two other
 * axes in increasing axis order, 17-19 exit face, 20-26 / 27-33 exit bins,
 * 34-41 attribute byte, 42 continues-previous flag, 43-47 curve index mod
 * 32. Key = (curve << 32) | position along the curve. *n_segments receives
 * the segment count; if it exceeds `capacity` the call returns
 * LVR_EOVERFLOW after counting and writes no segments (retry with a larger
 * buffer). Work runs on `cuda_stream` (a cudaStream_t, NULL: legacy default
 * stream) of the current device; the call waits for the count.
 *
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream
 * capture. The address is kept for the process: after a cudaDeviceReset of
 * that device the library must be reloaded before this call is used again. Every call on a device shares the one array, which keeps the
 * previous call's contents (the call clears what must start at zero):
 * calls that overlap on the GPU (from several streams or host threads)
 * race and must be serialised by the caller. Errors are reported by the
 * status code only. */
#define LVR_STATIC_MAX_VOXELS 2097152u
lvr_status lvr_voxelize_static(const float *xyz, const float *attr, const int64_t *curve_offsets,
                               int64_t n_curves, int64_t n_vertices, const lvr_grid_desc *grid,
                               uint32_t *offset, uint64_t *records, uint64_t *keys, int64_t capacity,
                               int64_t *n_segments, void *cuda_stream);

/* ------------------------------------------------------------------ density LoD
 * Sec. 3.4, Eq. 1: per voxel rho = sum over its segments of length * sigma,
 * sigma = sigma256[attribute byte] (host float32 [256], the transfer
 * function's opacity); then 2^3 pooling into `levels` levels (1..4),
 * dims ceil(d / 2). Each level stores sums: segment count (uint32), summed
 * length and summed length * sigma (float32); the density sampled at level
 * l is dens_l / 8^l, the paper's 2^3 average. Beside them the renderer's
 * sampling copy: 32 bytes per cell of each level padded by 1-3 cells per
 * side (a level with 2^32 - 1 or more padded cells: LVR_EINVAL). */
lvr_status lvr_build_lod(lvr_ctx *ctx, const lvr_lineset *ls, int levels,
                         const float *sigma256, lvr_lod **out);
typedef struct lvr_lod_info {
    int32_t levels;
    int32_t dims[4][3];
} lvr_lod_info;
lvr_status lvr_lod_info_get(const lvr_lod *lod, lvr_lod_info *info);
/* Sec. 5.3's second AO approach: occlusion over the whole sphere around each
 * voxel centre, precomputed per voxel and interpolated at hits (ao_mode 3).
 * Directions: `rays` spherical Fibonacci directions over the sphere (z_i =
 * 1 - (2i+1)/rays, phi_i = i pi (3 - sqrt 5)); along each, the level-0
 * density (cell-centred trilinear, zero outside the grid) summed at unit
 * steps 1 .. floor(radius) until it reaches 1; field = 1 - mean min(1, O).
 * rays 1..4096, radius 1..64 voxels (the paper: 100 rays, radius 5). At a
 * hit the field is interpolated trilinearly between voxel centres,
 * coordinates clamped to them. Stored with the LoD (float32 per voxel). */
lvr_status lvr_lod_ao_field(lvr_ctx *ctx, lvr_lod *lod, int rays, float radius);
/* The field, host or device float32 [voxels]. */
lvr_status lvr_export_ao_field(lvr_ctx *ctx, const lvr_lod *lod, float *field);
/* Representative lines (Sec. 3.4) for every level of `lod`, built from the
 * line set it was built from (same grid; EINVAL otherwise) and stored with
 * the LoD. Level 0: per voxel, its segments in canonical order, each flipped
 * when its direction makes an obtuse angle with the running average line
 * (sum of end points minus sum of start points); start and end points are
 * averaged separately and each average is snapped to the nearest face of the
 * cell (ties: the lower face id, -x +x -y +y -z +z) and the bin of that face
 * holding its projection. Level l + 1: per cell, the lines of its 2^3
 * children (z, y, x order), averaged the same way. After each level, two
 * neighbours' end points on their shared face (a line's start point first
 * when both lie there) both move to the bin of their average,
 * floor((b1 + b2 + 1) / 2) per coordinate. Integer arithmetic throughout;
 * results are exact. Used by lvr_render with shadows 2 (Sec. 5.2, first
 * approach). */
lvr_status lvr_lod_rep_lines(lvr_ctx *ctx, lvr_lod *lod, const lvr_lineset *ls);
/* The lines of one level, host or device uint8 [cells][8]: byte 0 = 1 when
 * the cell has a line, bytes 1-3 face, u, v of its start point, bytes 4-6 of
 * its end point, byte 7 = 0 (bins of the line set's N x N face grid). */
lvr_status lvr_export_rep_lines(lvr_ctx *ctx, const lvr_lod *lod, int level, uint8_t *out8);
/* Copy one level out; any pointer may be NULL; host or device; each
 * dims[level] product elements. */
lvr_status lvr_export_lod(lvr_ctx *ctx, const lvr_lod *lod, int level, uint32_t *cnt,
                          float *len, float *dens);
void lvr_free_lod(lvr_lod *lod);

/* ------------------------------------------------------------------ saving and restoring
 * The paper has no counterpart: a voxel model, a density LoD and a learned-AO
 * model in training can be written out (lvr_export_lineset, lvr_export_lod,
 * lvr_ao_model_state) and restored later without re-running the voxeliser or
 * the trainer.
 *
 * lvr_import_lineset: a line set from the arrays lvr_export_lineset writes.
 * info: res, bins, origin, scale, n_voxels (= res product) and n_segments
 * (bytes is ignored); offset: uint32 [n_voxels + 1]; fields: uint8
 * [n_segments * 8] (face_in, u_in, v_in, face_out, u_out, v_out, attribute
 * byte, continues flag); curve, ordinal: uint32 [n_segments]; all host or
 * device, only read. The arrays are checked (offsets from 0, non-decreasing,
 * ending at n_segments; faces < 6, bins < N, flag 0 or 1; within a voxel
 * strictly increasing (curve, ordinal), the voxeliser's order):
 * LVR_EINVAL otherwise, with nothing kept. Synchronises the stream. */
lvr_status lvr_import_lineset(lvr_ctx *ctx, const lvr_lineset_info *info, const uint32_t *offset,
                              const uint8_t *fields, const uint32_t *curve, const uint32_t *ordinal,
                              lvr_lineset **out);
/* lvr_import_lod: a LoD of `levels` levels (1..4) over a grid of dims0
 * voxels (level l: ceil(dims0 / 2^l) cells) from the per-level arrays
 * lvr_export_lod writes: cnt[l] uint32, len[l] and dens[l] float32 (finite,
 * >= 0, else LVR_EINVAL), each host or device. It renders exactly as the LoD
 * it was exported from. Synchronises the stream. */
lvr_status lvr_import_lod(lvr_ctx *ctx, int levels, const int32_t dims0[3], const uint32_t *const *cnt,
                          const float *const *len, const float *const *dens, lvr_lod **out);

/* ------------------------------------------------------------------ record layouts
 * The ray caster reads each segment as the packed 8-byte record of the
 * voxelisation (LVR_LAYOUT_AOS8) or, after lvr_lineset_layout, as a 16-byte
 * record holding the entry and exit face points as six IEEE half floats and
 * the attribute byte (LVR_LAYOUT_AOS16): more bytes per record, no bit
 * decoding. Face points are (2 bin + 1) / (2 N), exact in half precision
 * for the power-of-two bin counts N <= 128 the voxeliser accepts, so both
 * layouts give bit-identical images. The paper stores only the packed form
 * (Sec. 6.2). */
#define LVR_LAYOUT_AOS8 0
#define LVR_LAYOUT_AOS16 1
lvr_status lvr_lineset_layout(lvr_ctx *ctx, lvr_lineset *ls, int layout);

/* ------------------------------------------------------------------ camera at rest
 * Neighbour lists for the camera-at-rest mode (render desc `still`, Sec.
 * 4.1): per voxel, every segment of its 3 x 3 x 3 neighbourhood (itself
 * included) that comes within the tube radius plus a rounding margin of
 * 1e-4 radius + 1e-5 of the voxel. A tube farther away cannot enter it, so
 * testing only these gives the image the search over all 26 neighbours
 * gives. Kept in the line set (8 bytes per entry plus
 * 4 per voxel) and used by every later lvr_render at rest with a radius up
 * to `radius`; lvr_render builds them itself when they are missing or were
 * built for a smaller radius. Returns LVR_EOVERFLOW (nothing kept) when the
 * lists would hold more than 2^32 - 1 entries. Synchronises the stream. */
lvr_status lvr_lineset_neighbours(lvr_ctx *ctx, lvr_lineset *ls, float radius);

/* ------------------------------------------------------------------ rendering
 * Secs. 4-5. One ray per pixel (pinhole camera, pixel centres, row 0 at the
 * top) is traversed through the grid by 3D-DDA; the segments stored in each
 * visited non-empty voxel are intersected as tubes of radius `radius`
 * closed by spheres at their end points (Sec. 4.1); a voxel keeps the hits
 * whose entry point lies inside it and sorts them by depth (Sec. 4). Each
 * hit is shaded at its entry point (ambient + diffuse with the tube normal,
 * Sec. 5) and blended front to back with the transfer function's opacity
 * until the accumulated opacity reaches `ert_alpha` (Sec. 5.1); opaque mode
 * keeps the first hit. Optional soft shadows march the density LoD toward
 * a directional light, sampling coarser levels with distance (Sec. 5.2),
 * or (shadows 2, Sec. 5.2's first approach) test a half-line toward the
 * light, started one cell of level shadow_level away from the hit, against
 * the representative lines of the cells of that level it crosses: visibility
 * 0 when one passes within radius x 2^level of it, else 1;
 * optional ambient occlusion marches `ao_rays` hemisphere rays around the
 * normal up to `ao_radius` voxels (Sec. 5.3). Output pixel =
 * (C + (1 - A) * bg, A).
 *
 * Primary rays are float32 quantities built by a fixed sequence of float32
 * operations from the camera (see the implementation); light and camera
 * basis vectors are computed in float64 and rounded to float32.
 */
typedef struct lvr_view {
    float   eye[3];        /* camera position, grid (voxel) coordinates */
    float   at[3];         /* look-at point */
    float   up[3];         /* up hint */
    float   fovy_deg;      /* vertical field of view */
    int32_t width, height; /* full image size */
    int32_t crop[4];       /* x0, y0, w, h of the rendered rectangle; w = 0: full image */
    float   light_dir[3];  /* direction in which the light travels */
} lvr_view;

typedef struct lvr_render_desc {
    float   radius;        /* tube radius, voxel units, > 0 */
    float   tf_rgba[1024]; /* transfer function: RGBA per attribute byte */
    int32_t opaque;        /* 1: alpha = 1, first hit only (Sec. 5) */
    float   ert_alpha;     /* early ray termination threshold (> 1: off) */
    int32_t shadows;       /* 0 off, 1 soft shadows (density-marched, needs a LoD),
                              2 hard shadows against the representative lines of LoD level
                              shadow_level (needs lvr_lod_rep_lines) */
    int32_t ao_mode;       /* 0 off, 1 traced (density-marched, needs a LoD),
                              2 learned surrogate (needs an lvr_ao_model),
                              3 spherical per-voxel field (needs lvr_lod_ao_field) */
    int32_t ao_rays;       /* hemisphere rays per hit, 1..32 (16 typical) */
    float   ao_radius;     /* radius of influence, voxels (15 typical) */
    float   ka, kd;        /* ambient / diffuse weights (0.3 / 0.7 typical) */
    float   bg[3];         /* background colour */
    int32_t tile_w, tile_h;/* ray tile of one warp: 8x4 (0,0 = default), 4x8, 16x2, 32x1 */
    int32_t layout;        /* segment records read by the ray caster: LVR_LAYOUT_AOS8 (packed,
                              default) or LVR_LAYOUT_AOS16 (needs lvr_lineset_layout) */
    int32_t still;         /* 1: camera at rest (Sec. 4.1): each visited voxel also tests the
                              segments of its 26 neighbours (a hit still belongs to the voxel
                              holding its entry point; no tube piece is missed for radii up to
                              half a voxel) and blends only the first hit of each 5-bit line id
                              (curve index mod 32) per voxel. Reads the line set's neighbour
                              lists (lvr_lineset_neighbours; built on first use, the one call
                              that then allocates and synchronises). Not with ao_mode 2 or
                              batches. */
    int32_t shadow_level;  /* shadows 2: LoD level whose representative lines cast shadows */
} lvr_render_desc;

/* rgba: host or device float32 [h * w * 4] for the crop rectangle (row-major,
 * row 0 = top of the crop). counters: NULL, or host or device uint64 [4]
 * receiving voxels visited, records tested (at rest: the neighbour-list
 * entries of the visited voxels), LoD trilinear samples (with shadows 2 plus
 * the representative-line cells tested) and
 * composited hits over the whole rectangle (costs one extra reduction).
 * `lod` may be NULL unless shadows or AO are on; `ao` may be NULL unless
 * ao_mode == 2, where the call evaluates the model's per-voxel layer-1 term
 * for `lod` once and caches it in the model (the model is therefore not
 * const; a model must not be used by two overlapping calls). */
lvr_status lvr_render(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod,
                      const lvr_view *view, const lvr_render_desc *desc,
                      lvr_ao_model *ao, float *rgba, uint64_t *counters);

/* ------------------------------------------------------------------ rasterised comparison system
 * The paper's baseline (Secs. 1 and 5.1): tubes around the input polylines
 * rasterised into per-pixel fragment lists, sorted by depth and blended front
 * to back; opaque tubes by a depth test. No voxel model is involved.
 * Vertex i of a curve maps to p_i = fl32(fl32(v - origin) * scale) (the
 * voxeliser's float32 step without the fixed-point snap; grid->fit must be
 * 0, res and bins are ignored); each pair of consecutive vertices of a curve
 * is a capsule of radius desc->radius (the tube piece closed by spheres) with
 * attribute byte floor(((A_i + A_i+1) 255 + 65535) / 131070) of the two
 * vertices' 16-bit codes (attr_min / attr_max as for lvr_voxelize). Pixel
 * (i, j)'s primary ray is lvr_render's; it leaves one fragment per capsule it
 * enters (entry > 0; an eye inside a capsule sees none of it). Fragments are
 * sorted by (depth, capsule index), shaded as lvr_render does without shadows
 * or AO (ka + kd |n . L|) and blended front to back with the transfer
 * function's opacity until the float32 accumulated opacity reaches
 * ert_alpha (> 1: every fragment, as fragment lists do); opaque mode shows
 * the nearest fragment (ties: the lower capsule index). desc->shadows,
 * ao_mode and still must be 0; tile and layout are ignored.
 * xyz, attr (or NULL), curve_offsets: host or device, as for lvr_voxelize;
 * rgba: host or device float32 [h * w * 4] of the crop; stats: NULL or host.
 * Synchronises with the stream (the fragment count sizes the lists); the
 * lists live in a grow-only buffer of the context. */
typedef struct lvr_raster_stats {
    uint64_t fragments;      /* fragments over the crop */
    uint64_t max_per_pixel;  /* longest per-pixel list (transparent mode) */
    uint64_t list_bytes;     /* bytes of the lists: 12 per fragment (0 in opaque mode) */
} lvr_raster_stats;
lvr_status lvr_raster(lvr_ctx *ctx, const float *xyz, const float *attr, const int64_t *curve_offsets,
                      int64_t n_curves, int64_t n_vertices, const lvr_grid_desc *grid, const lvr_view *view,
                      const lvr_render_desc *desc, float *rgba, lvr_raster_stats *stats);


/* ------------------------------------------------------------------ batched rendering
 * Many views, possibly of different line sets, sizes and tile shapes, in one
 * CUDA graph (the paper renders one view at a time): views that fill the GPU
 * on their own (at least 8 tiles per resident warp of the single-view
 * kernel) get a launch of their own in the graph, as lvr_render would launch
 * them; the others share one persistent launch whose work queue is the
 * concatenation of their 32-ray tiles, largest views first, each warp taking
 * the next tile from one device counter. The graph (those launches, the
 * counter reset and the queue's kernel) is captured once and replayed by
 * lvr_batch_render. Each view renders exactly as lvr_render would render it
 * alone (bit-identical output). All items share one kind of AO: either all
 * ao_mode 2 (learned) or all ao_mode 0/1, and one record layout; rgba must
 * be device memory [h][w][4] for the view's crop and stay valid while the
 * batch exists. Items' line sets, LoDs and models must outlive the batch;
 * learned models are bound to their LoDs at creation. */
typedef struct lvr_batch lvr_batch;
typedef struct lvr_batch_item {
    const lvr_lineset     *ls;
    const lvr_lod         *lod;     /* may be NULL unless shadows or AO are on */
    lvr_view               view;
    const lvr_render_desc *desc;
    lvr_ao_model          *ao;      /* ao_mode 2 only */
    float                 *rgba;    /* device float32 [h][w][4] */
} lvr_batch_item;
lvr_status lvr_batch_create(lvr_ctx *ctx, const lvr_batch_item *items, int n, lvr_batch **out);
/* Launches the captured graph on the context's stream (asynchronous). */
lvr_status lvr_batch_render(lvr_ctx *ctx, lvr_batch *b);
/* Total 32-ray tiles and rays of the batch. */
lvr_status lvr_batch_size(const lvr_batch *b, int64_t *tiles, int64_t *rays);
void lvr_free_batch(lvr_batch *b);

/* Autotuner: renders the items as a batch with every candidate ray tile
 * (8x4, 4x8, 16x2, 32x1) and record layout (AOS8, and AOS16 when every
 * line set has its 16-byte records), `reps` timed replays each after one
 * warm-up, and reports the fastest. Items' own tile and layout are ignored
 * during the search; outputs are overwritten. ms[c] is the mean time of
 * candidate c = layout * 4 + tile index, or -1 when not run. */
typedef struct lvr_tune {
    int32_t tile_w, tile_h, layout;
    float   ms[8];
} lvr_tune;
lvr_status lvr_autotune(lvr_ctx *ctx, const lvr_batch_item *items, int n, int reps, lvr_tune *out);

/* ------------------------------------------------------------------ learned ambient occlusion
 * The paper has no counterpart: a small network that predicts the traced
 * AO of Sec. 5.3 (ao_mode 1) at a hit, used by lvr_render with ao_mode 2
 * in place of the marched AO rays.
 *
 * Model: 400 inputs, three hidden layers of 64 with ReLU, one sigmoid
 * output. Per-hit inputs 0..14: the hit segment's unit direction (entry ->
 * exit) with its first non-zero component made positive (3), the unit
 * tube normal at the hit (3), and for l = 0, 1, 2 the hit point's offset
 * inside the level-l LoD cell of its voxel v, p / 2^l - floor(v / 2^l) -
 * 1/2 per axis (9); input 15 is zero. Per-voxel inputs 16..390: for l = 0,
 * 1, 2 the 5^3 level-l cells around v's cell (dz, dy, dx in -2..2, x
 * fastest), log1p(8 rho), rho = dens_l / 8^l the density the AO march
 * samples, zero outside the level; inputs 391..399 are zero. The LoD needs
 * at least 3 levels. Parameters: float32 [lvr_ao_nparams()] = W1 [64][400],
 * b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64], W4 [64], b4
 * (row-major [out][in]), used as bfloat16 (round to nearest even) in every
 * product, with bfloat16 inputs and hidden activations and float32 sums;
 * the per-voxel part of layer 1 is summed per voxel and rounded to
 * bfloat16 before the per-hit part and b1 are added. */
int lvr_ao_nparams(void);
/* params: host float32 [lvr_ao_nparams()], copied; must be finite. */
lvr_status lvr_ao_model_create(lvr_ctx *ctx, const float *params, lvr_ao_model **out);
/* Current parameters into host or device float32 [lvr_ao_nparams()]. */
lvr_status lvr_ao_model_params(lvr_ctx *ctx, const lvr_ao_model *m, float *params);
void lvr_free_ao_model(lvr_ao_model *m);

/* Model output for n hits: voxel int32 [n] (level-0 linear index
 * x + X (y + Y z), in [0, voxels): LVR_EINVAL otherwise when host memory is
 * given; NaN output for that hit when device memory is given), dir float32
 * [n][3] (segment direction, any length, normalised as d / sqrt(d.d) in
 * float32; zero gives a zero direction input), pos float32 [n][3] (hit
 * point, grid coordinates, inside the voxel), normal float32 [n][3] (unit),
 * ao float32 [n]. Host or device buffers. The same device code as the fused
 * inference in lvr_render. */
lvr_status lvr_ao_infer(lvr_ctx *ctx, lvr_ao_model *m, const lvr_lod *lod, int64_t n,
                        const int32_t *voxel, const float *dir, const float *pos,
                        const float *normal, float *ao);
/* The model inputs of n hits as bfloat16 bit patterns, X uint16 [n][400];
 * device buffers only; arguments as for lvr_ao_infer (a voxel id out of
 * range gives an all-zero row). */
lvr_status lvr_ao_features(lvr_ctx *ctx, const lvr_lod *lod, int64_t n, const int32_t *voxel,
                           const float *dir, const float *pos, const float *normal, uint16_t *X);
/* Training samples of one view with traced AO (desc's ao_rays, ao_radius,
 * radius, transfer function, opaque and ert_alpha; shadows and ao_mode are
 * ignored). Per pixel of the crop rectangle the ray is composited as usual
 * and the hit of index k = h(seed, pixel) mod depth along it (0 = first) is
 * recorded, if the ray reaches it: voxel int32 (-1: none), dir float32 [3]
 * (unit entry -> exit direction of the hit segment), ao float32 (traced AO
 * factor); optionally (both or neither may be NULL) pos float32 [3] (hit
 * point, grid coordinates) and normal float32 [3] (unit tube normal there).
 * h is the lowbias32 integer hash of seed ^ (pixel * 0x9e3779b9), pixel =
 * row * crop width + column. Device buffers. */
lvr_status lvr_ao_samples(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod,
                          const lvr_view *view, const lvr_render_desc *desc, int32_t depth,
                          uint32_t seed, int32_t *voxel, float *dir, float *ao, float *pos,
                          float *normal);

/* Learned against traced AO over every hit the image composites: renders
 * like lvr_render with ao_mode 2 (rgba may be NULL; host or device) and
 * also traces desc->ao_rays AO rays at each hit. Shadows are off. */
typedef struct lvr_ao_error {
    uint64_t hits;          /* composited hits */
    double   mean_abs;      /* mean |learned - traced| */
    double   p99_abs;       /* 99th percentile of |learned - traced|, upper edge of a 1/4096 bin */
    double   max_abs;
    double   mean_traced, mean_learned;
} lvr_ao_error;
lvr_status lvr_ao_judge(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod,
                        const lvr_view *view, const lvr_render_desc *desc, lvr_ao_model *ao,
                        float *rgba, lvr_ao_error *err);
/* Training checkpoint of a model trained with lvr_ao_train_step: its float32
 * parameters, Adam moments m and v (float32 [lvr_ao_nparams()] each; zero
 * before the first Adam step) and the number of Adam steps taken, into host
 * or device buffers (synchronises). lvr_ao_model_set_state puts such a state
 * into a model (parameters finite; the cached per-voxel terms are dropped):
 * training continued from it takes the same steps as training that never
 * stopped. */
lvr_status lvr_ao_model_state(lvr_ctx *ctx, const lvr_ao_model *m, float *params, float *adam_m, float *adam_v,
                              int64_t *step);
lvr_status lvr_ao_model_set_state(lvr_ctx *ctx, lvr_ao_model *m, const float *params, const float *adam_m,
                                  const float *adam_v, int64_t step);
/* One step on a batch of n rows (1..2^20; device X bf16 bits [n][400],
 * device y float32 [n]): forward, mean squared error, backward, and, if
 * lr > 0, one Adam update (beta 0.9 / 0.999, eps 1e-8, bias-corrected)
 * of the float32 masters. loss (host, may be NULL): the batch MSE before
 * the update. grads (host or device float32 [lvr_ao_nparams()], may be
 * NULL): d MSE / d parameter, computed with the bf16 operands of the
 * forward pass (straight-through rounding). */
lvr_status lvr_ao_train_step(lvr_ctx *ctx, lvr_ao_model *m, int64_t n, const uint16_t *X,
                             const float *y, float lr, float *loss, float *grads);

typedef struct lvr_ao_train_desc {
    int64_t  n_samples;    /* samples over all sets, split evenly (>= 64) */
    int32_t  epochs;       /* passes over the samples */
    int32_t  batch;        /* rows per Adam step, multiple of 64, <= 65536 */
    float    lr;           /* Adam step size */
    uint64_t seed;         /* initial weights and sampling views */
    int32_t  view_size;    /* square sampling views, pixels (8..4096) */
    int32_t  depth;        /* hit index range of the samples (lvr_ao_samples) */
    const lvr_render_desc *render;   /* sampling render: radius, TF, ERT, AO rays / radius */
} lvr_ao_train_desc;
/* Trains a model on traced AO: for each line set (with its LoD), seeded
 * orbit views (40 degree field of view, distance 1.8 x half the grid
 * diagonal) are sampled with lvr_ao_samples until the set's share of
 * samples is collected; their inputs are built, the weights initialised
 * uniformly in +-1/sqrt(fan_in) (zero for the padding inputs) and `epochs`
 * passes of minibatch Adam run over a per-epoch stride permutation of the
 * samples, the step size decaying from lr to 0 along a half cosine. *out
 * receives the model; final_mse (host, may be NULL) its mean squared error
 * over all samples (training forward pass). */
lvr_status lvr_train_ao(lvr_ctx *ctx, const lvr_lineset *const *sets, const lvr_lod *const *lods,
                        int nsets, const lvr_ao_train_desc *td, lvr_ao_model **out, float *final_mse);

/* ------------------------------------------------------------------ test hooks
 * For tests of the failure paths; not for production use. Every device
 * allocation the library makes goes through one allocator:
 * lvr_test_fail_allocation(n) makes the allocation after the next n ones
 * fail once with LVR_ENOMEM (n < 0: off), and lvr_test_live_allocations()
 * returns how many of the library's device allocations are held right now
 * (a call that fails must leave it where it was, apart from the context's
 * grow-only buffers). Process-wide; not thread-safe with other calls. */
void lvr_test_fail_allocation(int64_t n);
int64_t lvr_test_live_allocations(void);

#ifdef __cplusplus
}
#endif
#endif
