// Ray casting of the voxelised line set (Secs. 4, 5): 3D-DDA traversal,
// ray-capsule tests against each visited voxel's own segments, per-voxel hit
// sorting, local illumination, front-to-back compositing with early ray
// termination, and density-LoD marches for soft shadows and ambient
// occlusion.
//
// Execution. A persistent kernel: every warp pulls warp-sized pixel tiles
// (8x4 by default) from a device counter. Launches that read no traversal
// counters (MODE_IMAGE_NC) drop the counting and the AO march's support
// tests. Per tile the warp alternates two
// phases until all its rays are finished:
//   A. traversal (one ray per lane): DDA, capsule tests, per-voxel sort and
//      front-to-back weighting. The compositing weight of a hit depends only
//      on the opacities in front of it, never on its lighting, so each hit's
//      weight and position are final here; they go to the lane's
//      shared-memory hit slots (KS per lane) with the record index, from
//      which phase B derives the normal and tube direction (one lane per
//      hit there, where the traversal has few lanes on hits). The warp steps
//      its lanes voxel by voxel until it holds ROUND_TARGET hits, or every
//      lane is full or finished; a full lane resumes inside the same voxel in
//      the next round. Lighting in small rounds keeps lanes in dense regions
//      from idling while a lane in a sparse region looks for hits.
//   B. lighting (whole warp): the warp's collected hits are lit together:
//      their geometry and shadow rays one lane per hit; the AO rays of one
//      hit on a group of
//      adjacent lanes, which sample the same neighbourhood at the same
//      distances (good cache locality, little divergence), their occlusion
//      summed by a fixed butterfly. Each hit's lit contribution is written
//      back to its slot, and the owning lane adds its slots in depth order.
//
// Precision. All device arithmetic is float32. The primary ray is a float32
// quantity built by a fixed sequence of correctly rounded operations. The
// ray state is a voxel index plus a local position; for every non-empty
// voxel the local origin is recomputed from the global ray in float-float
// (error-free product and sum), so intersections are solved with operands of
// magnitude ~1. Tube and sphere entries are solved around the closest
// approach, which does not cancel.
//
// Ownership. A voxel keeps a hit iff its entry point lies inside the voxel
// (in local coordinates, in [0,1)^3). DDA ties step in axis order x, y, z.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "ao_mlp.cuh"
#include "geom.cuh"
#include "lvr_internal.cuh"

namespace {

constexpr int RT = 128;       // threads per block (4 warps)
constexpr int KS = 3;         // hit slots per lane per lighting round
constexpr unsigned ROUND_TARGET = 16;   // a warp lights its hits once it holds this many
constexpr int MAX_AO = 32;
constexpr unsigned FULL = 0xffffffffu;

struct RenderParams {
    const uint32_t *offset;
    const uint64_t *rec;
    const uint4 *rec16;           // expanded 16-byte records (layout LAYOUT_AOS16), or null
    int32_t res[3];
    float invN;
    float r2;
    int32_t levels;
    int32_t ldims[4][3];
    const float4 *pk[4];          // corner-packed levels (32-byte cells), padded to cover the support
    uint32_t pstr[4][2];          //   their row and slice strides in cells
    uint32_t pbias[4];            //   the floor's bit offset and the padding, folded (see corner_cell)
    uint32_t pzero[4];            //   index of the all-zero cell past the last
    float lod_lo, lod_hi[3];      // support of the density field (level-0 voxels)
    float F[3], R[3], U[3], th, tw, eye[3];
    int32_t W, H, x0, y0, cw, ch;
    int32_t tile_w, tile_h, tiles_x, ntiles;
    float Lt[3];                  // toward the light, unit
    int32_t opaque;
    float ert;
    int32_t shadows, ao, ao_rays, nrays;
    int32_t ao_fast;              // 3 levels, AO radius in [12, 16): the unrolled AO march
    float ao_radius, ka, kd, bg[3];
    float aod[MAX_AO][3];         // hemisphere directions in the (T, B, n) frame
    const float4 *gtf;            // the transfer function in global memory (read through L1)
    float4 *out;                  // may be null (sample mode)
    unsigned long long *counters;
    unsigned *tile_counter;
    // learned AO (ao_mode 2)
    int32_t learned;
    const float *aof;             // ao_mode 3: spherical per-voxel AO field (level-0 voxels), else null
    int32_t still;                // camera at rest: neighbouring voxels, one hit per line id
    const uint32_t *halo_off;     // camera at rest: per voxel its neighbour-list entries
    const uint64_t *halo;         //   (neighbour << 32) | record
    // shadows 2: representative lines of one LoD level (Sec. 5.2, first approach)
    const uint64_t *rep;
    int32_t rep_dims[3];
    float rep_size, rep_inv, rep_r2;
    aomlp::Net net;
    const __nv_bfloat16 *vterm;
    // sample mode: per pixel the hit of index `target` (hash of seed and
    // pixel, mod depth) along the composited ray: voxel (-1: none), segment
    // direction, traced AO
    int32_t *samp_vox;
    float *samp_dir, *samp_ao;
    float *samp_pos, *samp_nrm;   // optional: hit point (grid coordinates), unit normal
    uint32_t samp_seed;
    int32_t samp_depth;
    // judge mode: learned vs traced AO statistics (see lvr_ao_judge)
    unsigned long long *judge;    // [4]: hits, sum |e|, sum traced, sum learned (x 2^32)
    unsigned *judge_max;          // max |e| as float bits
    unsigned *judge_hist;         // [JH] histogram of |e|
    // transfer function: RGBA per attribute byte (last: batched views copy
    // only the fields before it into shared memory). The kernels read it
    // through gtf: a single view's device copy written by the prep kernel,
    // or a queued view's copy inside the batch's item array.
    alignas(16) float tf[1024];
};
constexpr int HOT_BYTES = (int)((offsetof(RenderParams, tf) + 15) & ~(size_t)15);   // fields before tf

struct Vec { float x, y, z; };
__device__ __forceinline__ Vec mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ Vec sub(Vec a, Vec b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ float dot(Vec a, Vec b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ Vec cross(Vec a, Vec b) {
    return {fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x)};
}
__device__ __forceinline__ Vec axpy(float s, Vec d, Vec p) {
    return {fmaf(s, d.x, p.x), fmaf(s, d.y, p.y), fmaf(s, d.z, p.z)};
}
__device__ __forceinline__ Vec scale(Vec a, float s) { return {a.x * s, a.y * s, a.z * s}; }

// Face point (Sec. 3.2): face id -> axis and side, bins -> sub-square centres.
__device__ __forceinline__ Vec face_point(uint32_t face, uint32_t u, uint32_t v, float invN) {
    const uint32_t ax = face >> 1;
    const float side = (face & 1u) ? 1.0f : 0.0f;
    const float cu = ((float)u + 0.5f) * invN, cv = ((float)v + 0.5f) * invN;
    return {ax == 0 ? side : cu, ax == 1 ? side : (ax == 0 ? cu : cv), ax == 2 ? side : cv};
}

// Camera at rest: rounding margin of the neighbour lists' box cull: sqrt(r2) x (1 + 1e-4) + 1e-5.
__device__ __forceinline__ float cull_margin(float r2) { return sqrtf(r2) * 1.0001f + 1e-5f; }

// Neighbour `nc` (0..26, x fastest) of a voxel as an offset in voxels.
__device__ __forceinline__ Vec neighbour_offset(uint32_t nc) {
    return mk((float)((int)(nc % 3u) - 1), (float)((int)((nc / 3u) % 3u) - 1), (float)((int)(nc / 9u) - 1));
}

// First entry of ray p + s D into the sphere |x - c| = r; INF if none.
// Closest-approach form: the squared distance of the centre from the ray is
// taken from the perpendicular vector itself, which does not cancel.
__device__ __forceinline__ float sphere_entry(Vec p, Vec D, Vec c, float r2) {
    const Vec oc = sub(p, c);
    const float sc = -dot(oc, D);
    const Vec q = axpy(sc, D, oc);
    const float d2 = dot(q, q);
    return d2 > r2 ? INFINITY : sc - sqrtf(r2 - d2);
}

// First entry of ray p + s D into the capsule of radius sqrt(r2) around
// [a, b] (INF if none). The capsule is convex: its entry is the lateral entry
// into the infinite cylinder when that point lies between the end planes,
// otherwise the earlier of the two end-sphere entries. The lateral entry is
// solved in closest-approach form in the plane normal to the axis: closest
// approach parameter sc, perpendicular offset q, half chord
// sqrt((r^2 - |q|^2) / |D_perp|^2).
// The early reject of capsule_entry below as a predicate of its own: the
// record loops branch once around the whole test for the records it rejects
// (most of them), with the same decision as capsule_entry's own.
__device__ __forceinline__ bool capsule_rejects(Vec p, Vec D, Vec a, Vec b, float r2) {
    const Vec ba = sub(b, a);
    const float L2 = dot(ba, ba);
    const Vec c = cross(D, ba);
    const float c2 = dot(c, c);
    const float wc = dot(sub(a, p), c);
    return c2 > 1e-4f * L2 && wc * wc > 1.001f * r2 * c2;
}
__device__ __forceinline__ float capsule_entry(Vec p, Vec D, Vec a, Vec b, float r2) {
    const Vec ba = sub(b, a);
    const float L2 = dot(ba, ba);
    // Early reject: every point of the capsule lies within the radius of the
    // axis line, so a ray whose line passes farther from it misses. The
    // squared line distance is (w . c)^2 / |c|^2 with w = a - p, c = D x ba;
    // rejecting only beyond 1.001 r^2, and only when the lines are not
    // near-parallel (|c|^2 > 1e-4 L2, so c has a small relative error), keeps
    // every capsule the full test below accepts.
    const Vec c = cross(D, ba);
    const float c2 = dot(c, c);
    if (c2 > 1e-4f * L2) {
        const float wc = dot(sub(a, p), c);
        if (wc * wc > 1.001f * r2 * c2) return INFINITY;
    }
    if (L2 > 0.0f) {
        const float L = sqrtf(L2), iL = 1.0f / L;
        const Vec w = scale(ba, iL);
        const Vec oa = sub(p, a);
        const float dw = dot(D, w), ow = dot(oa, w);
        const Vec Dp = axpy(-dw, w, D), Op = axpy(-ow, w, oa);
        const float A = dot(Dp, Dp);
        if (A > 1e-12f) {
            const float sc = -dot(Dp, Op) / A;
            const Vec q = axpy(sc, Dp, Op);
            const float d2 = dot(q, q);
            if (d2 > r2) return INFINITY;              // misses the infinite cylinder
            const float t = sc - sqrtf((r2 - d2) / A);
            const float y = fmaf(t, dw, ow);
            if (y > 0.0f && y < L) return t;
        } else if (dot(Op, Op) > r2) {
            return INFINITY;
        }
        return fminf(sphere_entry(p, D, a, r2), sphere_entry(p, D, b, r2));
    }
    return sphere_entry(p, D, a, r2);
}

// Cell-centred trilinear density at level l, zero outside the grid: one
// 32-byte load of the corner-packed level (the x/y corners of slices iz and
// iz + 1, x differences precomputed), the same lerps in the same order as
// eight scalar corner loads would feed. The packed copy is padded to cover
// the support of the density field, so a point inside the support (which
// every caller checks) needs no range check.
//
// The cell is found without a conversion instruction: for |q| < 2^22,
// q + 1.5 * 2^23 rounded toward -infinity is the integer 1.5 * 2^23 +
// floor(q) exactly, and its bit pattern is 0x4B400000 + floor(q); the
// padded cell index is then a 32-bit sum of the three bit patterns times
// the strides, less a per-level constant (pbias) that removes the offsets
// and adds the padding. Subtracting the rounded sum back gives floor(q) as
// a float, so the fractions are q - floor(q), as with floorf.
constexpr float FLOOR_MAGIC = 12582912.0f;   // 1.5 * 2^23
__device__ __forceinline__ uint32_t corner_cell(const RenderParams &P, int l, Vec x, float &fx, float &fy,
                                                float &fz) {
    const float inv = __int_as_float((127 - l) << 23);         // 2^-l
    const float qx = fmaf(x.x, inv, -0.5f), qy = fmaf(x.y, inv, -0.5f), qz = fmaf(x.z, inv, -0.5f);
    const float tx = __fadd_rd(qx, FLOOR_MAGIC), ty = __fadd_rd(qy, FLOOR_MAGIC), tz = __fadd_rd(qz, FLOOR_MAGIC);
    fx = qx - (tx - FLOOR_MAGIC);
    fy = qy - (ty - FLOOR_MAGIC);
    fz = qz - (tz - FLOOR_MAGIC);
    return __float_as_uint(tx) + P.pstr[l][0] * __float_as_uint(ty) + P.pstr[l][1] * __float_as_uint(tz) -
           P.pbias[l];
}
// Cell i of level l (a: slice iz, b: slice iz + 1): two 16-byte loads at
// one address (two 16-byte loads issue faster here than one 32-byte load),
// marked to stay in L1 over the records and offsets the traversal streams
// through (the AO rays of nearby hits sample the same cells). The cell past
// the last (index pzero) is all zeros, the stand-in for a sample that is not
// taken.
__device__ __forceinline__ void load_cell(const RenderParams &P, int l, uint32_t i, float4 &a, float4 &b) {
    const float4 *c = P.pk[l] + 2 * (size_t)i;
    asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w)
        : "l"(c));
    asm("ld.global.nc.L1::evict_last.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(c + 1));
}
__device__ __forceinline__ float trilerp(float4 a, float4 b, float fx, float fy, float fz) {
    const float x00 = fmaf(fx, a.y, a.x), x10 = fmaf(fx, a.w, a.z);
    const float x01 = fmaf(fx, b.y, b.x), x11 = fmaf(fx, b.w, b.z);
    const float y0 = fmaf(fy, x10 - x00, x00), y1 = fmaf(fy, x11 - x01, x01);
    return fmaf(fz, y1 - y0, y0);
}
__device__ __forceinline__ float sample_level(const RenderParams &P, int l, Vec x) {
    float fx, fy, fz;
    float4 a, b;
    load_cell(P, l, corner_cell(P, l, x, fx, fy, fz), a, b);
    return trilerp(a, b, fx, fy, fz);
}

// Spherical AO field at x: cell-centred trilinear, coordinates clamped to
// the voxel centres (edge values hold outside).
__device__ __forceinline__ float sample_field(const RenderParams &P, Vec x) {
    const float xs[3] = {x.x, x.y, x.z};
    int i0[3], i1[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int d = P.ldims[0][a];
        const float q = fminf(fmaxf(xs[a] - 0.5f, 0.0f), (float)(d - 1));
        int fl = (int)floorf(q);
        if (fl > d - 2) fl = d - 2 < 0 ? 0 : d - 2;
        i0[a] = fl;
        i1[a] = fl + 1 < d ? fl + 1 : d - 1;
        f[a] = q - (float)fl;
    }
    const int dx = P.ldims[0][0], dy = P.ldims[0][1];
    auto at = [&](int X, int Y, int Z) { return __ldg(P.aof + (X + (int64_t)dx * (Y + (int64_t)dy * Z))); };
    const float x00 = fmaf(f[0], at(i1[0], i0[1], i0[2]) - at(i0[0], i0[1], i0[2]), at(i0[0], i0[1], i0[2]));
    const float x10 = fmaf(f[0], at(i1[0], i1[1], i0[2]) - at(i0[0], i1[1], i0[2]), at(i0[0], i1[1], i0[2]));
    const float x01 = fmaf(f[0], at(i1[0], i0[1], i1[2]) - at(i0[0], i0[1], i1[2]), at(i0[0], i0[1], i1[2]));
    const float x11 = fmaf(f[0], at(i1[0], i1[1], i1[2]) - at(i0[0], i1[1], i1[2]), at(i0[0], i1[1], i1[2]));
    const float y0 = fmaf(f[1], x10 - x00, x00), y1 = fmaf(f[1], x11 - x01, x01);
    return fmaf(f[2], y1 - y0, y0);
}

// A voxel owns a hit iff the entry point p + t D lies in its [0,1)^3 and in
// front of the ray's start (t > tmin).
__device__ __forceinline__ bool owned(Vec p, Vec D, float t, float tmin) {
    if (!(t < INFINITY) || !(t > tmin)) return false;
    const float x = fmaf(t, D.x, p.x), y = fmaf(t, D.y, p.y), z = fmaf(t, D.z, p.z);
    return x >= 0.0f && x < 1.0f && y >= 0.0f && y < 1.0f && z >= 0.0f && z < 1.0f;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ bool key_after(float t, uint32_t k, float lt, uint32_t lk) {
    return t > lt || (t == lt && k > lk);
}

// Kernel variants: image with traced or no AO; image with learned AO; hit
// samples (voxel, direction, traced AO) for the learned-AO trainer; image with
// learned AO that also traces AO at every hit and records the difference;
// image with the camera at rest (neighbouring voxels' segments, line ids).
// MODE_REP: the image mode with hard shadows against representative lines,
// a variant of its own so that the walk's registers do not weigh on the
// other image kernels
// MODE_IMAGE_NC is the image variant for launches that read no counters
// (the compiler drops the counting, and the AO march its support tests).
enum { MODE_IMAGE = 0, MODE_LEARNED = 1, MODE_SAMPLES = 2, MODE_JUDGE = 3, MODE_STILL = 4, MODE_REP = 5,
       MODE_IMAGE_NC = 6 };
constexpr int JH = 4096;          // judge histogram bins over |e| in [0, 1]

// Shared memory of one block: transfer function, per-lane sorted hit staging
// and per-lane hit slots (field-major, lane-minor: conflict-free). The hit's
// voxel id (last field) is kept only by the variants that need it, so the
// image variant stays within six resident blocks per SM.
enum { F_PX, F_PY, F_PZ, F_NX, F_NY, F_NZ, F_UX, F_UY, F_UZ, F_CR, F_CG, F_CB, F_AO, F_V, F_VID, NF };
// End points and attribute of record k in the given layout.
// `attr` receives the attribute byte in bits 0-7 and the 5-bit line id in bits 8-12.
template <int LAYOUT>
__device__ __forceinline__ void fetch_record(const RenderParams &P, uint32_t k, Vec &a, Vec &b, uint32_t &attr) {
    if constexpr (LAYOUT == 1) {
        const uint4 q = __ldg(P.rec16 + k);
        const __half2 h0 = *reinterpret_cast<const __half2 *>(&q.x), h1 = *reinterpret_cast<const __half2 *>(&q.y),
                      h2 = *reinterpret_cast<const __half2 *>(&q.z);
        a = mk(__low2float(h0), __high2float(h0), __low2float(h1));
        b = mk(__high2float(h1), __low2float(h2), __high2float(h2));
        attr = q.w;
    } else {
        const uint64_t r = __ldg(P.rec + k);
        a = face_point(rec_face_in(r), rec_u_in(r), rec_v_in(r), P.invN);
        b = face_point(rec_face_out(r), rec_u_out(r), rec_v_out(r), P.invN);
        attr = rec_attr(r) | (rec_line_id(r) << 8);
    }
}

// Hit geometry at the local entry point Pl on the tube around [a, b] (Sec. 5,
// reading S1): the unit normal n = Pl minus its closest point on the segment,
// and the unit tube direction u (zero for a point segment).
__device__ __forceinline__ void hit_geometry(Vec Pl, Vec a, Vec b, Vec &n, Vec &u) {
    const Vec ba = sub(b, a);
    const float L2 = dot(ba, ba);
    float h = 0.0f;
    u = mk(0.0f, 0.0f, 0.0f);
    if (L2 > 0.0f) {
        h = fminf(fmaxf(dot(sub(Pl, a), ba) / L2, 0.0f), 1.0f);
        u = scale(ba, 1.0f / sqrtf(L2));
    }
    n = sub(Pl, axpy(h, ba, a));
    n = scale(n, rsqrtf(dot(n, n)));
}

// Record layouts: the packed 8-byte record, or 16 bytes with the end points
// as six half floats (exact for power-of-two bin counts) and the attribute.
enum { LAYOUT_AOS8 = 0, LAYOUT_AOS16 = 1 };

template <int MODE, int LAYOUT, bool BATCH>
struct Smem {
    static constexpr int kMode = MODE;
    static constexpr int kLayout = LAYOUT;
    static constexpr bool kBatch = BATCH;   // the transfer function is read from global memory
    static constexpr bool kVid = MODE != MODE_IMAGE && MODE != MODE_IMAGE_NC && MODE != MODE_STILL && MODE != MODE_REP;
    static constexpr bool kStill = MODE == MODE_STILL;
    // the per-hit geometry (normal, tube direction) waits for the lighting
    // phase, where one lane takes one hit: the traversal stores the local
    // hit point in the normal's fields and the record index in the
    // direction's (at rest the record's neighbour offset would be needed
    // too, so that variant computes the geometry where it finds the hit)
    static constexpr bool kDefer = MODE != MODE_STILL;
    // one view with traced AO: the AO directions (lanes read different ones,
    // which the constant bank would serialise); batched views read them from
    // `hot`
    static constexpr bool kAod = !BATCH && MODE != MODE_LEARNED;
    float aod[kAod ? MAX_AO * 3 : 1];
    float4 hot[BATCH ? 4 : 1][BATCH ? HOT_BYTES / 16 : 1];   // batched: each warp's current view parameters
    // the staged (t, k) of each lane's current voxel, ascending: slot-major,
    // lane-minor columns; the single-view learned variant keeps them per
    // warp, because they are dead while a warp lights its hits and it
    // overlays the warp's activation tile on its own entries
    static constexpr bool kActTile = MODE == MODE_LEARNED;
    struct ColStage {
        float st[KS][RT];
        uint32_t sk[KS][RT];
    };
    struct WarpStage {
        union {
            struct {
                float st[KS][32];
                uint32_t sk[KS][32];
            };
            __align__(16) uint8_t act[aomlp::ACT_BYTES];
        };
    };
    std::conditional_t<kActTile, WarpStage[RT / 32], ColStage> stage;
    __device__ __forceinline__ float &st_(int q, int tid) {
        if constexpr (kActTile) return stage[tid >> 5].st[q][tid & 31];
        else return stage.st[q][tid];
    }
    __device__ __forceinline__ uint32_t &sk_(int q, int tid) {
        if constexpr (kActTile) return stage[tid >> 5].sk[q][tid & 31];
        else return stage.sk[q][tid];
    }
    // 32 words of warp `warp`'s staging entries (slot 0 of its lanes)
    __device__ __forceinline__ uint32_t *warp_words(int warp) { return reinterpret_cast<uint32_t *>(&st_(0, warp * 32)); }
    uint16_t sa[MODE == MODE_STILL ? KS : 1][MODE == MODE_STILL ? RT : 2];   // at rest: (line id << 5) | neighbour
    float slot[kVid ? NF : NF - 1][KS][RT];
    uint8_t item[4][32 * KS];     // per warp: (owner lane, slot) of each collected hit
    // judge and batched learned variant, per warp: per-hit inputs of 16 hits
    __align__(16) __nv_bfloat16 hin[MODE == MODE_JUDGE ? 4 * 16 * aomlp::HIN_STRIDE : 8];
};

struct Ray {
    Vec D;
    float invD[3];
    int v[3];
    float pl[3];
    float T;                      // ray parameter at the current voxel's entry
    float A, Cr, Cg, Cb;
    float rt;                     // resume key inside the current voxel
    uint32_t rk;
    bool resume;
    bool done;
    int hidx, target;             // sample mode: index of the next hit, index to record
    uint32_t idmask;              // camera at rest: line ids blended at the current voxel
};

// Phase A for one lane: traverse until KS hits are collected or the ray ends.
template <class SM>
__device__ __forceinline__ void voxel_step(const RenderParams &P, SM &sm, Ray &ray, int tid, unsigned &nvox,
                                           unsigned &nrec, unsigned &nhit, int &used) {
    const float Da[3] = {ray.D.x, ray.D.y, ray.D.z};
    do {
        // exit distance per axis, (face - pl) / D with the face at 1 for
        // D > 0 and at 0 for D < 0; an axis with D = 0 has 1 / D = inf, face
        // 1 and pl 0 (set at the ray's start), so its exit is inf
        float se = ((ray.invD[0] < 0.0f ? 0.0f : 1.0f) - ray.pl[0]) * ray.invD[0];
        int ax = 0;
#pragma unroll
        for (int a = 1; a < 3; a++) {
            const float e = ((ray.invD[a] < 0.0f ? 0.0f : 1.0f) - ray.pl[a]) * ray.invD[a];
            if (e < se) { se = e; ax = a; }
        }
        se = fmaxf(se, 0.0f);
        const uint32_t vid = (uint32_t)ray.v[0] + (uint32_t)P.res[0] * ((uint32_t)ray.v[1] + (uint32_t)P.res[1] * (uint32_t)ray.v[2]);
        // with the camera at rest (reading R2) the candidates are the voxel's
        // neighbour list: its own records and its neighbours' that reach into it
        const uint32_t *const offs = SM::kStill ? P.halo_off : P.offset;
        const uint32_t beg = __ldg(offs + vid), end = __ldg(offs + vid + 1);
        if (!ray.resume) {
            nvox++;
            nrec += end - beg;
        }
        if (end > beg) {
            // accurate local origin: eye + T D - v in float-float, rounded once
            float po[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float ph = __fmul_rn(ray.T, Da[a]);
                const float pe = __fmaf_rn(ray.T, Da[a], -ph);
                float sh, s2;
                two_sum(P.eye[a], ph, sh, s2);
                po[a] = __fadd_rn(__fsub_rn(sh, (float)ray.v[a]), __fadd_rn(s2, pe));
            }
            const Vec p = mk(po[0], po[1], po[2]);
            const int room = KS - used;
            int nh = 0;
            // stage one candidate: keep the `room` smallest (t, k), ascending;
            // at rest also only the smallest of each line id
            auto stage = [&](float t, uint32_t k, uint32_t aux) {
                if (!owned(p, ray.D, t, -ray.T)) return;
                if (ray.resume && !key_after(t, k, ray.rt, ray.rk)) return;
                if constexpr (SM::kStill) {
                    const uint32_t id = aux >> 5;
                    if ((ray.idmask >> id) & 1u) return;            // blended earlier at this voxel
                    int ns = nh < room ? nh : room;
                    for (int j = 0; j < ns; j++) {
                        if ((uint32_t)(sm.sa[j][tid] >> 5) != id) continue;
                        if (!key_after(sm.st_(j, tid), sm.sk_(j, tid), t, k)) return;   // staged one is first
                        for (int q = j; q + 1 < ns; q++) {                            // drop the staged one
                            sm.st_(q, tid) = sm.st_(q + 1, tid);
                            sm.sk_(q, tid) = sm.sk_(q + 1, tid);
                            sm.sa[q][tid] = sm.sa[q + 1][tid];
                        }
                        nh--;
                        break;
                    }
                }
                if (nh < room || t < sm.st_(room - 1, tid)) {
                    int q = nh < room ? nh : room - 1;
                    while (q > 0 && t < sm.st_(q - 1, tid)) {
                        sm.st_(q, tid) = sm.st_(q - 1, tid);
                        sm.sk_(q, tid) = sm.sk_(q - 1, tid);
                        if constexpr (SM::kStill) sm.sa[q][tid] = sm.sa[q - 1][tid];
                        q--;
                    }
                    sm.st_(q, tid) = t;
                    sm.sk_(q, tid) = k;
                    if constexpr (SM::kStill) sm.sa[q][tid] = (uint16_t)aux;
                }
                nh++;
            };
            if constexpr (SM::kStill) {
                for (uint32_t j = beg; j < end; j++) {
                    const uint64_t e = __ldg(P.halo + j);
                    const uint32_t k = (uint32_t)e, nc = (uint32_t)(e >> 32);
                    Vec a, b;
                    uint32_t attr;
                    fetch_record<SM::kLayout>(P, k, a, b, attr);
                    // the neighbour's face points in this voxel's frame (exact: binary fractions + integers)
                    const Vec o = neighbour_offset(nc);
                    a = mk(a.x + o.x, a.y + o.y, a.z + o.z);
                    b = mk(b.x + o.x, b.y + o.y, b.z + o.z);
                    if (capsule_rejects(p, ray.D, a, b, P.r2)) continue;
                    stage(capsule_entry(p, ray.D, a, b, P.r2), k, ((attr >> 8) << 5) | nc);
                }
            } else {
                for (uint32_t k = beg; k < end; k++) {
                    Vec a, b;
                    uint32_t attr;
                    fetch_record<SM::kLayout>(P, k, a, b, attr);
                    if (capsule_rejects(p, ray.D, a, b, P.r2)) continue;
                    stage(capsule_entry(p, ray.D, a, b, P.r2), k, 0u);
                }
            }
            const int take = nh < room ? nh : room;
            for (int q = 0; q < take; q++) {
                const float t = sm.st_(q, tid);
                const uint32_t k = sm.sk_(q, tid);
                Vec a, b;
                uint32_t attr;
                fetch_record<SM::kLayout>(P, k, a, b, attr);
                if constexpr (SM::kStill) {
                    const Vec o = neighbour_offset(sm.sa[q][tid] & 31u);
                    a = mk(a.x + o.x, a.y + o.y, a.z + o.z);
                    b = mk(b.x + o.x, b.y + o.y, b.z + o.z);
                    ray.idmask |= 1u << (attr >> 8);
                }
                attr &= 0xffu;
                const Vec Pl = axpy(t, ray.D, p);
                const float4 c = __ldg(P.gtf + attr);
                // front-to-back weight (Sec. 5.1); the opacity update is rounded
                // step by step so the termination test is reproducible:
                // A <- A + (1 - A) * alpha
                float w;
                if (P.opaque) {
                    w = 1.0f;
                    ray.A = 1.0f;
                    ray.done = true;
                } else {
                    w = __fmul_rn(__fsub_rn(1.0f, ray.A), c.w);
                    ray.A = __fadd_rn(ray.A, w);
                    if (ray.A >= P.ert) ray.done = true;
                }
                bool store = true;
                if constexpr (SM::kMode == MODE_SAMPLES) {   // only the target hit, then stop
                    store = ray.hidx == ray.target;
                    ray.hidx++;
                    if (store) ray.done = true;
                }
                if (P.nrays == 0) {
                    Vec n, u;
                    hit_geometry(Pl, a, b, n, u);
                    const Vec Lt = mk(P.Lt[0], P.Lt[1], P.Lt[2]);
                    const float kk = fmaf(P.kd, fabsf(dot(n, Lt)), P.ka);
                    ray.Cr = fmaf(w * c.x, kk, ray.Cr);
                    ray.Cg = fmaf(w * c.y, kk, ray.Cg);
                    ray.Cb = fmaf(w * c.z, kk, ray.Cb);
                } else if (store) {
                    sm.slot[F_PX][used][tid] = (float)ray.v[0] + Pl.x;
                    sm.slot[F_PY][used][tid] = (float)ray.v[1] + Pl.y;
                    sm.slot[F_PZ][used][tid] = (float)ray.v[2] + Pl.z;
                    if constexpr (SM::kDefer) {
                        sm.slot[F_NX][used][tid] = Pl.x;
                        sm.slot[F_NY][used][tid] = Pl.y;
                        sm.slot[F_NZ][used][tid] = Pl.z;
                        sm.slot[F_UX][used][tid] = __uint_as_float(k);
                    } else {
                        Vec n, u;
                        hit_geometry(Pl, a, b, n, u);
                        sm.slot[F_NX][used][tid] = n.x;
                        sm.slot[F_NY][used][tid] = n.y;
                        sm.slot[F_NZ][used][tid] = n.z;
                        sm.slot[F_UX][used][tid] = u.x;
                        sm.slot[F_UY][used][tid] = u.y;
                        sm.slot[F_UZ][used][tid] = u.z;
                    }
                    if constexpr (SM::kVid) sm.slot[F_VID][used][tid] = __uint_as_float(vid);
                    sm.slot[F_CR][used][tid] = w * c.x;
                    sm.slot[F_CG][used][tid] = w * c.y;
                    sm.slot[F_CB][used][tid] = w * c.z;
                    used++;
                }
                ray.rt = t;
                ray.rk = k;
                nhit++;
                if (ray.done) break;
            }
            if (ray.done) break;
            if (take < nh) {              // slots full inside this voxel: resume here
                ray.resume = true;
                break;
            }
        }
        ray.resume = false;
        ray.idmask = 0u;
        // step into the neighbour across face `ax`
        ray.T = __fadd_rn(ray.T, se);
#pragma unroll
        for (int a = 0; a < 3; a++) ray.pl[a] = fmaf(se, Da[a], ray.pl[a]);
#pragma unroll
        for (int a = 0; a < 3; a++) {       // constant indices keep the state in registers
            if (a != ax) continue;
            const int sg = Da[a] > 0.0f ? 1 : -1;
            ray.v[a] += sg;
            ray.pl[a] = sg > 0 ? 0.0f : 1.0f;
            if (ray.v[a] < 0 || ray.v[a] >= P.res[a]) ray.done = true;
        }
    } while (false);
}

template <class SM>
__device__ int traverse(const RenderParams &P, SM &sm, Ray &ray, int tid, unsigned &nvox, unsigned &nrec,
                        unsigned &nhit) {
    int used = 0;
    if (P.nrays == 0) {
        while (!ray.done) voxel_step(P, sm, ray, tid, nvox, nrec, nhit, used);
        return 0;
    }
    for (;;) {
        if (!ray.done && used < KS) voxel_step(P, sm, ray, tid, nvox, nrec, nhit, used);
        const unsigned tot = __reduce_add_sync(FULL, (unsigned)used);
        if (tot >= ROUND_TARGET || __all_sync(FULL, ray.done || used >= KS)) break;
    }
    return used;
}

// Hit frame for the AO hemisphere (reading S3): tangent = tube direction
// projected onto the tangent plane; fallback: the world axis least aligned
// with n.
__device__ __forceinline__ Vec ao_tangent(Vec n, Vec u) {
    const float un = dot(u, n);
    Vec T = axpy(-un, n, u);
    const float m = sqrtf(dot(T, T));
    if (m >= 1e-3f) return scale(T, 1.0f / m);
    const float ax = fabsf(n.x), ay = fabsf(n.y), az = fabsf(n.z);
    int e = 0;
    float best = ax;
    if (ay < best) { e = 1; best = ay; }
    if (az < best) { e = 2; }
    const float ne = e == 0 ? n.x : (e == 1 ? n.y : n.z);
    T = mk((e == 0 ? 1.0f : 0.0f) - ne * n.x, (e == 1 ? 1.0f : 0.0f) - ne * n.y, (e == 2 ? 1.0f : 0.0f) - ne * n.z);
    return scale(T, rsqrtf(dot(T, T)));
}

// Density march (Secs. 5.2, 5.3, readings S2 / S3): samples at s = 1, 2, 4,
// ... with step 2^l at level l = floor(log2 s) (capped); O += rho_l * 2^l
// with rho_l = dens_l / 8^l; the ray ends at O >= 1, beyond max_dist (if
// >= 0), or when the sample leaves the support of the density field.
// The march of an AO ray with 3 levels and a radius in [12, 16): the
// samples fall at s = 1, 2, 4, 8, 12 (levels 0, 1, 2, 2, 2), unrolled; the
// same samples, weights and sample count as march(), and the same
// min(1, O).
__device__ __forceinline__ bool in_support(const RenderParams &P, const Vec &x) {
    return !(x.x < P.lod_lo || x.y < P.lod_lo || x.z < P.lod_lo || x.x > P.lod_hi[0] || x.y > P.lod_hi[1] ||
             x.z > P.lod_hi[2]);
}
// Without counting (CNT false) the support tests are left out: the copy of
// the coarsest level is padded to hold every point within 12 voxels of the
// grid, which holds every sample of this march, and a sample outside the
// support has all eight corners outside the grid, so it reads the zeros the
// test would have given it.
template <bool CNT>
__device__ __forceinline__ float march_ao5(const RenderParams &P, Vec p, Vec d, unsigned &nsamp) {
    const int ss[5] = {1, 2, 4, 8, 12}, ll[5] = {0, 1, 2, 2, 2};
    // every sample's corners are requested before the first is used (one
    // memory round trip per ray instead of five); samples past the support
    // read the zero cell. The support is a box that holds p, and each
    // coordinate of the rounded p + s d is monotone in s, so the samples
    // inside it are a prefix of s = 1, 2, 4, 8, 12.
    float4 A[5], B[5];
    float fx[5], fy[5], fz[5];
    bool in[5];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const Vec x = axpy((float)ss[k], d, p);
        const uint32_t i = corner_cell(P, ll[k], x, fx[k], fy[k], fz[k]);
        if constexpr (CNT) {
            in[k] = in_support(P, x);
            load_cell(P, ll[k], in[k] ? i : P.pzero[ll[k]], A[k], B[k]);
        } else {
            load_cell(P, ll[k], i, A[k], B[k]);
        }
    }
    // the march stops at O >= 1 or when a sample leaves the support; terms
    // added after O >= 1 are non-negative and leave min(1, O) = 1, terms past
    // the support are zero, so summing all five gives the same min(1, O)
    float O = 0.0f;
#pragma unroll
    for (int k = 0; k < 5; k++) {
        if constexpr (CNT) nsamp += (in[k] && O < 1.0f) ? 1u : 0u;
        const float wl = __int_as_float((127 - 2 * ll[k]) << 23);   // 2^l / 8^l
        O = fmaf(trilerp(A[k], B[k], fx[k], fy[k], fz[k]), wl, O);
    }
    return O;
}

// The unbounded march (shadows) with 3 levels: s = 1, 2 (levels 0, 1), then
// s = 4, 8, 12, ... on level 2 until the sample leaves the density support
// or O reaches 1; the same samples, weights and sample count as march(), and
// the same min(1, O). The corners of four samples at a time are requested
// before the first of them is used.
template <int L0, int L1, int L2, int L3>
__device__ __forceinline__ void march4(const RenderParams &P, Vec p, Vec d, float s0, float s1, float s2, float s3,
                                       bool &alive, float &O, unsigned &nsamp) {
    constexpr int ll[4] = {L0, L1, L2, L3};
    const float ss[4] = {s0, s1, s2, s3};
    float4 A[4], B[4];
    float fx[4], fy[4], fz[4];
    bool in[4];
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const Vec x = axpy(ss[j], d, p);
        in[j] = (j == 0 ? alive : in[j - 1]) && in_support(P, x);
        const uint32_t i = corner_cell(P, ll[j], x, fx[j], fy[j], fz[j]);
        load_cell(P, ll[j], in[j] ? i : P.pzero[ll[j]], A[j], B[j]);
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        nsamp += (in[j] && O < 1.0f) ? 1u : 0u;
        const float wl = __int_as_float((127 - 2 * ll[j]) << 23);   // 2^l / 8^l
        O = fmaf(trilerp(A[j], B[j], fx[j], fy[j], fz[j]), wl, O);
    }
    alive = in[3] && O < 1.0f;
}
__device__ __forceinline__ float march_shadow3(const RenderParams &P, Vec p, Vec d, unsigned &nsamp) {
    float O = 0.0f;
    bool alive = true;
    // s = 1, 2, 4, 8 (levels 0, 1, 2, 2), then s = 12 + 16 g + 4 j on level 2
    march4<0, 1, 2, 2>(P, p, d, 1.0f, 2.0f, 4.0f, 8.0f, alive, O, nsamp);
    for (int s = 12; alive && s < (1 << 24); s += 16)
        march4<2, 2, 2, 2>(P, p, d, (float)s, (float)(s + 4), (float)(s + 8), (float)(s + 12), alive, O, nsamp);
    return O;
}

__device__ __forceinline__ float march(const RenderParams &P, Vec p, Vec d, float max_dist, unsigned &nsamp) {
    const int top = P.levels - 1;
    float O = 0.0f;
    int s = 1;
    for (;;) {
        if (max_dist >= 0.0f && (float)s > max_dist) break;
        const Vec x = axpy((float)s, d, p);
        if (x.x < P.lod_lo || x.y < P.lod_lo || x.z < P.lod_lo || x.x > P.lod_hi[0] || x.y > P.lod_hi[1] ||
            x.z > P.lod_hi[2])
            break;
        int l = 31 - __clz(s);
        l = l < top ? l : top;
        const float wl = __int_as_float((127 - 2 * l) << 23);   // 2^l / 8^l
        O = fmaf(sample_level(P, l, x), wl, O);
        nsamp++;
        if (O >= 1.0f) break;
        s += 1 << l;
    }
    return O;
}

// Squared distance between the half-line o + t d (t >= 0, |d| = 1) and the
// segment [a, b]: the least of the interior stationary point (when it lies
// in range) and the optima on the three boundaries t = 0, h = 0, h = 1.
// Every candidate is a pair of real points, so the result never falls below
// the true distance.
__device__ __forceinline__ float halfline_segment_d2(Vec o, Vec d, Vec a, Vec b) {
    const Vec ba = sub(b, a), ao = sub(a, o);
    const float L2 = dot(ba, ba), k = dot(d, ba), e = dot(d, ao), f = dot(ba, ao);
    auto at = [&](float t, float h) {
        const Vec q = sub(axpy(t, d, o), axpy(h, ba, a));
        return dot(q, q);
    };
    float best = at(0.0f, L2 > 0.0f ? fminf(1.0f, fmaxf(0.0f, __fdividef(-f, L2))) : 0.0f);
    best = fminf(best, at(fmaxf(0.0f, e), 0.0f));
    best = fminf(best, at(fmaxf(0.0f, e + k), 1.0f));
    const float det = L2 - k * k;
    if (L2 > 0.0f && det > 1e-6f * L2) {
        const float h = __fdividef(fmaf(k, e, -f), det), t = fmaf(h, k, e);
        if (t >= 0.0f && h >= 0.0f && h <= 1.0f) best = fminf(best, at(t, h));
    }
    return best;
}

// Does the line [a, b] pass within sqrt(r2) of the half-line o + t d? The
// distance between the two infinite lines, |w . c| / |c| with w = a - o and
// c = d x (b - a), bounds the answer from below and rejects most cells with
// one cross product and no division. When it does not, and the lines' closest
// points, t = (w x (b - a)) . c / |c|^2 and h = (w x d) . c / |c|^2, lie on
// the half-line and the segment, that distance is the answer; otherwise the
// optimum is on the boundary of the parameter range.
__device__ __forceinline__ bool rep_blocks(Vec o, Vec d, Vec a, Vec b, float r2) {
    const Vec ba = sub(b, a), c = cross(d, ba), w = sub(a, o);
    const float c2 = dot(c, c), wc = dot(w, c);
    if (wc * wc > r2 * c2) return false;
    if (c2 > 1e-6f * dot(ba, ba)) {
        const float t = dot(cross(w, ba), c), h = dot(cross(w, d), c);
        if (t >= 0.0f && h >= 0.0f && h <= c2) return true;
    }
    return halfline_segment_d2(o, d, a, b) <= r2;
}

template <class SM>
__device__ __forceinline__ int slot_owner(const SM &sm, int warp, int g) { return warp * 32 + (sm.item[warp][g] >> 3); }
template <class SM>
__device__ __forceinline__ int slot_index(const SM &sm, int warp, int g) { return sm.item[warp][g] & 7; }

// Hard shadow against the representative lines of one LoD level (Sec. 5.2,
// first approach): from one cell size toward the light, walk the level's
// cells (3D DDA, in cell units) and report 0 at the first cell whose line
// passes within the scaled radius of the half-line, else 1.
//
// The walk's parameter range [tnear, tfar) inside the level's grid is cut
// into pieces of REP_PIECE cell lengths (the last one open-ended) that are
// walked independently: piece k starts in the cell holding its first point
// and stops after the cell whose exit lies beyond its last, so the pieces
// cover the walk's cells (a cell at a seam may be tested twice) and the
// visibility is the minimum over the pieces. Each DDA step is decided by
// the current cell alone, so two walks in the same cell take the same path.
constexpr float REP_PIECE = 10.0f;

struct RepRay {
    float q[3], L[3], inv[3];
    float tnear, tfar;
};

__device__ __forceinline__ bool rep_ray(const RenderParams &P, Vec Pg, Vec Lt, RepRay &r) {
    const Vec q = scale(axpy(P.rep_size, Lt, Pg), P.rep_inv);
    r.q[0] = q.x; r.q[1] = q.y; r.q[2] = q.z;
    r.L[0] = Lt.x; r.L[1] = Lt.y; r.L[2] = Lt.z;
    r.tnear = 0.0f;
    r.tfar = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        r.inv[a] = __frcp_rn(r.L[a]);
        if (r.L[a] != 0.0f) {
            const float t1 = -r.q[a] * r.inv[a], t2 = ((float)P.rep_dims[a] - r.q[a]) * r.inv[a];
            r.tnear = fmaxf(r.tnear, fminf(t1, t2));
            r.tfar = fminf(r.tfar, fmaxf(t1, t2));
        } else if (r.q[a] < 0.0f || r.q[a] > (float)P.rep_dims[a]) {
            return false;
        }
    }
    return r.tnear < r.tfar;
}

__device__ __forceinline__ int rep_pieces(const RepRay &r) {
    return (int)fminf(32767.0f, ceilf((r.tfar - r.tnear) * (1.0f / REP_PIECE)));
}

// Walk piece `piece` of `pieces`: 0 if a line blocks, else 1. (The state
// arrays are only ever indexed by unrolled constants, so they stay in
// registers.)
__device__ __forceinline__ float rep_piece(const RenderParams &P, const RepRay &r, int piece, int pieces, unsigned &ntested) {
    const float t0 = fmaf(REP_PIECE, (float)piece, r.tnear);
    const float t1 = piece + 1 < pieces ? fmaf(REP_PIECE, (float)(piece + 1), r.tnear) : INFINITY;
    int v[3], st[3];
    float tm[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int vi = (int)floorf(fmaf(t0, r.L[a], r.q[a]));
        v[a] = min(max(vi, 0), P.rep_dims[a] - 1);
        st[a] = r.L[a] > 0.0f ? 1 : (r.L[a] < 0.0f ? -1 : 0);
        tm[a] = st[a] == 0 ? INFINITY : ((float)(st[a] > 0 ? v[a] + 1 : v[a]) - r.q[a]) * r.inv[a];
    }
    const unsigned long long *rep = reinterpret_cast<const unsigned long long *>(P.rep);
    const uint32_t sy = (uint32_t)P.rep_dims[0], sz = sy * (uint32_t)P.rep_dims[1];   // cells < 2^32
    const uint32_t stride[3] = {1u, sy, sz};
    uint32_t cell = (uint32_t)v[0] + sy * (uint32_t)v[1] + sz * (uint32_t)v[2];
    uint64_t w = __ldg(rep + cell);
    const Vec d = mk(r.L[0], r.L[1], r.L[2]);
    const int limit = P.rep_dims[0] + P.rep_dims[1] + P.rep_dims[2];
    for (int it = 0; it < limit; it++) {
        // the next cell, and its word loaded before this cell is tested
        const int ax = tm[0] <= tm[1] ? (tm[0] <= tm[2] ? 0 : 2) : (tm[1] <= tm[2] ? 1 : 2);
        bool more = false;
        int nv = 0;
        uint32_t ncell = cell;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (a != ax) continue;
            nv = v[a] + st[a];
            more = tm[a] < t1 && nv >= 0 && nv < P.rep_dims[a];
            ncell = st[a] > 0 ? cell + stride[a] : cell - stride[a];
        }
        const uint64_t nw = more ? __ldg(rep + ncell) : 0ull;
        ntested++;
        if (w & 1ull) {
            const uint32_t ps = (uint32_t)(w >> 8), pe = (uint32_t)(w >> 32);
            const Vec a = face_point(ps & 0xffu, (ps >> 8) & 0xffu, (ps >> 16) & 0xffu, P.invN);
            const Vec b = face_point(pe & 0xffu, (pe >> 8) & 0xffu, (pe >> 16) & 0xffu, P.invN);
            const Vec o = mk(r.q[0] - (float)v[0], r.q[1] - (float)v[1], r.q[2] - (float)v[2]);
            if (rep_blocks(o, d, a, b, P.rep_r2)) return 0.0f;
        }
        if (!more) break;
        cell = ncell;
        w = nw;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (a != ax) continue;
            v[a] = nv;
            tm[a] = ((float)(st[a] > 0 ? nv + 1 : nv) - r.q[a]) * r.inv[a];
        }
    }
    return 1.0f;
}

// The warp's hits' representative-line shadows, balanced over the lanes:
// every round, the hits still open (not blocked, pieces left; the first 32)
// get 32 / (their number) adjacent lanes each (a power of two), which walk
// the hit's next pieces side by side. Per-hit state lives in the staging
// arrays, which are dead while a warp lights its hits: sk holds (next piece
// << 16 | pieces) of hit g at [g / 32][warp * 32 + g % 32], st[0] the round's
// list of open hits.
template <class SM>
__device__ __forceinline__ void rep_shadows(const RenderParams &P, SM &sm, int warp, int lane, int total, Vec Lt, unsigned &nsamp) {
    auto hit_pos = [&](int g) {
        const int o = slot_owner(sm, warp, g), q = slot_index(sm, warp, g);
        return mk(sm.slot[F_PX][q][o], sm.slot[F_PY][q][o], sm.slot[F_PZ][q][o]);
    };
    for (int g = lane; g < total; g += 32) {
        RepRay r;
        const int n = rep_ray(P, hit_pos(g), Lt, r) ? rep_pieces(r) : 0;
        sm.sk_(g >> 5, warp * 32 + (g & 31)) = (uint32_t)n;
        sm.slot[F_V][slot_index(sm, warp, g)][slot_owner(sm, warp, g)] = 1.0f;
    }
    __syncwarp();
    uint32_t *list = sm.warp_words(warp);
    for (int round = 0; round < 65536; round++) {
        int K = 0;
        for (int g0 = 0; g0 < total && K < 32; g0 += 32) {
            const int g = g0 + lane;
            bool open = false;
            if (g < total) {
                const uint32_t s = sm.sk_(g >> 5, warp * 32 + (g & 31));
                open = (s >> 16) < (s & 0xffffu);   // a blocked hit's next piece is set past the end
            }
            const unsigned b = __ballot_sync(FULL, open);
            const int pos = K + __popc(b & ((1u << lane) - 1u));
            if (open && pos < 32) list[pos] = (uint32_t)g;
            K += __popc(b);
        }
        if (K == 0) break;
        K = min(K, 32);
        __syncwarp();
        int G = 1;
        while (2 * G * K <= 32) G <<= 1;
        const int i = lane / G, part = lane % G;
        float vis = 1.0f;
        int g = 0;
        uint32_t s = 0;
        if (i < K) {
            g = (int)list[i];
            s = sm.sk_(g >> 5, warp * 32 + (g & 31));
            const int piece = (int)(s >> 16) + part, pieces = (int)(s & 0xffffu);
            RepRay r;
            if (piece < pieces && rep_ray(P, hit_pos(g), Lt, r)) vis = rep_piece(P, r, piece, pieces, nsamp);
        }
        for (int x = G >> 1; x > 0; x >>= 1) vis = fminf(vis, __shfl_xor_sync(FULL, vis, x));
        __syncwarp();
        if (i < K && part == 0) {
            const uint32_t pieces = s & 0xffffu;
            uint32_t next = (s >> 16) + (uint32_t)G;
            if (vis == 0.0f) {
                sm.slot[F_V][slot_index(sm, warp, g)][slot_owner(sm, warp, g)] = 0.0f;
                next = pieces;
            }
            sm.sk_(g >> 5, warp * 32 + (g & 31)) = pieces | min(next, pieces) << 16;
        }
        __syncwarp();
    }
}


// Phase B: light the warp's collected hits.
//  - Shadows: one lane per hit, a march toward the light (Sec. 5.2).
//  - AO: the ao_rays hemisphere rays of one hit run on a group of adjacent
//    lanes (group = next power of two >= ao_rays), so a group samples one
//    neighbourhood at the same distances; occlusion is summed over the group
//    with a fixed butterfly, so the result does not depend on the schedule.
//  - Each hit's weighted colour is then scaled by ka * AO + kd * V * |n.L|.
template <class SM>
__device__ void light_hits(const RenderParams &P, SM &sm, int warp, int lane, int total, unsigned &nsamp,
                           unsigned long long js[4], float &jmax) {
    constexpr int MODE = SM::kMode;
    const Vec Lt = mk(P.Lt[0], P.Lt[1], P.Lt[2]);
    // the AO tangent frame replaces the tube direction at once where no
    // learned inputs or training samples read the direction afterwards
    constexpr bool kTmerge = SM::kDefer && MODE != MODE_LEARNED && MODE != MODE_JUDGE && MODE != MODE_SAMPLES;
    if constexpr (SM::kDefer) {   // the hits' geometry, one lane per hit (same operations as at the hit)
        for (int g = lane; g < total; g += 32) {
            const int o = slot_owner(sm, warp, g), q = slot_index(sm, warp, g);
            const Vec Pl = mk(sm.slot[F_NX][q][o], sm.slot[F_NY][q][o], sm.slot[F_NZ][q][o]);
            Vec a, b;
            uint32_t attr;
            fetch_record<SM::kLayout>(P, __float_as_uint(sm.slot[F_UX][q][o]), a, b, attr);
            Vec n, u;
            hit_geometry(Pl, a, b, n, u);
            if (kTmerge && P.ao) u = ao_tangent(n, u);
            sm.slot[F_NX][q][o] = n.x;
            sm.slot[F_NY][q][o] = n.y;
            sm.slot[F_NZ][q][o] = n.z;
            sm.slot[F_UX][q][o] = u.x;
            sm.slot[F_UY][q][o] = u.y;
            sm.slot[F_UZ][q][o] = u.z;
        }
        __syncwarp();
    }
    if (P.shadows == 1) {
        for (int g = lane; g < total; g += 32) {
            const int o = slot_owner(sm, warp, g), q = slot_index(sm, warp, g);
            const Vec Pg = mk(sm.slot[F_PX][q][o], sm.slot[F_PY][q][o], sm.slot[F_PZ][q][o]);
            sm.slot[F_V][q][o] =
                1.0f - fminf(1.0f, P.levels == 3 ? march_shadow3(P, Pg, Lt, nsamp) : march(P, Pg, Lt, -1.0f, nsamp));
        }
    } else if constexpr (MODE == MODE_REP) {
        rep_shadows(P, sm, warp, lane, total, Lt, nsamp);
    }
    if constexpr (MODE == MODE_LEARNED || MODE == MODE_JUDGE) {
        // learned AO (Sec. 5.3 surrogate), 16 hits per step: per-hit inputs
        // into a shared tile, then the model on tensor cores. The learned
        // variants (one view and batched) keep the activations in the warp's
        // tile, overlaid on its staging entries (short code that shares the
        // instruction cache with the traversal); the judge keeps them in
        // registers (fully unrolled). Both give the same bits. The judge
        // keeps its result in F_V (no shadows there) beside the traced AO.
        constexpr int FL = MODE == MODE_JUDGE ? F_V : F_AO;
        constexpr bool kAct = SM::kActTile;
        __nv_bfloat16 *h = sm.hin + (kAct ? 0 : warp * 16 * aomlp::HIN_STRIDE);
        uint8_t *act = nullptr;
        if constexpr (kAct) act = sm.stage[warp].act;
        const uint32_t rx = (uint32_t)P.res[0], ry = (uint32_t)P.res[1];
        for (int g0 = 0; g0 < total; g0 += 16) {
            if (lane < 16) {   // per-hit inputs of hit g0 + lane into row lane
                float hx[aomlp::NHIT];
                const int gi = g0 + lane;
                if (gi < total) {
                    const int o = slot_owner(sm, warp, gi), q = slot_index(sm, warp, gi);
                    const uint32_t vid = __float_as_uint(sm.slot[F_VID][q][o]);
                    aomlp::hit_inputs(sm.slot[F_UX][q][o], sm.slot[F_UY][q][o], sm.slot[F_UZ][q][o],
                                      sm.slot[F_NX][q][o], sm.slot[F_NY][q][o], sm.slot[F_NZ][q][o],
                                      sm.slot[F_PX][q][o], sm.slot[F_PY][q][o], sm.slot[F_PZ][q][o],
                                      (int)(vid % rx), (int)((vid / rx) % ry), (int)(vid / (rx * ry)), hx);
                } else {
#pragma unroll
                    for (int k = 0; k < aomlp::NHIT; k++) hx[k] = 0.0f;
                }
                if constexpr (kAct) aomlp::store_hit_inputs_act(hx, act, lane);
                else aomlp::store_hit_inputs(hx, h + lane * aomlp::HIN_STRIDE);
            }
            __syncwarp();
            const int gl = g0 + (lane >> 2), gh = gl + 8;
            const __nv_bfloat16 *vlo = nullptr, *vhi = nullptr;
            if (gl < total)
                vlo = P.vterm + (size_t)__float_as_uint(sm.slot[F_VID][slot_index(sm, warp, gl)][slot_owner(sm, warp, gl)]) * 64;
            if (gh < total)
                vhi = P.vterm + (size_t)__float_as_uint(sm.slot[F_VID][slot_index(sm, warp, gh)][slot_owner(sm, warp, gh)]) * 64;
            float lo, hi;
            if constexpr (kAct) aomlp::mlp_tile_smem(P.net, vlo, vhi, act, lo, hi);
            else aomlp::mlp_tile(P.net, vlo, vhi, h, lo, hi);
            if ((lane & 3) == 0) {
                const int g = lane >> 2;
                if (g0 + g < total) sm.slot[FL][slot_index(sm, warp, g0 + g)][slot_owner(sm, warp, g0 + g)] = lo;
                if (g0 + g + 8 < total) sm.slot[FL][slot_index(sm, warp, g0 + g + 8)][slot_owner(sm, warp, g0 + g + 8)] = hi;
            }
            __syncwarp();
        }
    }
    if (MODE != MODE_LEARNED && P.aof) {   // spherical AO field (Sec. 5.3, second approach)
        for (int g = lane; g < total; g += 32) {
            const int o = slot_owner(sm, warp, g), q = slot_index(sm, warp, g);
            sm.slot[F_AO][q][o] = sample_field(P, mk(sm.slot[F_PX][q][o], sm.slot[F_PY][q][o], sm.slot[F_PZ][q][o]));
        }
    }
    if (MODE != MODE_LEARNED && P.ao) {
        int G = 1;
        while (G < P.ao_rays) G <<= 1;
        const int per = 32 / G, sub = lane / G, ray = lane % G;
        // each hit's tangent once, one lane per hit, in place of its tube
        // direction (read after this only by the training-sample mode, which
        // keeps it and takes the tangent per ray)
        constexpr bool kTpre = MODE != MODE_SAMPLES;
        if constexpr (kTpre && !kTmerge) {
            for (int g = lane; g < total; g += 32) {
                const int ow = slot_owner(sm, warp, g), q = slot_index(sm, warp, g);
                const Vec T = ao_tangent(mk(sm.slot[F_NX][q][ow], sm.slot[F_NY][q][ow], sm.slot[F_NZ][q][ow]),
                                         mk(sm.slot[F_UX][q][ow], sm.slot[F_UY][q][ow], sm.slot[F_UZ][q][ow]));
                sm.slot[F_UX][q][ow] = T.x;
                sm.slot[F_UY][q][ow] = T.y;
                sm.slot[F_UZ][q][ow] = T.z;
            }
            __syncwarp();
        }
        const float *aod = SM::kBatch ? &P.aod[0][0] : sm.aod;
        for (int m = 0; m < total; m += per) {
            const int g = m + sub;
            float o = 0.0f;
            if (g < total && ray < P.ao_rays) {
                const int ow = slot_owner(sm, warp, g), q = slot_index(sm, warp, g);
                const Vec Pg = mk(sm.slot[F_PX][q][ow], sm.slot[F_PY][q][ow], sm.slot[F_PZ][q][ow]);
                const Vec n = mk(sm.slot[F_NX][q][ow], sm.slot[F_NY][q][ow], sm.slot[F_NZ][q][ow]);
                const Vec u = mk(sm.slot[F_UX][q][ow], sm.slot[F_UY][q][ow], sm.slot[F_UZ][q][ow]);
                const Vec T = kTpre ? u : ao_tangent(n, u);
                const Vec B = cross(n, T);
                const float dx = aod[3 * ray], dy = aod[3 * ray + 1], dz = aod[3 * ray + 2];
                const Vec d = mk(fmaf(T.x, dx, fmaf(B.x, dy, n.x * dz)), fmaf(T.y, dx, fmaf(B.y, dy, n.y * dz)),
                                 fmaf(T.z, dx, fmaf(B.z, dy, n.z * dz)));
                o = fminf(1.0f, P.ao_fast ? march_ao5<MODE != MODE_IMAGE_NC>(P, Pg, d, nsamp)
                                           : march(P, Pg, d, P.ao_radius, nsamp));
            }
            for (int x = G >> 1; x > 0; x >>= 1) o += __shfl_xor_sync(FULL, o, x);
            if (ray == 0 && g < total) {
                const int ow = slot_owner(sm, warp, g), q = slot_index(sm, warp, g);
                sm.slot[F_AO][q][ow] = 1.0f - o / (float)P.ao_rays;
            }
        }
    }
    __syncwarp();
    for (int g = lane; g < total; g += 32) {
        const int o = slot_owner(sm, warp, g), q = slot_index(sm, warp, g);
        const Vec n = mk(sm.slot[F_NX][q][o], sm.slot[F_NY][q][o], sm.slot[F_NZ][q][o]);
        float AO, V;
        if constexpr (MODE == MODE_JUDGE) {
            const float tr = sm.slot[F_AO][q][o], le = sm.slot[F_V][q][o], e = fabsf(le - tr);
            js[0] += 1ull;
            js[1] += (unsigned long long)(e * 4294967296.0f);
            js[2] += (unsigned long long)(tr * 4294967296.0f);
            js[3] += (unsigned long long)(le * 4294967296.0f);
            jmax = fmaxf(jmax, e);
            atomicAdd(P.judge_hist + (e < 1.0f ? (int)(e * (float)JH) : JH - 1), 1u);   // NaN: last bin
            AO = le;
            V = 1.0f;
        } else {
            AO = (P.ao || P.aof || MODE == MODE_LEARNED) ? sm.slot[F_AO][q][o] : 1.0f;
            V = P.shadows ? sm.slot[F_V][q][o] : 1.0f;
        }
        const float kk = fmaf(P.ka, AO, P.kd * V * fabsf(dot(n, Lt)));
        sm.slot[F_CR][q][o] *= kk;
        sm.slot[F_CG][q][o] *= kk;
        sm.slot[F_CB][q][o] *= kk;
    }
}

// Per-block counters of the traversal and the judge.
struct Stats {
    unsigned nvox = 0, nrec = 0, nsamp = 0, nhit = 0;
    unsigned long long js[4] = {0ull, 0ull, 0ull, 0ull};
    float jmax = 0.0f;
};

// One 32-ray tile (one warp) of one view, from primary rays to output pixels.
template <class SM>
__device__ __forceinline__ void render_tile(const RenderParams &P, SM &sm, unsigned tile, int tid, int warp,
                                            int lane, Stats &S) {
    constexpr int MODE = SM::kMode;
    const int px = (int)(tile % (unsigned)P.tiles_x) * P.tile_w + lane % P.tile_w;
    const int py = (int)(tile / (unsigned)P.tiles_x) * P.tile_h + lane / P.tile_w;
    const bool valid = px < P.cw && py < P.ch;
    Ray ray;
    ray.hidx = ray.target = 0;
    ray.idmask = 0u;
    if (MODE == MODE_SAMPLES && valid) {
        const int64_t pix = (int64_t)py * P.cw + px;
        P.samp_vox[pix] = -1;
        uint32_t hsh = P.samp_seed ^ (uint32_t)pix * 0x9e3779b9u;   // integer hash (lowbias32)
        hsh ^= hsh >> 16; hsh *= 0x7feb352du; hsh ^= hsh >> 15; hsh *= 0x846ca68bu; hsh ^= hsh >> 16;
        ray.target = (int)(hsh % (uint32_t)P.samp_depth);
    }
    ray.A = ray.Cr = ray.Cg = ray.Cb = 0.0f;
    ray.done = !valid;
    ray.resume = false;
    ray.rt = 0.0f;
    ray.rk = 0;
    ray.T = 0.0f;
    if (valid) {
        const int i = P.x0 + px, j = P.y0 + py;
        // primary ray: float32 contract, each step correctly rounded
        const float sx = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * i + 1), (float)P.W), 1.0f), P.tw);
        const float sy = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * j + 1), (float)P.H), 1.0f), P.th);
        float d[3];
#pragma unroll
        for (int a = 0; a < 3; a++)
            d[a] = __fsub_rn(__fadd_rn(P.F[a], __fmul_rn(sx, P.R[a])), __fmul_rn(sy, P.U[a]));
        const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])), __fmul_rn(d[2], d[2]));
        const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
        ray.D = mk(__fmul_rn(d[0], inv), __fmul_rn(d[1], inv), __fmul_rn(d[2], inv));
        const float Da[3] = {ray.D.x, ray.D.y, ray.D.z};
        // slab test: only the entry parameter is needed, approximately
        float tnear = 0.0f, tfar = INFINITY;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (Da[a] != 0.0f) {
                const float ia = 1.0f / Da[a];
                const float t1 = (0.0f - P.eye[a]) * ia, t2 = ((float)P.res[a] - P.eye[a]) * ia;
                tnear = fmaxf(tnear, fminf(t1, t2));
                tfar = fminf(tfar, fmaxf(t1, t2));
            } else if (P.eye[a] < 0.0f || P.eye[a] > (float)P.res[a]) {
                tnear = INFINITY;
            }
        }
        if (!(tnear < tfar)) {
            ray.done = true;
        } else {
            // entry point in float-float, split into voxel index + local position
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float ph = __fmul_rn(tnear, Da[a]);
                const float pe = __fmaf_rn(tnear, Da[a], -ph);
                float sh, s2;
                two_sum(P.eye[a], ph, sh, s2);
                const float lo = __fadd_rn(s2, pe);
                float fl = floorf(sh);
                float f = __fadd_rn(__fsub_rn(sh, fl), lo);
                if (f < 0.0f) { fl -= 1.0f; f += 1.0f; }
                else if (f >= 1.0f) { fl += 1.0f; f -= 1.0f; }
                int vi = (int)fl;
                if (vi < 0) { f += (float)vi; vi = 0; }
                if (vi > P.res[a] - 1) { f += (float)(vi - (P.res[a] - 1)); vi = P.res[a] - 1; }
                ray.v[a] = vi;
                ray.pl[a] = Da[a] != 0.0f ? f : 0.0f;   // never stepped along a: pl only keeps its exit at inf
                ray.invD[a] = Da[a] != 0.0f ? 1.0f / Da[a] : INFINITY;
            }
            ray.T = tnear;
        }
    }
    // alternate traversal and lighting until every ray of the tile is finished
    for (;;) {
        const int used = traverse(P, sm, ray, tid, S.nvox, S.nrec, S.nhit);
        if (P.nrays > 0) {
            // list the warp's hits: (owner lane, slot), lane-major
            int pre = used;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, pre, o);
                if (lane >= o) pre += y;
            }
            const int total = __shfl_sync(FULL, pre, 31);
            pre -= used;
            for (int q = 0; q < used; q++) sm.item[warp][pre + q] = (uint8_t)((lane << 3) | q);
            __syncwarp();
            if (total > 0) {
                light_hits(P, sm, warp, lane, total, S.nsamp, S.js, S.jmax);
                __syncwarp();
                for (int q = 0; q < used; q++) {
                    ray.Cr += sm.slot[F_CR][q][tid];
                    ray.Cg += sm.slot[F_CG][q][tid];
                    ray.Cb += sm.slot[F_CB][q][tid];
                }
                if constexpr (MODE == MODE_SAMPLES) {   // the one stored hit
                  if (used > 0) {
                    const int64_t pix = (int64_t)py * P.cw + px;
                    P.samp_vox[pix] = (int32_t)__float_as_uint(sm.slot[F_VID][0][tid]);
                    P.samp_dir[3 * pix] = sm.slot[F_UX][0][tid];
                    P.samp_dir[3 * pix + 1] = sm.slot[F_UY][0][tid];
                    P.samp_dir[3 * pix + 2] = sm.slot[F_UZ][0][tid];
                    P.samp_ao[pix] = sm.slot[F_AO][0][tid];
                    if (P.samp_pos) {
                        P.samp_pos[3 * pix] = sm.slot[F_PX][0][tid];
                        P.samp_pos[3 * pix + 1] = sm.slot[F_PY][0][tid];
                        P.samp_pos[3 * pix + 2] = sm.slot[F_PZ][0][tid];
                        P.samp_nrm[3 * pix] = sm.slot[F_NX][0][tid];
                        P.samp_nrm[3 * pix + 1] = sm.slot[F_NY][0][tid];
                        P.samp_nrm[3 * pix + 2] = sm.slot[F_NZ][0][tid];
                    }
                  }
                }
            }
            __syncwarp();
        }
        if (__all_sync(FULL, ray.done)) break;
    }
    if (valid && P.out) {
        const float4 o = make_float4(fmaf(1.0f - ray.A, P.bg[0], ray.Cr), fmaf(1.0f - ray.A, P.bg[1], ray.Cg),
                                     fmaf(1.0f - ray.A, P.bg[2], ray.Cb), ray.A);
        P.out[(int64_t)py * P.cw + px] = o;
    }
}

template <int MODE>
__device__ __forceinline__ void flush_stats(const RenderParams &P, int lane, Stats &S) {
    if (MODE != MODE_IMAGE_NC && P.counters) {
        const unsigned c0 = __reduce_add_sync(FULL, S.nvox), c1 = __reduce_add_sync(FULL, S.nrec),
                       c2 = __reduce_add_sync(FULL, S.nsamp), c3 = __reduce_add_sync(FULL, S.nhit);
        if (lane == 0) {
            atomicAdd(P.counters + 0, (unsigned long long)c0);
            atomicAdd(P.counters + 1, (unsigned long long)c1);
            atomicAdd(P.counters + 2, (unsigned long long)c2);
            atomicAdd(P.counters + 3, (unsigned long long)c3);
        }
    }
    if constexpr (MODE == MODE_JUDGE) {
#pragma unroll
        for (int c = 0; c < 4; c++)
            for (int o = 16; o > 0; o >>= 1) S.js[c] += __shfl_xor_sync(FULL, S.js[c], o);
        for (int o = 16; o > 0; o >>= 1) S.jmax = fmaxf(S.jmax, __shfl_xor_sync(FULL, S.jmax, o));
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < 4; c++) atomicAdd(P.judge + c, S.js[c]);
            atomicMax(P.judge_max, __float_as_uint(S.jmax));
        }
    }
}

constexpr int min_blocks(int mode) {
    return mode == MODE_IMAGE || mode == MODE_IMAGE_NC
               ? 7
               : (mode == MODE_JUDGE ? 4 : (mode == MODE_STILL ? 5 : 6));
}
// batched: the image variant reads its view from shared memory and needs 80
// registers; the learned one keeps 96 (at 80 it spills)
constexpr int min_blocks_batch(int mode) {
    return mode == MODE_IMAGE || mode == MODE_IMAGE_NC ? 6 : (mode == MODE_LEARNED ? 5 : min_blocks(mode));
}

// One view: a persistent grid takes 32-ray tiles from a global counter.
template <int MODE, int LAYOUT>
__global__ void __launch_bounds__(RT, min_blocks(MODE))
render_kernel(const __grid_constant__ RenderParams P) {
    __shared__ Smem<MODE, LAYOUT, false> sm;
    if constexpr (decltype(sm)::kAod)
        for (int i = threadIdx.x; i < MAX_AO * 3; i += RT) sm.aod[i] = P.aod[i / 3][i % 3];
    __syncthreads();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    Stats S;
    for (;;) {
        unsigned tile = 0;
        if (lane == 0) tile = atomicAdd(P.tile_counter, 1u);
        tile = __shfl_sync(FULL, tile, 0);
        if (tile >= (unsigned)P.ntiles) break;
        render_tile(P, sm, tile, tid, warp, lane, S);
    }
    flush_stats<MODE>(P, lane, S);
}

// Many views in one persistent launch: the work queue is the concatenation
// of the views' tile lists (largest views first); a warp takes the next tile
// from one global counter and finds its view by binary search over the
// views' first-tile offsets. Each view's parameters live in global memory.
struct BatchParams {
    const RenderParams *items;
    const unsigned *tile0;        // [n + 1]: first tile of each view, total last
    int32_t n;
    unsigned *counter;
};

template <int MODE, int LAYOUT>
__global__ void __launch_bounds__(RT, min_blocks_batch(MODE))
render_batch_kernel(const __grid_constant__ BatchParams B) {
    __shared__ Smem<MODE, LAYOUT, true> sm;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned total = __ldg(B.tile0 + B.n);
    int cur = -1;
    Stats S;
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(B.counter, 1u);
        t = __shfl_sync(FULL, t, 0);
        if (t >= total) break;
        int lo = 0, hi = B.n - 1;   // last view with tile0 <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(B.tile0 + mid) <= t) lo = mid;
            else hi = mid - 1;
        }
        if (lo != cur) {   // this warp's view changed: copy its parameters (all but the TF)
            __syncwarp();
            const float4 *src = reinterpret_cast<const float4 *>(B.items + lo);
            for (int i = lane; i < HOT_BYTES / 16; i += 32) sm.hot[warp][i] = __ldg(src + i);
            __syncwarp();
            cur = lo;
        }
        render_tile(*reinterpret_cast<const RenderParams *>(sm.hot[warp]), sm, t - __ldg(B.tile0 + lo), tid, warp,
                    lane, S);
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
static void norm3(double *a) {
    const double l = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= l; a[1] /= l; a[2] /= l;
}

// Validates the arguments and fills the launch parameters (all but outputs).
// `judge`: learned AO for the image plus traced AO at every hit (ao_rays).
// Camera basis (forward, right, up) and half-extents of the image plane in
// float64, rounded to float32; Lt = toward the light. False: degenerate.
bool camera_basis(const lvr_view *view, float F[3], float R[3], float U[3], float *th, float *tw, float Lt[3]) {
    double f[3], up[3], r[3], u[3];
    for (int a = 0; a < 3; a++) {
        f[a] = (double)view->at[a] - (double)view->eye[a];
        up[a] = view->up[a];
    }
    norm3(f);
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    if (!(fabs(r[0]) + fabs(r[1]) + fabs(r[2]) > 0.0)) return false;
    norm3(r);
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    const double tanh_ = tan((double)view->fovy_deg * M_PI / 360.0);
    for (int a = 0; a < 3; a++) {
        F[a] = (float)f[a];
        R[a] = (float)r[a];
        U[a] = (float)u[a];
    }
    *th = (float)tanh_;
    *tw = (float)(tanh_ * (double)view->width / (double)view->height);
    double ld[3] = {view->light_dir[0], view->light_dir[1], view->light_dir[2]};
    norm3(ld);
    for (int a = 0; a < 3; a++) Lt[a] = (float)(-ld[a]);
    return true;
}

// ------------------------------------------------------------------ camera at rest: neighbour lists
// One thread per voxel: the records of the 27 voxels around it (neighbour
// order x fastest, records ascending) whose segment comes within the cull
// margin of it (a box test first, then the exact distance). Count pass (halo null): per voxel the number into
// cnt and the sum into *total; fill pass: the entries at halo + hoff[voxel].
// Face points and the offsets are binary fractions and small integers, so
// the shifted end points are exact. A hit's entry point lies on its tube and
// inside the voxel up to rounding far below the margin, so every record that
// can give the voxel a hit stays in its list.
__global__ void __launch_bounds__(256) neighbours_kernel(const uint32_t *__restrict__ offset,
                                                         const uint64_t *__restrict__ rec, int rx, int ry, int rz,
                                                         float invN, float r2, uint32_t *__restrict__ cnt,
                                                         unsigned long long *total,
                                                         const uint32_t *__restrict__ hoff,
                                                         uint64_t *__restrict__ halo) {
    const int64_t nvox = (int64_t)rx * ry * rz;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t n = 0;
    if (v < nvox) {
        const float rm = cull_margin(r2);
        const int x = (int)(v % rx), y = (int)((v / rx) % ry), z = (int)(v / ((int64_t)rx * ry));
        uint64_t *out = halo ? halo + hoff[v] : nullptr;
        for (uint32_t nc = 0; nc < 27; nc++) {
            const int X = x + (int)(nc % 3u) - 1, Y = y + (int)((nc / 3u) % 3u) - 1, Z = z + (int)(nc / 9u) - 1;
            if ((unsigned)X >= (unsigned)rx || (unsigned)Y >= (unsigned)ry || (unsigned)Z >= (unsigned)rz) continue;
            const int64_t nv = X + (int64_t)rx * (Y + (int64_t)ry * Z);
            const uint32_t nb = offset[nv], ne = offset[nv + 1];
            const Vec o = neighbour_offset(nc);
            for (uint32_t k = nb; k < ne; k++) {
                const uint64_t r = rec[k];
                Vec a = face_point(rec_face_in(r), rec_u_in(r), rec_v_in(r), invN);
                Vec b = face_point(rec_face_out(r), rec_u_out(r), rec_v_out(r), invN);
                a = mk(a.x + o.x, a.y + o.y, a.z + o.z);
                b = mk(b.x + o.x, b.y + o.y, b.z + o.z);
                if (fmaxf(a.x, b.x) + rm < 0.0f || fminf(a.x, b.x) - rm > 1.0f || fmaxf(a.y, b.y) + rm < 0.0f ||
                    fminf(a.y, b.y) - rm > 1.0f || fmaxf(a.z, b.z) + rm < 0.0f || fminf(a.z, b.z) - rm > 1.0f)
                    continue;
                if (nc != 13) {
                    const float pa[3] = {a.x, a.y, a.z}, pb[3] = {b.x, b.y, b.z};
                    if (lvr_geom::segment_box_dist2(pa, pb) > rm * rm) continue;
                }
                if (out) out[n] = (uint64_t)nc << 32 | k;
                n++;
            }
        }
        if (!halo) cnt[v] = n;
    }
    if (!halo) {
        const unsigned long long w = __reduce_add_sync(0xffffffffu, n);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(total, w);
    }
}

lvr_status ensure_neighbours(lvr_ctx *ctx, lvr_lineset *ls, float r2) {
    if (ls->halo_off && ls->halo_r2 >= r2) return LVR_OK;
    cudaStream_t s = ctx->stream;
    dev_free(ctx, ls->halo_off);
    dev_free(ctx, ls->halo);
    ls->halo_off = nullptr;
    ls->halo = nullptr;
    ls->halo_n = 0;
    ls->halo_r2 = 0.0f;
    const int64_t nvox = ls->nvox;
    const size_t cnt_bytes = ((size_t)nvox * 4 + 255) & ~(size_t)255;
    lvr_status st = ensure_scratch(ctx, cnt_bytes + (size_t)scan_tile_count(nvox) * 8);
    if (st != LVR_OK) return st;
    uint32_t *cnt = (uint32_t *)ctx->scratch;
    unsigned long long *tiles = (unsigned long long *)((char *)ctx->scratch + cnt_bytes);
    uint32_t *hoff = nullptr;
    if ((st = dev_alloc(ctx, (void **)&hoff, (size_t)(nvox + 1) * 4)) != LVR_OK) return st;
    unsigned long long *total = ctx->d_u64 + 6;
    LVR_CUDA(ctx, cudaMemsetAsync(total, 0, 8, s));
    const unsigned grid = grid1d(nvox, 256);
    neighbours_kernel<<<grid, 256, 0, s>>>(ls->offset, ls->rec, ls->res[0], ls->res[1], ls->res[2],
                                           1.0f / (float)ls->bins, r2, cnt, total, nullptr, nullptr);
    LVR_CUDA(ctx, cudaGetLastError());
    // the total decides overflow here, so the scan's overflow bit goes to a
    // word of its own instead of the context's status
    scan_counts(s, cnt, nvox, tiles, hoff, ctx->d_status + 2);
    LVR_CUDA(ctx, cudaGetLastError());
    unsigned long long *h = (unsigned long long *)ctx->h_pinned;
    LVR_CUDA(ctx, cudaMemcpyAsync(h, total, 8, cudaMemcpyDeviceToHost, s));
    LVR_CUDA(ctx, cudaStreamSynchronize(s));
    const unsigned long long n = h[0];
    if (n > 0xffffffffull) {
        dev_free(ctx, hoff);
        return set_err(ctx, LVR_EOVERFLOW, "neighbour lists: %llu entries (more than 2^32 - 1)", n);
    }
    uint64_t *halo = nullptr;
    if (n > 0 && (st = dev_alloc(ctx, (void **)&halo, (size_t)n * 8)) != LVR_OK) {
        dev_free(ctx, hoff);
        return st;
    }
    if (n > 0) {
        neighbours_kernel<<<grid, 256, 0, s>>>(ls->offset, ls->rec, ls->res[0], ls->res[1], ls->res[2],
                                               1.0f / (float)ls->bins, r2, nullptr, nullptr, hoff, halo);
        LVR_CUDA(ctx, cudaGetLastError());
    }
    ls->halo_off = hoff;
    ls->halo = halo;
    ls->halo_n = (int64_t)n;
    ls->halo_r2 = r2;
    return LVR_OK;
}

extern "C" lvr_status lvr_lineset_neighbours(lvr_ctx *ctx, lvr_lineset *ls, float radius) {
    if (!ctx) return LVR_EINVAL;
    if (!ls) return set_err(ctx, LVR_EINVAL, "lvr_lineset_neighbours: null line set");
    if (!(radius > 0.0f) || !(radius < 1e3f)) return set_err(ctx, LVR_EINVAL, "radius must be > 0");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    lvr_status st = ensure_neighbours(ctx, ls, radius * radius);
    if (st != LVR_OK) return st;
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LVR_OK;
}

static lvr_status setup(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod, const lvr_view *view,
                        const lvr_render_desc *desc, lvr_ao_model *ao, RenderParams &P, bool judge = false) {
    if (!ls || !view || !desc) return set_err(ctx, LVR_EINVAL, "lvr_render: null argument");
    if (view->width < 1 || view->height < 1) return set_err(ctx, LVR_EINVAL, "image size must be >= 1");
    int x0 = 0, y0 = 0, cw = view->width, ch = view->height;
    if (view->crop[2] > 0) {
        x0 = view->crop[0]; y0 = view->crop[1]; cw = view->crop[2]; ch = view->crop[3];
        if (x0 < 0 || y0 < 0 || ch < 1 || x0 + cw > view->width || y0 + ch > view->height)
            return set_err(ctx, LVR_EINVAL, "crop outside the image");
    }
    if (!(desc->radius > 0.0f) || !(desc->radius < 1e3f)) return set_err(ctx, LVR_EINVAL, "radius must be > 0");
    if (!(view->fovy_deg > 0.0f && view->fovy_deg < 180.0f)) return set_err(ctx, LVR_EINVAL, "fovy out of (0,180)");
    if (desc->ao_mode < 0 || desc->ao_mode > 3) return set_err(ctx, LVR_EINVAL, "bad ao_mode");
    if (desc->ao_mode == 3 && !(lod && lod->aof)) return set_err(ctx, LVR_EINVAL, "ao_mode 3 needs lvr_lod_ao_field");
    if (desc->ao_mode == 2 && !ao) return set_err(ctx, LVR_EINVAL, "learned AO needs a model");
    if (desc->still && desc->ao_mode == 2) return set_err(ctx, LVR_EINVAL, "the camera-at-rest mode has no learned-AO variant");
    if ((desc->ao_mode == 2 || judge) && lod && lod->levels < 3)
        return set_err(ctx, LVR_EINVAL, "learned AO needs a LoD of >= 3 levels");
    if (desc->shadows < 0 || desc->shadows > 2) return set_err(ctx, LVR_EINVAL, "bad shadows mode");
    if (desc->shadows == 2 && (desc->ao_mode == 2 || desc->still))
        return set_err(ctx, LVR_EINVAL, "shadows 2 has no learned-AO or camera-at-rest variant");
    if (desc->shadows == 2 && !(lod && desc->shadow_level >= 0 && desc->shadow_level < lod->levels &&
                                lod->rep[desc->shadow_level] && lod->rep_bins == ls->bins))
        return set_err(ctx, LVR_EINVAL, "shadows 2 needs lvr_lod_rep_lines and a shadow_level of the LoD");
    const bool need_lod = desc->shadows || desc->ao_mode != 0;
    if (need_lod && !lod) return set_err(ctx, LVR_EINVAL, "shadows / AO need a LoD");
    if ((desc->ao_mode == 1 || judge) && (desc->ao_rays < 1 || desc->ao_rays > MAX_AO))
        return set_err(ctx, LVR_EINVAL, "ao_rays must be in [1,32]");
    if (lod && (lod->dims[0][0] != ls->res[0] || lod->dims[0][1] != ls->res[1] || lod->dims[0][2] != ls->res[2]))
        return set_err(ctx, LVR_EINVAL, "LoD does not belong to this line set");
    if (desc->layout != LAYOUT_AOS8 && desc->layout != LAYOUT_AOS16) return set_err(ctx, LVR_EINVAL, "bad layout");
    if (desc->layout == LAYOUT_AOS16 && !ls->rec16 && ls->nseg > 0)
        return set_err(ctx, LVR_EINVAL, "16-byte records not built (lvr_lineset_layout)");
    int tw = desc->tile_w, th = desc->tile_h;
    if (tw == 0 && th == 0) { tw = 8; th = 4; }
    if (tw * th != 32 || tw < 1 || th < 1) return set_err(ctx, LVR_EINVAL, "tile must have 32 pixels");

    memset(&P, 0, sizeof P);
    P.offset = ls->offset;
    P.rec = ls->rec;
    P.rec16 = (const uint4 *)ls->rec16;
    for (int a = 0; a < 3; a++) P.res[a] = ls->res[a];
    P.invN = 1.0f / (float)ls->bins;
    P.r2 = desc->radius * desc->radius;
    if (lod) {
        P.levels = lod->levels;
        for (int l = 0; l < lod->levels; l++) {
            for (int a = 0; a < 3; a++) P.ldims[l][a] = lod->dims[l][a];
            P.pk[l] = lod->pk[l];
            P.pstr[l][0] = (uint32_t)lod->pstride[l][0];
            P.pstr[l][1] = (uint32_t)lod->pstride[l][1];
            P.pbias[l] = lod->pbias[l];
            P.pzero[l] = lod->pzero[l];
        }
        const float cell = (float)(1 << (lod->levels - 1));
        P.lod_lo = -0.5f * cell;
        for (int a = 0; a < 3; a++) P.lod_hi[a] = ((float)lod->dims[lod->levels - 1][a] + 0.5f) * cell;
    }
    if (!camera_basis(view, P.F, P.R, P.U, &P.th, &P.tw, P.Lt)) return set_err(ctx, LVR_EINVAL, "degenerate camera");
    for (int a = 0; a < 3; a++) P.eye[a] = view->eye[a];
    P.W = view->width; P.H = view->height; P.x0 = x0; P.y0 = y0; P.cw = cw; P.ch = ch;
    P.tile_w = tw; P.tile_h = th;
    P.tiles_x = (cw + tw - 1) / tw;
    P.ntiles = P.tiles_x * ((ch + th - 1) / th);
    P.opaque = desc->opaque ? 1 : 0;
    P.ert = desc->ert_alpha;
    P.shadows = desc->shadows;
    if (P.shadows == 2) {
        const int l = desc->shadow_level;
        P.rep = lod->rep[l];
        for (int a = 0; a < 3; a++) P.rep_dims[a] = lod->dims[l][a];
        P.rep_size = (float)(1 << l);
        P.rep_inv = 1.0f / P.rep_size;
        P.rep_r2 = desc->radius * desc->radius;   // radius x 2^l in cells of 2^l voxels
    }
    P.ao = desc->ao_mode == 1 || judge ? 1 : 0;
    P.ao_rays = P.ao ? desc->ao_rays : 0;
    P.learned = desc->ao_mode == 2 ? 1 : 0;
    P.aof = desc->ao_mode == 3 && !judge ? lod->aof : nullptr;
    P.still = desc->still ? 1 : 0;
    if (P.still) {
        // the line set's neighbour lists are a cache inside the handle
        lvr_status st = ensure_neighbours(ctx, const_cast<lvr_lineset *>(ls), P.r2);
        if (st != LVR_OK) return st;
        P.halo_off = ls->halo_off;
        P.halo = ls->halo;
    }
    if (judge) P.shadows = 0;   // the judge keeps the learned AO where the visibility would go
    P.nrays = (P.shadows ? 1 : 0) + P.ao_rays + P.learned + (P.aof ? 1 : 0);
    P.ao_radius = desc->ao_radius;
    P.ao_fast = lod && lod->levels == 3 && desc->ao_radius >= 12.0f && desc->ao_radius < 16.0f;
    P.ka = desc->ka;
    P.kd = desc->kd;
    for (int a = 0; a < 3; a++) P.bg[a] = desc->bg[a];
    if (P.ao) {   // spherical-Fibonacci hemisphere directions
        const double golden = M_PI * (3.0 - sqrt(5.0));
        for (int i = 0; i < desc->ao_rays; i++) {
            const double z = 1.0 - (i + 0.5) / desc->ao_rays, rr = sqrt(1.0 - z * z), ph = i * golden;
            P.aod[i][0] = (float)(rr * cos(ph));
            P.aod[i][1] = (float)(rr * sin(ph));
            P.aod[i][2] = (float)z;
        }
    }
    memcpy(P.tf, desc->tf_rgba, sizeof P.tf);
    if (P.learned) {
        const void *vt = nullptr;
        lvr_status st = ao_bind(ctx, ao, lod, &vt);
        if (st != LVR_OK) return st;
        P.net = ao_net(ao);
        P.vterm = (const __nv_bfloat16 *)vt;
    }
    return LVR_OK;
}

typedef void (*RenderKernel)(RenderParams);

static RenderKernel pick_kernel(int mode, int layout) {
    switch (mode * 2 + layout) {
    case MODE_IMAGE * 2: return render_kernel<MODE_IMAGE, LAYOUT_AOS8>;
    case MODE_IMAGE * 2 + 1: return render_kernel<MODE_IMAGE, LAYOUT_AOS16>;
    case MODE_LEARNED * 2: return render_kernel<MODE_LEARNED, LAYOUT_AOS8>;
    case MODE_LEARNED * 2 + 1: return render_kernel<MODE_LEARNED, LAYOUT_AOS16>;
    case MODE_SAMPLES * 2: return render_kernel<MODE_SAMPLES, LAYOUT_AOS8>;
    case MODE_JUDGE * 2: return render_kernel<MODE_JUDGE, LAYOUT_AOS8>;
    case MODE_STILL * 2: return render_kernel<MODE_STILL, LAYOUT_AOS8>;
    case MODE_STILL * 2 + 1: return render_kernel<MODE_STILL, LAYOUT_AOS16>;
    case MODE_REP * 2: return render_kernel<MODE_REP, LAYOUT_AOS8>;
    case MODE_REP * 2 + 1: return render_kernel<MODE_REP, LAYOUT_AOS16>;
    case MODE_IMAGE_NC * 2: return render_kernel<MODE_IMAGE_NC, LAYOUT_AOS8>;
    case MODE_IMAGE_NC * 2 + 1: return render_kernel<MODE_IMAGE_NC, LAYOUT_AOS16>;
    default: return nullptr;
    }
}

static int kernel_mode(const RenderParams &P) {
    return P.judge ? MODE_JUDGE
                   : (P.learned ? MODE_LEARNED
                                : (P.samp_vox ? MODE_SAMPLES
                                              : (P.still ? MODE_STILL
                                                        : (P.shadows == 2 ? MODE_REP
                                                                          : (P.counters ? MODE_IMAGE : MODE_IMAGE_NC)))));
}

// Persistent grid size of a kernel: SMs x resident blocks (cached per variant).
static lvr_status grid_blocks(lvr_ctx *ctx, int slot, const void *kern, int *blocks) {
    int &b = ctx->render_blocks[slot];
    if (!b) {
        int sms = 0, per_sm = 0;
        LVR_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        LVR_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RT, 0));
        b = sms * (per_sm > 0 ? per_sm : 1);
    }
    *blocks = b;
    return LVR_OK;
}

// Before a single-view launch: the transfer function, passed by value, into
// the context's device copy (the kernels read it through L1, each lane its
// own entry: from shared memory it would cost 4 KB per block, from the
// constant bank its divergent reads would serialise), and the tile counter
// to zero. Stream-ordered, so back-to-back launches on the context's stream
// each see their own.
struct TfParam {
    float v[1024];
};
__global__ void __launch_bounds__(256) render_prep_kernel(const __grid_constant__ TfParam t, float *dst,
                                                          unsigned *tile_counter) {
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) dst[i] = t.v[i];
    if (threadIdx.x == 0) *tile_counter = 0u;
}

// A single-view launch in two parts: everything that may fail or allocate
// (the transfer function's device copy, the kernel, its persistent grid),
// then the stream work alone (the prep kernel and the render), which a
// batch also records into its graph.
struct ViewLaunch {
    RenderKernel kern = nullptr;
    int grid = 0;
};
static lvr_status prepare_view(lvr_ctx *ctx, RenderParams &P, int layout, ViewLaunch &L) {
    lvr_status st;
    if (!ctx->d_tf && (st = dev_alloc(ctx, (void **)&ctx->d_tf, 4096)) != LVR_OK) return st;
    P.tile_counter = ctx->d_status + 1;
    P.gtf = reinterpret_cast<const float4 *>(ctx->d_tf);
    const int mode = kernel_mode(P);
    L.kern = pick_kernel(mode, layout);
    if (!L.kern) return set_err(ctx, LVR_EINVAL, "this render mode has no 16-byte record variant");
    int blocks;
    if ((st = grid_blocks(ctx, mode * 2 + layout, (const void *)L.kern, &blocks)) != LVR_OK) return st;
    const int need = (P.ntiles + RT / 32 - 1) / (RT / 32);
    L.grid = need < blocks ? need : blocks;
    return LVR_OK;
}
static void enqueue_view(lvr_ctx *ctx, const RenderParams &P, const ViewLaunch &L) {
    TfParam t;
    memcpy(t.v, P.tf, sizeof(t.v));
    render_prep_kernel<<<1, 256, 0, ctx->stream>>>(t, ctx->d_tf, P.tile_counter);
    L.kern<<<L.grid, RT, 0, ctx->stream>>>(P);
}
static lvr_status launch(lvr_ctx *ctx, RenderParams &P, int layout) {
    ViewLaunch L;
    lvr_status st = prepare_view(ctx, P, layout, L);
    if (st != LVR_OK) return st;
    enqueue_view(ctx, P, L);
    LVR_CUDA(ctx, cudaGetLastError());
    return LVR_OK;
}

extern "C" lvr_status lvr_render(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod,
                                 const lvr_view *view, const lvr_render_desc *desc,
                                 lvr_ao_model *ao, float *rgba, uint64_t *counters) {
    if (!ctx) return LVR_EINVAL;
    if (!rgba) return set_err(ctx, LVR_EINVAL, "lvr_render: null output");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    RenderParams P;
    lvr_status st = setup(ctx, ls, lod, view, desc, ao, P);
    if (st != LVR_OK) return st;
    cudaStream_t s = ctx->stream;
    const size_t out_bytes = (size_t)P.cw * P.ch * 16;
    const bool host_out = !is_device_ptr(rgba);
    const bool host_cnt = counters && !is_device_ptr(counters);
    if (host_out && (st = ensure_stage_out(ctx, out_bytes)) != LVR_OK) return st;
    P.out = host_out ? (float4 *)ctx->stage_out : (float4 *)rgba;
    if (counters) {
        P.counters = host_cnt ? (unsigned long long *)ctx->d_u64 : (unsigned long long *)counters;
        LVR_CUDA(ctx, cudaMemsetAsync(P.counters, 0, 32, s));
    }
    if ((st = launch(ctx, P, desc->layout)) != LVR_OK) return st;
    if (host_out) LVR_CUDA(ctx, cudaMemcpyAsync(rgba, P.out, out_bytes, cudaMemcpyDeviceToHost, s));
    if (host_cnt) LVR_CUDA(ctx, cudaMemcpyAsync(counters, P.counters, 32, cudaMemcpyDeviceToHost, s));
    if (host_out || host_cnt) LVR_CUDA(ctx, cudaStreamSynchronize(s));
    return LVR_OK;
}

// Hit samples of one view for the learned-AO trainer: per pixel of the crop
// (device buffers) the hit of index hash(seed, pixel) mod depth along the ray,
// composited as `desc` says, with traced AO: voxel (-1: none), unit segment
// direction (entry -> exit) and traced AO.
lvr_status render_samples(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod, const lvr_view *view,
                          const lvr_render_desc *desc, int32_t depth, uint32_t seed, int32_t *vox, float *dir,
                          float *ao, float *pos, float *nrm) {
    if (depth < 1) return set_err(ctx, LVR_EINVAL, "sample depth must be >= 1");
    RenderParams P;
    lvr_render_desc d = *desc;
    d.ao_mode = 1;
    d.shadows = 0;
    d.still = 0;
    lvr_status st = setup(ctx, ls, lod, view, &d, nullptr, P);
    if (st != LVR_OK) return st;
    P.samp_vox = vox;
    P.samp_dir = dir;
    P.samp_ao = ao;
    P.samp_seed = seed;
    P.samp_depth = depth;
    P.samp_pos = pos && nrm ? pos : nullptr;
    P.samp_nrm = pos && nrm ? nrm : nullptr;
    return launch(ctx, P, LAYOUT_AOS8);
}

extern "C" lvr_status lvr_ao_samples(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod, const lvr_view *view,
                                     const lvr_render_desc *desc, int32_t depth, uint32_t seed, int32_t *voxel,
                                     float *dir, float *ao, float *pos, float *normal) {
    if (!ctx) return LVR_EINVAL;
    if (!voxel || !dir || !ao) return set_err(ctx, LVR_EINVAL, "lvr_ao_samples: null output");
    if (!is_device_ptr(voxel) || !is_device_ptr(dir) || !is_device_ptr(ao) || (pos && !is_device_ptr(pos)) ||
        (normal && !is_device_ptr(normal)))
        return set_err(ctx, LVR_EINVAL, "lvr_ao_samples takes device buffers");
    if (!pos != !normal) return set_err(ctx, LVR_EINVAL, "lvr_ao_samples: pos and normal go together");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    return render_samples(ctx, ls, lod, view, desc, depth, seed, voxel, dir, ao, pos, normal);
}

extern "C" lvr_status lvr_ao_judge(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod, const lvr_view *view,
                                   const lvr_render_desc *desc, lvr_ao_model *ao, float *rgba, lvr_ao_error *err) {
    if (!ctx) return LVR_EINVAL;
    if (!err || !ao) return set_err(ctx, LVR_EINVAL, "lvr_ao_judge: null argument");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    RenderParams P;
    lvr_render_desc d = *desc;
    d.ao_mode = 2;
    d.still = 0;
    lvr_status st = setup(ctx, ls, lod, view, &d, ao, P, true);
    if (st != LVR_OK) return st;
    cudaStream_t s = ctx->stream;
    const size_t out_bytes = (size_t)P.cw * P.ch * 16;
    const bool host_out = rgba && !is_device_ptr(rgba);
    if (host_out && (st = ensure_stage_out(ctx, out_bytes)) != LVR_OK) return st;
    P.out = host_out ? (float4 *)ctx->stage_out : (float4 *)rgba;
    unsigned *hist = nullptr;
    if ((st = dev_alloc(ctx, (void **)&hist, JH * 4 + 64)) != LVR_OK) return st;
    P.judge_hist = hist;
    P.judge = (unsigned long long *)(hist + JH);
    P.judge_max = hist + JH + 8;
    cudaError_t e = cudaMemsetAsync(hist, 0, JH * 4 + 64, s);
    if (e == cudaSuccess) {
        st = launch(ctx, P, LAYOUT_AOS8);
        e = cudaGetLastError();
    }
    std::vector<unsigned> h(JH + 16);
    if (st == LVR_OK && e == cudaSuccess) e = cudaMemcpyAsync(h.data(), hist, JH * 4 + 64, cudaMemcpyDeviceToHost, s);
    if (st == LVR_OK && e == cudaSuccess && host_out) e = cudaMemcpyAsync(rgba, P.out, out_bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(ctx, hist);
    if (st != LVR_OK) return st;
    if (e != cudaSuccess) return cuda_err(ctx, e, "lvr_ao_judge");
    unsigned long long js[4];
    memcpy(js, h.data() + JH, sizeof js);
    unsigned mx = h[JH + 8];
    memset(err, 0, sizeof *err);
    err->hits = js[0];
    if (js[0]) {
        const double sc = 1.0 / 4294967296.0 / (double)js[0];
        err->mean_abs = (double)js[1] * sc;
        err->mean_traced = (double)js[2] * sc;
        err->mean_learned = (double)js[3] * sc;
        float m;
        memcpy(&m, &mx, 4);
        err->max_abs = m;
        const unsigned long long want = (js[0] * 99 + 99) / 100;   // ceil(0.99 hits)
        unsigned long long acc = 0;
        for (int b = 0; b < JH; b++) {
            acc += h[b];
            if (acc >= want) { err->p99_abs = (double)(b + 1) / JH; break; }
        }
        if (err->p99_abs > err->max_abs) err->p99_abs = err->max_abs;
    }
    return LVR_OK;
}

// ------------------------------------------------------------------ record layouts
namespace {

// 16-byte records: end points as six halves (exact: (2 bin + 1) / (2N) with
// N a power of two <= 1024 has at most 11 significant bits) and the attribute.
__global__ void expand_records_kernel(const uint64_t *__restrict__ rec, int64_t n, float invN, uint4 *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t r = rec[i];
        const Vec a = face_point(rec_face_in(r), rec_u_in(r), rec_v_in(r), invN);
        const Vec b = face_point(rec_face_out(r), rec_u_out(r), rec_v_out(r), invN);
        const __half2 h0 = __floats2half2_rn(a.x, a.y), h1 = __floats2half2_rn(a.z, b.x),
                      h2 = __floats2half2_rn(b.y, b.z);
        uint4 q;
        q.x = *reinterpret_cast<const uint32_t *>(&h0);
        q.y = *reinterpret_cast<const uint32_t *>(&h1);
        q.z = *reinterpret_cast<const uint32_t *>(&h2);
        q.w = rec_attr(r) | (rec_line_id(r) << 8);
        out[i] = q;
    }
}

}  // namespace

extern "C" lvr_status lvr_lineset_layout(lvr_ctx *ctx, lvr_lineset *ls, int layout) {
    if (!ctx) return LVR_EINVAL;
    if (!ls) return set_err(ctx, LVR_EINVAL, "lvr_lineset_layout: null line set");
    if (layout == LAYOUT_AOS8) return LVR_OK;
    if (layout != LAYOUT_AOS16) return set_err(ctx, LVR_EINVAL, "bad layout");
    if (ls->bins < 1 || ls->bins > 1024 || (ls->bins & (ls->bins - 1)))
        return set_err(ctx, LVR_EINVAL, "16-byte records need a power-of-two bin count <= 1024");
    if (ls->rec16 || ls->nseg == 0) return LVR_OK;
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    lvr_status st = dev_alloc(ctx, &ls->rec16, (size_t)ls->nseg * 16);
    if (st != LVR_OK) return st;
    const unsigned g = grid1d(ls->nseg, 256) > 65535 ? 65535 : grid1d(ls->nseg, 256);
    expand_records_kernel<<<g, 256, 0, ctx->stream>>>(ls->rec, ls->nseg, 1.0f / (float)ls->bins, (uint4 *)ls->rec16);
    LVR_CUDA(ctx, cudaGetLastError());
    return LVR_OK;
}

// ------------------------------------------------------------------ batched rendering
struct lvr_batch {
    lvr_ctx *ctx = nullptr;
    int n = 0;
    int mode = 0, layout = 0;
    int64_t tiles = 0, rays = 0;
    RenderParams *d_items = nullptr;
    unsigned *d_tile0 = nullptr;
    unsigned *d_counter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

typedef void (*BatchKernel)(BatchParams);

BatchKernel pick_batch_kernel(int mode, int layout) {
    switch (mode * 2 + layout) {
    case MODE_IMAGE_NC * 2: return render_batch_kernel<MODE_IMAGE_NC, LAYOUT_AOS8>;
    case MODE_IMAGE_NC * 2 + 1: return render_batch_kernel<MODE_IMAGE_NC, LAYOUT_AOS16>;
    case MODE_REP * 2: return render_batch_kernel<MODE_REP, LAYOUT_AOS8>;
    case MODE_REP * 2 + 1: return render_batch_kernel<MODE_REP, LAYOUT_AOS16>;
    case MODE_LEARNED * 2: return render_batch_kernel<MODE_LEARNED, LAYOUT_AOS8>;
    case MODE_LEARNED * 2 + 1: return render_batch_kernel<MODE_LEARNED, LAYOUT_AOS16>;
    default: return nullptr;
    }
}

// Builds a batch; `tile` / `layout` >= 0 override every item's own choice.
lvr_status batch_build(lvr_ctx *ctx, const lvr_batch_item *items, int n, int tile_w, int tile_h, int layout,
                       lvr_batch **out) {
    *out = nullptr;
    if (n < 1 || !items) return set_err(ctx, LVR_EINVAL, "batch needs at least one item");
    std::vector<RenderParams> P(n);
    std::vector<int> order(n);
    int mode = -1, lay = -1;
    for (int i = 0; i < n; i++) {
        const lvr_batch_item &it = items[i];
        if (!it.desc || !it.rgba) return set_err(ctx, LVR_EINVAL, "batch item %d: null desc or output", i);
        if (!is_device_ptr(it.rgba)) return set_err(ctx, LVR_EINVAL, "batch item %d: rgba must be device memory", i);
        lvr_render_desc d = *it.desc;
        if (d.still) return set_err(ctx, LVR_EINVAL, "batch item %d: batches render with the camera in motion", i);
        if (tile_w > 0) { d.tile_w = tile_w; d.tile_h = tile_h; }
        if (layout >= 0) d.layout = layout;
        lvr_status st = setup(ctx, it.ls, it.lod, &it.view, &d, it.ao, P[i]);
        if (st != LVR_OK) return st;
        const int m = P[i].learned ? MODE_LEARNED : (P[i].shadows == 2 ? MODE_REP : MODE_IMAGE_NC);   // no counters
        if (mode >= 0 && (m != mode || d.layout != lay))
            return set_err(ctx, LVR_EINVAL,
                           "batch items must share the AO kind, representative-line shadows or not, and the "
                           "record layout");
        mode = m;
        lay = d.layout;
        P[i].out = (float4 *)it.rgba;
        order[i] = i;
    }
    // every item's voxel term must still be bound (a model caches a limited number of LoDs)
    for (int i = 0; i < n; i++) {
        if (!P[i].learned) continue;
        if (ao_cached(items[i].ao, items[i].lod) != (const void *)P[i].vterm)
            return set_err(ctx, LVR_EINVAL, "a model is used with more than %d LoDs in one batch",
                           lvr_ao_model::kBound);
    }
    // largest views first, so the queue ends with small tiles lists
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return P[a].ntiles > P[b].ntiles; });
    lvr_batch *B = new lvr_batch();
    B->ctx = ctx;
    B->n = n;
    B->mode = mode;
    B->layout = lay;
    std::vector<RenderParams> sorted(n);
    for (int i = 0; i < n; i++) {
        sorted[i] = P[order[i]];
        B->rays += (int64_t)sorted[i].cw * sorted[i].ch;
        B->tiles += sorted[i].ntiles;
    }
    // Views that fill the GPU on their own (at least 8 tiles per resident
    // warp of the single-view kernel) get their own launch in the graph: the
    // single-view kernel takes its view's parameters from the constant bank,
    // where the queue kernel reads them from shared memory at every use. The
    // queue holds the rest, the largest (sorted first) excluded.
    std::vector<ViewLaunch> own(n);
    int nl = 0;
    for (; nl < n; nl++) {
        RenderParams q = sorted[nl];
        lvr_status st = prepare_view(ctx, q, lay, own[nl]);
        if (st != LVR_OK) {
            delete B;
            return st;
        }
        if ((int64_t)sorted[nl].ntiles < 8LL * own[nl].grid * (RT / 32)) break;
        sorted[nl] = q;   // its tile counter and transfer-function copy are the context's
    }
    const int nq = n - nl;
    std::vector<unsigned> tile0(nq + 1);
    int64_t tot = 0;
    for (int i = 0; i < nq; i++) {
        tile0[i] = (unsigned)tot;
        tot += sorted[nl + i].ntiles;
    }
    if (tot >= (int64_t)0xffffffffu) {
        delete B;
        return set_err(ctx, LVR_EINVAL, "batch too large");
    }
    tile0[nq] = (unsigned)tot;
    cudaStream_t s = ctx->stream;
    lvr_status st = LVR_OK;
    auto fail = [&](lvr_status e) { lvr_free_batch(B); return e; };
    if ((st = dev_alloc(ctx, (void **)&B->d_items, sizeof(RenderParams) * n)) != LVR_OK) return fail(st);
    std::vector<RenderParams> queued(sorted.begin() + nl, sorted.end());
    for (int i = 0; i < nq; i++) queued[i].gtf = reinterpret_cast<const float4 *>(B->d_items[i].tf);
    if ((st = dev_alloc(ctx, (void **)&B->d_tile0, sizeof(unsigned) * (n + 1) + 256)) != LVR_OK) return fail(st);
    B->d_counter = B->d_tile0 + ((n + 1 + 63) & ~63);
    cudaError_t e = cudaSuccess;
    if (nq > 0) {
        e = cudaMemcpyAsync(B->d_items, queued.data(), sizeof(RenderParams) * nq, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(B->d_tile0, tile0.data(), sizeof(unsigned) * (nq + 1), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // host vectors go out of scope
    if (e != cudaSuccess) return fail(cuda_err(ctx, e, "lvr_batch_create"));
    const BatchKernel kern = pick_batch_kernel(mode, lay);
    int blocks;
    if ((st = grid_blocks(ctx, 16 + mode * 2 + lay, (const void *)kern, &blocks)) != LVR_OK) return fail(st);
    const int64_t need = (tot + RT / 32 - 1) / (RT / 32);
    const int grid = need < blocks ? (int)need : blocks;
    BatchParams bp;
    bp.items = B->d_items;
    bp.tile0 = B->d_tile0;
    bp.n = nq;
    bp.counter = B->d_counter;
    // capture: the views with a launch of their own, then the queue's counter
    // reset and its persistent launch
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int i = 0; i < nl; i++) enqueue_view(ctx, sorted[i], own[i]);
        if (nq > 0) {
            cudaMemsetAsync(B->d_counter, 0, 4, s);
            kern<<<grid, RT, 0, s>>>(bp);
        }
        e = cudaStreamEndCapture(s, &B->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
    if (e != cudaSuccess) return fail(cuda_err(ctx, e, "lvr_batch_create (graph)"));
    *out = B;
    return LVR_OK;
}

}  // namespace

extern "C" lvr_status lvr_batch_create(lvr_ctx *ctx, const lvr_batch_item *items, int n, lvr_batch **out) {
    if (!ctx) return LVR_EINVAL;
    if (!out) return set_err(ctx, LVR_EINVAL, "lvr_batch_create: null output");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    return batch_build(ctx, items, n, -1, -1, -1, out);
}

extern "C" lvr_status lvr_batch_render(lvr_ctx *ctx, lvr_batch *b) {
    if (!ctx) return LVR_EINVAL;
    if (!b || b->ctx != ctx) return set_err(ctx, LVR_EINVAL, "lvr_batch_render: bad batch");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    LVR_CUDA(ctx, cudaGraphLaunch(b->exec, ctx->stream));
    return LVR_OK;
}

extern "C" lvr_status lvr_batch_size(const lvr_batch *b, int64_t *tiles, int64_t *rays) {
    if (!b) return LVR_EINVAL;
    if (tiles) *tiles = b->tiles;
    if (rays) *rays = b->rays;
    return LVR_OK;
}

extern "C" void lvr_free_batch(lvr_batch *b) {
    if (!b) return;
    lvr_ctx *ctx = b->ctx;
    cudaSetDevice(ctx->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    dev_free(ctx, b->d_items);
    dev_free(ctx, b->d_tile0);
    delete b;
}

extern "C" lvr_status lvr_autotune(lvr_ctx *ctx, const lvr_batch_item *items, int n, int reps, lvr_tune *out) {
    if (!ctx) return LVR_EINVAL;
    if (!out || reps < 1) return set_err(ctx, LVR_EINVAL, "lvr_autotune: bad argument");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    static const int tiles[4][2] = {{8, 4}, {4, 8}, {16, 2}, {32, 1}};
    bool aos16 = n > 0 && items;
    for (int i = 0; aos16 && i < n; i++) aos16 = items[i].ls && (items[i].ls->rec16 || items[i].ls->nseg == 0);
    cudaStream_t s = ctx->stream;
    cudaEvent_t e0, e1;
    LVR_CUDA(ctx, cudaEventCreate(&e0));
    LVR_CUDA(ctx, cudaEventCreate(&e1));
    memset(out, 0, sizeof *out);
    float best = INFINITY;
    lvr_status st = LVR_OK;
    for (int c = 0; c < 8 && st == LVR_OK; c++) {
        out->ms[c] = -1.0f;
        const int layout = c / 4, ti = c % 4;
        if (layout == LAYOUT_AOS16 && !aos16) continue;
        lvr_batch *B = nullptr;
        if ((st = batch_build(ctx, items, n, tiles[ti][0], tiles[ti][1], layout, &B)) != LVR_OK) break;
        cudaError_t e = cudaGraphLaunch(B->exec, s);   // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && e == cudaSuccess; r++) e = cudaGraphLaunch(B->exec, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        lvr_free_batch(B);
        if (e != cudaSuccess) {
            st = cuda_err(ctx, e, "lvr_autotune");
            break;
        }
        out->ms[c] = ms / reps;
        if (out->ms[c] < best) {
            best = out->ms[c];
            out->tile_w = tiles[ti][0];
            out->tile_h = tiles[ti][1];
            out->layout = layout;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}
