/*
 * Plain FP64 CPU oracle for the voxel-based line ray-caster (arXiv 1801.01155).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this code: only the tests, the smoke check and the benchmark's CPU
 * baseline use it. It shares no code, headers, tables or constants with the
 * CUDA library; the two meet only in the seeded inputs.
 *
 * It restates the paper's algorithm step by step, slowly and plainly:
 *   - curve voxelisation: clip every edge at the voxel faces in order of
 *     occurrence, keep one linear segment per voxel between consecutive face
 *     points, drop the partial pieces before the first and after the last
 *     face point (Sec. 3.1);
 *   - quantisation of each face point to the centre of one of N x N
 *     sub-squares of its face, with a 3-bit face id (Sec. 3.2);
 *   - per-voxel segment lists stored contiguously behind an offset table
 *     (Sec. 3.3);
 *   - the density LoD rho = sum length * sigma (Eq. 1) with 2^3 pooling
 *     (Sec. 3.4);
 *   - ray casting: 3D-DDA from voxel to voxel, ray-tube tests against the
 *     voxel's own segments, per-voxel hit sorting, local illumination and
 *     front-to-back alpha compositing with early ray termination
 *     (Secs. 4, 5, 5.1);
 *   - soft shadows by cone-marching the density LoD toward a directional
 *     light (Sec. 5.2) and ambient occlusion by marching the density along
 *     hemisphere rays within a radius of influence (Sec. 5.3).
 * Where the paper is silent the oracle follows the readings listed in the
 * repository's design notes; each is named where it is used.
 */
#ifndef LVR_ORACLE_H
#define LVR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* -------------------------------------------------------------- grid */
typedef struct orc_grid {
    int32_t res[3];      /* voxels per axis */
    int32_t bins;        /* N: sub-squares per face edge (power of two, 2..128) */
    float   origin[3];   /* world point mapped to grid (0,0,0) */
    float   scale;       /* grid units per world unit */
    float   attr_min, attr_max;
} orc_grid;

/* One stored per-voxel segment, fields decoded. */
typedef struct orc_seg {
    uint32_t voxel;      /* x + res_x * (y + res_y * z) */
    uint32_t curve;      /* input curve index */
    uint32_t ordinal;    /* index of the segment along its curve (all segments counted) */
    uint8_t  face_in, u_in, v_in;     /* entry face id (0=-x,1=+x,2=-y,3=+y,4=-z,5=+z), bins */
    uint8_t  face_out, u_out, v_out;  /* exit face id, bins */
    uint8_t  attr;       /* attribute byte */
    uint8_t  cont;       /* 1 iff the previous segment of the curve is stored too */
} orc_seg;

typedef struct orc_voxset {
    orc_grid  grid;
    int64_t   nvox;
    int64_t   nseg;
    uint32_t *offset;    /* [nvox + 1] exclusive prefix of per-voxel counts */
    orc_seg  *seg;       /* [nseg] voxel-major, then (curve, ordinal) */
} orc_voxset;

/* Error codes (0 = ok). */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_EOVERFLOW = 4 };

const char *orc_last_error(void);

/* Bits and bytes of the paper's packed line record for N bins per face edge:
 * 2 face ids of 3 bits, 2 endpoints of 2*log2(N) bin bits, 8 attribute bits,
 * 5 local-id bits; bytes = ceil(bits / 8) (Sec. 6.2, memory statistics). */
int orc_record_bits(int bins);
int orc_record_bytes(int bins);

/* World -> grid fixed point (reading V1): p = fl32(fl32(v - o) * s) and
 * X = round_half_even(p * 2^16) as int32. Fails on non-finite p or |p| >= 2^14. */
int orc_fixed_point(const float *xyz, int64_t nv, const orc_grid *g, int32_t *X);
/* Attribute to 16-bit code (reading V5). attr may be NULL (all zero). */
int orc_attr16(const float *attr, int64_t nv, float amin, float amax, uint16_t *A);
/* Grid fitted to the bounding box keeping its aspect ratio (Sec. 3.1). */
int orc_fit_grid(const float *xyz, int64_t nv, int32_t rmax, int32_t bins, orc_grid *out);

int  orc_voxelize(const float *xyz, const float *attr, const int64_t *curve_offsets,
                  int64_t n_curves, int64_t n_vertices, const orc_grid *g, orc_voxset **out);
void orc_voxset_free(orc_voxset *vs);
int64_t orc_voxset_nseg(const orc_voxset *vs);
int64_t orc_voxset_nvox(const orc_voxset *vs);
/* fields: [nseg * 8] = face_in,u_in,v_in,face_out,u_out,v_out,attr,cont */
void orc_voxset_export(const orc_voxset *vs, uint32_t *offset, uint8_t *fields,
                       uint32_t *curve, uint32_t *ordinal);

/* -------------------------------------------------------------- LoD */
#define ORC_MAX_LEVELS 4
typedef struct orc_lod {
    int      levels;
    int32_t  dims[ORC_MAX_LEVELS][3];
    uint32_t *cnt[ORC_MAX_LEVELS];
    double   *len[ORC_MAX_LEVELS];
    double   *dens[ORC_MAX_LEVELS];  /* sums; density as sampled = dens / 8^level */
} orc_lod;

int  orc_build_lod(const orc_voxset *vs, int levels, const float *sigma256, orc_lod **out);
void orc_lod_free(orc_lod *lod);
void orc_lod_dims(const orc_lod *lod, int level, int32_t *dims3);
void orc_lod_export(const orc_lod *lod, int level, uint32_t *cnt, double *len, double *dens);

/* -------------------------------------------------------------- rendering */
typedef struct orc_view {
    float   eye[3], at[3], up[3];
    float   fovy_deg;
    int32_t width, height;
    float   light_dir[3];       /* direction in which light travels */
} orc_view;

/* ---- representative lines (reading R3; replines.c) ---- */
typedef struct orc_reps {
    int      levels;
    int32_t  dims[ORC_MAX_LEVELS][3];
    uint8_t *rep[ORC_MAX_LEVELS];   /* per cell: valid, face_a, u_a, v_a, face_b, u_b, v_b */
} orc_reps;
int    orc_reps_build(const orc_voxset *vs, int levels, orc_reps **out);
void   orc_reps_free(orc_reps *reps);
void   orc_reps_export(const orc_reps *reps, int level, uint8_t *out7);
void   orc_rep_world(const orc_reps *reps, int level, int64_t cell, int N, double a[3], double b[3]);
double orc_halfline_segment_distance(const double o[3], const double d[3], const double a[3],
                                     const double b[3]);
/* visibility (0 or 1) of point P toward the light direction Lt (unit, toward
 * the light) against the representative lines of `level` (reading S5) */
double orc_shadow_reps_visibility(const orc_voxset *vs, const orc_reps *reps, float radius, int level,
                                  const double P[3], const double Lt[3]);

typedef struct orc_rdesc {
    float   radius;             /* tube radius, voxel units */
    float   tf[1024];           /* RGBA per attribute byte */
    int32_t opaque;             /* 1: alpha = 1, first hit only */
    float   ert_alpha;          /* early termination threshold (>= 1: never) */
    int32_t shadows;            /* soft shadow cone march */
    int32_t ao;                 /* 1: traced (density-marched) AO; 2: learned surrogate */
    int32_t ao_rays;            /* hemisphere rays per hit */
    float   ao_radius;          /* radius of influence, voxels */
    float   ka, kd;             /* ambient and diffuse weights */
    float   bg[3];              /* background colour */
    const float *ao_params;     /* learned AO parameters (ao == 2), see orc_ao_mlp */
    int32_t still;              /* 1: camera at rest (reading R2): also test the 26
                                   neighbouring voxels' segments; one hit per line id
                                   per voxel */
    const double *ao_field;     /* ao == 3: per-voxel spherical AO (orc_ao_sphere_field) */
    const orc_reps *reps;       /* shadows == 2: representative lines (reading S5) */
    int32_t shadow_level;       /* their level */
} orc_rdesc;

/* counters[0..3]: voxels visited, records tested, LoD trilinear samples,
 * composited hits (summed over the listed pixels). */
enum { ORC_RENDER_DDA = 0, ORC_RENDER_BRUTE = 1 };
/* tie: per-pixel bit mask of near-tie decisions (may be NULL): 1 silhouette
 * graze, 2 voxel ownership, 4 depth order, 16 AO frame, 32 slab entry, 64 a
 * hit's hard-shadow visibility (shadows 2); margin: per pixel, the smallest
 * decision margin in units of its tie threshold (may be NULL); flip: per
 * pixel, the sum over hits whose hard-shadow visibility is a near-tie of
 * w kd |n.L| max(rgb), the most a flip of each can move any colour channel
 * (may be NULL); alt (may be NULL): per pixel whose only near-tie is one
 * pair of hits closer in depth than their error bounds, the RGBA with that
 * pair composited in the other order (the other right answer); NaN
 * elsewhere (DDA mode only). */
int orc_render(const orc_voxset *vs, const orc_lod *lod, const orc_view *view,
               const orc_rdesc *rd, const int32_t *pix, int64_t npix, int mode,
               double *rgba, uint8_t *tie, double *margin, double *flip, double *alt,
               uint64_t *counters, int nthreads);

/* Reading K1, the rasterised comparison system: every capsule between two
 * consecutive vertices of the input polylines (float32 grid coordinates, no
 * voxel model), one fragment per capsule a pixel's ray enters, sorted by
 * (entry, capsule index) and blended front to back (S1 shading, no shadows
 * or AO) until the float32 opacity reaches ert_alpha; opaque: the nearest.
 * counters[0..1]: fragments, blended fragments. alt (may be NULL): as for
 * orc_render, the pixel with its one near-tie pair of fragments blended in
 * the other order, NaN elsewhere. */
int orc_raster(const float *xyz, const float *attr, const int64_t *offsets, int64_t nc, const orc_grid *g,
               const orc_view *view, const orc_rdesc *rd, const int32_t *pix, int64_t npix, double *rgba,
               uint8_t *tie, double *alt, uint64_t *counters, int nthreads);

/* ---- pieces exposed for pin tests ---- */
/* Primary ray of pixel (i, j) under the single-precision ray contract (reading R0). */
void orc_primary_ray(const orc_view *view, int32_t i, int32_t j, float org[3], float dir[3]);
/* First entry t > 0 of ray (o, d) into the capsule of radius r around segment
 * [a, b]; returns 0 if none. dist = distance from the ray line to the segment. */
int orc_capsule_entry(const double o[3], const double d[3], const double a[3],
                      const double b[3], double r, double *t, double *dist);
/* Density march from p along unit dir (max_dist < 0: unbounded); returns the
 * accumulated optical depth O. */
double orc_march(const orc_lod *lod, const double p[3], const double dir[3], double max_dist);
/* Trilinear density sample at level l, grid position x (level-0 voxel units). */
double orc_sample(const orc_lod *lod, int level, const double x[3]);
/* Hemisphere directions around normal n with tangent hint u (reading S3). */
void orc_ao_dirs(const double n[3], const double u[3], int k, double *dirs);

/* ---- spherical per-voxel AO (reading S4) ---- */
/* field[v] = 1 - mean over `rays` sphere directions of min(1, O), O the
 * level-0 density summed at distances 1, 2, ..., radius from voxel v's centre. */
void   orc_ao_sphere_field(const orc_lod *lod, int rays, double radius, double *field);
/* trilinear value of a cell-centred field at x, coordinates clamped to the
 * voxel centres (the field holds its edge values outside). */
double orc_ao_field_sample(const double *field, const int32_t dims[3], const double x[3]);

/* ---- learned AO surrogate (reading L1; aomlp.c) ---- */
int    orc_ao_nparams(void);
int    orc_ao_ninputs(void);
double orc_bf16(double x);
void   orc_ao_tangent(const double a[3], const double b[3], double t[3]);
/* x: [orc_ao_ninputs()]; t tangent, n unit normal, p hit point (grid
 * coordinates); returns -1 if the LoD has fewer than 3 levels. */
int    orc_ao_features(const orc_lod *lod, int64_t voxel, const double t[3], const double n[3],
                       const double p[3], double *x);
double orc_ao_mlp(const float *params, const double *x);

#ifdef __cplusplus
}
#endif
#endif
