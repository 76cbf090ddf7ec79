/*
 * Oracle voxeliser (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Curve voxelisation (Sec. 3.1), face-point quantisation (Sec. 3.2) and the
 * compact per-voxel storage (Sec. 3.3), written out plainly:
 *   1. every vertex goes to fixed point on the grid (reading V1);
 *   2. for each curve, edge by edge, list the voxel planes the edge crosses,
 *      ordered by their exact rational edge parameter t (reading V2);
 *   3. consecutive face points bound one segment in the voxel between them;
 *      pieces before the first / after the last face point are dropped
 *      (Sec. 3.1); segments outside the grid are dropped (reading V3);
 *   4. each face point is quantised to the centre of one of N x N
 *      sub-squares of its face (Sec. 3.2, reading V4) and the attribute is
 *      interpolated to it (Sec. 3.1, reading V5);
 *   5. segments are grouped per voxel behind an offset table (Sec. 3.3);
 *      the grouping is a stable counting sort of the generation order, so
 *      each voxel lists its segments by (curve, ordinal) (reading V6).
 * All decisions are exact integer arithmetic.
 */
#include "oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define FX 65536            /* fixed-point units per voxel */
#define FX_SHIFT 16

static __thread char g_err[256];
const char *orc_last_error(void) { return g_err; }
static int fail(int code, const char *msg) {
    snprintf(g_err, sizeof g_err, "%s", msg);
    return code;
}

int orc_record_bits(int bins) {
    int lg = 0;
    while ((1 << lg) < bins) lg++;
    return 2 * 3 + 2 * (2 * lg) + 8 + 5;
}
int orc_record_bytes(int bins) { return (orc_record_bits(bins) + 7) / 8; }

static int64_t floordiv(int64_t a, int64_t b) {   /* b > 0 */
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

static int valid_bins(int n) {
    if (n < 2 || n > 128) return 0;
    return (n & (n - 1)) == 0;
}

int orc_fixed_point(const float *xyz, int64_t nv, const orc_grid *g, int32_t *X) {
    for (int64_t i = 0; i < nv; i++) {
        for (int a = 0; a < 3; a++) {
            float d = xyz[3 * i + a] - g->origin[a];   /* one float32 rounding */
            float p = d * g->scale;                     /* one float32 rounding */
            if (!(fabsf(p) < 16384.0f))
                return fail(ORC_EINVAL, "vertex not finite or outside +-2^14 voxels");
            float q = p * 65536.0f;                     /* exact: power-of-two scaling */
            X[3 * i + a] = (int32_t)lrintf(q);          /* round half to even */
        }
    }
    return ORC_OK;
}

int orc_attr16(const float *attr, int64_t nv, float amin, float amax, uint16_t *A) {
    if (!attr || !(amax > amin)) {
        memset(A, 0, sizeof(uint16_t) * (size_t)nv);
        return ORC_OK;
    }
    float span = amax - amin;
    for (int64_t i = 0; i < nv; i++) {
        float a = attr[i];
        if (!isfinite(a)) return fail(ORC_EINVAL, "attribute not finite");
        float q = (a - amin) / span;
        if (q < 0.0f) q = 0.0f;
        if (q > 1.0f) q = 1.0f;
        float s = q * 65535.0f;
        A[i] = (uint16_t)lrintf(s);
    }
    return ORC_OK;
}

int orc_fit_grid(const float *xyz, int64_t nv, int32_t rmax, int32_t bins, orc_grid *out) {
    if (nv <= 0 || rmax < 1 || !valid_bins(bins)) return fail(ORC_EINVAL, "bad fit arguments");
    float mn[3], mx[3];
    for (int a = 0; a < 3; a++) { mn[a] = xyz[a]; mx[a] = xyz[a]; }
    for (int64_t i = 0; i < nv; i++)
        for (int a = 0; a < 3; a++) {
            float v = xyz[3 * i + a];
            if (!isfinite(v)) return fail(ORC_EINVAL, "vertex not finite");
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    double ext[3], emax = 0.0;
    for (int a = 0; a < 3; a++) {
        ext[a] = (double)mx[a] - (double)mn[a];
        if (ext[a] > emax) emax = ext[a];
    }
    if (!(emax > 0.0)) return fail(ORC_EINVAL, "degenerate bounding box");
    memset(out, 0, sizeof *out);
    for (int a = 0; a < 3; a++) {
        double r = ceil(ext[a] * (double)rmax / emax);
        out->res[a] = r < 1.0 ? 1 : (int32_t)r;
        out->origin[a] = mn[a];
    }
    out->scale = (float)((double)rmax / emax);
    out->bins = bins;
    return ORC_OK;
}

/* ------------------------------------------------------------ segment generation */
typedef struct { orc_seg *v; int64_t n, cap; } segvec;

static int push(segvec *s, const orc_seg *x) {
    if (s->n == s->cap) {
        int64_t nc = s->cap ? s->cap * 2 : 1024;
        orc_seg *p = (orc_seg *)realloc(s->v, sizeof(orc_seg) * (size_t)nc);
        if (!p) return 0;
        s->v = p;
        s->cap = nc;
    }
    s->v[s->n++] = *x;
    return 1;
}

/* Face point state: face id, two bins, 16-bit attribute. */
typedef struct { int face, u, v; int64_t A; } fpoint;

/* Bin of coordinate X0 + t * D (t = n / d, d > 0) on the face of voxel index vb,
 * counted in units of 1/N of a voxel: floor(N * rem / FX), clamped to N - 1. */
static int bin_of(int64_t X0b, int64_t Db, int64_t vb, int64_t n, int64_t d, int N) {
    int64_t rem_d = (X0b - vb * FX) * d + n * Db;      /* rem * d, in [0, FX * d] */
    if (rem_d < 0 || rem_d > (int64_t)FX * d) {
        fprintf(stderr, "oracle: face point outside its voxel (internal error)\n");
        abort();
    }
    int64_t b = ((int64_t)N * rem_d) / ((int64_t)FX * d);
    if (b > N - 1) b = N - 1;
    return (int)b;
}

/* Voxelise curve c (vertices [v0, v1)) and append its stored segments in order. */
static int curve_segments(const int32_t *X, const uint16_t *A, int64_t v0, int64_t v1,
                          uint32_t c, const orc_grid *g, segvec *out) {
    if (v1 - v0 < 2) return 1;
    const int N = g->bins;
    int64_t cur[3];
    for (int a = 0; a < 3; a++) cur[a] = floordiv(X[3 * v0 + a], FX);
    int have_prev = 0, prev_stored = 0;
    fpoint prev = {0, 0, 0, 0};
    uint32_t k = 0;                               /* segment ordinal along the curve */
    for (int64_t e = v0; e + 1 < v1; e++) {
        int64_t P0[3], D[3];
        for (int a = 0; a < 3; a++) {
            P0[a] = X[3 * e + a];
            D[a] = (int64_t)X[3 * (e + 1) + a] - P0[a];
        }
        /* next crossing per axis: plane index, t = num / den */
        int64_t next_plane[3], last_plane[3], den[3];
        int active[3];
        for (int a = 0; a < 3; a++) {
            int64_t f0 = floordiv(P0[a], FX), f1 = floordiv(P0[a] + D[a], FX);
            if (D[a] > 0) {
                next_plane[a] = f0 + 1; last_plane[a] = f1; den[a] = D[a];
                active[a] = next_plane[a] <= last_plane[a];
            } else if (D[a] < 0) {
                next_plane[a] = f0; last_plane[a] = f1 + 1; den[a] = -D[a];
                active[a] = next_plane[a] >= last_plane[a];
            } else {
                active[a] = 0; den[a] = 1; next_plane[a] = last_plane[a] = 0;
            }
        }
        for (;;) {
            /* pick the axis whose next crossing has the smallest t; ties x, y, z */
            int best = -1;
            int64_t bn = 0, bd = 1;
            for (int a = 0; a < 3; a++) {
                if (!active[a]) continue;
                int64_t n = D[a] > 0 ? next_plane[a] * FX - P0[a] : P0[a] - next_plane[a] * FX;
                if (best < 0 || n * bd < bn * den[a]) { best = a; bn = n; bd = den[a]; }
            }
            if (best < 0) break;
            const int a = best;
            const int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;   /* other axes, increasing */
            fpoint here;
            here.face = 2 * a + (D[a] > 0 ? 1 : 0);                /* exit face of cur */
            here.u = bin_of(P0[b0], D[b0], cur[b0], bn, bd, N);
            here.v = bin_of(P0[b1], D[b1], cur[b1], bn, bd, N);
            {
                int64_t A0 = A[e], A1 = A[e + 1];
                here.A = A0 + floordiv((A1 - A0) * bn, bd);
            }
            if (have_prev) {
                int stored = cur[0] >= 0 && cur[0] < g->res[0] && cur[1] >= 0 &&
                             cur[1] < g->res[1] && cur[2] >= 0 && cur[2] < g->res[2];
                if (stored) {
                    orc_seg s;
                    s.voxel = (uint32_t)(cur[0] + (int64_t)g->res[0] * (cur[1] + (int64_t)g->res[1] * cur[2]));
                    s.curve = c;
                    s.ordinal = k;
                    s.face_in = (uint8_t)prev.face; s.u_in = (uint8_t)prev.u; s.v_in = (uint8_t)prev.v;
                    s.face_out = (uint8_t)here.face; s.u_out = (uint8_t)here.u; s.v_out = (uint8_t)here.v;
                    s.attr = (uint8_t)(((prev.A + here.A) * 255 + 65535) / 131070);
                    s.cont = (uint8_t)(prev_stored ? 1 : 0);
                    if (!push(out, &s)) return 0;
                }
                prev_stored = stored;
                k++;
            }
            /* step into the neighbour; the same physical point is its entry point */
            cur[a] += D[a] > 0 ? 1 : -1;
            prev.face = 2 * a + (D[a] > 0 ? 0 : 1);
            prev.u = here.u; prev.v = here.v; prev.A = here.A;
            have_prev = 1;
            if (D[a] > 0) { next_plane[a]++; active[a] = next_plane[a] <= last_plane[a]; }
            else          { next_plane[a]--; active[a] = next_plane[a] >= last_plane[a]; }
        }
    }
    return 1;
}

int orc_voxelize(const float *xyz, const float *attr, const int64_t *curve_offsets,
                 int64_t n_curves, int64_t n_vertices, const orc_grid *g, orc_voxset **out) {
    *out = NULL;
    if (!valid_bins(g->bins)) return fail(ORC_EINVAL, "bins must be a power of two in [2,128]");
    for (int a = 0; a < 3; a++)
        if (g->res[a] < 1 || g->res[a] > 4096) return fail(ORC_EINVAL, "resolution out of range");
    if (!(g->scale > 0.0f) || !isfinite(g->scale)) return fail(ORC_EINVAL, "scale must be > 0");
    int64_t nvox = (int64_t)g->res[0] * g->res[1] * g->res[2];
    if (nvox >= 4294967295LL) return fail(ORC_EINVAL, "grid too large");
    if (n_curves < 0 || n_vertices < 0) return fail(ORC_EINVAL, "negative size");
    if (n_curves > 0xffffffffLL) return fail(ORC_EINVAL, "too many curves");
    if (curve_offsets[0] != 0 || curve_offsets[n_curves] != n_vertices)
        return fail(ORC_EINVAL, "curve offsets must start at 0 and end at n_vertices");
    for (int64_t c = 0; c < n_curves; c++)
        if (curve_offsets[c + 1] < curve_offsets[c]) return fail(ORC_EINVAL, "offsets not monotone");

    int32_t *X = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(n_vertices ? n_vertices : 1));
    uint16_t *A = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(n_vertices ? n_vertices : 1));
    if (!X || !A) { free(X); free(A); return fail(ORC_ENOMEM, "out of memory"); }
    int rc = orc_fixed_point(xyz, n_vertices, g, X);
    if (rc == ORC_OK) rc = orc_attr16(attr, n_vertices, g->attr_min, g->attr_max, A);
    if (rc != ORC_OK) { free(X); free(A); return rc; }

    /* segments in generation order = (curve, ordinal) order */
    segvec gen = {NULL, 0, 0};
    for (int64_t c = 0; c < n_curves; c++) {
        if (!curve_segments(X, A, curve_offsets[c], curve_offsets[c + 1], (uint32_t)c, g, &gen)) {
            free(X); free(A); free(gen.v);
            return fail(ORC_ENOMEM, "out of memory");
        }
        if (gen.n > 0xffffffffLL) {
            free(X); free(A); free(gen.v);
            return fail(ORC_EOVERFLOW, "more than 2^32-1 segments");
        }
    }
    free(X);
    free(A);

    orc_voxset *vs = (orc_voxset *)calloc(1, sizeof *vs);
    uint32_t *offset = (uint32_t *)calloc((size_t)nvox + 1, sizeof(uint32_t));
    orc_seg *seg = (orc_seg *)malloc(sizeof(orc_seg) * (size_t)(gen.n ? gen.n : 1));
    uint32_t *cursor = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)nvox);
    if (!vs || !offset || !seg || !cursor) {
        free(vs); free(offset); free(seg); free(cursor); free(gen.v);
        return fail(ORC_ENOMEM, "out of memory");
    }
    /* stable counting sort by voxel: count, exclusive prefix sum, scatter */
    for (int64_t i = 0; i < gen.n; i++) offset[gen.v[i].voxel + 1]++;
    for (int64_t v = 0; v < nvox; v++) offset[v + 1] += offset[v];
    memcpy(cursor, offset, sizeof(uint32_t) * (size_t)nvox);
    for (int64_t i = 0; i < gen.n; i++) seg[cursor[gen.v[i].voxel]++] = gen.v[i];
    free(cursor);
    free(gen.v);

    vs->grid = *g;
    vs->nvox = nvox;
    vs->nseg = (int64_t)offset[nvox];
    vs->offset = offset;
    vs->seg = seg;
    *out = vs;
    return ORC_OK;
}

void orc_voxset_free(orc_voxset *vs) {
    if (!vs) return;
    free(vs->offset);
    free(vs->seg);
    free(vs);
}
int64_t orc_voxset_nseg(const orc_voxset *vs) { return vs->nseg; }
int64_t orc_voxset_nvox(const orc_voxset *vs) { return vs->nvox; }

void orc_voxset_export(const orc_voxset *vs, uint32_t *offset, uint8_t *fields,
                       uint32_t *curve, uint32_t *ordinal) {
    if (offset) memcpy(offset, vs->offset, sizeof(uint32_t) * (size_t)(vs->nvox + 1));
    for (int64_t i = 0; i < vs->nseg; i++) {
        const orc_seg *s = &vs->seg[i];
        if (fields) {
            uint8_t *f = fields + 8 * i;
            f[0] = s->face_in; f[1] = s->u_in; f[2] = s->v_in;
            f[3] = s->face_out; f[4] = s->u_out; f[5] = s->v_out;
            f[6] = s->attr; f[7] = s->cont;
        }
        if (curve) curve[i] = s->curve;
        if (ordinal) ordinal[i] = s->ordinal;
    }
}
