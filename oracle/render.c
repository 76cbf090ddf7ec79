/*
 * Oracle ray-caster (TEST INFRASTRUCTURE ONLY; see oracle.h). FP64 throughout,
 * except where a float decides a discrete outcome that the kernel decides in
 * float32 (the early-termination test), which is then taken in float32 too.
 *
 *   primary rays ........ reading R0 (single-precision ray contract)
 *   traversal ........... Sec. 4: 3D-DDA from voxel face to voxel face; empty
 *                         voxels skipped; ties stepped in axis order x, y, z
 *   intersection ........ Sec. 4 / 4.1: tubes of a user radius around each
 *                         segment, closed by spheres at the joints (capsules);
 *                         a voxel only tests its own segments (interactive
 *                         mode, Sec. 4.1) and owns the hits whose entry point
 *                         lies in it (reading R1)
 *   per-voxel sort ...... Sec. 4: hits sorted in visibility order
 *   shading ............. Sec. 5: normal at the entering intersection and a
 *                         local illumination model (reading S1)
 *   compositing ......... Sec. 5.1: front-to-back alpha blending, opacity from
 *                         the transfer function, alpha termination
 *   shadows ............. Sec. 5.2, second approach: one ray toward the light
 *                         sampling the density LoD, coarser with distance
 *                         (cone opening of one finest voxel; reading S2)
 *   ambient occlusion ... Sec. 5.3, first approach: hemisphere rays around the
 *                         normal accumulate density until it reaches 1, the
 *                         ray passes the radius of influence or leaves the
 *                         domain; averaged over rays (reading S3)
 *
 * Tie flags: where a decision margin of the FP64 computation is so small that
 * a float32 evaluation of the same decision may go the other way, the pixel
 * is flagged (bit mask) and parity tests exclude and count it.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TIE_GRAZE 1
#define TIE_OWNER 2
#define TIE_SORT  4
#define TIE_FRAME 16
#define TIE_SLAB  32
#define TIE_SHADOW 64   /* a hit's binary visibility (shadows 2) is a near-tie */

static const double EPS_G = 7.5e-7;   /* |distance - radius| at a silhouette */
static const double EPS_T = 7.5e-7;   /* entry parameter vs voxel faces / other hits */
static const double ERR_Q = 7.5e-8;   /* float32 error of a squared distance, scaling the root term */
static const double EPS_F = 1e-5;     /* AO frame switch */
static const double FRAME_MIN = 1e-3; /* tangent shorter than this: axis fallback */

/* ------------------------------------------------------------------ vectors */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static void norm3(double *a) {
    double l = sqrt(dot3(a, a));
    a[0] /= l; a[1] /= l; a[2] /= l;
}

/* ------------------------------------------------------------------ camera (R0) */
typedef struct { float F[3], R[3], U[3], th, tw, eye[3]; int W, H; } cam32;

static void cam_setup(const orc_view *v, cam32 *c) {
    double f[3], up[3], r[3], u[3];
    for (int a = 0; a < 3; a++) {
        f[a] = (double)v->at[a] - (double)v->eye[a];
        up[a] = v->up[a];
    }
    norm3(f);
    cross3(f, up, r);
    norm3(r);
    cross3(r, f, u);
    double th = tan((double)v->fovy_deg * M_PI / 360.0);
    double tw = th * (double)v->width / (double)v->height;
    for (int a = 0; a < 3; a++) {
        c->F[a] = (float)f[a];
        c->R[a] = (float)r[a];
        c->U[a] = (float)u[a];
        c->eye[a] = v->eye[a];
    }
    c->th = (float)th;
    c->tw = (float)tw;
    c->W = v->width;
    c->H = v->height;
}

/* Single-precision ray of pixel (i, j): every operation rounds to float32 in
 * the order written (the library builds the identical float32 ray). */
static void cam_ray(const cam32 *c, int32_t i, int32_t j, float org[3], float dir[3]) {
    float px = (float)(2 * i + 1) / (float)c->W;
    float sx = (px - 1.0f) * c->tw;
    float py = (float)(2 * j + 1) / (float)c->H;
    float sy = (py - 1.0f) * c->th;
    float d[3];
    for (int a = 0; a < 3; a++) {
        float t = sx * c->R[a];
        float s = c->F[a] + t;
        float w = sy * c->U[a];
        d[a] = s - w;
    }
    float n2 = d[0] * d[0];
    float y2 = d[1] * d[1];
    n2 = n2 + y2;
    float z2 = d[2] * d[2];
    n2 = n2 + z2;
    float inv = 1.0f / sqrtf(n2);
    for (int a = 0; a < 3; a++) {
        dir[a] = d[a] * inv;
        org[a] = c->eye[a];
    }
}

void orc_primary_ray(const orc_view *view, int32_t i, int32_t j, float org[3], float dir[3]) {
    cam32 c;
    cam_setup(view, &c);
    cam_ray(&c, i, j, org, dir);
}

/* ------------------------------------------------------------------ segments */
static void face_point(int face, int u, int v, int N, double q[3]) {
    int a = face / 2;
    int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
    q[a] = (face & 1) ? 1.0 : 0.0;
    q[b0] = (u + 0.5) / N;             /* sub-square centre (Sec. 3.2) */
    q[b1] = (v + 0.5) / N;
}

static void seg_world(const orc_voxset *vs, const orc_seg *s, double a[3], double b[3]) {
    const int32_t *R = vs->grid.res;
    int64_t vid = s->voxel;
    double base[3] = {(double)(vid % R[0]), (double)((vid / R[0]) % R[1]), (double)(vid / ((int64_t)R[0] * R[1]))};
    face_point(s->face_in, s->u_in, s->v_in, vs->grid.bins, a);
    face_point(s->face_out, s->u_out, s->v_out, vs->grid.bins, b);
    for (int k = 0; k < 3; k++) { a[k] += base[k]; b[k] += base[k]; }
}

static int same_geometry(const orc_seg *x, const orc_seg *y) {
    return x->voxel == y->voxel && x->face_in == y->face_in && x->u_in == y->u_in &&
           x->v_in == y->v_in && x->face_out == y->face_out && x->u_out == y->u_out &&
           x->v_out == y->v_out;
}

/* Distance from the line o + t d to the segment [a, b]; *tc = line parameter
 * of the closest approach. The direction need not be unit: primary rays
 * carry a float32 direction whose length differs from 1 by ~1e-7. */
static double line_segment_distance(const double *o, const double *d, const double *a,
                                    const double *b, double *tc) {
    double ba[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double ao[3] = {a[0] - o[0], a[1] - o[1], a[2] - o[2]};
    double L2 = dot3(ba, ba), dd = dot3(d, d), k = dot3(d, ba);
    double h = 0.0;
    if (L2 > 0.0) {
        double det = dd * L2 - k * k;
        if (det > 1e-14 * dd * L2) {
            /* minimise |o + t d - a - h ba|^2 over t, h */
            double e = dot3(d, ao), f = dot3(ba, ao);
            h = (k * e - dd * f) / det;
        }
        if (h < 0.0) h = 0.0;
        if (h > 1.0) h = 1.0;
    }
    double c[3] = {a[0] + h * ba[0], a[1] + h * ba[1], a[2] + h * ba[2]};
    double co[3] = {c[0] - o[0], c[1] - o[1], c[2] - o[2]};
    double t = dot3(co, d) / dd;
    double p[3] = {o[0] + t * d[0] - c[0], o[1] + t * d[1] - c[1], o[2] + t * d[2] - c[2]};
    *tc = t;
    return sqrt(dot3(p, p));
}

/* Smaller root of |o + t d - c|^2 = r^2, solved around the closest approach
 * t_c = -(o - c).d / |d|^2: the squared distance of the centre from the line
 * is taken from the perpendicular vector itself, which does not cancel even
 * for an origin hundreds of radii away. *g = half chord length. */
static int sphere_entry(const double *o, const double *d, const double *c, double r,
                        double *t, double *g) {
    double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
    double dd = dot3(d, d);
    double tc = -dot3(oc, d) / dd;
    double q[3] = {oc[0] + tc * d[0], oc[1] + tc * d[1], oc[2] + tc * d[2]};
    double h = r * r - dot3(q, q);
    if (h < 0.0) return 0;
    *g = sqrt(h);
    *t = tc - *g / sqrt(dd);
    return 1;
}

/* Which surface a capsule entry lies on: its lateral body, or one of the
 * end spheres (then `c` is the sphere centre). `ymargin` is how far the body
 * candidate's axial coordinate lies from the end planes, i.e. how close the
 * body / sphere choice came to going the other way. */
typedef struct { double t, sens, c[3], ymargin; int part; } entry;

/* Capsule entry: the capsule is the union of the finite cylinder and the two
 * end spheres, so its first entry is the smallest of: the lateral entry into
 * the infinite cylinder when that point lies between the end planes, and the
 * entries into the two spheres. sens = 1 / (|d_perp| g), g the half chord,
 * scales the float32 error of the root. */
static int capsule_entry_s(const double *o, const double *d, const double *a, const double *b,
                           double r, entry *E) {
    double tc;
    if (line_segment_distance(o, d, a, b, &tc) > r) return 0;
    /* ray origin inside the capsule: no entering intersection ahead */
    {
        double ba[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, oa[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
        double L2 = dot3(ba, ba), h = L2 > 0.0 ? dot3(oa, ba) / L2 : 0.0;
        if (h < 0.0) h = 0.0;
        if (h > 1.0) h = 1.0;
        double q[3] = {oa[0] - h * ba[0], oa[1] - h * ba[1], oa[2] - h * ba[2]};
        if (dot3(q, q) <= r * r) return 0;
    }
    int found = 0;
    double ymargin = 1e300;
    double ba[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double L2 = dot3(ba, ba);
    if (L2 > 0.0) {
        double L = sqrt(L2);
        double w[3] = {ba[0] / L, ba[1] / L, ba[2] / L};
        double oa[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
        double dw = dot3(d, w), mw = dot3(oa, w);
        double dp[3] = {d[0] - dw * w[0], d[1] - dw * w[1], d[2] - dw * w[2]};
        double mp[3] = {oa[0] - mw * w[0], oa[1] - mw * w[1], oa[2] - mw * w[2]};
        /* |mp + t dp| = r, around the closest approach to the axis */
        double A = dot3(dp, dp);
        if (A > 0.0) {
            double tca = -dot3(dp, mp) / A;
            double q[3] = {mp[0] + tca * dp[0], mp[1] + tca * dp[1], mp[2] + tca * dp[2]};
            double h = r * r - dot3(q, q);
            if (h >= 0.0) {
                double s = sqrt(A), g = sqrt(h);
                double t = tca - g / s;
                double y = mw + t * dw;             /* axial coordinate of the entry point */
                ymargin = fmin(fabs(y), fabs(y - L));
                if (y >= 0.0 && y <= L) {
                    found = 1;
                    E->t = t;
                    E->part = 0;
                    E->sens = 1.0 / fmax(s * g, 1e-12);
                }
            }
        }
    }
    const double *cs[2] = {a, b};
    for (int k = 0; k < 2; k++) {
        double ts, g;
        if (sphere_entry(o, d, cs[k], r, &ts, &g) && (!found || ts < E->t)) {
            found = 1;
            E->t = ts;
            E->part = 1 + k;
            E->sens = 1.0 / fmax(g, 1e-12);
            for (int c = 0; c < 3; c++) E->c[c] = cs[k][c];
        }
    }
    E->ymargin = ymargin;
    if (!found || !(E->t > 0.0)) return 0;
    return 1;
}

int orc_capsule_entry(const double o[3], const double d[3], const double a[3],
                      const double b[3], double r, double *t, double *dist) {
    double tc;
    entry E;
    *dist = line_segment_distance(o, d, a, b, &tc);
    if (!capsule_entry_s(o, d, a, b, r, &E)) return 0;
    *t = E.t;
    return 1;
}

/* ------------------------------------------------------------------ LoD marches */
double orc_sample(const orc_lod *L, int l, const double x[3]) {
    double s = ldexp(1.0, l);
    double q[3], f[3];
    int64_t i0[3];
    for (int a = 0; a < 3; a++) {
        q[a] = x[a] / s - 0.5;                   /* cell-centred samples */
        double fl = floor(q[a]);
        i0[a] = (int64_t)fl;
        f[a] = q[a] - fl;
    }
    const int32_t *dm = L->dims[l];
    double acc = 0.0;
    for (int c = 0; c < 8; c++) {
        int64_t idx[3];
        double w = 1.0;
        int inside = 1;
        for (int a = 0; a < 3; a++) {
            int bit = (c >> a) & 1;
            idx[a] = i0[a] + bit;
            w *= bit ? f[a] : 1.0 - f[a];
            if (idx[a] < 0 || idx[a] >= dm[a]) inside = 0;   /* zero outside the grid */
        }
        if (inside) acc += w * L->dens[l][idx[0] + (int64_t)dm[0] * (idx[1] + (int64_t)dm[1] * idx[2])];
    }
    return acc / ldexp(1.0, 3 * l);              /* sum of 8^l voxels -> average */
}

/* Reading S4 (Sec. 5.3, second approach): occlusion over the whole sphere
 * around each voxel centre, from the level-0 density, in a pre-process.
 * Directions: spherical Fibonacci set over the sphere, z_i = 1 - (2i+1)/K,
 * phi_i = i pi (3 - sqrt 5); samples at unit steps s = 1 .. radius. */
void orc_ao_sphere_field(const orc_lod *L, int rays, double radius, double *field) {
    const int32_t *dm = L->dims[0];
    const int64_t n = (int64_t)dm[0] * dm[1] * dm[2];
    const double golden = M_PI * (3.0 - sqrt(5.0));
    double *dirs = (double *)malloc(sizeof(double) * 3 * (size_t)rays);
    for (int i = 0; i < rays; i++) {
        const double z = 1.0 - (2.0 * i + 1.0) / rays, rr = sqrt(1.0 - z * z), ph = i * golden;
        dirs[3 * i] = rr * cos(ph);
        dirs[3 * i + 1] = rr * sin(ph);
        dirs[3 * i + 2] = z;
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t v = 0; v < n; v++) {
        const double c[3] = {v % dm[0] + 0.5, (v / dm[0]) % dm[1] + 0.5, v / ((int64_t)dm[0] * dm[1]) + 0.5};
        double occ = 0.0;
        for (int k = 0; k < rays; k++) {
            double O = 0.0;
            for (int s = 1; s <= radius; s++) {
                const double x[3] = {c[0] + s * dirs[3 * k], c[1] + s * dirs[3 * k + 1], c[2] + s * dirs[3 * k + 2]};
                O += orc_sample(L, 0, x);
                if (O >= 1.0) break;
            }
            occ += fmin(1.0, O);
        }
        field[v] = 1.0 - occ / rays;
    }
    free(dirs);
}

double orc_ao_field_sample(const double *field, const int32_t dm[3], const double x[3]) {
    double f[3];
    int64_t i0[3];
    for (int a = 0; a < 3; a++) {
        double q = x[a] - 0.5;
        if (q < 0.0) q = 0.0;
        if (q > dm[a] - 1) q = dm[a] - 1;
        double fl = floor(q);
        if (fl > dm[a] - 2) fl = dm[a] - 2 < 0 ? 0 : dm[a] - 2;
        i0[a] = (int64_t)fl;
        f[a] = q - fl;
    }
    double acc = 0.0;
    for (int c = 0; c < 8; c++) {
        int64_t idx[3];
        double w = 1.0;
        for (int a = 0; a < 3; a++) {
            int bit = (c >> a) & 1;
            idx[a] = i0[a] + bit;
            if (idx[a] > dm[a] - 1) idx[a] = dm[a] - 1;
            w *= bit ? f[a] : 1.0 - f[a];
        }
        acc += w * field[idx[0] + (int64_t)dm[0] * (idx[1] + (int64_t)dm[1] * idx[2])];
    }
    return acc;
}

static int level_of(int64_t s, int levels) {
    int l = 0;
    while (((int64_t)2 << l) <= s) l++;          /* floor(log2 s) */
    return l < levels - 1 ? l : levels - 1;
}

/* Reading S2: start one voxel from the point, sample level l = floor(log2 s)
 * (capped at the coarsest level), add density * step, step 2^l; stop at
 * O >= 1, past max_dist, or once the sample point has left the domain of the
 * density field: the grid enlarged by half a coarsest-level cell, beyond
 * which every level's trilinear sample is exactly zero (a ray that has left
 * this convex box never re-enters it, so stopping there changes nothing). */
static double march(const orc_lod *L, const double *p, const double *dir,
                    double max_dist, uint64_t *nsamples) {
    const int top = L->levels - 1;
    const double cell = ldexp(1.0, top);
    double lo = -0.5 * cell, hi[3];
    for (int a = 0; a < 3; a++) hi[a] = ((double)L->dims[top][a] + 0.5) * cell;
    double O = 0.0;
    int64_t s = 1;
    for (;;) {
        if (max_dist >= 0.0 && (double)s > max_dist) break;
        double x[3];
        int outside = 0;
        for (int a = 0; a < 3; a++) {
            x[a] = p[a] + (double)s * dir[a];
            if (x[a] < lo || x[a] > hi[a]) outside = 1;
        }
        if (outside) break;
        int l = level_of(s, L->levels);
        O += orc_sample(L, l, x) * ldexp(1.0, l);
        (*nsamples)++;
        if (O >= 1.0) break;
        s += (int64_t)1 << l;
    }
    return O;
}

double orc_march(const orc_lod *L, const double p[3], const double dir[3], double max_dist) {
    uint64_t n = 0;
    return march(L, p, dir, max_dist, &n);
}

/* Reading S3: spherical-Fibonacci directions on the hemisphere around n, in
 * the frame whose tangent is the tube axis projected onto the tangent plane
 * (fallback: the world axis least aligned with n). */
static void ao_dirs_t(const double *n, const double *u, int k, double *dirs, double *fmargin) {
    double un = dot3(u, n);
    double T[3] = {u[0] - un * n[0], u[1] - un * n[1], u[2] - un * n[2]};
    double m = sqrt(dot3(T, T));
    *fmargin = fabs(m - FRAME_MIN) / EPS_F;
    if (m >= FRAME_MIN) {
        T[0] /= m; T[1] /= m; T[2] /= m;
    } else {
        double an[3] = {fabs(n[0]), fabs(n[1]), fabs(n[2])};
        int e = 0;
        for (int a = 1; a < 3; a++) if (an[a] < an[e]) e = a;
        for (int a = 0; a < 3; a++)
            if (a != e) *fmargin = fmin(*fmargin, fabs(an[a] - an[e]) / EPS_F);
        double E[3] = {0, 0, 0};
        E[e] = 1.0;
        double en = dot3(E, n);
        for (int a = 0; a < 3; a++) T[a] = E[a] - en * n[a];
        norm3(T);
    }
    double B[3];
    cross3(n, T, B);
    const double golden = M_PI * (3.0 - sqrt(5.0));
    for (int i = 0; i < k; i++) {
        double z = 1.0 - (i + 0.5) / k;
        double rr = sqrt(1.0 - z * z);
        double ph = i * golden;
        double x = rr * cos(ph), y = rr * sin(ph);
        for (int a = 0; a < 3; a++) dirs[3 * i + a] = T[a] * x + B[a] * y + n[a] * z;
    }
}

void orc_ao_dirs(const double n[3], const double u[3], int k, double *dirs) {
    double fm;
    ao_dirs_t(n, u, k, dirs, &fm);
}

/* ------------------------------------------------------------------ per-pixel state */
typedef struct {
    double C[3], A;
    float A32;          /* the termination decision, in float32 */
    int done;
    int tie;
    double margin;      /* smallest decision margin, in units of its tie threshold */
    double flip;        /* shadows 2: sum over hits whose visibility is a near-tie of
                           the most a flip of it can move the pixel's colour */
    uint64_t nvox, nrec, nsamp, nhit;
    /* depth-sort near-ties: how many, and where the last one was (the voxel's
       ordinal along the ray and the pair's position in its sorted hits) */
    int nsort;
    int64_t sort_vox, sort_i;
    /* input of a second pass: swap the sorted pair (swap_i, swap_i + 1) of
       voxel ordinal swap_vox (-1: none) */
    int64_t swap_vox, swap_i;
} pixstate;

static void note(pixstate *ps, double m, int bit) {
    if (m < ps->margin) ps->margin = m;
    if (m < 1.0) ps->tie |= bit;
}

typedef struct { double t, eps; int64_t k; entry e; } hit;

static int hit_cmp(const void *x, const void *y) {
    const hit *a = (const hit *)x, *b = (const hit *)y;
    if (a->t < b->t) return -1;
    if (a->t > b->t) return 1;
    return (a->k > b->k) - (a->k < b->k);
}

/* Reading S5: hard shadow against the representative lines of one level.
 * The half-line starts one cell size of that level toward the light and
 * crosses that level's cells; blocked if it comes within radius x 2^level
 * of the line of a crossed cell. Near-grazes and near-edge crossings are
 * flagged. */
/* Reading S5's visibility is binary, and the library finds hit points in
 * float32: the hit point v + p_local is rounded once to float32 (half an ulp,
 * 1.5e-5 voxel below 256 and 3e-5 below 512, far above the float-float
 * local point's own error) and the walk's start point, the hit plus one cell
 * toward the light, once more; the distance tests on O(1) cell coordinates
 * add about 1e-6. A pixel is a tie when a visited cell's line lies within
 * EPS_SH x (cell size of the level) of the threshold distance, or when the
 * walk's cell sequence is decided by less than EPS_SH (level cell units: the
 * start cell, or two crossings of one step) and one of the cells the other
 * choice would visit holds a line within that margin of blocking. EPS_SH =
 * 1e-4 is 3x the error bound for grids up to 256^3 and 1.6x up to 512^3. */
static const double EPS_SH = 1e-4;
/* a quarter of the 2e-3 per-channel tolerance the parity tests use */
static const double FLIP_MIN = 5e-4;

/* distance from the half-line S + t Lt to the line of cell (x, y, z), or
 * +inf when the cell is outside the level or has no line */
static double rep_cell_distance(const orc_reps *R, int l, int N, const int64_t v[3], const double *S,
                                const double *Lt) {
    const int32_t *dm = R->dims[l];
    for (int a = 0; a < 3; a++)
        if (v[a] < 0 || v[a] >= dm[a]) return 1e300;
    const int64_t cell = v[0] + (int64_t)dm[0] * (v[1] + (int64_t)dm[1] * v[2]);
    if (!R->rep[l][7 * cell]) return 1e300;
    double a[3], b[3];
    orc_rep_world(R, l, cell, N, a, b);
    return orc_halfline_segment_distance(S, Lt, a, b);
}

/* flag an owner tie when a cell that the other choice visits could block */
static void note_alt(pixstate *ps, const orc_reps *R, int l, int N, const int64_t v[3], const double *S,
                     const double *Lt, double rl, double tol) {
    if (rep_cell_distance(R, l, N, v, S, Lt) <= rl + tol) note(ps, 0.0, TIE_OWNER);
}

static double shadow_reps(const orc_voxset *vs, const orc_rdesc *rd, const double *P, const double *Lt,
                          pixstate *ps) {
    const orc_reps *R = rd->reps;
    const int l = rd->shadow_level;
    const double size = ldexp(1.0, l), rl = rd->radius * size, tol = EPS_SH * size;
    const int32_t *dm = R->dims[l];
    const int N = vs->grid.bins;
    double S[3], q[3];
    for (int a = 0; a < 3; a++) {
        S[a] = P[a] + size * Lt[a];
        q[a] = S[a] / size;                       /* level-l cell coordinates */
    }
    /* enter the level's grid */
    double tnear = 0.0, tfar = 1e300;
    for (int a = 0; a < 3; a++) {
        if (Lt[a] != 0.0) {
            double t1 = (0.0 - q[a]) / Lt[a], t2 = ((double)dm[a] - q[a]) / Lt[a];
            tnear = fmax(tnear, fmin(t1, t2));
            tfar = fmin(tfar, fmax(t1, t2));
        } else if (q[a] < 0.0 || q[a] > dm[a]) {
            return 1.0;
        }
    }
    if (!(tnear < tfar)) return 1.0;
    int64_t v[3], step[3];
    double tmax[3], x[3];
    for (int a = 0; a < 3; a++) {
        x[a] = q[a] + tnear * Lt[a];
        int64_t vi = (int64_t)floor(x[a]);
        if (vi < 0) vi = 0;
        if (vi > dm[a] - 1) vi = dm[a] - 1;
        v[a] = vi;
        step[a] = Lt[a] > 0.0 ? 1 : (Lt[a] < 0.0 ? -1 : 0);
        tmax[a] = step[a] == 0 ? 1e300 : ((double)(step[a] > 0 ? vi + 1 : vi) - q[a]) / Lt[a];
    }
    /* the start cell: a coordinate within EPS_SH of a cell boundary */
    for (int a = 0; a < 3; a++) {
        const double fr = x[a] - floor(x[a]);
        if (fr < EPS_SH || fr > 1.0 - EPS_SH) {
            int64_t w[3] = {v[0], v[1], v[2]};
            w[a] += fr < EPS_SH ? -1 : 1;
            note_alt(ps, R, l, N, w, S, Lt, rl, tol);
        }
    }
    for (;;) {
        const double dist = rep_cell_distance(R, l, N, v, S, Lt);
        if (dist < 1e299) {
            note(ps, fabs(dist - rl) / tol, TIE_GRAZE);
            if (dist <= rl) return 0.0;
        }
        int ax = 0;
        for (int a = 1; a < 3; a++) if (tmax[a] < tmax[ax]) ax = a;
        /* near-simultaneous crossings: the other orders visit v + e_a (and,
         * with three, v + e_a + e_b) instead of v + e_ax */
        int tied[3], nt = 0;
        for (int a = 0; a < 3; a++)
            if (tmax[a] < 1e299 && fabs(tmax[a] - tmax[ax]) < EPS_SH) tied[nt++] = a;
        if (nt > 1)
            for (int m = 1; m < (1 << nt) - 1; m++) {
                int64_t w[3] = {v[0], v[1], v[2]};
                for (int i = 0; i < nt; i++)
                    if (m >> i & 1) w[tied[i]] += step[tied[i]];
                note_alt(ps, R, l, N, w, S, Lt, rl, tol);
            }
        v[ax] += step[ax];
        if (v[ax] < 0 || v[ax] >= dm[ax]) break;
        tmax[ax] = ((double)(step[ax] > 0 ? v[ax] + 1 : v[ax]) - q[ax]) / Lt[ax];
    }
    return 1.0;
}

double orc_shadow_reps_visibility(const orc_voxset *vs, const orc_reps *reps, float radius, int level,
                                  const double P[3], const double Lt[3]) {
    orc_rdesc rd;
    memset(&rd, 0, sizeof rd);
    rd.radius = radius;
    rd.reps = reps;
    rd.shadow_level = level;
    pixstate ps;
    memset(&ps, 0, sizeof ps);
    ps.margin = 1e300;
    return shadow_reps(vs, &rd, P, Lt, &ps);
}

/* Shade one hit (reading S1) and composite it front to back (Sec. 5.1). */
static void shade_composite(const orc_voxset *vs, const orc_lod *L, const orc_rdesc *rd,
                            const double *O, const double *D, const double *Lt,
                            const hit *h, pixstate *ps) {
    const orc_seg *s = &vs->seg[h->k];
    double a[3], b[3];
    seg_world(vs, s, a, b);
    double P[3] = {O[0] + h->t * D[0], O[1] + h->t * D[1], O[2] + h->t * D[2]};
    double ba[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double L2 = dot3(ba, ba), hh = 0.0;
    if (L2 > 0.0) {
        double pa[3] = {P[0] - a[0], P[1] - a[1], P[2] - a[2]};
        hh = dot3(pa, ba) / L2;
        if (hh < 0.0) hh = 0.0;
        if (hh > 1.0) hh = 1.0;
    }
    double n[3] = {P[0] - (a[0] + hh * ba[0]), P[1] - (a[1] + hh * ba[1]), P[2] - (a[2] + hh * ba[2])};
    norm3(n);
    const float *tf = rd->tf + 4 * s->attr;
    double alpha = rd->opaque ? 1.0 : (double)tf[3];

    double V = 1.0, AO = 1.0;
    if (rd->shadows == 2 && rd->reps) {
        /* the visibility is binary and enters only this hit's diffuse term
         * (S1), so a flip of it moves the pixel by at most w kd |n.L| max(rgb)
         * (w: its compositing weight); near-ties add that to the pixel's flip
         * budget, and those whose flip reaches FLIP_MIN also flag the pixel */
        pixstate sh = *ps;
        sh.tie = 0;
        sh.margin = 1e300;
        V = shadow_reps(vs, rd, P, Lt, &sh);
        const double w = rd->opaque ? 1.0 : (1.0 - ps->A) * alpha;
        const double cmax = fmax((double)tf[0], fmax((double)tf[1], (double)tf[2]));
        const double dmax = w * rd->kd * fabs(dot3(n, Lt)) * cmax;
        if (sh.tie) ps->flip += dmax;
        if (dmax >= FLIP_MIN) {
            if (sh.tie) ps->tie |= TIE_SHADOW;
            ps->margin = fmin(ps->margin, sh.margin);
        }
    } else if (rd->shadows && L) V = 1.0 - fmin(1.0, march(L, P, Lt, -1.0, &ps->nsamp));
    if (rd->ao == 3 && L && rd->ao_field) {
        AO = orc_ao_field_sample(rd->ao_field, L->dims[0], P);
    } else if (rd->ao == 2 && L && rd->ao_params) {
        double t[3], x[512];
        orc_ao_tangent(a, b, t);
        if (orc_ao_features(L, s->voxel, t, n, P, x) == 0) AO = orc_ao_mlp(rd->ao_params, x);
        else AO = NAN;
    } else if (rd->ao && L && rd->ao_rays > 0) {
        double u[3] = {ba[0], ba[1], ba[2]};
        if (L2 > 0.0) { double l = sqrt(L2); u[0] /= l; u[1] /= l; u[2] /= l; }
        double *dirs = (double *)malloc(sizeof(double) * 3 * (size_t)rd->ao_rays);
        double fm;
        ao_dirs_t(n, u, rd->ao_rays, dirs, &fm);
        note(ps, fm, TIE_FRAME);
        double occ = 0.0;
        for (int i = 0; i < rd->ao_rays; i++)
            occ += fmin(1.0, march(L, P, dirs + 3 * i, rd->ao_radius, &ps->nsamp));
        free(dirs);
        AO = 1.0 - occ / rd->ao_rays;
    }
    double diff = fabs(dot3(n, Lt));
    double k = rd->ka * AO + rd->kd * V * diff;
    ps->nhit++;
    if (rd->opaque) {
        for (int c = 0; c < 3; c++) ps->C[c] = tf[c] * k;
        ps->A = 1.0;
        ps->done = 1;
        return;
    }
    double w = (1.0 - ps->A) * alpha;
    for (int c = 0; c < 3; c++) ps->C[c] += w * tf[c] * k;
    ps->A += w;
    float t1 = 1.0f - ps->A32;
    float t2 = t1 * tf[3];
    ps->A32 = ps->A32 + t2;
    if (ps->A32 >= rd->ert_alpha) ps->done = 1;
}

/* Two hits closer in depth than their error bounds may swap under float32 -
 * unless they are one surface: two capsules entered through the same joint
 * sphere give bit-identical roots on both sides and keep index order. */
static const double YMARGIN = 1e-4;
static void flag_sorted_ties(const orc_voxset *vs, const hit *hs, int nh, pixstate *ps) {
    for (int i = 0; i + 1 < nh; i++) {
        const hit *x = &hs[i], *y = &hs[i + 1];
        if (same_geometry(&vs->seg[x->k], &vs->seg[y->k])) continue;
        if (x->e.part && y->e.part && x->e.c[0] == y->e.c[0] && x->e.c[1] == y->e.c[1] &&
            x->e.c[2] == y->e.c[2] && x->e.ymargin > YMARGIN && y->e.ymargin > YMARGIN)
            continue;
        const double m = (y->t - x->t) / (x->eps + y->eps);
        note(ps, m, TIE_SORT);
        if (m < 1.0) {
            ps->nsort++;
            ps->sort_vox = (int64_t)ps->nvox;
            ps->sort_i = i;
        }
    }
}

/* Sec. 4.1's line-id rule (reading R2): among one voxel's hits, sorted by
 * (depth, index), keep only the first of each local line id (curve index
 * mod 32, the record's 5-bit id). Returns the new count. */
static int dedup_line_ids(const orc_voxset *vs, hit *hs, int nh) {
    uint32_t seen = 0;
    int m = 0;
    for (int i = 0; i < nh; i++) {
        const uint32_t id = 1u << (vs->seg[hs[i].k].curve & 31u);
        if (seen & id) continue;
        seen |= id;
        hs[m++] = hs[i];
    }
    return m;
}

/* One ray by DDA traversal (Sec. 4). */
static void trace_dda(const orc_voxset *vs, const orc_lod *L, const orc_rdesc *rd,
                      const double *O, const double *D, const double *Lt, pixstate *ps,
                      hit **buf, int *bufcap) {
    const int32_t *R = vs->grid.res;
    double tnear = -1e300, tfar = 1e300;
    for (int a = 0; a < 3; a++) {
        if (D[a] != 0.0) {
            double t1 = (0.0 - O[a]) / D[a], t2 = ((double)R[a] - O[a]) / D[a];
            tnear = fmax(tnear, fmin(t1, t2));
            tfar = fmin(tfar, fmax(t1, t2));
        } else if (O[a] < 0.0 || O[a] > R[a]) {
            return;
        }
    }
    if (tnear < 0.0) tnear = 0.0;
    note(ps, fabs(tfar - tnear) / 1e-5, TIE_SLAB);
    if (!(tnear < tfar)) return;
    int64_t v[3], step[3];
    double tmax[3];
    for (int a = 0; a < 3; a++) {
        double p = O[a] + tnear * D[a];
        int64_t vi = (int64_t)floor(p);
        if (vi < 0) vi = 0;
        if (vi > R[a] - 1) vi = R[a] - 1;
        v[a] = vi;
        step[a] = D[a] > 0.0 ? 1 : (D[a] < 0.0 ? -1 : 0);
    }
    for (int a = 0; a < 3; a++)
        tmax[a] = step[a] == 0 ? 1e300
                : ((double)(step[a] > 0 ? v[a] + 1 : v[a]) - O[a]) / D[a];
    double t0 = tnear;
    const double r = rd->radius;
    while (!ps->done) {
        int ax = 0;
        for (int a = 1; a < 3; a++) if (tmax[a] < tmax[ax]) ax = a;
        double t1 = tmax[ax];
        ps->nvox++;
        /* candidate segments: those stored in this voxel, or (camera at rest,
         * reading R2) in this voxel and its 26 neighbours */
        const int reach = rd->still ? 1 : 0;
        int nh = 0;
        for (int dz = -reach; dz <= reach; dz++)
            for (int dy = -reach; dy <= reach; dy++)
                for (int dx = -reach; dx <= reach; dx++) {
                    const int64_t X = v[0] + dx, Y = v[1] + dy, Z = v[2] + dz;
                    if (X < 0 || Y < 0 || Z < 0 || X >= R[0] || Y >= R[1] || Z >= R[2]) continue;
                    const int64_t vid = X + (int64_t)R[0] * (Y + (int64_t)R[1] * Z);
                    const uint32_t beg = vs->offset[vid], end = vs->offset[vid + 1];
                    if (end == beg) continue;
                    ps->nrec += end - beg;
                    if (nh + (int)(end - beg) > *bufcap) {
                        *bufcap = nh + (int)(end - beg) + 64;
                        *buf = (hit *)realloc(*buf, sizeof(hit) * (size_t)*bufcap);
                    }
                    for (uint32_t k = beg; k < end; k++) {
                        double a[3], b[3], tc;
                        entry E;
                        seg_world(vs, &vs->seg[k], a, b);
                        double dist = line_segment_distance(O, D, a, b, &tc);
                        if (tc > t0 - 0.01 && tc < t1 + 0.01) note(ps, fabs(dist - r) / EPS_G, TIE_GRAZE);
                        if (!capsule_entry_s(O, D, a, b, r, &E)) continue;
                        double t = E.t, eps = EPS_T + ERR_Q * E.sens;
                        note(ps, fmin(fabs(t - t0), fabs(t - t1)) / eps, TIE_OWNER);
                        if (t >= t0 && t < t1) {
                            (*buf)[nh].t = t; (*buf)[nh].eps = eps; (*buf)[nh].k = k; (*buf)[nh].e = E;
                            nh++;
                        }
                    }
                }
        if (nh > 0) {
            qsort(*buf, (size_t)nh, sizeof(hit), hit_cmp);
            flag_sorted_ties(vs, *buf, nh, ps);
            if ((int64_t)ps->nvox == ps->swap_vox && ps->swap_i + 1 < nh) {   /* the other order of a near-tie */
                const hit x = (*buf)[ps->swap_i];
                (*buf)[ps->swap_i] = (*buf)[ps->swap_i + 1];
                (*buf)[ps->swap_i + 1] = x;
            }
            if (rd->still) nh = dedup_line_ids(vs, *buf, nh);
            for (int i = 0; i < nh && !ps->done; i++) shade_composite(vs, L, rd, O, D, Lt, &(*buf)[i], ps);
        }
        if (ps->done) break;
        t0 = t1;
        v[ax] += step[ax];
        if (v[ax] < 0 || v[ax] >= R[ax]) break;
        tmax[ax] = ((double)(step[ax] > 0 ? v[ax] + 1 : v[ax]) - O[ax]) / D[ax];
    }
}

/* One ray by brute force with the camera at rest (reading R2): every capsule
 * of every voxel; a hit belongs to the grid cell that holds its entry point
 * (dropped outside the grid); per cell the first hit of each line id is
 * kept; globally sorted by depth. */
static void trace_brute_still(const orc_voxset *vs, const orc_lod *L, const orc_rdesc *rd,
                              const double *O, const double *D, const double *Lt, pixstate *ps) {
    const int32_t *R = vs->grid.res;
    const double r = rd->radius;
    int64_t cap = 64, nh = 0;
    hit *hs = (hit *)malloc(sizeof(hit) * (size_t)cap);
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    for (int64_t k = 0; k < vs->nseg; k++) {
        double a[3], b[3], tc;
        entry E;
        seg_world(vs, &vs->seg[k], a, b);
        double dist = line_segment_distance(O, D, a, b, &tc);
        note(ps, fabs(dist - r) / EPS_G, TIE_GRAZE);
        if (!capsule_entry_s(O, D, a, b, r, &E)) continue;
        double t = E.t, eps = EPS_T + ERR_Q * E.sens;
        double P[3] = {O[0] + t * D[0], O[1] + t * D[1], O[2] + t * D[2]};
        int64_t c[3];
        int inside = 1;
        double margin = 1e300;
        for (int a3 = 0; a3 < 3; a3++) {
            c[a3] = (int64_t)floor(P[a3]);
            if (c[a3] < 0 || c[a3] >= R[a3]) inside = 0;
            if (D[a3] != 0.0) {
                margin = fmin(margin, fabs(P[a3] - c[a3]) / fabs(D[a3]));
                margin = fmin(margin, fabs(P[a3] - (c[a3] + 1)) / fabs(D[a3]));
            }
        }
        note(ps, margin / eps, TIE_OWNER);
        if (!inside) continue;
        if (nh == cap) {
            cap *= 2;
            hs = (hit *)realloc(hs, sizeof(hit) * (size_t)cap);
            cell = (int64_t *)realloc(cell, sizeof(int64_t) * (size_t)cap);
        }
        hs[nh].t = t; hs[nh].eps = eps; hs[nh].k = k; hs[nh].e = E;
        nh++;
    }
    qsort(hs, (size_t)nh, sizeof(hit), hit_cmp);
    flag_sorted_ties(vs, hs, (int)nh, ps);
    /* first hit of each (cell, line id) */
    int64_t m = 0;
    for (int64_t i = 0; i < nh; i++) {
        const double *t_ = &hs[i].t;
        double P[3] = {O[0] + *t_ * D[0], O[1] + *t_ * D[1], O[2] + *t_ * D[2]};
        const int64_t ci = (int64_t)floor(P[0]) + (int64_t)R[0] * ((int64_t)floor(P[1]) + (int64_t)R[1] * (int64_t)floor(P[2]));
        const uint32_t id = vs->seg[hs[i].k].curve & 31u;
        int dup = 0;
        for (int64_t j = 0; j < m; j++)
            if (cell[j] == ci && (vs->seg[hs[j].k].curve & 31u) == id) { dup = 1; break; }
        if (dup) continue;
        cell[m] = ci;
        hs[m++] = hs[i];
    }
    for (int64_t i = 0; i < m && !ps->done; i++) shade_composite(vs, L, rd, O, D, Lt, &hs[i], ps);
    free(hs);
    free(cell);
}

/* One ray by brute force: every capsule of every voxel, kept iff its entry
 * point lies in the voxel that stores it; globally sorted by depth. */
static void trace_brute(const orc_voxset *vs, const orc_lod *L, const orc_rdesc *rd,
                        const double *O, const double *D, const double *Lt, pixstate *ps) {
    const int32_t *R = vs->grid.res;
    const double r = rd->radius;
    int64_t cap = 64, nh = 0;
    hit *hs = (hit *)malloc(sizeof(hit) * (size_t)cap);
    for (int64_t vid = 0; vid < vs->nvox; vid++) {
        uint32_t beg = vs->offset[vid], end = vs->offset[vid + 1];
        if (beg == end) continue;
        int64_t vx = vid % R[0], vy = (vid / R[0]) % R[1], vz = vid / ((int64_t)R[0] * R[1]);
        int64_t vv[3] = {vx, vy, vz};
        for (uint32_t k = beg; k < end; k++) {
            double a[3], b[3], tc;
            entry E;
            seg_world(vs, &vs->seg[k], a, b);
            double dist = line_segment_distance(O, D, a, b, &tc);
            {
                /* only matters if the grazing point is in this voxel */
                double P[3] = {O[0] + tc * D[0], O[1] + tc * D[1], O[2] + tc * D[2]};
                int near = 1;
                for (int c = 0; c < 3; c++)
                    if (P[c] < vv[c] - 0.01 || P[c] > vv[c] + 1.01) near = 0;
                if (near) note(ps, fabs(dist - r) / EPS_G, TIE_GRAZE);
            }
            if (!capsule_entry_s(O, D, a, b, r, &E)) continue;
            double t = E.t, eps = EPS_T + ERR_Q * E.sens;
            double P[3] = {O[0] + t * D[0], O[1] + t * D[1], O[2] + t * D[2]};
            int own = 1;
            double margin = 1e300;
            for (int c = 0; c < 3; c++) {
                if (P[c] < vv[c] || P[c] >= vv[c] + 1) own = 0;
                if (D[c] != 0.0) {
                    margin = fmin(margin, fabs(P[c] - vv[c]) / fabs(D[c]));
                    margin = fmin(margin, fabs(P[c] - (vv[c] + 1)) / fabs(D[c]));
                }
            }
            note(ps, margin / eps, TIE_OWNER);
            if (!own) continue;
            if (nh == cap) { cap *= 2; hs = (hit *)realloc(hs, sizeof(hit) * (size_t)cap); }
            hs[nh].t = t; hs[nh].eps = eps; hs[nh].k = k; hs[nh].e = E;
            nh++;
        }
    }
    qsort(hs, (size_t)nh, sizeof(hit), hit_cmp);
    flag_sorted_ties(vs, hs, (int)nh, ps);
    for (int64_t i = 0; i < nh && !ps->done; i++) shade_composite(vs, L, rd, O, D, Lt, &hs[i], ps);
    free(hs);
}

int orc_render(const orc_voxset *vs, const orc_lod *L, const orc_view *view,
               const orc_rdesc *rd, const int32_t *pix, int64_t npix, int mode,
               double *rgba, uint8_t *tie, double *margin, double *flip, double *alt,
               uint64_t *counters, int nthreads) {
    if ((rd->shadows == 1 || rd->ao) && !L) return ORC_EINVAL;
    if (rd->shadows == 2 && (!rd->reps || rd->shadow_level < 0 || rd->shadow_level >= rd->reps->levels))
        return ORC_EINVAL;
    if (rd->ao == 3 && !rd->ao_field) return ORC_EINVAL;
    if (view->width < 1 || view->height < 1 || !(rd->radius > 0.0f)) return ORC_EINVAL;
    cam32 cam;
    cam_setup(view, &cam);
    double Lt[3];
    {
        double ld[3] = {view->light_dir[0], view->light_dir[1], view->light_dir[2]};
        norm3(ld);
        /* toward the light, rounded to float32 like the library's copy */
        for (int a = 0; a < 3; a++) Lt[a] = (double)(float)(-ld[a]);
    }
    uint64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(+ : c0, c1, c2, c3)
#endif
    {
        hit *buf = NULL;
        int bufcap = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t p = 0; p < npix; p++) {
            float o32[3], d32[3];
            cam_ray(&cam, pix[2 * p], pix[2 * p + 1], o32, d32);
            double O[3] = {o32[0], o32[1], o32[2]}, D[3] = {d32[0], d32[1], d32[2]};
            pixstate ps;
            memset(&ps, 0, sizeof ps);
            ps.margin = 1e300;
            ps.swap_vox = -1;
            if (mode == ORC_RENDER_BRUTE && rd->still) trace_brute_still(vs, L, rd, O, D, Lt, &ps);
            else if (mode == ORC_RENDER_BRUTE) trace_brute(vs, L, rd, O, D, Lt, &ps);
            else trace_dda(vs, L, rd, O, D, Lt, &ps, &buf, &bufcap);
            for (int c = 0; c < 3; c++) rgba[4 * p + c] = ps.C[c] + (1.0 - ps.A) * rd->bg[c];
            rgba[4 * p + 3] = ps.A;
            if (alt) {
                /* a pixel whose only near-tie is one depth order has two
                 * right answers: the second composites that pair the other
                 * way round */
                for (int c = 0; c < 4; c++) alt[4 * p + c] = NAN;
                if (mode != ORC_RENDER_BRUTE && ps.tie == TIE_SORT && ps.nsort == 1) {
                    pixstate ps2;
                    memset(&ps2, 0, sizeof ps2);
                    ps2.margin = 1e300;
                    ps2.swap_vox = ps.sort_vox;
                    ps2.swap_i = ps.sort_i;
                    trace_dda(vs, L, rd, O, D, Lt, &ps2, &buf, &bufcap);
                    for (int c = 0; c < 3; c++) alt[4 * p + c] = ps2.C[c] + (1.0 - ps2.A) * rd->bg[c];
                    alt[4 * p + 3] = ps2.A;
                }
            }
            if (tie) tie[p] = (uint8_t)ps.tie;
            if (margin) margin[p] = ps.margin;
            if (flip) flip[p] = ps.flip;
            c0 += ps.nvox; c1 += ps.nrec; c2 += ps.nsamp; c3 += ps.nhit;
        }
        free(buf);
    }
    if (counters) { counters[0] = c0; counters[1] = c1; counters[2] = c2; counters[3] = c3; }
    return ORC_OK;
}

/* ------------------------------------------------------------------ rasterised comparison system
 * Reading K1 (the paper's comparison system: tubes built around the input
 * lines by the rasteriser, per-pixel fragment lists sorted by depth and
 * blended front to back, Secs. 1 and 5.1). The input polylines are used
 * directly (no voxel model). Vertex i of a curve maps to grid coordinates
 * p = fl32(fl32(v - origin) * scale) (the voxeliser's float32 step, without
 * its fixed-point snap); consecutive vertices (v_i, v_i+1) form one capsule
 * of radius r (the tube piece closed by spheres at both ends), with the
 * attribute byte floor(((A_i + A_i+1) 255 + 65535) / 131070) of the two
 * vertices' 16-bit codes. A pixel's ray leaves one fragment per capsule it
 * enters (entry parameter > 0, origin outside), with no voxel ownership;
 * the fragments are sorted by (entry parameter, capsule index) and blended
 * front to back with S1's shading (no shadows or AO) until the float32
 * accumulated opacity reaches ert_alpha (> 1: every fragment, as the paper's
 * lists do); opaque mode keeps the nearest fragment. */
typedef struct { double a[3], b[3]; uint8_t attr; } rseg;

static int raster_segments(const float *xyz, const float *attr, const int64_t *offsets, int64_t nc,
                           const orc_grid *g, rseg **out, int64_t *nout) {
    const int64_t nv = offsets[nc];
    uint16_t *A = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)(nv > 0 ? nv : 1));
    if (!A) return ORC_ENOMEM;
    int st = orc_attr16(attr, nv, g->attr_min, g->attr_max, A);
    if (st) { free(A); return st; }
    int64_t n = 0;
    for (int64_t c = 0; c < nc; c++)
        if (offsets[c + 1] - offsets[c] > 1) n += offsets[c + 1] - offsets[c] - 1;
    rseg *S = (rseg *)malloc(sizeof(rseg) * (size_t)(n > 0 ? n : 1));
    if (!S) { free(A); return ORC_ENOMEM; }
    int64_t k = 0;
    for (int64_t c = 0; c < nc; c++)
        for (int64_t i = offsets[c]; i + 1 < offsets[c + 1]; i++) {
            rseg *s = &S[k++];
            for (int a = 0; a < 3; a++) {
                float d0 = xyz[3 * i + a] - g->origin[a], d1 = xyz[3 * (i + 1) + a] - g->origin[a];
                float p0 = d0 * g->scale, p1 = d1 * g->scale;
                s->a[a] = p0;
                s->b[a] = p1;
            }
            s->attr = (uint8_t)(((int64_t)(A[i] + A[i + 1]) * 255 + 65535) / 131070);
        }
    free(A);
    *out = S;
    *nout = n;
    return ORC_OK;
}

static int raster_hit_cmp(const void *x, const void *y) { return hit_cmp(x, y); }

/* S1 shading of capsule s entered at depth t: rgb * (ka + kd |n . Lt|) */
static void raster_color(const rseg *s, const orc_rdesc *rd, const double *O, const double *D, double t,
                         const double *Lt, double c[3]) {
    double P[3] = {O[0] + t * D[0], O[1] + t * D[1], O[2] + t * D[2]};
    double ba[3] = {s->b[0] - s->a[0], s->b[1] - s->a[1], s->b[2] - s->a[2]};
    double L2 = dot3(ba, ba), h = 0.0;
    if (L2 > 0.0) {
        double pa[3] = {P[0] - s->a[0], P[1] - s->a[1], P[2] - s->a[2]};
        h = dot3(pa, ba) / L2;
        if (h < 0.0) h = 0.0;
        if (h > 1.0) h = 1.0;
    }
    double n[3] = {P[0] - (s->a[0] + h * ba[0]), P[1] - (s->a[1] + h * ba[1]), P[2] - (s->a[2] + h * ba[2])};
    norm3(n);
    const float *tf = rd->tf + 4 * s->attr;
    const double kk = rd->ka + rd->kd * fabs(dot3(n, Lt));
    for (int q = 0; q < 3; q++) c[q] = tf[q] * kk;
}

/* a quarter of the 2e-3 per-channel tolerance the parity tests use */
static const double SWAP_MIN = 5e-4;

/* Blend the sorted fragments of one pixel front to back (opaque: the
 * nearest); swap >= 1 blends fragments swap - 1 and swap in the other order.
 * Only decisions about the blended fragments matter: two neighbours in depth
 * order (the second may be the first one not blended) closer than their
 * error bounds may swap, unless both entered one joint sphere
 * (bit-identical roots); a swap moves the pixel by T a_i a_i+1 (c_i -
 * c_i+1), flagged from SWAP_MIN on (opaque: c_0 - c_1). Returns the number
 * of fragments blended. */
static int64_t raster_blend(const rseg *S, hit *hs, int64_t nh, const orc_rdesc *rd, const double *O,
                            const double *D, const double *Lt, pixstate *ps, int64_t swap) {
    if (swap >= 1 && swap < nh) {
        const hit x = hs[swap - 1];
        hs[swap - 1] = hs[swap];
        hs[swap] = x;
    }
    int64_t m = 0;   /* fragments blended */
    double Tprev = 1.0, cprev[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i <= nh; i++) {
        double c[3] = {0.0, 0.0, 0.0};
        const float *tf = i < nh ? rd->tf + 4 * S[hs[i].k].attr : NULL;
        if (i < nh) raster_color(&S[hs[i].k], rd, O, D, hs[i].t, Lt, c);
        if (i > 0 && i < nh) {
            const entry *x = &hs[i - 1].e, *y = &hs[i].e;
            const int same = x->part && y->part && x->c[0] == y->c[0] && x->c[1] == y->c[1] &&
                             x->c[2] == y->c[2];
            const double aa = rd->opaque ? 1.0 : (double)rd->tf[4 * S[hs[i - 1].k].attr + 3] * tf[3];
            double dc = 0.0;
            for (int q = 0; q < 3; q++) dc = fmax(dc, fabs(c[q] - cprev[q]));
            if (!same && Tprev * aa * dc >= SWAP_MIN) {
                const double mg = (hs[i].t - hs[i - 1].t) / (hs[i - 1].eps + hs[i].eps);
                note(ps, mg, TIE_SORT);
                if (mg < 1.0) {
                    ps->nsort++;
                    ps->sort_i = i;
                }
            }
        }
        if (i == nh || ps->done) break;
        m++;
        ps->nhit++;
        for (int q = 0; q < 3; q++) cprev[q] = c[q];
        Tprev = 1.0 - ps->A;
        if (rd->opaque) {
            for (int q = 0; q < 3; q++) ps->C[q] = c[q];
            ps->A = 1.0;
            ps->done = 1;
            continue;
        }
        const double w = (1.0 - ps->A) * (double)tf[3];
        for (int q = 0; q < 3; q++) ps->C[q] += w * c[q];
        ps->A += w;
        float t1 = 1.0f - ps->A32;
        float t2 = t1 * tf[3];
        ps->A32 = ps->A32 + t2;
        if (ps->A32 >= rd->ert_alpha) ps->done = 1;
    }
    if (swap >= 1 && swap < nh) {   /* restore the sorted order */
        const hit x = hs[swap - 1];
        hs[swap - 1] = hs[swap];
        hs[swap] = x;
    }
    return m;
}

int orc_raster(const float *xyz, const float *attr, const int64_t *offsets, int64_t nc, const orc_grid *g,
               const orc_view *view, const orc_rdesc *rd, const int32_t *pix, int64_t npix, double *rgba,
               uint8_t *tie, double *alt, uint64_t *counters, int nthreads) {
    if (nc < 0 || !offsets || (!xyz && offsets[nc] > 0)) return ORC_EINVAL;
    if (view->width < 1 || view->height < 1 || !(rd->radius > 0.0f)) return ORC_EINVAL;
    rseg *S = NULL;
    int64_t ns = 0;
    int st = raster_segments(xyz, attr, offsets, nc, g, &S, &ns);
    if (st) return st;
    cam32 cam;
    cam_setup(view, &cam);
    double Lt[3];
    {
        double ld[3] = {view->light_dir[0], view->light_dir[1], view->light_dir[2]};
        norm3(ld);
        for (int a = 0; a < 3; a++) Lt[a] = (double)(float)(-ld[a]);
    }
    const double r = rd->radius;
    uint64_t c0 = 0, c1 = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel reduction(+ : c0, c1)
#endif
    {
        int64_t cap = 64;
        hit *hs = (hit *)malloc(sizeof(hit) * (size_t)cap);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t p = 0; p < npix; p++) {
            float o32[3], d32[3];
            cam_ray(&cam, pix[2 * p], pix[2 * p + 1], o32, d32);
            double O[3] = {o32[0], o32[1], o32[2]}, D[3] = {d32[0], d32[1], d32[2]};
            pixstate ps;
            memset(&ps, 0, sizeof ps);
            ps.margin = 1e300;
            int64_t nh = 0;
            double graze_t = 1e300, graze_m = 1e300;   /* nearest grazing approach and its margin */
            for (int64_t k = 0; k < ns; k++) {
                double tc;
                const double dist = line_segment_distance(O, D, S[k].a, S[k].b, &tc);
                const double gm = fabs(dist - r) / EPS_G;
                if (gm < 1.0 && tc < graze_t) { graze_t = tc; graze_m = gm; }
                entry E;
                if (!capsule_entry_s(O, D, S[k].a, S[k].b, r, &E)) continue;
                if (nh == cap) {
                    cap *= 2;
                    hs = (hit *)realloc(hs, sizeof(hit) * (size_t)cap);
                }
                hs[nh].t = E.t;
                hs[nh].eps = EPS_T + ERR_Q * E.sens;
                hs[nh].k = k;
                hs[nh].e = E;
                nh++;
            }
            qsort(hs, (size_t)nh, sizeof(hit), raster_hit_cmp);
            const int64_t m = raster_blend(S, hs, nh, rd, O, D, Lt, &ps, -1);
            /* a capsule grazed in front of the last blended fragment may
             * appear or vanish */
            if (graze_m < 1.0 && (m == nh || graze_t <= hs[m - 1].t + 1e-3)) note(&ps, graze_m, TIE_GRAZE);
            for (int c = 0; c < 3; c++) rgba[4 * p + c] = ps.C[c] + (1.0 - ps.A) * rd->bg[c];
            rgba[4 * p + 3] = ps.A;
            if (tie) tie[p] = (uint8_t)ps.tie;
            if (alt) {   /* one near-tie in depth order: the pair blended the other way round */
                for (int c = 0; c < 4; c++) alt[4 * p + c] = NAN;
                if (ps.tie == TIE_SORT && ps.nsort == 1) {
                    pixstate ps2;
                    memset(&ps2, 0, sizeof ps2);
                    ps2.margin = 1e300;
                    raster_blend(S, hs, nh, rd, O, D, Lt, &ps2, ps.sort_i);
                    for (int c = 0; c < 3; c++) alt[4 * p + c] = ps2.C[c] + (1.0 - ps2.A) * rd->bg[c];
                    alt[4 * p + 3] = ps2.A;
                }
            }
            c0 += (uint64_t)nh;
            c1 += ps.nhit;
        }
        free(hs);
    }
    free(S);
    if (counters) { counters[0] = c0; counters[1] = c1; }
    return ORC_OK;
}
