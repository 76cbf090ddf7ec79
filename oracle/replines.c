/*
 * Representative lines of the LoD and shadows against them (TEST
 * INFRASTRUCTURE ONLY; see oracle.h). Secs. 3.4 and 5.2 (first shadow
 * approach).
 *
 * Reading R3 (representative lines):
 *  - level 0: per voxel, the stored segments in canonical order; a segment
 *    whose direction makes an obtuse angle with the running average line
 *    (sum of end points minus sum of start points so far) is flipped; the
 *    start points and the end points are averaged separately;
 *  - each average point is snapped to the nearest face of the cell (ties:
 *    the lower face id, -x, +x, -y, +y, -z, +z) and to the bin of that face
 *    holding its projection (N bins per face edge, clamped);
 *  - connectivity: for each axis x, y, z in turn and each cell in linear
 *    order, if the cell's line has an end point on its +axis face and the
 *    neighbour's line one on its -axis face (start point checked first),
 *    both move to the bin that holds the average of the two points;
 *  - level l + 1: per cell, the lines of its 2^3 children (z, y, x order) in
 *    the parent's coordinates, averaged and snapped the same way, then
 *    connected.
 * Face points are kept as integers in units of 1 / (2N) (level 0) or
 * 1 / (4N) (children in a parent), so every decision is exact.
 *
 * Reading S5 (first shadow approach): from the hit point, a half-line toward
 * the light crosses the cells of level `shadow_level` (starting one cell
 * size of that level away from the hit); it is blocked if it passes within
 * radius x 2^level of the representative line of a cell it crosses;
 * visibility is 0 or 1.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* integer coordinates (units 1/(2N)) of face point (f, u, v) of a cell */
static void face_q(int f, int u, int v, int64_t N, int64_t q[3]) {
    int ax = f >> 1, b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
    q[ax] = (f & 1) ? 2 * N : 0;
    q[b0] = 2 * u + 1;
    q[b1] = 2 * v + 1;
}

/* snap the average S / n (units 1/U per cell edge) to a face point */
static void snap(const int64_t S[3], int64_t n, int64_t U, int64_t N, uint8_t *f, uint8_t *u, uint8_t *v) {
    int best = 0;
    int64_t bd = 0;
    for (int face = 0; face < 6; face++) {
        int ax = face >> 1;
        int64_t d = (face & 1) ? U * n - S[ax] : S[ax];
        if (face == 0 || d < bd) { bd = d; best = face; }
    }
    int ax = best >> 1, b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
    int64_t bins[2];
    int bx[2] = {b0, b1};
    for (int i = 0; i < 2; i++) {
        int64_t s = S[bx[i]] < 0 ? 0 : S[bx[i]];
        int64_t b = (s * N) / (U * n);
        bins[i] = b > N - 1 ? N - 1 : b;
    }
    *f = (uint8_t)best;
    *u = (uint8_t)bins[0];
    *v = (uint8_t)bins[1];
}

/* accumulate one line (a, b) into the running sums with the flip rule */
static void accumulate(int64_t a[3], int64_t b[3], int64_t SA[3], int64_t SB[3], int64_t *n) {
    if (*n > 0) {
        int64_t dot = 0;
        for (int c = 0; c < 3; c++) dot += (b[c] - a[c]) * (SB[c] - SA[c]);
        if (dot < 0)
            for (int c = 0; c < 3; c++) { int64_t t = a[c]; a[c] = b[c]; b[c] = t; }
    }
    for (int c = 0; c < 3; c++) { SA[c] += a[c]; SB[c] += b[c]; }
    (*n)++;
}

static void connect(uint8_t *rep, const int32_t *dm) {
    for (int ax = 0; ax < 3; ax++) {
        for (int64_t z = 0; z < dm[2]; z++)
            for (int64_t y = 0; y < dm[1]; y++)
                for (int64_t x = 0; x < dm[0]; x++) {
                    int64_t p[3] = {x, y, z};
                    int64_t c = x + dm[0] * (y + (int64_t)dm[1] * z);
                    if (!rep[7 * c]) continue;
                    p[ax]++;
                    if (p[ax] >= dm[ax]) continue;
                    int64_t w = p[0] + dm[0] * (p[1] + (int64_t)dm[1] * p[2]);
                    if (!rep[7 * w]) continue;
                    uint8_t *rc = rep + 7 * c, *rw = rep + 7 * w;
                    int ec = rc[1] == 2 * ax + 1 ? 1 : (rc[4] == 2 * ax + 1 ? 4 : 0);
                    int ew = rw[1] == 2 * ax ? 1 : (rw[4] == 2 * ax ? 4 : 0);
                    if (!ec || !ew) continue;
                    uint8_t u = (uint8_t)((rc[ec + 1] + rw[ew + 1] + 1) >> 1);
                    uint8_t v = (uint8_t)((rc[ec + 2] + rw[ew + 2] + 1) >> 1);
                    rc[ec + 1] = rw[ew + 1] = u;
                    rc[ec + 2] = rw[ew + 2] = v;
                }
    }
}

int orc_reps_build(const orc_voxset *vs, int levels, orc_reps **out) {
    if (levels < 1 || levels > ORC_MAX_LEVELS) return ORC_EINVAL;
    orc_reps *R = (orc_reps *)calloc(1, sizeof(orc_reps));
    R->levels = levels;
    const int64_t N = vs->grid.bins;
    for (int a = 0; a < 3; a++) R->dims[0][a] = vs->grid.res[a];
    for (int l = 1; l < levels; l++)
        for (int a = 0; a < 3; a++) R->dims[l][a] = (R->dims[l - 1][a] + 1) / 2;
    for (int l = 0; l < levels; l++) {
        int64_t n = (int64_t)R->dims[l][0] * R->dims[l][1] * R->dims[l][2];
        R->rep[l] = (uint8_t *)calloc((size_t)n, 7);
    }
    /* level 0 from the segments */
    for (int64_t v = 0; v < vs->nvox; v++) {
        int64_t SA[3] = {0, 0, 0}, SB[3] = {0, 0, 0}, n = 0;
        for (uint32_t k = vs->offset[v]; k < vs->offset[v + 1]; k++) {
            const orc_seg *s = &vs->seg[k];
            int64_t a[3], b[3];
            face_q(s->face_in, s->u_in, s->v_in, N, a);
            face_q(s->face_out, s->u_out, s->v_out, N, b);
            accumulate(a, b, SA, SB, &n);
        }
        if (!n) continue;
        uint8_t *r = R->rep[0] + 7 * v;
        r[0] = 1;
        snap(SA, n, 2 * N, N, r + 1, r + 2, r + 3);
        snap(SB, n, 2 * N, N, r + 4, r + 5, r + 6);
    }
    connect(R->rep[0], R->dims[0]);
    /* coarser levels from the children's lines */
    for (int l = 1; l < levels; l++) {
        const int32_t *cd = R->dims[l - 1], *pd = R->dims[l];
        for (int64_t z = 0; z < pd[2]; z++)
            for (int64_t y = 0; y < pd[1]; y++)
                for (int64_t x = 0; x < pd[0]; x++) {
                    int64_t SA[3] = {0, 0, 0}, SB[3] = {0, 0, 0}, n = 0;
                    for (int dz = 0; dz < 2; dz++)
                        for (int dy = 0; dy < 2; dy++)
                            for (int dx = 0; dx < 2; dx++) {
                                int64_t X = 2 * x + dx, Y = 2 * y + dy, Z = 2 * z + dz;
                                if (X >= cd[0] || Y >= cd[1] || Z >= cd[2]) continue;
                                const uint8_t *c = R->rep[l - 1] + 7 * (X + cd[0] * (Y + (int64_t)cd[1] * Z));
                                if (!c[0]) continue;
                                int64_t a[3], b[3], off[3] = {dx, dy, dz};
                                face_q(c[1], c[2], c[3], N, a);
                                face_q(c[4], c[5], c[6], N, b);
                                for (int q = 0; q < 3; q++) {
                                    a[q] += off[q] * 2 * N;
                                    b[q] += off[q] * 2 * N;
                                }
                                accumulate(a, b, SA, SB, &n);
                            }
                    if (!n) continue;
                    uint8_t *r = R->rep[l] + 7 * (x + pd[0] * (y + (int64_t)pd[1] * z));
                    r[0] = 1;
                    snap(SA, n, 4 * N, N, r + 1, r + 2, r + 3);
                    snap(SB, n, 4 * N, N, r + 4, r + 5, r + 6);
                }
        connect(R->rep[l], R->dims[l]);
    }
    *out = R;
    return ORC_OK;
}

void orc_reps_free(orc_reps *R) {
    if (!R) return;
    for (int l = 0; l < R->levels; l++) free(R->rep[l]);
    free(R);
}

void orc_reps_export(const orc_reps *R, int level, uint8_t *out7) {
    int64_t n = (int64_t)R->dims[level][0] * R->dims[level][1] * R->dims[level][2];
    memcpy(out7, R->rep[level], (size_t)n * 7);
}

/* distance between the half-line o + t d (t >= 0) and the segment [a, b] */
double orc_halfline_segment_distance(const double o[3], const double d[3], const double a[3],
                                     const double b[3]) {
    double ba[3], ao[3];
    for (int c = 0; c < 3; c++) { ba[c] = b[c] - a[c]; ao[c] = a[c] - o[c]; }
    double L2 = ba[0] * ba[0] + ba[1] * ba[1] + ba[2] * ba[2];
    double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double k = d[0] * ba[0] + d[1] * ba[1] + d[2] * ba[2];
    double e = d[0] * ao[0] + d[1] * ao[1] + d[2] * ao[2];
    double f = ba[0] * ao[0] + ba[1] * ao[1] + ba[2] * ao[2];
    /* candidate (t, h) pairs: the free optimum and the boundary optima */
    double cand[4][2];
    int nc = 0;
    double det = dd * L2 - k * k;
    if (L2 > 0.0 && det > 1e-14 * dd * L2) {
        double h = (k * e - dd * f) / det, t = (e + h * k) / dd;
        if (t >= 0.0 && h >= 0.0 && h <= 1.0) { cand[nc][0] = t; cand[nc][1] = h; nc++; }
    }
    {   /* t = 0 */
        double h = L2 > 0.0 ? -f / L2 : 0.0;
        if (h < 0.0) h = 0.0;
        if (h > 1.0) h = 1.0;
        cand[nc][0] = 0.0; cand[nc][1] = h; nc++;
    }
    for (int hh = 0; hh < 2; hh++) {   /* h = 0, h = 1 */
        double t = (e + hh * k) / dd;
        if (t < 0.0) t = 0.0;
        cand[nc][0] = t; cand[nc][1] = hh; nc++;
    }
    double best = 1e300;
    for (int i = 0; i < nc; i++) {
        double t = cand[i][0], h = cand[i][1], p2 = 0.0;
        for (int c = 0; c < 3; c++) {
            double p = o[c] + t * d[c] - (a[c] + h * ba[c]);
            p2 += p * p;
        }
        if (p2 < best) best = p2;
    }
    return sqrt(best);
}

/* world end points of the representative line of cell c at `level` */
void orc_rep_world(const orc_reps *R, int level, int64_t cell, int N, double a[3], double b[3]) {
    const int32_t *dm = R->dims[level];
    const uint8_t *r = R->rep[level] + 7 * cell;
    const double size = ldexp(1.0, level);
    const int64_t p[3] = {cell % dm[0], (cell / dm[0]) % dm[1], cell / ((int64_t)dm[0] * dm[1])};
    int64_t qa[3], qb[3];
    face_q(r[1], r[2], r[3], N, qa);
    face_q(r[4], r[5], r[6], N, qb);
    for (int c = 0; c < 3; c++) {
        a[c] = (p[c] + qa[c] / (2.0 * N)) * size;
        b[c] = (p[c] + qb[c] / (2.0 * N)) * size;
    }
}
