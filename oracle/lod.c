/*
 * Oracle density LoD (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * Sec. 3.4, Eq. 1: per voxel rho = sum over its lines of length(l_i) * sigma_i,
 * then an octree built bottom-up by pooling 2^3 voxels into one coarser voxel.
 * Reading: each level stores *sums* (line count, summed length, summed
 * length * sigma) so that counts stay integers; the density sampled at
 * level l is dens_l / 8^l, which is the paper's 2^3 average. Coarser
 * dimensions are ceil(dim / 2).
 *
 * Segment endpoints are face-bin centres; in units of 1/(2N) voxel every
 * coordinate is an integer (0 or 2N on the face axis, 2j+1 on the other two),
 * so length = sqrt(I) / (2N) with I an integer.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* endpoint of a face point in units of 1/(2N) voxel */
static void face_point_2n(int face, int u, int v, int N, int64_t q[3]) {
    int a = face / 2;
    int b0 = a == 0 ? 1 : 0, b1 = a == 2 ? 1 : 2;
    q[a] = (face & 1) ? 2 * N : 0;
    q[b0] = 2 * u + 1;
    q[b1] = 2 * v + 1;
}

double orc_seg_length(const orc_seg *s, int N);
double orc_seg_length(const orc_seg *s, int N) {
    int64_t p[3], q[3];
    face_point_2n(s->face_in, s->u_in, s->v_in, N, p);
    face_point_2n(s->face_out, s->u_out, s->v_out, N, q);
    int64_t I = 0;
    for (int a = 0; a < 3; a++) I += (q[a] - p[a]) * (q[a] - p[a]);
    return sqrt((double)I) / (2.0 * N);
}

int orc_build_lod(const orc_voxset *vs, int levels, const float *sigma256, orc_lod **out) {
    *out = NULL;
    if (levels < 1 || levels > ORC_MAX_LEVELS) return ORC_EINVAL;
    orc_lod *L = (orc_lod *)calloc(1, sizeof *L);
    if (!L) return ORC_ENOMEM;
    L->levels = levels;
    for (int l = 0; l < levels; l++) {
        for (int a = 0; a < 3; a++)
            L->dims[l][a] = l == 0 ? vs->grid.res[a] : (L->dims[l - 1][a] + 1) / 2;
        size_t n = (size_t)L->dims[l][0] * L->dims[l][1] * L->dims[l][2];
        L->cnt[l] = (uint32_t *)calloc(n, sizeof(uint32_t));
        L->len[l] = (double *)calloc(n, sizeof(double));
        L->dens[l] = (double *)calloc(n, sizeof(double));
        if (!L->cnt[l] || !L->len[l] || !L->dens[l]) { orc_lod_free(L); return ORC_ENOMEM; }
    }
    const int N = vs->grid.bins;
    for (int64_t v = 0; v < vs->nvox; v++) {
        for (uint32_t i = vs->offset[v]; i < vs->offset[v + 1]; i++) {
            double len = orc_seg_length(&vs->seg[i], N);
            L->cnt[0][v] += 1;
            L->len[0][v] += len;
            L->dens[0][v] += len * (double)sigma256[vs->seg[i].attr];    /* Eq. 1 */
        }
    }
    for (int l = 1; l < levels; l++) {
        const int32_t *dc = L->dims[l - 1], *dp = L->dims[l];
        for (int z = 0; z < dp[2]; z++)
            for (int y = 0; y < dp[1]; y++)
                for (int x = 0; x < dp[0]; x++) {
                    size_t p = (size_t)x + (size_t)dp[0] * ((size_t)y + (size_t)dp[1] * z);
                    for (int dz = 0; dz < 2; dz++)
                        for (int dy = 0; dy < 2; dy++)
                            for (int dx = 0; dx < 2; dx++) {
                                int cx = 2 * x + dx, cy = 2 * y + dy, cz = 2 * z + dz;
                                if (cx >= dc[0] || cy >= dc[1] || cz >= dc[2]) continue;
                                size_t c = (size_t)cx + (size_t)dc[0] * ((size_t)cy + (size_t)dc[1] * cz);
                                L->cnt[l][p] += L->cnt[l - 1][c];
                                L->len[l][p] += L->len[l - 1][c];
                                L->dens[l][p] += L->dens[l - 1][c];
                            }
                }
    }
    *out = L;
    return ORC_OK;
}

void orc_lod_free(orc_lod *L) {
    if (!L) return;
    for (int l = 0; l < ORC_MAX_LEVELS; l++) {
        free(L->cnt[l]);
        free(L->len[l]);
        free(L->dens[l]);
    }
    free(L);
}

void orc_lod_dims(const orc_lod *L, int level, int32_t *dims3) {
    for (int a = 0; a < 3; a++) dims3[a] = L->dims[level][a];
}

void orc_lod_export(const orc_lod *L, int level, uint32_t *cnt, double *len, double *dens) {
    size_t n = (size_t)L->dims[level][0] * L->dims[level][1] * L->dims[level][2];
    if (cnt) memcpy(cnt, L->cnt[level], n * sizeof(uint32_t));
    if (len) memcpy(len, L->len[level], n * sizeof(double));
    if (dens) memcpy(dens, L->dens[level], n * sizeof(double));
}
