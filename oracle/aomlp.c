/*
 * Oracle of the learned ambient-occlusion surrogate (TEST INFRASTRUCTURE
 * ONLY; see oracle.h). Not part of the paper: the surrogate replaces the
 * traced density AO of Sec. 5.3 by a small network trained on that AO.
 *
 * Reading L1 (model definition), restated from the build's specification:
 *  - inputs (256): the hit segment's direction, sign-normalised so that its
 *    first non-zero component is positive (3 values; zero for a zero-length
 *    segment), then for the 5^3 level-0 voxels around the hit voxel
 *    (dz, dy, dx in -2..2, x fastest) log1p(count) and log1p(summed length),
 *    zero outside the grid (250 values), then 3 zeros;
 *  - three hidden layers of 64 with ReLU, one sigmoid output;
 *  - parameters as float32, used as bfloat16 (round to nearest even):
 *    W1 [64][256], b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64],
 *    W4 [64], b4 [1];
 *  - bfloat16 values enter every product: the inputs, the weights, the
 *    hidden activations after ReLU; biases and sums stay float;
 *  - the neighbourhood part of layer 1 (inputs 3..255) depends only on the
 *    hit voxel; it is summed first and stored as bfloat16, then the
 *    direction part and the bias are added.
 * The oracle evaluates these steps in float64.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <string.h>

enum { NIN = 256, NH = 64 };
enum { OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
       OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NH, NPARAM = OB4 + 1 };

int orc_ao_nparams(void) { return NPARAM; }

/* float64 -> float32 (nearest) -> bfloat16 (nearest even), returned as float64 */
double orc_bf16(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {       /* finite: round */
        u += 0x7fffu + ((u >> 16) & 1u);
        u &= 0xffff0000u;
    }
    memcpy(&f, &u, 4);
    return (double)f;
}

void orc_ao_tangent(const double a[3], const double b[3], double t[3]) {
    double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(l > 0.0)) { t[0] = t[1] = t[2] = 0.0; return; }
    double s = 1.0;
    for (int c = 0; c < 3; c++)
        if (d[c] != 0.0) { s = d[c] > 0.0 ? 1.0 : -1.0; break; }
    for (int c = 0; c < 3; c++) t[c] = s * d[c] / l;
}

void orc_ao_features(const orc_lod *L, int64_t voxel, const double t[3], double *x) {
    const int32_t *dm = L->dims[0];
    int64_t vx = voxel % dm[0], vy = (voxel / dm[0]) % dm[1], vz = voxel / ((int64_t)dm[0] * dm[1]);
    memset(x, 0, sizeof(double) * NIN);
    x[0] = t[0]; x[1] = t[1]; x[2] = t[2];
    for (int dz = -2; dz <= 2; dz++)
        for (int dy = -2; dy <= 2; dy++)
            for (int dx = -2; dx <= 2; dx++) {
                int n = (dz + 2) * 25 + (dy + 2) * 5 + (dx + 2);
                int64_t X = vx + dx, Y = vy + dy, Z = vz + dz;
                if (X < 0 || Y < 0 || Z < 0 || X >= dm[0] || Y >= dm[1] || Z >= dm[2]) continue;
                int64_t i = X + (int64_t)dm[0] * (Y + (int64_t)dm[1] * Z);
                x[3 + 2 * n] = log1p((double)L->cnt[0][i]);
                x[4 + 2 * n] = log1p(L->len[0][i]);
            }
}

static double relu(double v) { return v > 0.0 ? v : 0.0; }

double orc_ao_mlp(const float *p, const double *x) {
    double xb[NIN], h1[NH], h2[NH], h3[NH];
    for (int k = 0; k < NIN; k++) xb[k] = orc_bf16(x[k]);
    for (int f = 0; f < NH; f++) {
        double nb = 0.0, dir = 0.0;
        for (int k = 3; k < NIN; k++) nb += orc_bf16(p[OW1 + f * NIN + k]) * xb[k];
        for (int k = 0; k < 3; k++) dir += orc_bf16(p[OW1 + f * NIN + k]) * xb[k];
        h1[f] = orc_bf16(relu(orc_bf16(nb) + dir + p[OB1 + f]));
    }
    for (int f = 0; f < NH; f++) {
        double z = p[OB2 + f];
        for (int k = 0; k < NH; k++) z += orc_bf16(p[OW2 + f * NH + k]) * h1[k];
        h2[f] = orc_bf16(relu(z));
    }
    for (int f = 0; f < NH; f++) {
        double z = p[OB3 + f];
        for (int k = 0; k < NH; k++) z += orc_bf16(p[OW3 + f * NH + k]) * h2[k];
        h3[f] = orc_bf16(relu(z));
    }
    double z = p[OB4];
    for (int k = 0; k < NH; k++) z += orc_bf16(p[OW4 + k]) * h3[k];
    return 1.0 / (1.0 + exp(-z));
}
