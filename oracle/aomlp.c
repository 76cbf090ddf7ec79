/*
 * Oracle of the learned ambient-occlusion surrogate (TEST INFRASTRUCTURE
 * ONLY; see oracle.h). Not part of the paper: the surrogate replaces the
 * traced density AO of Sec. 5.3 by a small network trained on that AO.
 *
 * Reading L1 (model definition):
 *  - 400 inputs. Per hit (0..14): the hit segment's unit direction with
 *    its first non-zero component made positive (3; zero for a zero-length
 *    segment), the unit tube normal at the hit (3), and for levels
 *    l = 0, 1, 2 the hit point's offset inside the level-l cell of its
 *    voxel, p / 2^l - floor(v / 2^l) - 1/2 per axis (9); input 15 is zero.
 *    Per voxel (16..390): for l = 0, 1, 2 the 5^3 level-l cells around
 *    that cell (dz, dy, dx in -2..2, x fastest), log1p(8 rho) with
 *    rho = dens_l / 8^l the density the AO march samples there (Eq. 1),
 *    zero outside the level's grid; inputs 391..399 are zero.
 *  - three hidden layers of 64 with ReLU, one sigmoid output;
 *  - parameters as float32, used as bfloat16 (round to nearest even):
 *    W1 [64][400], b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64],
 *    W4 [64], b4 [1];
 *  - bfloat16 values enter every product: the inputs, the weights, the
 *    hidden activations after ReLU; biases and sums stay float;
 *  - the per-voxel part of layer 1 (inputs 16..399) depends only on the
 *    hit voxel; it is summed first and stored as bfloat16, then the per-hit
 *    part and the bias are added.
 * The oracle evaluates these steps in float64. The LoD needs >= 3 levels.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <string.h>

enum { NIN = 400, NH = 64, NHIT = 15, VOFF = 16, NVOXIN = 375 };
enum { OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
       OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NH, NPARAM = OB4 + 1 };

int orc_ao_nparams(void) { return NPARAM; }
int orc_ao_ninputs(void) { return NIN; }

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

int orc_ao_features(const orc_lod *L, int64_t voxel, const double t[3], const double n[3],
                    const double p[3], double *x) {
    if (L->levels < 3) return -1;
    const int32_t *d0 = L->dims[0];
    const int64_t v[3] = {voxel % d0[0], (voxel / d0[0]) % d0[1], voxel / ((int64_t)d0[0] * d0[1])};
    memset(x, 0, sizeof(double) * NIN);
    for (int c = 0; c < 3; c++) {
        x[c] = t[c];
        x[3 + c] = n[c];
    }
    for (int l = 0; l < 3; l++) {
        const double cell = (double)(1 << l);
        for (int c = 0; c < 3; c++) x[6 + 3 * l + c] = p[c] / cell - (double)(v[c] >> l) - 0.5;
    }
    for (int l = 0; l < 3; l++) {
        const int32_t *dm = L->dims[l];
        const int64_t cx = v[0] >> l, cy = v[1] >> l, cz = v[2] >> l;
        const double inv = 1.0 / pow(8.0, l);
        for (int dz = -2; dz <= 2; dz++)
            for (int dy = -2; dy <= 2; dy++)
                for (int dx = -2; dx <= 2; dx++) {
                    const int slot = (dz + 2) * 25 + (dy + 2) * 5 + (dx + 2);
                    const int64_t X = cx + dx, Y = cy + dy, Z = cz + dz;
                    if (X < 0 || Y < 0 || Z < 0 || X >= dm[0] || Y >= dm[1] || Z >= dm[2]) continue;
                    const double rho = L->dens[l][X + (int64_t)dm[0] * (Y + (int64_t)dm[1] * Z)] * inv;
                    x[VOFF + 125 * l + slot] = log1p(8.0 * rho);
                }
    }
    return 0;
}

static double relu(double v) { return v > 0.0 ? v : 0.0; }

double orc_ao_mlp(const float *p, const double *x) {
    double xb[NIN], h1[NH], h2[NH], h3[NH];
    for (int k = 0; k < NIN; k++) xb[k] = orc_bf16(x[k]);
    for (int f = 0; f < NH; f++) {
        double vox = 0.0, hit = 0.0;
        for (int k = VOFF; k < NIN; k++) vox += orc_bf16(p[OW1 + f * NIN + k]) * xb[k];
        for (int k = 0; k < VOFF; k++) hit += orc_bf16(p[OW1 + f * NIN + k]) * xb[k];
        h1[f] = orc_bf16(relu(orc_bf16(vox) + hit + p[OB1 + f]));
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
