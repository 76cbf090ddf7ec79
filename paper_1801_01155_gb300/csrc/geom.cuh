// Geometry shared by the camera-at-rest neighbour lists and their host test.
// Compiles as CUDA (host and device) and as plain C++ (the test builds it
// with the host compiler).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define LVR_HD __host__ __device__
#else
#define LVR_HD
#endif

namespace lvr_geom {

// Squared distance from the segment a + s (b - a), 0 <= s <= 1, to the unit
// box [0, 1]^3. Along the segment the squared distance is a convex piecewise
// quadratic whose pieces end where a coordinate crosses 0 or 1; on each piece
// the axes outside the box are fixed, and its minimum is the piece's
// stationary point clamped to the piece. Every candidate is evaluated with
// the true distance, so rounding can only move the result by a few units in
// the last place.
LVR_HD inline float segment_box_dist2(const float a[3], const float b[3]) {
    const float d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    auto f = [&](float s) {
        float q = 0.0f;
        for (int i = 0; i < 3; i++) {
            const float x = fmaf(s, d[i], a[i]);
            const float e = fmaxf(fmaxf(-x, x - 1.0f), 0.0f);
            q = fmaf(e, e, q);
        }
        return q;
    };
    float bp[8];
    int nb = 0;
    bp[nb++] = 0.0f;
    bp[nb++] = 1.0f;
    for (int i = 0; i < 3; i++) {
        if (d[i] == 0.0f) continue;
        for (int c = 0; c < 2; c++) {
            const float sb = ((float)c - a[i]) / d[i];
            if (sb > 0.0f && sb < 1.0f) bp[nb++] = sb;
        }
    }
    for (int i = 1; i < nb; i++)   // insertion sort of at most 8 values
        for (int j = i; j > 0 && bp[j] < bp[j - 1]; j--) {
            const float tmp = bp[j];
            bp[j] = bp[j - 1];
            bp[j - 1] = tmp;
        }
    float best = f(1.0f);
    for (int k = 0; k + 1 < nb; k++) {
        const float s0 = bp[k], s1 = bp[k + 1], mid = 0.5f * (s0 + s1);
        best = fminf(best, f(s0));
        float num = 0.0f, den = 0.0f;
        for (int i = 0; i < 3; i++) {
            const float x = fmaf(mid, d[i], a[i]);
            if (x < 0.0f || x > 1.0f) {
                const float c = x < 0.0f ? 0.0f : 1.0f;
                num = fmaf(d[i], c - a[i], num);
                den = fmaf(d[i], d[i], den);
            }
        }
        if (den > 0.0f) best = fminf(best, f(fminf(fmaxf(num / den, s0), s1)));
    }
    return best;
}

}  // namespace lvr_geom
