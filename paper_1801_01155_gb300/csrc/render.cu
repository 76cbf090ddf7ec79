// Ray casting of the voxelised line set (Secs. 4, 5): 3D-DDA traversal,
// ray-capsule tests against each visited voxel's own segments, per-voxel hit
// sorting, local illumination, front-to-back compositing with early ray
// termination, and density-LoD marches for soft shadows and ambient
// occlusion.
//
// Precision. All device arithmetic is float32. The primary ray is a float32
// quantity built by a fixed sequence of correctly rounded operations. The
// ray's position is kept in voxel-local coordinates: the box entry point is
// computed once in float-float (error-free product and sum), and from then
// on the ray state is the voxel index plus a local position in [0,1]^3, so
// every intersection is solved with operands of magnitude about 1 instead
// of the camera distance. Tube-axis distances use cross products, which do
// not cancel.
//
// Ownership. A voxel keeps a hit iff its entry point lies inside the voxel:
// in local coordinates, iff the entry parameter s satisfies
// 0 <= s < s_exit. Ties between faces step in axis order x, y, z.
#include <math.h>
#include <string.h>

#include "lvr_internal.cuh"

namespace {

constexpr int RT = 128;       // threads per block (4 warps)
constexpr int HMAX = 8;       // hits per voxel staged in shared memory per ray
constexpr int MAX_AO = 32;

struct RenderParams {
    const uint32_t *offset;
    const uint64_t *rec;
    int32_t res[3];
    float invN;
    float r2;
    int32_t levels;
    int32_t ldims[4][3];
    const float *dens[4];
    float lod_lo, lod_hi[3];      // support of the density field (level-0 voxels)
    float F[3], R[3], U[3], th, tw, eye[3];
    int32_t W, H, x0, y0, cw, ch;
    int32_t tile_w, tile_h;
    float Lt[3];                  // toward the light, unit
    int32_t opaque;
    float ert;
    int32_t shadows, ao, ao_rays;
    float ao_radius, ka, kd, bg[3];
    float aod[MAX_AO][3];         // hemisphere directions in the (T, B, n) frame
    float tf[1024];
    float4 *out;
    unsigned long long *counters;
};

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

// Face point (Sec. 3.2): face id -> axis and side, bins -> sub-square centres.
__device__ __forceinline__ Vec face_point(uint32_t face, uint32_t u, uint32_t v, float invN) {
    const uint32_t ax = face >> 1;
    const float side = (face & 1u) ? 1.0f : 0.0f;
    const float cu = ((float)u + 0.5f) * invN, cv = ((float)v + 0.5f) * invN;
    return {ax == 0 ? side : cu, ax == 1 ? side : (ax == 0 ? cu : cv), ax == 2 ? side : cv};
}

// First entry of ray p + s D (|D| = 1) into the sphere |x - c| = r; INF if
// none. Closest-approach form: the squared distance of the centre from the
// ray is taken from the perpendicular vector itself, which does not cancel.
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
__device__ __forceinline__ float capsule_entry(Vec p, Vec D, Vec a, Vec b, float r2) {
    const Vec ba = sub(b, a);
    const float L2 = dot(ba, ba);
    if (L2 > 0.0f) {
        const float L = sqrtf(L2), iL = 1.0f / L;
        const Vec w = mk(ba.x * iL, ba.y * iL, ba.z * iL);
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

// Cell-centred trilinear density at level l, zero outside the grid.
__device__ __forceinline__ float sample_level(const RenderParams &P, int l, Vec x) {
    const float inv = __int_as_float((127 - l) << 23);         // 2^-l
    const float qx = fmaf(x.x, inv, -0.5f), qy = fmaf(x.y, inv, -0.5f), qz = fmaf(x.z, inv, -0.5f);
    const float fx0 = floorf(qx), fy0 = floorf(qy), fz0 = floorf(qz);
    const int ix = (int)fx0, iy = (int)fy0, iz = (int)fz0;
    const float fx = qx - fx0, fy = qy - fy0, fz = qz - fz0;
    const int dx = P.ldims[l][0], dy = P.ldims[l][1], dz = P.ldims[l][2];
    const float *__restrict__ d = P.dens[l];
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        const int X = ix + (c & 1), Y = iy + ((c >> 1) & 1), Z = iz + ((c >> 2) & 1);
        if ((unsigned)X < (unsigned)dx && (unsigned)Y < (unsigned)dy && (unsigned)Z < (unsigned)dz) {
            const float w = ((c & 1) ? fx : 1.0f - fx) * (((c >> 1) & 1) ? fy : 1.0f - fy) *
                            (((c >> 2) & 1) ? fz : 1.0f - fz);
            acc = fmaf(w, __ldg(d + (X + (int64_t)dx * (Y + (int64_t)dy * Z))), acc);
        }
    }
    return acc;
}

// Density march (Secs. 5.2, 5.3): samples at s = 1, 2, 4, ... with step 2^l
// at level l = floor(log2 s) (capped); optical depth O += rho_l * 2^l with
// rho_l = dens_l / 8^l; stops at O >= 1, beyond max_dist (if >= 0), or when
// the sample leaves the support of the density field.
__device__ float march(const RenderParams &P, Vec p, Vec d, float max_dist, unsigned &nsamp) {
    float O = 0.0f;
    int s = 1;
    const int top = P.levels - 1;
    for (;;) {
        if (max_dist >= 0.0f && (float)s > max_dist) break;
        const Vec x = axpy((float)s, d, p);
        if (x.x < P.lod_lo || x.y < P.lod_lo || x.z < P.lod_lo || x.x > P.lod_hi[0] ||
            x.y > P.lod_hi[1] || x.z > P.lod_hi[2])
            break;
        int l = 31 - __clz(s);
        l = l < top ? l : top;
        const float w = __int_as_float((127 - 2 * l) << 23);   // 2^l / 8^l
        O = fmaf(sample_level(P, l, x), w, O);
        nsamp++;
        if (O >= 1.0f) break;
        s += 1 << l;
    }
    return O;
}

struct RayState {
    float Cr, Cg, Cb, A;
    bool done;
    unsigned nvox, nrec, nsamp, nhit;
};

// Shade one hit at local parameter t of voxel (vx,vy,vz) and composite it.
__device__ void shade_hit(const RenderParams &P, const float4 *s_tf, uint64_t r, float t, Vec p, Vec D,
                          int vx, int vy, int vz, RayState &S) {
    const Vec a = face_point(rec_face_in(r), rec_u_in(r), rec_v_in(r), P.invN);
    const Vec b = face_point(rec_face_out(r), rec_u_out(r), rec_v_out(r), P.invN);
    const Vec Pl = axpy(t, D, p);
    const Vec ba = sub(b, a);
    const float L2 = dot(ba, ba);
    float h = 0.0f;
    if (L2 > 0.0f) h = fminf(fmaxf(dot(sub(Pl, a), ba) / L2, 0.0f), 1.0f);
    Vec n = sub(Pl, axpy(h, ba, a));
    const float nl = rsqrtf(dot(n, n));
    n = mk(n.x * nl, n.y * nl, n.z * nl);
    const float4 c = s_tf[rec_attr(r)];
    const float alpha = P.opaque ? 1.0f : c.w;
    const Vec Lt = mk(P.Lt[0], P.Lt[1], P.Lt[2]);
    const Vec Pg = mk((float)vx + Pl.x, (float)vy + Pl.y, (float)vz + Pl.z);
    float V = 1.0f, AO = 1.0f;
    if (P.shadows) V = 1.0f - fminf(1.0f, march(P, Pg, Lt, -1.0f, S.nsamp));
    if (P.ao) {
        Vec u = mk(0.0f, 0.0f, 0.0f);
        if (L2 > 0.0f) {
            const float il = 1.0f / sqrtf(L2);
            u = mk(ba.x * il, ba.y * il, ba.z * il);
        }
        const float un = dot(u, n);
        Vec T = mk(u.x - un * n.x, u.y - un * n.y, u.z - un * n.z);
        const float m = sqrtf(dot(T, T));
        if (m >= 1e-3f) {
            T = mk(T.x / m, T.y / m, T.z / m);
        } else {
            const float ax = fabsf(n.x), ay = fabsf(n.y), az = fabsf(n.z);
            int e = 0;
            float best = ax;
            if (ay < best) { e = 1; best = ay; }
            if (az < best) { e = 2; }
            const float ne = e == 0 ? n.x : (e == 1 ? n.y : n.z);
            T = mk((e == 0 ? 1.0f : 0.0f) - ne * n.x, (e == 1 ? 1.0f : 0.0f) - ne * n.y,
                   (e == 2 ? 1.0f : 0.0f) - ne * n.z);
            const float tl = rsqrtf(dot(T, T));
            T = mk(T.x * tl, T.y * tl, T.z * tl);
        }
        const Vec B = cross(n, T);
        float occ = 0.0f;
        for (int i = 0; i < P.ao_rays; i++) {
            const float dx = P.aod[i][0], dy = P.aod[i][1], dz = P.aod[i][2];
            const Vec d = mk(fmaf(T.x, dx, fmaf(B.x, dy, n.x * dz)), fmaf(T.y, dx, fmaf(B.y, dy, n.y * dz)),
                             fmaf(T.z, dx, fmaf(B.z, dy, n.z * dz)));
            occ += fminf(1.0f, march(P, Pg, d, P.ao_radius, S.nsamp));
        }
        AO = 1.0f - occ / (float)P.ao_rays;
    }
    const float k = fmaf(P.ka, AO, P.kd * V * fabsf(dot(n, Lt)));
    S.nhit++;
    if (P.opaque) {
        S.Cr = c.x * k;
        S.Cg = c.y * k;
        S.Cb = c.z * k;
        S.A = 1.0f;
        S.done = true;
        return;
    }
    // front-to-back blending (Sec. 5.1); the opacity update is rounded step by
    // step so the termination test is reproducible: A <- A + (1 - A) * alpha
    const float w = __fmul_rn(__fsub_rn(1.0f, S.A), alpha);
    S.Cr = fmaf(w, c.x * k, S.Cr);
    S.Cg = fmaf(w, c.y * k, S.Cg);
    S.Cb = fmaf(w, c.z * k, S.Cb);
    S.A = __fadd_rn(S.A, w);
    if (S.A >= P.ert) S.done = true;
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

__global__ void __launch_bounds__(RT)
render_kernel(const __grid_constant__ RenderParams P) {
    __shared__ float4 s_tf[256];
    __shared__ float s_ht[HMAX][RT];
    __shared__ uint32_t s_hk[HMAX][RT];
    for (int i = threadIdx.x; i < 256; i += RT)
        s_tf[i] = make_float4(P.tf[4 * i], P.tf[4 * i + 1], P.tf[4 * i + 2], P.tf[4 * i + 3]);
    __syncthreads();

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int px = blockIdx.x * (2 * P.tile_w) + (warp & 1) * P.tile_w + lane % P.tile_w;
    const int py = blockIdx.y * (2 * P.tile_h) + (warp >> 1) * P.tile_h + lane / P.tile_w;
    if (px >= P.cw || py >= P.ch) return;
    const int i = P.x0 + px, j = P.y0 + py;

    // primary ray: float32 contract, each step correctly rounded
    const float sx = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * i + 1), (float)P.W), 1.0f), P.tw);
    const float sy = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * j + 1), (float)P.H), 1.0f), P.th);
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; a++) d[a] = __fsub_rn(__fadd_rn(P.F[a], __fmul_rn(sx, P.R[a])), __fmul_rn(sy, P.U[a]));
    const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])), __fmul_rn(d[2], d[2]));
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    const Vec D = mk(__fmul_rn(d[0], inv), __fmul_rn(d[1], inv), __fmul_rn(d[2], inv));
    const float Da[3] = {D.x, D.y, D.z};

    RayState S = {0.0f, 0.0f, 0.0f, 0.0f, false, 0u, 0u, 0u, 0u};
    // slab test: only the entry parameter is needed, approximately
    float tnear = 0.0f, tfar = INFINITY;
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (Da[a] != 0.0f) {
            const float ia = 1.0f / Da[a];
            const float t1 = (0.0f - P.eye[a]) * ia, t2 = ((float)P.res[a] - P.eye[a]) * ia;
            tnear = fmaxf(tnear, fminf(t1, t2));
            tfar = fminf(tfar, fmaxf(t1, t2));
        } else if (P.eye[a] < 0.0f || P.eye[a] > (float)P.res[a]) {
            miss = true;
        }
    }
    if (!miss && tnear < tfar) {
        // entry point in float-float, split into voxel index + local position
        int v[3];
        float pl[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float ph = __fmul_rn(tnear, Da[a]);
            const float pe = __fmaf_rn(tnear, Da[a], -ph);
            float sh, se;
            two_sum(P.eye[a], ph, sh, se);
            const float lo = __fadd_rn(se, pe);
            float fl = floorf(sh);
            float f = __fadd_rn(__fsub_rn(sh, fl), lo);
            if (f < 0.0f) { fl -= 1.0f; f += 1.0f; }
            else if (f >= 1.0f) { fl += 1.0f; f -= 1.0f; }
            int vi = (int)fl;
            if (vi < 0) { f += (float)vi; vi = 0; }
            if (vi > P.res[a] - 1) { f += (float)(vi - (P.res[a] - 1)); vi = P.res[a] - 1; }
            v[a] = vi;
            pl[a] = f;
        }
        const float invD[3] = {Da[0] != 0.0f ? 1.0f / Da[0] : INFINITY, Da[1] != 0.0f ? 1.0f / Da[1] : INFINITY,
                               Da[2] != 0.0f ? 1.0f / Da[2] : INFINITY};
        const float r2 = P.r2;
        float T = tnear;              // ray parameter at the current voxel's entry
        float(*ht)[RT] = s_ht;
        uint32_t(*hk)[RT] = s_hk;
        for (;;) {
            // exit parameter of the current voxel, ties in axis order x, y, z
            float se = INFINITY;
            int ax = 0;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                float e = Da[a] > 0.0f ? (1.0f - pl[a]) * invD[a] : (Da[a] < 0.0f ? (0.0f - pl[a]) * invD[a] : INFINITY);
                if (e < se) { se = e; ax = a; }
            }
            se = fmaxf(se, 0.0f);
            const uint32_t vid = (uint32_t)v[0] + (uint32_t)P.res[0] * ((uint32_t)v[1] + (uint32_t)P.res[1] * (uint32_t)v[2]);
            const uint32_t beg = __ldg(P.offset + vid), end = __ldg(P.offset + vid + 1);
            S.nvox++;
            if (end > beg) {
                S.nrec += end - beg;
                // accurate local origin: eye + T D - v in float-float, rounded once
                float po[3];
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const float ph = __fmul_rn(T, Da[a]);
                    const float pe = __fmaf_rn(T, Da[a], -ph);
                    float sh, s2;
                    two_sum(P.eye[a], ph, sh, s2);
                    po[a] = __fadd_rn(__fsub_rn(sh, (float)v[a]), __fadd_rn(s2, pe));
                }
                const Vec p = mk(po[0], po[1], po[2]);
                int nh = 0;
                for (uint32_t k = beg; k < end; k++) {
                    const uint64_t r = __ldg(P.rec + k);
                    const Vec a = face_point(rec_face_in(r), rec_u_in(r), rec_v_in(r), P.invN);
                    const Vec b = face_point(rec_face_out(r), rec_u_out(r), rec_v_out(r), P.invN);
                    const float t = capsule_entry(p, D, a, b, r2);
                    if (!owned(p, D, t, -T)) continue;
                    // bounded insertion: keep the HMAX smallest (t, k), in order
                    if (nh < HMAX || t < ht[HMAX - 1][tid]) {
                        int q = nh < HMAX ? nh : HMAX - 1;
                        while (q > 0 && t < ht[q - 1][tid]) {
                            ht[q][tid] = ht[q - 1][tid];
                            hk[q][tid] = hk[q - 1][tid];
                            q--;
                        }
                        ht[q][tid] = t;
                        hk[q][tid] = k;
                    }
                    nh++;
                }
                const int nl = nh < HMAX ? nh : HMAX;
                for (int q = 0; q < nl && !S.done; q++)
                    shade_hit(P, s_tf, __ldg(P.rec + hk[q][tid]), ht[q][tid], p, D, v[0], v[1], v[2], S);
                if (nh > HMAX && !S.done) {
                    // more hits than staged: select the next (t, k) one at a time
                    float lt = ht[HMAX - 1][tid];
                    uint32_t lk = hk[HMAX - 1][tid];
                    while (!S.done) {
                        float bt = INFINITY;
                        uint32_t bk = 0xffffffffu;
                        for (uint32_t k = beg; k < end; k++) {
                            const uint64_t r = __ldg(P.rec + k);
                            const Vec a = face_point(rec_face_in(r), rec_u_in(r), rec_v_in(r), P.invN);
                            const Vec b = face_point(rec_face_out(r), rec_u_out(r), rec_v_out(r), P.invN);
                            const float t = capsule_entry(p, D, a, b, r2);
                            if (!owned(p, D, t, -T)) continue;
                            const bool after = t > lt || (t == lt && k > lk);
                            const bool before = t < bt || (t == bt && k < bk);
                            if (after && before) { bt = t; bk = k; }
                        }
                        if (bk == 0xffffffffu) break;
                        shade_hit(P, s_tf, __ldg(P.rec + bk), bt, p, D, v[0], v[1], v[2], S);
                        lt = bt;
                        lk = bk;
                    }
                }
            }
            if (S.done) break;
            T = __fadd_rn(T, se);
            // step into the neighbour across face `ax`
#pragma unroll
            for (int a = 0; a < 3; a++) pl[a] = fmaf(se, Da[a], pl[a]);
            const int sg = Da[ax] > 0.0f ? 1 : -1;
            v[ax] += sg;
            pl[ax] = sg > 0 ? 0.0f : 1.0f;
            if (v[ax] < 0 || v[ax] >= P.res[ax]) break;
        }
    }
    const float4 o = make_float4(fmaf(1.0f - S.A, P.bg[0], S.Cr), fmaf(1.0f - S.A, P.bg[1], S.Cg),
                                 fmaf(1.0f - S.A, P.bg[2], S.Cb), S.A);
    P.out[(int64_t)py * P.cw + px] = o;
    if (P.counters) {
        const unsigned mask = __activemask();
        const unsigned c0 = __reduce_add_sync(mask, S.nvox), c1 = __reduce_add_sync(mask, S.nrec),
                       c2 = __reduce_add_sync(mask, S.nsamp), c3 = __reduce_add_sync(mask, S.nhit);
        if (lane == __ffs(mask) - 1) {
            atomicAdd(P.counters + 0, (unsigned long long)c0);
            atomicAdd(P.counters + 1, (unsigned long long)c1);
            atomicAdd(P.counters + 2, (unsigned long long)c2);
            atomicAdd(P.counters + 3, (unsigned long long)c3);
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ host side
static void norm3(double *a) {
    const double l = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    a[0] /= l; a[1] /= l; a[2] /= l;
}

extern "C" lvr_status lvr_render(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod,
                                 const lvr_view *view, const lvr_render_desc *desc,
                                 const lvr_ao_model *ao, float *rgba, uint64_t *counters) {
    if (!ctx) return LVR_EINVAL;
    if (!ls || !view || !desc || !rgba) return set_err(ctx, LVR_EINVAL, "lvr_render: null argument");
    if (view->width < 1 || view->height < 1) return set_err(ctx, LVR_EINVAL, "image size must be >= 1");
    int x0 = 0, y0 = 0, cw = view->width, ch = view->height;
    if (view->crop[2] > 0) {
        x0 = view->crop[0]; y0 = view->crop[1]; cw = view->crop[2]; ch = view->crop[3];
        if (x0 < 0 || y0 < 0 || ch < 1 || x0 + cw > view->width || y0 + ch > view->height)
            return set_err(ctx, LVR_EINVAL, "crop outside the image");
    }
    if (!(desc->radius > 0.0f) || !(desc->radius < 1e3f)) return set_err(ctx, LVR_EINVAL, "radius must be > 0");
    if (!(view->fovy_deg > 0.0f && view->fovy_deg < 180.0f)) return set_err(ctx, LVR_EINVAL, "fovy out of (0,180)");
    if (desc->ao_mode < 0 || desc->ao_mode > 2) return set_err(ctx, LVR_EINVAL, "bad ao_mode");
    if (desc->ao_mode == 2) return set_err(ctx, LVR_EINVAL, "learned AO model not available in this build");
    (void)ao;
    const bool need_lod = desc->shadows || desc->ao_mode == 1;
    if (need_lod && !lod) return set_err(ctx, LVR_EINVAL, "shadows / traced AO need a LoD");
    if (desc->ao_mode == 1 && (desc->ao_rays < 1 || desc->ao_rays > 32))
        return set_err(ctx, LVR_EINVAL, "ao_rays must be in [1,32]");
    if (lod && (lod->dims[0][0] != ls->res[0] || lod->dims[0][1] != ls->res[1] || lod->dims[0][2] != ls->res[2]))
        return set_err(ctx, LVR_EINVAL, "LoD does not belong to this line set");
    int tw = desc->tile_w, th = desc->tile_h;
    if (tw == 0 && th == 0) { tw = 8; th = 4; }
    if (tw * th != 32 || tw < 1 || th < 1) return set_err(ctx, LVR_EINVAL, "tile must have 32 pixels");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;

    RenderParams P;
    memset(&P, 0, sizeof P);
    P.offset = ls->offset;
    P.rec = ls->rec;
    for (int a = 0; a < 3; a++) P.res[a] = ls->res[a];
    P.invN = 1.0f / (float)ls->bins;
    P.r2 = desc->radius * desc->radius;
    if (lod) {
        P.levels = lod->levels;
        for (int l = 0; l < lod->levels; l++) {
            for (int a = 0; a < 3; a++) P.ldims[l][a] = lod->dims[l][a];
            P.dens[l] = lod->dens[l];
        }
        const float cell = (float)(1 << (lod->levels - 1));
        P.lod_lo = -0.5f * cell;
        for (int a = 0; a < 3; a++) P.lod_hi[a] = ((float)lod->dims[lod->levels - 1][a] + 0.5f) * cell;
    }
    // camera basis in float64, rounded to float32
    double f[3], up[3], r[3], u[3];
    for (int a = 0; a < 3; a++) {
        f[a] = (double)view->at[a] - (double)view->eye[a];
        up[a] = view->up[a];
    }
    norm3(f);
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    norm3(r);
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    if (!(fabs(r[0]) + fabs(r[1]) + fabs(r[2]) > 0.0)) return set_err(ctx, LVR_EINVAL, "degenerate camera");
    const double tanh_ = tan((double)view->fovy_deg * M_PI / 360.0);
    for (int a = 0; a < 3; a++) {
        P.F[a] = (float)f[a];
        P.R[a] = (float)r[a];
        P.U[a] = (float)u[a];
        P.eye[a] = view->eye[a];
    }
    P.th = (float)tanh_;
    P.tw = (float)(tanh_ * (double)view->width / (double)view->height);
    P.W = view->width; P.H = view->height; P.x0 = x0; P.y0 = y0; P.cw = cw; P.ch = ch;
    P.tile_w = tw; P.tile_h = th;
    double ld[3] = {view->light_dir[0], view->light_dir[1], view->light_dir[2]};
    norm3(ld);
    for (int a = 0; a < 3; a++) P.Lt[a] = (float)(-ld[a]);
    P.opaque = desc->opaque ? 1 : 0;
    P.ert = desc->ert_alpha;
    P.shadows = desc->shadows ? 1 : 0;
    P.ao = desc->ao_mode == 1 ? 1 : 0;
    P.ao_rays = desc->ao_rays;
    P.ao_radius = desc->ao_radius;
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

    const size_t out_bytes = (size_t)cw * ch * 16;
    const bool host_out = !is_device_ptr(rgba);
    const bool host_cnt = counters && !is_device_ptr(counters);
    lvr_status st = LVR_OK;
    if (host_out && (st = ensure_stage_out(ctx, out_bytes)) != LVR_OK) return st;
    P.out = host_out ? (float4 *)ctx->stage_out : (float4 *)rgba;
    if (counters) {
        P.counters = host_cnt ? (unsigned long long *)ctx->d_u64 : (unsigned long long *)counters;
        LVR_CUDA(ctx, cudaMemsetAsync(P.counters, 0, 32, s));
    }
    dim3 grid((cw + 2 * tw - 1) / (2 * tw), (ch + 2 * th - 1) / (2 * th));
    render_kernel<<<grid, RT, 0, s>>>(P);
    LVR_CUDA(ctx, cudaGetLastError());
    if (host_out) LVR_CUDA(ctx, cudaMemcpyAsync(rgba, P.out, out_bytes, cudaMemcpyDeviceToHost, s));
    if (host_cnt) LVR_CUDA(ctx, cudaMemcpyAsync(counters, P.counters, 32, cudaMemcpyDeviceToHost, s));
    if (host_out || host_cnt) LVR_CUDA(ctx, cudaStreamSynchronize(s));
    return LVR_OK;
}
