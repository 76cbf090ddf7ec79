// Rasterised comparison system (the paper's baseline, Secs. 1 and 5.1):
// tubes around the input polylines, per-pixel fragment lists sorted by depth
// and blended front to back; opaque tubes by a depth test.
//
// Geometry: vertex i of a curve maps to p_i = fl32(fl32(v - origin) * scale);
// each pair (p_i, p_i+1) of one curve is a capsule of radius r (the tube
// piece with spherical ends), identified by i (so capsule order = input
// order), with attribute byte floor(((A_i + A_i+1) 255 + 65535) / 131070).
// A pixel's primary ray (the ray caster's float32 construction) leaves one
// fragment per capsule it enters (entry > 0), with no voxel model involved.
//
// GPU design. Capsules are rasterised one thread each over the pixels of
// their conservative screen rectangle (the two end spheres' bounds):
//   transparent: pass 1 counts fragments per pixel (atomics), an exclusive
//   scan places each pixel's list, pass 2 writes (depth, capsule) pairs into
//   it; one warp per pixel then sorts its list (ascending-only bitonic
//   network, in shared memory up to 512 entries, in place in global memory
//   beyond), finds the termination index with the float32 opacity
//   recurrence, shades the blended fragments across the lanes and sums them
//   with a warp prefix product of (1 - alpha) (float32);
//   opaque: pass 1 takes the 64-bit minimum of the depth per pixel, pass 2
//   the smallest capsule id among the fragments at that depth, and a thread
//   per pixel shades the winner.
// Depths are float-float sums T + s (no float64 on the device): T a float32
// ray parameter near the surface part hit, s the float32 entry computed from
// a local origin built in float-float (as the ray caster does per voxel),
// normalised to hi + lo and ordered as one 64-bit integer key. Sphere entries
// use a frame anchored at the sphere's centre, so the two capsules sharing a
// joint give bit-identical depths there and keep capsule order.
#include <math.h>
#include <string.h>

#include "lvr_internal.cuh"

namespace {

constexpr int RS_CAP = 512;     // per-pixel lists sorted in shared memory up to this length
constexpr int RS_WARPS = 4;     // resolve kernel: warps per block, one pixel per warp at a time
constexpr unsigned FULLW = 0xffffffffu;

struct V3 { float x, y, z; };
__device__ __forceinline__ V3 v3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ V3 vsub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ float vdot(V3 a, V3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ V3 vaxpy(float s, V3 d, V3 p) { return {fmaf(s, d.x, p.x), fmaf(s, d.y, p.y), fmaf(s, d.z, p.z)}; }
__device__ __forceinline__ V3 vscale(V3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }

struct RasterParams {
    const float4 *sa, *sb;      // slot i: (p_i, attribute byte) and (p_i+1, 1 if a capsule starts at i)
    int64_t nslot;
    float F[3], R[3], U[3], eye[3], Lt[3];
    float tw, th;
    int32_t W, H, x0, y0, cw, ch;
    float r, r2;
    float ert, ka, kd, bg[3];
    uint32_t *count;            // per pixel: fragments (pass 1), then the write cursor
    const uint32_t *offset;     // [npix + 1]
    unsigned long long *ft;     // fragment depth keys
    uint32_t *fid;              // fragment capsules
    unsigned long long *zbuf;   // opaque: minimum depth bits per pixel
    uint32_t *zid;              // opaque: smallest capsule at that depth
    float4 *out;
    float4 *dirs;               // per crop pixel: its primary ray direction
    unsigned long long *stats;  // [0] longest list, [1] fragments (opaque)
    uint32_t *status;
    float tf[1024];
};

// x + y exactly as s + e (Knuth)
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// primary ray direction of pixel (i, j): float32 contract, each step rounded
__device__ __forceinline__ V3 ray_dir(const RasterParams &P, int i, int j) {
    const float sx = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * i + 1), (float)P.W), 1.0f), P.tw);
    const float sy = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * j + 1), (float)P.H), 1.0f), P.th);
    float d[3];
#pragma unroll
    for (int a = 0; a < 3; a++) d[a] = __fsub_rn(__fadd_rn(P.F[a], __fmul_rn(sx, P.R[a])), __fmul_rn(sy, P.U[a]));
    const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])), __fmul_rn(d[2], d[2]));
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    return v3(__fmul_rn(d[0], inv), __fmul_rn(d[1], inv), __fmul_rn(d[2], inv));
}

// eye + T D - c in float-float, rounded once
__device__ __forceinline__ V3 local_origin(const RasterParams &P, V3 D, float T, V3 c) {
    const float Da[3] = {D.x, D.y, D.z}, ca[3] = {c.x, c.y, c.z};
    float p[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float ph = __fmul_rn(T, Da[a]);
        const float pe = __fmaf_rn(T, Da[a], -ph);
        float sh, s2;
        two_sum_f(P.eye[a], ph, sh, s2);
        p[a] = __fadd_rn(__fsub_rn(sh, ca[a]), __fadd_rn(s2, pe));
    }
    return v3(p[0], p[1], p[2]);
}

// A depth hi + lo (|lo| <= ulp(hi) / 2) as a 64-bit key ordered like the
// value: the order-preserving images of hi and lo side by side.
constexpr unsigned long long KEY_NONE = ~0ull;
__device__ __forceinline__ uint32_t ford(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unford(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
// key of T + s, or KEY_NONE unless the sum is positive
__device__ __forceinline__ unsigned long long depth_key(float T, float s) {
    float hi, lo;
    two_sum_f(T, s, hi, lo);
    lo = __fadd_rn(lo, 0.0f);   // -0 -> +0
    if (!(hi > 0.0f || (hi == 0.0f && lo > 0.0f))) return KEY_NONE;
    return ((unsigned long long)ford(hi) << 32) | ford(lo);
}

// first entry of p + s D into the sphere of radius sqrt(r2) around the origin
__device__ __forceinline__ float sphere_entry0(V3 p, V3 D, float r2) {
    const float sc = -vdot(p, D);
    const V3 q = vaxpy(sc, D, p);
    const float d2 = vdot(q, q);
    return d2 > r2 ? INFINITY : sc - sqrtf(r2 - d2);
}

__device__ __forceinline__ unsigned long long sphere_depth(const RasterParams &P, V3 D, V3 c) {
    const float T = vdot(vsub(c, v3(P.eye[0], P.eye[1], P.eye[2])), D);
    const float s = sphere_entry0(local_origin(P, D, T, c), D, P.r2);
    return s < INFINITY ? depth_key(T, s) : KEY_NONE;
}

// Depth key of the ray's entry into capsule [a, b], or KEY_NONE.
__device__ __forceinline__ unsigned long long capsule_depth(const RasterParams &P, V3 D, V3 a, V3 b) {
    unsigned long long best = KEY_NONE;
    const V3 ba = vsub(b, a);
    const float L2 = vdot(ba, ba);
    if (L2 > 0.0f) {
        // lateral surface, in a frame anchored at a
        const float Ta = vdot(vsub(a, v3(P.eye[0], P.eye[1], P.eye[2])), D);
        const V3 p = local_origin(P, D, Ta, a);
        const float L = sqrtf(L2), iL = 1.0f / L;
        const V3 w = vscale(ba, iL);
        const float dw = vdot(D, w), ow = vdot(p, w);
        const V3 Dp = vaxpy(-dw, w, D), Op = vaxpy(-ow, w, p);
        const float A = vdot(Dp, Dp);
        if (A > 1e-12f) {
            const float sc = -vdot(Dp, Op) / A;
            const V3 q = vaxpy(sc, Dp, Op);
            const float d2 = vdot(q, q);
            if (d2 > P.r2) return KEY_NONE;              // misses the infinite cylinder
            const float s = sc - sqrtf((P.r2 - d2) / A);
            const float y = fmaf(s, dw, ow);
            if (y > 0.0f && y < L) best = depth_key(Ta, s);
        } else if (vdot(Op, Op) > P.r2) {
            return KEY_NONE;
        }
        best = min(best, sphere_depth(P, D, b));
    }
    return min(best, sphere_depth(P, D, a));
}

// Conservative pixel rectangle of the capsule (both end spheres); false if
// it lies behind the camera or off the crop.
__device__ bool capsule_rect(const RasterParams &P, V3 a, V3 b, int &i0, int &i1, int &j0, int &j1) {
    float sxl = INFINITY, sxh = -INFINITY, syl = INFINITY, syh = -INFINITY;
    bool near = false, front = false;
    const V3 e = v3(P.eye[0], P.eye[1], P.eye[2]);
    const V3 F = v3(P.F[0], P.F[1], P.F[2]), R = v3(P.R[0], P.R[1], P.R[2]), U = v3(P.U[0], P.U[1], P.U[2]);
    for (int k = 0; k < 2; k++) {
        const V3 rel = vsub(k ? b : a, e);
        const float z = vdot(rel, F), x = vdot(rel, R), y = -vdot(rel, U);
        if (z + P.r > 0.0f) front = true;
        if (z - P.r <= 1e-3f) { near = true; continue; }
        const float zl = z - P.r, zh = z + P.r;
        sxl = fminf(sxl, fminf((x - P.r) / zl, (x - P.r) / zh));
        sxh = fmaxf(sxh, fmaxf((x + P.r) / zl, (x + P.r) / zh));
        syl = fminf(syl, fminf((y - P.r) / zl, (y - P.r) / zh));
        syh = fmaxf(syh, fmaxf((y + P.r) / zl, (y + P.r) / zh));
    }
    if (!front) return false;
    if (near) {   // reaches the camera plane: the whole crop
        i0 = P.x0; i1 = P.x0 + P.cw - 1; j0 = P.y0; j1 = P.y0 + P.ch - 1;
        return true;
    }
    // pixel i has sx = ((2i + 1) / W - 1) tw: i = ((sx / tw + 1) W - 1) / 2; one pixel of margin
    const float fi0 = ((sxl / P.tw + 1.0f) * (float)P.W - 1.0f) * 0.5f, fi1 = ((sxh / P.tw + 1.0f) * (float)P.W - 1.0f) * 0.5f;
    const float fj0 = ((syl / P.th + 1.0f) * (float)P.H - 1.0f) * 0.5f, fj1 = ((syh / P.th + 1.0f) * (float)P.H - 1.0f) * 0.5f;
    const float lo_x = (float)P.x0, hi_x = (float)(P.x0 + P.cw - 1), lo_y = (float)P.y0, hi_y = (float)(P.y0 + P.ch - 1);
    const float ci0 = fmaxf(floorf(fi0) - 1.0f, lo_x), ci1 = fminf(ceilf(fi1) + 1.0f, hi_x);
    const float cj0 = fmaxf(floorf(fj0) - 1.0f, lo_y), cj1 = fminf(ceilf(fj1) + 1.0f, hi_y);
    if (!(ci0 <= ci1) || !(cj0 <= cj1)) return false;
    i0 = (int)ci0; i1 = (int)ci1; j0 = (int)cj0; j1 = (int)cj1;
    return true;
}

__global__ void __launch_bounds__(256)
rs_rays_kernel(const __grid_constant__ RasterParams P) {
    const int64_t npix = (int64_t)P.cw * P.ch;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const V3 D = ray_dir(P, (int)(p % P.cw) + P.x0, (int)(p / P.cw) + P.y0);
        P.dirs[p] = make_float4(D.x, D.y, D.z, 0.0f);
    }
}

// Per curve: grid coordinates and 16-bit attribute codes of its vertices,
// one slot per vertex (the last vertex of a curve starts no capsule).
__global__ void __launch_bounds__(256)
rs_prep_kernel(const float *__restrict__ xyz, const float *__restrict__ attr, const int64_t *__restrict__ off,
               int64_t nc, int64_t nv, float o0, float o1, float o2, float s, float amin, float aspan,
               float4 *__restrict__ sa, float4 *__restrict__ sb, uint32_t *status) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t beg = off[c], end = off[c + 1];
        if (beg < 0 || end < beg || end > nv || (c == 0 && beg != 0) || (c == nc - 1 && end != nv)) {
            atomicOr(status, ST_BAD_OFFSETS);
            continue;
        }
        float px = 0.0f, py = 0.0f, pz = 0.0f;
        int A0 = 0;
        for (int64_t i = beg; i < end; i++) {
            const float x = __fmul_rn(__fsub_rn(xyz[3 * i], o0), s);
            const float y = __fmul_rn(__fsub_rn(xyz[3 * i + 1], o1), s);
            const float z = __fmul_rn(__fsub_rn(xyz[3 * i + 2], o2), s);
            if (!(fabsf(x) < 16384.0f && fabsf(y) < 16384.0f && fabsf(z) < 16384.0f)) atomicOr(status, ST_BAD_VERTEX);
            int A = 0;
            if (attr) {
                const float av = attr[i];
                if (!isfinite(av)) atomicOr(status, ST_BAD_ATTR);
                float q = __fdiv_rn(__fsub_rn(av, amin), aspan);
                q = fminf(fmaxf(q, 0.0f), 1.0f);
                A = __float2int_rn(__fmul_rn(q, 65535.0f));
            }
            if (i > beg) {
                const int byte = (int)(((int64_t)(A0 + A) * 255 + 65535) / 131070);
                sa[i - 1] = make_float4(px, py, pz, __int_as_float(byte));
                sb[i - 1] = make_float4(x, y, z, 1.0f);
            }
            px = x; py = y; pz = z;
            A0 = A;
        }
        if (end > beg) {
            sa[end - 1] = make_float4(px, py, pz, __int_as_float(0));
            sb[end - 1] = make_float4(px, py, pz, 0.0f);
        }
    }
}

enum { PASS_COUNT = 0, PASS_WRITE = 1, PASS_DEPTH = 2, PASS_ID = 3 };

// One thread per capsule over its pixel rectangle.
template <int PASS>
__global__ void __launch_bounds__(256)
rs_frag_kernel(const __grid_constant__ RasterParams P) {
    unsigned long long nfrag = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P.nslot;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float4 B = P.sb[k];
        if (B.w == 0.0f) continue;
        const float4 Aw = P.sa[k];
        const V3 a = v3(Aw.x, Aw.y, Aw.z), b = v3(B.x, B.y, B.z);
        {   // the eye inside the capsule: no entering intersection
            const V3 ba = vsub(b, a), ea = vsub(v3(P.eye[0], P.eye[1], P.eye[2]), a);
            const float L2 = vdot(ba, ba);
            const float h = L2 > 0.0f ? fminf(1.0f, fmaxf(0.0f, vdot(ea, ba) / L2)) : 0.0f;
            const V3 q = vaxpy(-h, ba, ea);
            if (vdot(q, q) <= P.r2) continue;
        }
        int i0, i1, j0, j1;
        if (!capsule_rect(P, a, b, i0, i1, j0, j1)) continue;
        // bounding sphere of the capsule, for a cheap conservative reject
        const V3 mrel = vsub(v3(0.5f * (a.x + b.x), 0.5f * (a.y + b.y), 0.5f * (a.z + b.z)),
                             v3(P.eye[0], P.eye[1], P.eye[2]));
        const V3 hb = vsub(b, a);
        const float Rb = 0.5f * sqrtf(vdot(hb, hb)) + P.r;
        const float Rb2 = (Rb * 1.0001f + 1e-3f) * (Rb * 1.0001f + 1e-3f);
        for (int j = j0; j <= j1; j++)
            for (int i = i0; i <= i1; i++) {
                const int64_t pix = (int64_t)(j - P.y0) * P.cw + (i - P.x0);
                const float4 Dw = P.dirs[pix];
                const V3 D = v3(Dw.x, Dw.y, Dw.z);
                const V3 perp = vaxpy(-vdot(mrel, D), D, mrel);
                if (vdot(perp, perp) > Rb2) continue;
                const unsigned long long t = capsule_depth(P, D, a, b);
                if (t == KEY_NONE) continue;
                if constexpr (PASS == PASS_COUNT) {
                    atomicAdd(P.count + pix, 1u);
                } else if constexpr (PASS == PASS_WRITE) {
                    // the same decision as the counting pass; checked all the same
                    const uint32_t q = atomicAdd(P.count + pix, 1u);
                    if (q < P.offset[pix + 1] - P.offset[pix]) {
                        P.ft[P.offset[pix] + q] = t;
                        P.fid[P.offset[pix] + q] = (uint32_t)k;
                    } else {
                        atomicOr(P.status, ST_INTERNAL);
                    }
                } else if constexpr (PASS == PASS_DEPTH) {
                    atomicMin(P.zbuf + pix, t);
                    nfrag++;
                } else {
                    if (t == P.zbuf[pix]) atomicMin(P.zid + pix, (uint32_t)k);
                }
            }
    }
    if constexpr (PASS == PASS_DEPTH) {
        for (int o = 16; o > 0; o >>= 1) nfrag += __shfl_xor_sync(FULLW, nfrag, o);
        if ((threadIdx.x & 31) == 0 && nfrag) atomicAdd(P.stats + 1, nfrag);
    }
}

// Shading of a fragment (S1: ka + kd |n . L|, no shadows or AO): colour
// times the lighting factor in rgb, opacity in w.
__device__ __forceinline__ float4 shade(const RasterParams &P, const float4 *tf, V3 D, unsigned long long t,
                                        uint32_t k) {
    const float4 Aw = P.sa[k], B = P.sb[k];
    const V3 a = v3(Aw.x, Aw.y, Aw.z), ba = vsub(v3(B.x, B.y, B.z), a);
    const float Ta = vdot(vsub(a, v3(P.eye[0], P.eye[1], P.eye[2])), D);
    const float hi = unford((uint32_t)(t >> 32)), lo = unford((uint32_t)t);
    const V3 pl = vaxpy(__fadd_rn(__fsub_rn(hi, Ta), lo), D, local_origin(P, D, Ta, a));   // entry point - a
    const float L2 = vdot(ba, ba);
    const float h = L2 > 0.0f ? fminf(1.0f, fmaxf(0.0f, vdot(pl, ba) / L2)) : 0.0f;
    V3 n = vaxpy(-h, ba, pl);
    n = vscale(n, rsqrtf(fmaxf(vdot(n, n), 1e-30f)));
    const float kk = fmaf(P.kd, fabsf(n.x * P.Lt[0] + n.y * P.Lt[1] + n.z * P.Lt[2]), P.ka);
    const float4 c = tf[__float_as_int(Aw.w) & 255];
    return make_float4(c.x * kk, c.y * kk, c.z * kk, c.w);
}

__device__ __forceinline__ bool frag_less(unsigned long long ka, uint32_t ia, unsigned long long kb, uint32_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

// Ascending-only bitonic network over n entries (entries at or past n act as
// +inf and are never touched): for each block size k, compare i with its
// mirror i ^ (k - 1), then half-cleaners at strides k/4 .. 1.
template <class T, class I>
__device__ __forceinline__ void warp_sort(T *t, I *id, int n, int lane) {
    int S = 1;
    while (S < n) S <<= 1;
    for (int k = 2; k <= S; k <<= 1) {
        for (int m = k; m >= 2; m >>= 1) {
            const int mask = m == k ? k - 1 : m >> 1;
            for (int i = lane; i < S; i += 32) {
                const int j = i ^ mask;
                if (j > i && j < n) {
                    const unsigned long long ti = t[i], tj = t[j];
                    const uint32_t ii = id[i], ij = id[j];
                    if (frag_less(tj, ij, ti, ii)) {
                        t[i] = tj; t[j] = ti;
                        id[i] = ij; id[j] = ii;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// One warp per pixel: sort its list, find the termination index, shade and
// blend the fragments before it.
__global__ void __launch_bounds__(RS_WARPS * 32)
rs_resolve_kernel(const __grid_constant__ RasterParams P) {
    __shared__ unsigned long long st[RS_WARPS][RS_CAP];
    __shared__ uint32_t si[RS_WARPS][RS_CAP];
    __shared__ float4 tf[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        tf[i] = make_float4(P.tf[4 * i], P.tf[4 * i + 1], P.tf[4 * i + 2], P.tf[4 * i + 3]);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t npix = (int64_t)P.cw * P.ch;
    unsigned longest = 0;
    for (int64_t p = blockIdx.x * (int64_t)RS_WARPS + warp; p < npix; p += (int64_t)gridDim.x * RS_WARPS) {
        const uint32_t beg = P.offset[p];
        const int n = (int)(P.offset[p + 1] - beg);
        longest = max(longest, (unsigned)n);
        unsigned long long *t;
        uint32_t *id;
        if (n <= RS_CAP) {
            for (int i = lane; i < n; i += 32) {
                st[warp][i] = P.ft[beg + i];
                si[warp][i] = P.fid[beg + i];
            }
            __syncwarp();
            t = st[warp];
            id = si[warp];
        } else {
            t = P.ft + beg;
            id = P.fid + beg;
        }
        warp_sort(t, id, n, lane);
        // termination: the float32 opacity recurrence over the sorted list
        int m = n;
        if (P.ert <= 1.0f && lane == 0) {
            float A32 = 0.0f;
            for (int k = 0; k < n; k++) {
                const float al = tf[__float_as_int(P.sa[id[k]].w) & 255].w;
                A32 = __fadd_rn(A32, __fmul_rn(__fsub_rn(1.0f, A32), al));
                if (A32 >= P.ert) { m = k + 1; break; }
            }
        }
        m = __shfl_sync(FULLW, m, 0);
        // blend fragments 0 .. m-1: weight = alpha x prod of (1 - alpha) before it
        const float4 Dw = P.dirs[p];
        const V3 D = v3(Dw.x, Dw.y, Dw.z);
        float carry = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, Asum = 0.0f;
        for (int k0 = 0; k0 < m; k0 += 32) {
            const int k = k0 + lane;
            float4 c = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (k < m) c = shade(P, tf, D, t[k], id[k]);
            float x = 1.0f - c.w;              // inclusive prefix product of (1 - alpha)
            for (int o = 1; o < 32; o <<= 1) {
                const float y = __shfl_up_sync(FULLW, x, o);
                if (lane >= o) x *= y;
            }
            float before = __shfl_up_sync(FULLW, x, 1);
            if (lane == 0) before = 1.0f;
            const float w = k < m ? carry * before * c.w : 0.0f;
            C0 = fmaf(w, c.x, C0); C1 = fmaf(w, c.y, C1); C2 = fmaf(w, c.z, C2); Asum += w;
            carry *= __shfl_sync(FULLW, x, 31);
        }
        for (int o = 16; o > 0; o >>= 1) {
            C0 += __shfl_xor_sync(FULLW, C0, o);
            C1 += __shfl_xor_sync(FULLW, C1, o);
            C2 += __shfl_xor_sync(FULLW, C2, o);
            Asum += __shfl_xor_sync(FULLW, Asum, o);
        }
        if (lane == 0) {
            const float rest = 1.0f - Asum;
            P.out[p] = make_float4(fmaf(rest, P.bg[0], C0), fmaf(rest, P.bg[1], C1), fmaf(rest, P.bg[2], C2), Asum);
        }
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) longest = max(longest, __shfl_xor_sync(FULLW, longest, o));
    if (lane == 0) atomicMax(P.stats, (unsigned long long)longest);
}

// Opaque: shade each pixel's nearest fragment.
__global__ void __launch_bounds__(256)
rs_opaque_kernel(const __grid_constant__ RasterParams P) {
    __shared__ float4 tf[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        tf[i] = make_float4(P.tf[4 * i], P.tf[4 * i + 1], P.tf[4 * i + 2], P.tf[4 * i + 3]);
    __syncthreads();
    const int64_t npix = (int64_t)P.cw * P.ch;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = P.zid[p];
        if (k == 0xffffffffu) {
            P.out[p] = make_float4(P.bg[0], P.bg[1], P.bg[2], 0.0f);
            continue;
        }
        const float4 Dw = P.dirs[p];
        const float4 c = shade(P, tf, v3(Dw.x, Dw.y, Dw.z), P.zbuf[p], k);
        P.out[p] = make_float4(c.x, c.y, c.z, 1.0f);
    }
}

}  // namespace

extern "C" lvr_status lvr_raster(lvr_ctx *ctx, const float *xyz, const float *attr, const int64_t *curve_offsets,
                                 int64_t n_curves, int64_t n_vertices, const lvr_grid_desc *g,
                                 const lvr_view *view, const lvr_render_desc *desc, float *rgba,
                                 lvr_raster_stats *stats) {
    if (!ctx) return LVR_EINVAL;
    if (!g || !view || !desc || !rgba || !curve_offsets) return set_err(ctx, LVR_EINVAL, "lvr_raster: null argument");
    if (n_curves < 1 || n_vertices < 0 || n_vertices > 0xfffffffeLL)
        return set_err(ctx, LVR_EINVAL, "need >= 1 curve and < 2^32 - 1 vertices");
    if (n_vertices > 0 && !xyz) return set_err(ctx, LVR_EINVAL, "xyz is null");
    if (g->fit) return set_err(ctx, LVR_EINVAL, "lvr_raster takes an explicit grid (origin, scale)");
    if (!(g->scale > 0.0f) || !isfinite(g->scale)) return set_err(ctx, LVR_EINVAL, "scale must be > 0");
    if (!(desc->radius > 0.0f) || !(desc->radius < 1e3f)) return set_err(ctx, LVR_EINVAL, "radius must be > 0");
    if (desc->shadows || desc->ao_mode || desc->still)
        return set_err(ctx, LVR_EINVAL, "the rasterised comparison system shades locally (no shadows, AO or still mode)");
    if (view->width < 1 || view->height < 1) return set_err(ctx, LVR_EINVAL, "image size must be >= 1");
    if (!(view->fovy_deg > 0.0f && view->fovy_deg < 180.0f)) return set_err(ctx, LVR_EINVAL, "fovy out of (0,180)");
    int x0 = 0, y0 = 0, cw = view->width, ch = view->height;
    if (view->crop[2] > 0) {
        x0 = view->crop[0]; y0 = view->crop[1]; cw = view->crop[2]; ch = view->crop[3];
        if (x0 < 0 || y0 < 0 || ch < 1 || x0 + cw > view->width || y0 + ch > view->height)
            return set_err(ctx, LVR_EINVAL, "crop outside the image");
    }
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;

    RasterParams P;
    memset(&P, 0, sizeof P);
    if (!camera_basis(view, P.F, P.R, P.U, &P.th, &P.tw, P.Lt)) return set_err(ctx, LVR_EINVAL, "degenerate camera");
    for (int a = 0; a < 3; a++) P.eye[a] = view->eye[a];
    P.W = view->width; P.H = view->height; P.x0 = x0; P.y0 = y0; P.cw = cw; P.ch = ch;
    P.r = desc->radius;
    P.r2 = desc->radius * desc->radius;
    P.ert = desc->opaque ? 0.0f : desc->ert_alpha;
    P.ka = desc->ka;
    P.kd = desc->kd;
    for (int a = 0; a < 3; a++) P.bg[a] = desc->bg[a];
    memcpy(P.tf, desc->tf_rgba, sizeof P.tf);
    const int64_t npix = (int64_t)cw * ch;

    // inputs: host data staged
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t bx = (size_t)n_vertices * 12, ba = attr ? (size_t)n_vertices * 4 : 0, bo = (size_t)(n_curves + 1) * 8;
    lvr_status st = LVR_OK;
    if ((n_vertices > 0 && !is_device_ptr(xyz)) || (attr && !is_device_ptr(attr)) || !is_device_ptr(curve_offsets))
        if ((st = ensure_stage_in(ctx, al(bx) + al(ba) + al(bo))) != LVR_OK) return st;
    const void *dx = xyz, *da = attr, *dof = curve_offsets;
    if ((st = stage_input(ctx, xyz, bx, 0, &dx)) != LVR_OK) return st;
    if ((st = stage_input(ctx, attr, ba, al(bx), &da)) != LVR_OK) return st;
    if ((st = stage_input(ctx, curve_offsets, bo, al(bx) + al(ba), &dof)) != LVR_OK) return st;

    // scratch: slots | counts | offsets | scan tiles | opaque depth and id | staged output
    const int64_t nslot = n_vertices > 0 ? n_vertices : 1;
    const int64_t ntiles = scan_tile_count(npix);
    const bool host_out = !is_device_ptr(rgba);
    const size_t b_slot = al((size_t)nslot * 16), b_cnt = al((size_t)npix * 4), b_off = al((size_t)(npix + 1) * 4),
                 b_tiles = al((size_t)ntiles * 8), b_z = al((size_t)npix * 8), b_zid = al((size_t)npix * 4),
                 b_dir = al((size_t)npix * 16),
                 b_out = host_out ? al((size_t)npix * 16) : 0;
    if ((st = ensure_scratch(ctx, 2 * b_slot + b_cnt + b_off + b_tiles + b_z + b_zid + b_dir + b_out)) != LVR_OK)
        return st;
    char *sp = (char *)ctx->scratch;
    float4 *sa = (float4 *)sp; sp += b_slot;
    float4 *sb = (float4 *)sp; sp += b_slot;
    uint32_t *count = (uint32_t *)sp; sp += b_cnt;
    uint32_t *offset = (uint32_t *)sp; sp += b_off;
    unsigned long long *tiles = (unsigned long long *)sp; sp += b_tiles;
    unsigned long long *zbuf = (unsigned long long *)sp; sp += b_z;
    uint32_t *zid = (uint32_t *)sp; sp += b_zid;
    float4 *dirs = (float4 *)sp; sp += b_dir;
    float4 *out = host_out ? (float4 *)sp : (float4 *)rgba;
    P.sa = sa; P.sb = sb; P.nslot = n_vertices;
    P.count = count; P.offset = offset; P.zbuf = zbuf; P.zid = zid; P.out = out; P.dirs = dirs;
    P.stats = ctx->d_u64;
    P.status = ctx->d_status;

    LVR_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, 4, s));
    LVR_CUDA(ctx, cudaMemsetAsync(ctx->d_u64, 0, 16, s));
    const float aspan = g->attr_max - g->attr_min;
    LVR_CUDA(ctx, cudaMemsetAsync(sb, 0, (size_t)nslot * 16, s));   // every slot defined, capsule flags off
    rs_prep_kernel<<<grid1d(n_curves, 256), 256, 0, s>>>(
        (const float *)dx, (da && g->attr_max > g->attr_min) ? (const float *)da : nullptr, (const int64_t *)dof,
        n_curves, n_vertices, g->origin[0], g->origin[1], g->origin[2], g->scale, g->attr_min, aspan, sa, sb,
        ctx->d_status);
    rs_rays_kernel<<<grid1d(npix, 256), 256, 0, s>>>(P);
    LVR_CUDA(ctx, cudaGetLastError());
    const unsigned gslot = grid1d(n_vertices, 256);
    uint32_t *h32 = (uint32_t *)ctx->h_pinned;
    unsigned long long *h64 = (unsigned long long *)((char *)ctx->h_pinned + 64);
    uint64_t nfrag = 0, longest = 0;
    if (desc->opaque) {
        LVR_CUDA(ctx, cudaMemsetAsync(zbuf, 0xff, (size_t)npix * 8, s));
        LVR_CUDA(ctx, cudaMemsetAsync(zid, 0xff, (size_t)npix * 4, s));
        if (n_vertices > 0) {
            rs_frag_kernel<PASS_DEPTH><<<gslot, 256, 0, s>>>(P);
            rs_frag_kernel<PASS_ID><<<gslot, 256, 0, s>>>(P);
        }
        rs_opaque_kernel<<<grid1d(npix, 256), 256, 0, s>>>(P);
        LVR_CUDA(ctx, cudaGetLastError());
        LVR_CUDA(ctx, cudaMemcpyAsync(h32, ctx->d_status, 4, cudaMemcpyDeviceToHost, s));
        LVR_CUDA(ctx, cudaMemcpyAsync(h64, ctx->d_u64, 16, cudaMemcpyDeviceToHost, s));
        LVR_CUDA(ctx, cudaStreamSynchronize(s));
        nfrag = h64[1];
    } else {
        LVR_CUDA(ctx, cudaMemsetAsync(count, 0, (size_t)npix * 4, s));
        if (n_vertices > 0) rs_frag_kernel<PASS_COUNT><<<gslot, 256, 0, s>>>(P);
        scan_counts(s, count, npix, tiles, offset, ctx->d_status);
        LVR_CUDA(ctx, cudaGetLastError());
        LVR_CUDA(ctx, cudaMemcpyAsync(h32, ctx->d_status, 4, cudaMemcpyDeviceToHost, s));
        LVR_CUDA(ctx, cudaMemcpyAsync(h32 + 1, offset + npix, 4, cudaMemcpyDeviceToHost, s));
        LVR_CUDA(ctx, cudaStreamSynchronize(s));
        if (h32[0] & ST_OVERFLOW) return set_err(ctx, LVR_EOVERFLOW, "more than 2^32 - 1 fragments");
        if (h32[0] & (ST_BAD_OFFSETS | ST_BAD_VERTEX | ST_BAD_ATTR)) return set_err(ctx, LVR_EINVAL, "bad input: %s",
            h32[0] & ST_BAD_OFFSETS ? "curve offsets must start at 0, not decrease and end at n_vertices"
            : h32[0] & ST_BAD_VERTEX ? "vertex not finite or outside +-2^14 voxels of the grid" : "attribute not finite");
        nfrag = h32[1];
        if (nfrag > ctx->frag_cap) {
            dev_free(ctx, ctx->frag_t);
            dev_free(ctx, ctx->frag_id);
            ctx->frag_t = nullptr;
            ctx->frag_id = nullptr;
            ctx->frag_cap = 0;
            const size_t cap = (size_t)nfrag + nfrag / 8 + 1024;
            if ((st = dev_alloc(ctx, (void **)&ctx->frag_t, cap * 8)) != LVR_OK) return st;
            if ((st = dev_alloc(ctx, (void **)&ctx->frag_id, cap * 4)) != LVR_OK) return st;
            ctx->frag_cap = cap;
        }
        P.ft = (unsigned long long *)ctx->frag_t;
        P.fid = ctx->frag_id;
        LVR_CUDA(ctx, cudaMemsetAsync(count, 0, (size_t)npix * 4, s));
        if (n_vertices > 0) rs_frag_kernel<PASS_WRITE><<<gslot, 256, 0, s>>>(P);
        int sms = 0;
        LVR_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        const int64_t want = (npix + RS_WARPS - 1) / RS_WARPS;
        const unsigned grid = (unsigned)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
        rs_resolve_kernel<<<grid, RS_WARPS * 32, 0, s>>>(P);
        LVR_CUDA(ctx, cudaGetLastError());
        LVR_CUDA(ctx, cudaMemcpyAsync(h64, ctx->d_u64, 8, cudaMemcpyDeviceToHost, s));
        LVR_CUDA(ctx, cudaMemcpyAsync(h32, ctx->d_status, 4, cudaMemcpyDeviceToHost, s));
        LVR_CUDA(ctx, cudaStreamSynchronize(s));
        longest = h64[0];
        if (h32[0] & ST_INTERNAL) return set_err(ctx, LVR_ECUDA, "rasteriser: passes disagree on a fragment count");
    }
    if (h32[0] & ST_BAD_OFFSETS)
        return set_err(ctx, LVR_EINVAL, "curve offsets must start at 0, not decrease and end at n_vertices");
    if (h32[0] & ST_BAD_VERTEX) return set_err(ctx, LVR_EINVAL, "vertex not finite or outside +-2^14 voxels of the grid");
    if (h32[0] & ST_BAD_ATTR) return set_err(ctx, LVR_EINVAL, "attribute not finite");
    if (host_out && (st = copy_out(ctx, rgba, out, (size_t)npix * 16)) != LVR_OK) return st;
    if (stats) {
        stats->fragments = nfrag;
        stats->max_per_pixel = longest;
        stats->list_bytes = desc->opaque ? 0 : nfrag * 12;
    }
    return LVR_OK;
}
