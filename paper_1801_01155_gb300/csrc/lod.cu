// Density LoD (Sec. 3.4, Eq. 1): per voxel rho = sum length * sigma over its
// segments, then 2^3 pooling. Levels store sums (count, length, length*sigma);
// the density sampled at level l is dens_l / 8^l.
//
// Segment lengths are exact: endpoints are face-bin centres, integer in
// units of 1/(2N), so length = sqrt(I) / (2N) with I < 2^24 an integer;
// float32 sqrt of I is correctly rounded and the division by 2N is exact.
// Sums run in the canonical segment order (level 0) and in the fixed child
// order z, y, x (coarser levels), so results are deterministic.
#include <algorithm>
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "lvr_internal.cuh"

namespace {

__device__ __forceinline__ void face_point_2n(uint32_t face, uint32_t u, uint32_t v, int twoN, int q[3]) {
    const int ax = (int)(face >> 1);
    const int side = (face & 1u) ? twoN : 0;
    const int cu = 2 * (int)u + 1, cv = 2 * (int)v + 1;
    q[0] = ax == 0 ? side : cu;
    q[1] = ax == 1 ? side : (ax == 0 ? cu : cv);
    q[2] = ax == 2 ? side : cv;
}

__global__ void __launch_bounds__(256)
lod_level0_kernel(const uint32_t *__restrict__ offset, const uint64_t *__restrict__ rec, int64_t nvox,
                  int N, const float *__restrict__ sigma_g, uint32_t *cnt, float *len, float *dens) {
    __shared__ float sigma[256];
    sigma[threadIdx.x] = sigma_g[threadIdx.x];
    __syncthreads();
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const uint32_t beg = offset[v], end = offset[v + 1];
    const int twoN = 2 * N;
    const float inv2N = 1.0f / (float)twoN;      // power of two: exact
    float L = 0.0f, R = 0.0f;
    for (uint32_t i = beg; i < end; i++) {
        const uint64_t r = __ldg(rec + i);
        int a[3], b[3];
        face_point_2n(rec_face_in(r), rec_u_in(r), rec_v_in(r), twoN, a);
        face_point_2n(rec_face_out(r), rec_u_out(r), rec_v_out(r), twoN, b);
        const int I = (b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) +
                      (b[2] - a[2]) * (b[2] - a[2]);
        const float l = __fmul_rn(__fsqrt_rn((float)I), inv2N);
        L = __fadd_rn(L, l);
        R = __fmaf_rn(l, sigma[rec_attr(r)], R);
    }
    cnt[v] = end - beg;
    len[v] = L;
    dens[v] = R;
}

__global__ void __launch_bounds__(256)
lod_pool_kernel(int cx, int cy, int cz, const uint32_t *__restrict__ ccnt, const float *__restrict__ clen,
                const float *__restrict__ cdens, int px, int py, int pz, uint32_t *pcnt, float *plen,
                float *pdens) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t np = (int64_t)px * py * pz;
    if (p >= np) return;
    const int x = (int)(p % px), y = (int)((p / px) % py), z = (int)(p / ((int64_t)px * py));
    uint32_t c = 0;
    float L = 0.0f, R = 0.0f;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                const int X = 2 * x + dx, Y = 2 * y + dy, Z = 2 * z + dz;
                if (X >= cx || Y >= cy || Z >= cz) continue;
                const int64_t i = X + (int64_t)cx * (Y + (int64_t)cy * Z);
                c += ccnt[i];
                L = __fadd_rn(L, clen[i]);
                R = __fadd_rn(R, cdens[i]);
            }
    pcnt[p] = c;
    plen[p] = L;
    pdens[p] = R;
}

// Corner-packed copy of one level for trilinear sampling: padded cell
// (i, j, k) -> X = i - lo, Y = j - lo, Z = k - lo; per z-slice Z and Z + 1 a
// float4 (v(X, Y), v(X+1, Y) - v(X, Y), v(X, Y+1), v(X+1, Y+1) - v(X, Y+1)),
// zero outside the grid; the two slices of a cell are adjacent (32 bytes).
__global__ void __launch_bounds__(256)
lod_pack_kernel(const float *__restrict__ d, int dx, int dy, int dz, int lo, int px, int py, int pz, float4 *pk) {
    const int64_t np = (int64_t)px * py * pz;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < np; c += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(c % px) - lo, Y = (int)((c / px) % py) - lo, Z = (int)(c / ((int64_t)px * py)) - lo;
        auto v = [&](int x, int y, int z) {
            return (x >= 0 && y >= 0 && z >= 0 && x < dx && y < dy && z < dz)
                       ? __ldg(d + (x + (int64_t)dx * (y + (int64_t)dy * z))) : 0.0f;
        };
        float4 s[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const float v00 = v(X, Y, Z + h), v10 = v(X + 1, Y, Z + h), v01 = v(X, Y + 1, Z + h),
                        v11 = v(X + 1, Y + 1, Z + h);
            s[h] = make_float4(v00, v10 - v00, v01, v11 - v01);
        }
        pk[2 * c] = s[0];
        pk[2 * c + 1] = s[1];
    }
}

// One sample of the spherical AO stencil: integer part and fraction of s d.
struct AoStep {
    int32_t ix, iy, iz;
    float fx, fy, fz;
    int32_t pad[2];
};

// Spherical per-voxel AO (Sec. 5.3, second approach): per voxel centre, for
// each direction, the level-0 density summed at unit steps (cell-centred
// trilinear samples, zero outside the grid) until it reaches 1; AO = 1 -
// mean min(1, O). A sample at c + s d has the same fractional position in
// every voxel, so the stencil (integer offsets, fractions) is one table.
__global__ void __launch_bounds__(256)
ao_field_kernel(const float4 *__restrict__ pk0, int64_t px, int64_t sz, int dx, int dy, int dz,
                const AoStep *__restrict__ tab, int rays, int steps, float *field) {
    const int64_t n = (int64_t)dx * dy * dz;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int vx = (int)(v % dx), vy = (int)((v / dx) % dy), vz = (int)(v / ((int64_t)dx * dy));
        float occ = 0.0f;
        for (int k = 0; k < rays; k++) {
            float O = 0.0f;
            for (int s = 0; s < steps; s++) {
                const AoStep e = tab[k * steps + s];
                const int ix = vx + e.ix, iy = vy + e.iy, iz = vz + e.iz;
                float val = 0.0f;
                if ((unsigned)(ix + 1) <= (unsigned)dx && (unsigned)(iy + 1) <= (unsigned)dy &&
                    (unsigned)(iz + 1) <= (unsigned)dz) {
                    const float4 *c = pk0 + 2 * (ix + px * iy + sz * iz);
                    const float4 a = __ldg(c), b = __ldg(c + 1);
                    const float x00 = fmaf(e.fx, a.y, a.x), x10 = fmaf(e.fx, a.w, a.z);
                    const float x01 = fmaf(e.fx, b.y, b.x), x11 = fmaf(e.fx, b.w, b.z);
                    const float y0 = fmaf(e.fy, x10 - x00, x00), y1 = fmaf(e.fy, x11 - x01, x01);
                    val = fmaf(e.fz, y1 - y0, y0);
                }
                O += val;
                if (O >= 1.0f) break;
            }
            occ += fminf(1.0f, O);
        }
        field[v] = 1.0f - occ / (float)rays;
    }
}

constexpr int AOT_MAX_TAPS = 640;                  // stencil entries passed as a kernel parameter

// Two voxels per thread: a block covers 64 x 4 x 2 voxels, a thread the x
// neighbours 2i and 2i + 1, whose trilinear corners share a column (the
// upper x corners of the first are the lower ones of the second), so a tap
// costs 12 shared loads for two voxels instead of 16. Even and odd tile
// columns are stored in separate planes, so a warp's loads stay on distinct
// banks. The density of the tile grown by H cells per side (zero outside the
// grid) is staged once per block; the stencil (corner column offsets and
// trilinear weights) comes from the constant bank. O is not cut off at 1:
// min(1, O) is the same either way since density >= 0.
constexpr int AOP_X = 64, AOP_Y = 4, AOP_Z = 2;

struct AoPairTap {
    float4 wa, wb;         // corner (x, y, z) bits -> weight (bit 0 x, bit 1 y, bit 2 z): corners 0-3, 4-7
    int32_t off[3];        // per corner column d = 0, 1, 2: plane * plane size + offset in the plane
    int32_t pad;
};
struct AoPairTaps {
    AoPairTap t[AOT_MAX_TAPS];
};

template <int STEPS>
__global__ void __launch_bounds__(AOP_X / 2 * AOP_Y * AOP_Z)
ao_field_pair_kernel(const float *__restrict__ dens, int dx, int dy, int dz, const __grid_constant__ AoPairTaps tab,
                     int rays, int H, float *field) {
    extern __shared__ float tile[];
    const int TX = AOP_X + 2 * H, TY = AOP_Y + 2 * H, TZ = AOP_Z + 2 * H;
    const int TXh = (TX + 1) / 2, PS = TXh * TY * TZ;
    const int tx0 = blockIdx.x * AOP_X, ty0 = blockIdx.y * AOP_Y, tz0 = blockIdx.z * AOP_Z;
    for (int i = threadIdx.x; i < TX * TY * TZ; i += blockDim.x) {
        const int X = i % TX, Y = (i / TX) % TY, Z = i / (TX * TY);
        const int gx = tx0 - H + X, gy = ty0 - H + Y, gz = tz0 - H + Z;
        tile[(X & 1) * PS + (X >> 1) + TXh * (Y + TY * Z)] =
            (gx >= 0 && gy >= 0 && gz >= 0 && gx < dx && gy < dy && gz < dz)
                ? __ldg(dens + (gx + (int64_t)dx * (gy + (int64_t)dy * gz))) : 0.0f;
    }
    __syncthreads();
    const int lx = threadIdx.x % (AOP_X / 2), ly = (threadIdx.x / (AOP_X / 2)) % AOP_Y,
              lz = threadIdx.x / (AOP_X / 2 * AOP_Y);
    const int vx = tx0 + 2 * lx, vy = ty0 + ly, vz = tz0 + lz;
    if (vx >= dx || vy >= dy || vz >= dz) return;
    const float *cb = tile + lx + TXh * ((ly + H) + TY * (lz + H));
    const int sy = TXh, sz = TXh * TY;
    float occ0 = 0.0f, occ1 = 0.0f;
    for (int k = 0; k < rays; k++) {
        float O0 = 0.0f, O1 = 0.0f;
#pragma unroll
        for (int s = 0; s < STEPS; s++) {
            const AoPairTap &e = tab.t[k * STEPS + s];
            const float4 wa = e.wa, wb = e.wb;
            const float *c0 = cb + e.off[0], *c1 = cb + e.off[1], *c2 = cb + e.off[2];
            const float p0 = c0[0], p1 = c1[0], p2 = c2[0];
            const float q0 = c0[sy], q1 = c1[sy], q2 = c2[sy];
            const float r0 = c0[sz], r1 = c1[sz], r2 = c2[sz];
            const float u0 = c0[sz + sy], u1 = c1[sz + sy], u2 = c2[sz + sy];
            O0 = fmaf(wa.x, p0, O0);
            O0 = fmaf(wa.y, p1, O0);
            O0 = fmaf(wa.z, q0, O0);
            O0 = fmaf(wa.w, q1, O0);
            O0 = fmaf(wb.x, r0, O0);
            O0 = fmaf(wb.y, r1, O0);
            O0 = fmaf(wb.z, u0, O0);
            O0 = fmaf(wb.w, u1, O0);
            O1 = fmaf(wa.x, p1, O1);
            O1 = fmaf(wa.y, p2, O1);
            O1 = fmaf(wa.z, q1, O1);
            O1 = fmaf(wa.w, q2, O1);
            O1 = fmaf(wb.x, r1, O1);
            O1 = fmaf(wb.y, r2, O1);
            O1 = fmaf(wb.z, u1, O1);
            O1 = fmaf(wb.w, u2, O1);
        }
        occ0 += fminf(1.0f, O0);
        occ1 += fminf(1.0f, O1);
    }
    const int64_t o = vx + (int64_t)dx * (vy + (int64_t)dy * vz);
    field[o] = 1.0f - occ0 / (float)rays;
    if (vx + 1 < dx) field[o + 1] = 1.0f - occ1 / (float)rays;
}

}  // namespace

// ------------------------------------------------------------------ representative lines
// Sec. 3.4: one average line per cell of every level. Level 0 averages the
// start points and the end points of a voxel's segments separately, in the
// canonical segment order, flipping a segment first when it points against
// the running average (sum of end points minus sum of start points); each
// average is snapped to the nearest face of the cell (ties: the lower face
// id) and the bin holding its projection. Coarser cells average their
// children's lines (children in z, y, x order) the same way. After each
// level, a line end point on a face shared with a neighbour's line end point
// (start point taken first when both lie on that face) moves, with it, to
// the bin of their average. Points are integers in units of 1/(2N) of a
// cell (children: 1/(4N) of the parent), so every decision is exact.
//
// Joining is a gather: a face pair only changes the two end points on that
// face, so each cell reads its neighbours from the unjoined copy and writes
// its own word; the result equals joining the pairs one after another.
namespace {

__device__ __forceinline__ uint32_t rep_point(uint64_t w, int e) { return (uint32_t)(w >> (8 + 24 * e)) & 0xffffffu; }

// nearest face and bins of the average point S / n (S in units 1 / U per cell edge)
__device__ __forceinline__ uint32_t rep_snap(const long long S[3], long long n, long long U, long long N) {
    int best = 0;
    long long bd = S[0];
    for (int f = 1; f < 6; f++) {
        const long long d = (f & 1) ? U * n - S[f >> 1] : S[f >> 1];
        if (d < bd) { bd = d; best = f; }
    }
    const int ax = best >> 1, b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
    uint32_t bin[2];
    const int bx[2] = {b0, b1};
    for (int i = 0; i < 2; i++) {
        const long long s = S[bx[i]] < 0 ? 0 : S[bx[i]];
        const long long b = (s * N) / (U * n);
        bin[i] = (uint32_t)(b > N - 1 ? N - 1 : b);
    }
    return (uint32_t)best | bin[0] << 8 | bin[1] << 16;
}

__device__ __forceinline__ void rep_accumulate(int a[3], int b[3], long long SA[3], long long SB[3], long long &n) {
    if (n > 0) {
        long long dot = 0;
        for (int c = 0; c < 3; c++) dot += (long long)(b[c] - a[c]) * (SB[c] - SA[c]);
        if (dot < 0)
            for (int c = 0; c < 3; c++) { const int t = a[c]; a[c] = b[c]; b[c] = t; }
    }
    for (int c = 0; c < 3; c++) { SA[c] += a[c]; SB[c] += b[c]; }
    n++;
}

__device__ __forceinline__ uint64_t rep_word(uint32_t ps, uint32_t pe) {
    return 1ull | (uint64_t)ps << 8 | (uint64_t)pe << 32;
}

__global__ void __launch_bounds__(256)
rep_level0_kernel(const uint32_t *__restrict__ offset, const uint64_t *__restrict__ rec, int64_t nvox, int N,
                  uint64_t *__restrict__ out) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const uint32_t beg = offset[v], end = offset[v + 1];
    long long SA[3] = {0, 0, 0}, SB[3] = {0, 0, 0}, n = 0;
    for (uint32_t k = beg; k < end; k++) {
        const uint64_t r = rec[k];
        int a[3], b[3];
        face_point_2n(rec_face_in(r), rec_u_in(r), rec_v_in(r), 2 * N, a);
        face_point_2n(rec_face_out(r), rec_u_out(r), rec_v_out(r), 2 * N, b);
        rep_accumulate(a, b, SA, SB, n);
    }
    out[v] = n ? rep_word(rep_snap(SA, n, 2 * N, N), rep_snap(SB, n, 2 * N, N)) : 0ull;
}

__global__ void __launch_bounds__(256)
rep_pool_kernel(const uint64_t *__restrict__ child, int cx, int cy, int cz, uint64_t *__restrict__ out,
                int px, int py, int pz, int N) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= (int64_t)px * py * pz) return;
    const int x = (int)(c % px), y = (int)((c / px) % py), z = (int)(c / ((int64_t)px * py));
    long long SA[3] = {0, 0, 0}, SB[3] = {0, 0, 0}, n = 0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                const int X = 2 * x + dx, Y = 2 * y + dy, Z = 2 * z + dz;
                if (X >= cx || Y >= cy || Z >= cz) continue;
                const uint64_t w = child[X + (int64_t)cx * (Y + (int64_t)cy * Z)];
                if (!(w & 1ull)) continue;
                int a[3], b[3];
                const uint32_t ps = rep_point(w, 0), pe = rep_point(w, 1);
                face_point_2n(ps & 0xffu, (ps >> 8) & 0xffu, ps >> 16, 2 * N, a);
                face_point_2n(pe & 0xffu, (pe >> 8) & 0xffu, pe >> 16, 2 * N, b);
                const int off[3] = {dx, dy, dz};
                for (int q = 0; q < 3; q++) {
                    a[q] += off[q] * 2 * N;
                    b[q] += off[q] * 2 * N;
                }
                rep_accumulate(a, b, SA, SB, n);
            }
    out[c] = n ? rep_word(rep_snap(SA, n, 4 * N, N), rep_snap(SB, n, 4 * N, N)) : 0ull;
}

// which end point (0 start, 1 end) of line word w lies on face f, start first; -1: none
__device__ __forceinline__ int rep_end_on(uint64_t w, uint32_t f) {
    if ((rep_point(w, 0) & 0xffu) == f) return 0;
    if ((rep_point(w, 1) & 0xffu) == f) return 1;
    return -1;
}

__global__ void __launch_bounds__(256)
rep_join_kernel(const uint64_t *__restrict__ in, uint64_t *__restrict__ out, int dx, int dy, int dz) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= (int64_t)dx * dy * dz) return;
    uint64_t w = in[c];
    if (w & 1ull) {
        const int dm[3] = {dx, dy, dz};
        const int p[3] = {(int)(c % dx), (int)((c / dx) % dy), (int)(c / ((int64_t)dx * dy))};
        const int64_t stride[3] = {1, dx, (int64_t)dx * dy};
        uint64_t res = w;
        for (int e = 0; e < 2; e++) {
            const uint32_t pt = rep_point(w, e), f = pt & 0xffu;
            if (rep_end_on(w, f) != e) continue;   // the other end point on this face joins
            const int ax = (int)(f >> 1), side = (int)(f & 1u);
            const int q = p[ax] + (side ? 1 : -1);
            if (q < 0 || q >= dm[ax]) continue;
            const uint64_t nw = in[c + (side ? stride[ax] : -stride[ax])];
            if (!(nw & 1ull)) continue;
            const int ne = rep_end_on(nw, f ^ 1u);
            if (ne < 0) continue;
            const uint32_t np = rep_point(nw, ne);
            const uint32_t u = (((pt >> 8) & 0xffu) + ((np >> 8) & 0xffu) + 1u) >> 1;
            const uint32_t v = ((pt >> 16) + (np >> 16) + 1u) >> 1;
            const int sh = 8 + 24 * e;
            res = (res & ~(0xffffffull << sh)) | (uint64_t)(f | u << 8 | v << 16) << sh;
        }
        w = res;
    }
    out[c] = w;
}

}  // namespace

extern "C" lvr_status lvr_lod_rep_lines(lvr_ctx *ctx, lvr_lod *lod, const lvr_lineset *ls) {
    if (!ctx) return LVR_EINVAL;
    if (!lod || !ls) return set_err(ctx, LVR_EINVAL, "lvr_lod_rep_lines: null argument");
    for (int a = 0; a < 3; a++)
        if (lod->dims[0][a] != ls->res[a]) return set_err(ctx, LVR_EINVAL, "LoD does not belong to this line set");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    lvr_status st = LVR_OK;
    for (int l = 0; l < lod->levels && st == LVR_OK; l++)
        if (!lod->rep[l]) {
            const size_t n = (size_t)lod->dims[l][0] * lod->dims[l][1] * lod->dims[l][2];
            st = dev_alloc(ctx, (void **)&lod->rep[l], n * 8);
        }
    uint64_t *tmp = nullptr;
    const int64_t n0 = (int64_t)ls->res[0] * ls->res[1] * ls->res[2];
    if (st == LVR_OK) st = dev_alloc(ctx, (void **)&tmp, (size_t)n0 * 8);
    if (st != LVR_OK) return st;
    const int N = ls->bins;
    rep_level0_kernel<<<grid1d(n0, 256), 256, 0, s>>>(ls->offset, ls->rec, n0, N, tmp);
    rep_join_kernel<<<grid1d(n0, 256), 256, 0, s>>>(tmp, lod->rep[0], ls->res[0], ls->res[1], ls->res[2]);
    for (int l = 1; l < lod->levels; l++) {
        const int32_t *c = lod->dims[l - 1], *p = lod->dims[l];
        const int64_t np = (int64_t)p[0] * p[1] * p[2];
        rep_pool_kernel<<<grid1d(np, 256), 256, 0, s>>>(lod->rep[l - 1], c[0], c[1], c[2], tmp, p[0], p[1], p[2], N);
        rep_join_kernel<<<grid1d(np, 256), 256, 0, s>>>(tmp, lod->rep[l], p[0], p[1], p[2]);
    }
    const cudaError_t e = cudaGetLastError();
    dev_free(ctx, tmp);   // stream-ordered
    if (e != cudaSuccess) return cuda_err(ctx, e, "lvr_lod_rep_lines");
    lod->rep_bins = N;
    return LVR_OK;
}

extern "C" lvr_status lvr_export_rep_lines(lvr_ctx *ctx, const lvr_lod *lod, int level, uint8_t *out8) {
    if (!ctx) return LVR_EINVAL;
    if (!lod || level < 0 || level >= lod->levels || !lod->rep[level] || !out8)
        return set_err(ctx, LVR_EINVAL, "no representative lines at this level");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t n = (size_t)lod->dims[level][0] * lod->dims[level][1] * lod->dims[level][2];
    return copy_out(ctx, out8, lod->rep[level], n * 8);
}

extern "C" lvr_status lvr_lod_ao_field(lvr_ctx *ctx, lvr_lod *lod, int rays, float radius) {
    if (!ctx) return LVR_EINVAL;
    if (!lod) return set_err(ctx, LVR_EINVAL, "lvr_lod_ao_field: null LoD");
    if (rays < 1 || rays > 4096 || !(radius >= 1.0f) || radius > 64.0f)
        return set_err(ctx, LVR_EINVAL, "rays must be in [1,4096] and the radius in [1,64] voxels");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    const int steps = (int)floorf(radius);
    // the stencil: spherical Fibonacci directions, samples at unit steps
    std::vector<AoStep> tab((size_t)rays * steps);
    const double golden = M_PI * (3.0 - sqrt(5.0));
    for (int k = 0; k < rays; k++) {
        const double z = 1.0 - (2.0 * k + 1.0) / rays, rr = sqrt(1.0 - z * z), ph = k * golden;
        const double d[3] = {rr * cos(ph), rr * sin(ph), z};
        for (int s = 1; s <= steps; s++) {
            AoStep &e = tab[(size_t)k * steps + s - 1];
            int32_t *ip[3] = {&e.ix, &e.iy, &e.iz};
            float *fp[3] = {&e.fx, &e.fy, &e.fz};
            for (int a = 0; a < 3; a++) {
                const double o = s * d[a], fl = floor(o);
                *ip[a] = (int32_t)fl;
                *fp[a] = (float)(o - fl);
            }
            e.pad[0] = e.pad[1] = 0;
        }
    }
    const int32_t *dm = lod->dims[0];
    const int64_t n = (int64_t)dm[0] * dm[1] * dm[2];
    lvr_status st = LVR_OK;
    if (!lod->aof && (st = dev_alloc(ctx, (void **)&lod->aof, (size_t)n * 4)) != LVR_OK) return st;
    const size_t tb = tab.size() * sizeof(AoStep);
    if ((st = ensure_stage_in(ctx, tb)) != LVR_OK) return st;
    LVR_CUDA(ctx, cudaMemcpyAsync(ctx->stage_in, tab.data(), tb, cudaMemcpyHostToDevice, ctx->stream));
    const int H = steps + 1;   // samples reach floor(s d) in [-steps, steps] plus one corner
    const int PX = AOP_X + 2 * H, PY = AOP_Y + 2 * H, PZ = AOP_Z + 2 * H, PXh = (PX + 1) / 2;
    const size_t pair_bytes = (size_t)2 * PXh * PY * PZ * 4;
    if (steps == 5 && pair_bytes <= 200 * 1024 && tab.size() <= (size_t)AOT_MAX_TAPS) {
        static AoPairTaps taps;   // host staging of the kernel parameter (copied at launch)
        static std::mutex mu;
        std::lock_guard<std::mutex> lk(mu);
        const int PS = PXh * PY * PZ;
        for (size_t i = 0; i < tab.size(); i++) {
            const AoStep &e = tab[i];
            AoPairTap &t = taps.t[i];
            const int m = H + e.ix;   // >= 1: column of the first corner, relative to 2 x (thread's x)
            for (int d = 0; d < 3; d++)
                t.off[d] = ((m + d) & 1) * PS + ((m + d) >> 1) + PXh * (e.iy + PY * e.iz);
            float w[8];
            for (int c = 0; c < 8; c++)
                w[c] = (c & 1 ? e.fx : 1.0f - e.fx) * (c & 2 ? e.fy : 1.0f - e.fy) * (c & 4 ? e.fz : 1.0f - e.fz);
            t.wa = make_float4(w[0], w[1], w[2], w[3]);
            t.wb = make_float4(w[4], w[5], w[6], w[7]);
            t.pad = 0;
        }
        LVR_CUDA(ctx, cudaFuncSetAttribute(ao_field_pair_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)pair_bytes));
        const dim3 grid((dm[0] + AOP_X - 1) / AOP_X, (dm[1] + AOP_Y - 1) / AOP_Y, (dm[2] + AOP_Z - 1) / AOP_Z);
        ao_field_pair_kernel<5><<<grid, AOP_X / 2 * AOP_Y * AOP_Z, pair_bytes, ctx->stream>>>(
            lod->dens[0], dm[0], dm[1], dm[2], taps, rays, H, lod->aof);
    } else {
        const unsigned g = grid1d(n, 256) > 65535 ? 65535 : grid1d(n, 256);
        ao_field_kernel<<<g, 256, 0, ctx->stream>>>(lod->pk0[0], lod->pstride[0][0], lod->pstride[0][1], dm[0], dm[1],
                                                    dm[2], (const AoStep *)ctx->stage_in,
                                                   rays, steps, lod->aof);
    }
    LVR_CUDA(ctx, cudaGetLastError());
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // the table lives in host memory until copied
    return LVR_OK;
}

extern "C" lvr_status lvr_export_ao_field(lvr_ctx *ctx, const lvr_lod *lod, float *field) {
    if (!ctx) return LVR_EINVAL;
    if (!lod || !lod->aof || !field) return set_err(ctx, LVR_EINVAL, "no spherical AO field");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t n = (size_t)lod->dims[0][0] * lod->dims[0][1] * lod->dims[0][2];
    return copy_out(ctx, field, lod->aof, n * 4);
}

// A LoD handle with its level arrays and padded sampling copies allocated
// (contents undefined): dims of level l = ceil(dims0 / 2^l).
lvr_status lod_alloc(lvr_ctx *ctx, int levels, const int32_t dims0[3], lvr_lod **out) {
    static uint64_t next_gen = 0;
    lvr_lod *L = new lvr_lod();
    L->ctx = ctx;
    L->gen = __atomic_add_fetch(&next_gen, 1, __ATOMIC_RELAXED);
    L->levels = levels;
    lvr_status st = LVR_OK;
    for (int l = 0; l < levels && st == LVR_OK; l++) {
        for (int a = 0; a < 3; a++) L->dims[l][a] = l == 0 ? dims0[a] : (L->dims[l - 1][a] + 1) / 2;
        const size_t n = (size_t)L->dims[l][0] * L->dims[l][1] * L->dims[l][2];
        if ((st = dev_alloc(ctx, (void **)&L->cnt[l], n * 4)) != LVR_OK) break;
        if ((st = dev_alloc(ctx, (void **)&L->len[l], n * 4)) != LVR_OK) break;
        st = dev_alloc(ctx, (void **)&L->dens[l], n * 4);
    }
    // padding of the sampling copies: the support of the density field is
    // [-c/2, (top + 1/2) c] per axis in level-0 units (c = 2^(levels-1), top =
    // the coarsest level's dims); at level l its sample points fall in cells
    // floor(x / 2^l - 1/2), whose corners reach one cell further
    for (int l = 0; l < levels && st == LVR_OK; l++) {
        const double m = ldexp(1.0, levels - 1 - l);
        L->pad_lo[l] = -(int)floor(-0.5 * m - 0.5);
        int64_t pd[3];
        // with 3 levels the coarsest copy also holds every point within 13
        // voxels of the grid: the AO march of radius 12 then needs no support
        // test (its samples there read zeros)
        const bool reach = levels == 3 && l == 2;
        if (reach) L->pad_lo[l] = std::max(L->pad_lo[l], -(int)floor(-13.0 / 4.0 - 0.5));
        for (int a = 0; a < 3; a++) {
            int64_t hi = (int64_t)floor(((double)L->dims[levels - 1][a] + 0.5) * m - 0.5) + 1;
            if (reach) hi = std::max(hi, (int64_t)floor(((double)dims0[a] + 13.0) / 4.0 - 0.5));
            L->pad_hi[l][a] = (int32_t)(hi - (L->dims[l][a] - 1));
            pd[a] = (int64_t)L->dims[l][a] + L->pad_lo[l] + L->pad_hi[l][a];
        }
        L->pstride[l][0] = pd[0];
        L->pstride[l][1] = pd[0] * pd[1];
        const int64_t ncell = pd[0] * pd[1] * pd[2];
        if (ncell >= ((int64_t)1 << 32) - 1) {
            st = set_err(ctx, LVR_EINVAL, "LoD: a padded level must have fewer than 2^32 - 1 cells");
            break;
        }
        L->pzero[l] = (uint32_t)ncell;
        st = dev_alloc(ctx, (void **)&L->pk[l], (size_t)(ncell + 1) * 32);
        if (st == LVR_OK) {
            const int64_t c0 = L->pad_lo[l] * (1 + L->pstride[l][0] + L->pstride[l][1]);
            L->pk0[l] = L->pk[l] + 2 * c0;
            L->pbias[l] = (uint32_t)((0x4B400000u - (uint32_t)L->pad_lo[l]) *
                                     (uint32_t)(1 + L->pstride[l][0] + L->pstride[l][1]));
        }
    }
    if (st != LVR_OK) {
        lvr_free_lod(L);
        return st;
    }
    *out = L;
    return LVR_OK;
}

// The corner-packed sampling copy of every level from its densities.
lvr_status lod_pack(lvr_ctx *ctx, lvr_lod *L) {
    for (int l = 0; l < L->levels; l++) {
        const int32_t *dm = L->dims[l];
        const int lo = L->pad_lo[l];
        const int px = dm[0] + lo + L->pad_hi[l][0], py = dm[1] + lo + L->pad_hi[l][1], pz = dm[2] + lo + L->pad_hi[l][2];
        const int64_t np = (int64_t)px * py * pz;
        const unsigned g = grid1d(np, 256) > 65535 ? 65535 : grid1d(np, 256);
        lod_pack_kernel<<<g, 256, 0, ctx->stream>>>(L->dens[l], dm[0], dm[1], dm[2], lo, px, py, pz, L->pk[l]);
        LVR_CUDA(ctx, cudaMemsetAsync(L->pk[l] + 2 * (size_t)np, 0, 32, ctx->stream));   // the zero cell
    }
    LVR_CUDA(ctx, cudaGetLastError());
    return LVR_OK;
}

extern "C" lvr_status lvr_build_lod(lvr_ctx *ctx, const lvr_lineset *ls, int levels,
                                    const float *sigma256, lvr_lod **out) {
    if (!ctx) return LVR_EINVAL;
    if (!ls || !out || !sigma256) return set_err(ctx, LVR_EINVAL, "lvr_build_lod: null argument");
    *out = nullptr;
    if (levels < 1 || levels > 4) return set_err(ctx, LVR_EINVAL, "levels must be in [1,4]");
    for (int i = 0; i < 256; i++)
        if (!(sigma256[i] >= 0.0f) || !(sigma256[i] < 1e30f))
            return set_err(ctx, LVR_EINVAL, "sigma must be finite and >= 0");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    lvr_lod *L = nullptr;
    lvr_status st = lod_alloc(ctx, levels, ls->res, &L);
    if (st == LVR_OK) st = ensure_stage_in(ctx, 1024);
    if (st != LVR_OK) {
        lvr_free_lod(L);
        return st;
    }
    float *dsig = (float *)ctx->stage_in;
    cudaError_t e = cudaMemcpyAsync(dsig, sigma256, 1024, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        lod_level0_kernel<<<grid1d(ls->nvox, 256), 256, 0, s>>>(ls->offset, ls->rec, ls->nvox, ls->bins,
                                                                 dsig, L->cnt[0], L->len[0], L->dens[0]);
        for (int l = 1; l < levels; l++) {
            const int32_t *c = L->dims[l - 1], *p = L->dims[l];
            const int64_t np = (int64_t)p[0] * p[1] * p[2];
            lod_pool_kernel<<<grid1d(np, 256), 256, 0, s>>>(c[0], c[1], c[2], L->cnt[l - 1], L->len[l - 1],
                                                             L->dens[l - 1], p[0], p[1], p[2], L->cnt[l],
                                                             L->len[l], L->dens[l]);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        st = lod_pack(ctx, L);
    } else {
        st = cuda_err(ctx, e, "lvr_build_lod");
    }
    if (st != LVR_OK) {
        lvr_free_lod(L);
        return st;
    }
    *out = L;
    return LVR_OK;
}

extern "C" lvr_status lvr_lod_info_get(const lvr_lod *lod, lvr_lod_info *info) {
    if (!lod || !info) return LVR_EINVAL;
    info->levels = lod->levels;
    for (int l = 0; l < 4; l++)
        for (int a = 0; a < 3; a++) info->dims[l][a] = l < lod->levels ? lod->dims[l][a] : 0;
    return LVR_OK;
}

extern "C" lvr_status lvr_export_lod(lvr_ctx *ctx, const lvr_lod *lod, int level, uint32_t *cnt,
                                     float *len, float *dens) {
    if (!ctx) return LVR_EINVAL;
    if (!lod || level < 0 || level >= lod->levels) return set_err(ctx, LVR_EINVAL, "bad LoD level");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t n = (size_t)lod->dims[level][0] * lod->dims[level][1] * lod->dims[level][2];
    lvr_status st = copy_out(ctx, cnt, lod->cnt[level], n * 4);
    if (st == LVR_OK) st = copy_out(ctx, len, lod->len[level], n * 4);
    if (st == LVR_OK) st = copy_out(ctx, dens, lod->dens[level], n * 4);
    return st;
}

extern "C" void lvr_free_lod(lvr_lod *lod) {
    if (!lod) return;
    cudaSetDevice(lod->ctx->device);
    for (int l = 0; l < 4; l++) {
        dev_free(lod->ctx, lod->cnt[l]);
        dev_free(lod->ctx, lod->len[l]);
        dev_free(lod->ctx, lod->dens[l]);
        dev_free(lod->ctx, lod->pk[l]);
    }
    dev_free(lod->ctx, lod->aof);
    for (int l = 0; l < 4; l++) dev_free(lod->ctx, lod->rep[l]);
    delete lod;
}
