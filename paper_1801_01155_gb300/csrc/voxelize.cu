// Device voxeliser: curve clipping, face-point quantisation and the compact
// per-voxel segment store (Secs. 3.1-3.3).
//
// The paper builds the store on the GPU in three stages: curves write their
// per-voxel segments to an append buffer tagged with voxel ids, the buffer
// is sorted by voxel id, and an exclusive prefix sum gives each voxel's
// start index (Sec. 3.3). Here the same store is built without a global
// sort: one warp per curve (its edges on the lanes) counts its segments per
// voxel (atomics), an exclusive scan turns the counts into the offset table,
// a second pass scatters the packed records to their voxel's range, and a
// short per-voxel sort by (curve, ordinal) makes every list's order
// canonical.
//
// Every decision is exact integer arithmetic on the fixed-point vertices:
// plane crossings are ordered by their rational edge parameter t = n / d
// (compared by 64-bit cross products), bins are floor(N * position) computed
// as one integer division, and attribute interpolation uses floor division.
#include <float.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "lvr_internal.cuh"

namespace {

constexpr int FXS = 16;                 // fixed point: 2^16 units per voxel
constexpr int64_t FX = 1 << FXS;
constexpr int SMALL_LIST = 16;          // lists up to this length: sorted in one thread
constexpr int SMEM_LIST = 2048;         // lists up to this length: sorted in shared memory

struct VoxParams {
    const float *xyz;
    const float *attr;                  // nullptr: all attribute codes 0
    const int64_t *offs;
    int64_t nc, nv;
    float o[3], s;
    float amin, aspan;
    int32_t res[3];
    int32_t N;
    uint32_t *status;
};

// World -> grid fixed point: p = fl32(fl32(v - o) * s), X = rint_even(p * 2^16).
__device__ __forceinline__ bool load_vertex(const VoxParams &P, int64_t i, int64_t X[3], int64_t &A) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        float d = __fsub_rn(__ldg(P.xyz + 3 * i + a), P.o[a]);
        float p = __fmul_rn(d, P.s);
        if (!(fabsf(p) < 16384.0f)) {
            ok = false;
            p = 0.0f;
        }
        X[a] = (int64_t)__float2int_rn(__fmul_rn(p, 65536.0f));
    }
    A = 0;
    if (P.attr) {
        float a = __ldg(P.attr + i);
        if (!isfinite(a)) {
            atomicOr(P.status, ST_BAD_ATTR);
        } else {
            float q = __fdiv_rn(__fsub_rn(a, P.amin), P.aspan);
            q = fminf(fmaxf(q, 0.0f), 1.0f);
            A = (int64_t)__float2int_rn(__fmul_rn(q, 65535.0f));
        }
    }
    return ok;
}

// floor(num / den) for 0 <= num < 2^62, 0 < den, quotient below 2^24: a
// float32 estimate (relative error < 2^-22, so off by at most one) corrected
// with exact 64-bit products. Replaces a 64-bit division routine.
__device__ __forceinline__ int64_t udiv_small(int64_t num, int64_t den) {
    int64_t q = (int64_t)floorf(__fdividef((float)num, (float)den));
    if (q < 0) q = 0;
    while (q > 0 && q * den > num) q--;
    while ((q + 1) * den <= num) q++;
    return q;
}

__device__ __forceinline__ int64_t floor_div(int64_t a, int64_t b) {   // b > 0, |a / b| < 2^24
    return a >= 0 ? udiv_small(a, b) : -udiv_small(b - 1 - a, b);
}

// Bin of the face point on an axis b whose coordinate is X0b + Db * n / d,
// relative to voxel index vb: floor(N * rem / FX), clamped to N - 1.
__device__ __forceinline__ uint32_t face_bin(int64_t X0b, int64_t Db, int64_t vb, int64_t n,
                                             int64_t d, int N, uint32_t *status) {
    int64_t rem_d = (X0b - vb * FX) * d + n * Db;
    int64_t lim = FX * d;
    if (rem_d < 0 || rem_d > lim) {
        atomicOr(status, ST_INTERNAL);
        rem_d = rem_d < 0 ? 0 : lim;
    }
    int64_t b = udiv_small((int64_t)N * rem_d, lim);
    return (uint32_t)(b > N - 1 ? N - 1 : b);
}

// One warp per curve, its edges spread over the lanes 32 at a time. Each
// lane takes one edge (v_e, v_e+1): how many planes it crosses and its last
// crossing (face point, attribute, the voxel before it) follow in closed
// form; a warp scan numbers the crossings along the curve, each lane learns
// the crossing before its first one from the nearest lower lane with one
// (or from the previous window), and then walks its edge's crossings in the
// sequential order (earliest first, ties x, y, z), emitting the segment
// that ends at each. The voxel at the start of an edge is floor(v_e) on every
// axis (the sequential walk's state there), so the result is the same
// segment sequence, ordinals and flags as one thread walking the curve.
// COUNT: per-voxel segment counts and the total stored. SCATTER: each
// segment goes into its voxel's range at an atomic cursor, as one 32-byte
// slot holding the (record, key) pair when `pair` is given (one whole sector
// per scattered segment, written by one store: the cache never fills a
// partly written sector from DRAM; the sort then writes the arrays), else
// into rec / key directly.
// The scatter target of one segment: its record and key in the first half of
// a 32-byte sector.
struct __align__(32) PairSlot {
    unsigned long long r, k, pad0, pad1;
};
__device__ __forceinline__ void store_slot(PairSlot *p, uint64_t r, uint64_t k) {
    // streaming store (read once, by the sort): it should not push the cursors out of L2
    asm volatile("st.global.cs.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"((uint32_t)r),
                 "r"((uint32_t)(r >> 32)), "r"((uint32_t)k), "r"((uint32_t)(k >> 32)), "r"(0u), "r"(0u), "r"(0u),
                 "r"(0u)
                 : "memory");
}

template <bool SCATTER>
__global__ void __launch_bounds__(256)
vox_warp_kernel(VoxParams P, uint32_t *cnt, const uint32_t *__restrict__ offset, uint64_t *__restrict__ rec,
                uint64_t *__restrict__ key, PairSlot *__restrict__ pair, unsigned long long *total) {
    const unsigned FULLM = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int N = P.N;
    unsigned long long nstored_all = 0;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < P.nc; c += nwarps) {
        const int64_t v0 = P.offs[c], v1 = P.offs[c + 1];
        if (!SCATTER) {
            bool bad = v0 < 0 || v1 < v0 || v1 > P.nv;
            if (c == 0 && v0 != 0) bad = true;
            if (c == P.nc - 1 && v1 != P.nv) bad = true;
            if (bad) {
                if (lane == 0) atomicOr(P.status, ST_BAD_OFFSETS);
                continue;
            }
        }
        if (v1 - v0 < 2) {
            if (!SCATTER && v1 - v0 == 1 && lane == 0) {
                int64_t X[3], A;
                if (!load_vertex(P, v0, X, A)) atomicOr(P.status, ST_BAD_VERTEX);
            }
            continue;
        }
        // carried along the curve: crossings so far, the last one as the next segment's entry point
        int64_t ncross = 0;
        uint32_t cf = 0, cu = 0, cv = 0;
        int64_t cA = 0;
        bool cstored = false;          // the segment ending at the last crossing was stored
        bool bad_vertex = false;
        for (int64_t base = v0; base + 1 < v1; base += 32) {
            const int64_t e = base + lane;
            const bool has_edge = e + 1 < v1;
            int64_t X0[3] = {0, 0, 0}, X1[3] = {0, 0, 0}, A0 = 0, A1 = 0;
            if (has_edge) {
                bad_vertex |= !load_vertex(P, e, X0, A0);
                bad_vertex |= !load_vertex(P, e + 1, X1, A1);
            }
            int64_t D[3], den[3], nextp[3], lastp[3];
            bool act[3];
            int m = 0;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                D[a] = X1[a] - X0[a];
                const int64_t f0 = X0[a] >> FXS, f1 = X1[a] >> FXS;
                if (D[a] > 0) {
                    nextp[a] = f0 + 1; lastp[a] = f1; den[a] = D[a]; act[a] = nextp[a] <= lastp[a];
                    if (act[a]) m += (int)(lastp[a] - nextp[a] + 1);
                } else if (D[a] < 0) {
                    nextp[a] = f0; lastp[a] = f1 + 1; den[a] = -D[a]; act[a] = nextp[a] >= lastp[a];
                    if (act[a]) m += (int)(nextp[a] - lastp[a] + 1);
                } else {
                    nextp[a] = lastp[a] = 0; den[a] = 1; act[a] = false;
                }
            }
            if (!has_edge) m = 0;
            // the edge's last crossing: the latest plane, ties to the higher axis (crossed last)
            uint32_t lf = 0, lu = 0, lv = 0;
            int64_t lA = 0;
            bool lin = false;              // the voxel before it lies in the grid
            if (m > 0) {
                int ax = -1;
                int64_t bn = 0, bd = 1;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    if (!act[a]) continue;
                    const int64_t n = D[a] > 0 ? lastp[a] * FX - X0[a] : X0[a] - lastp[a] * FX;
                    if (ax < 0 || n * bd >= bn * den[a]) { ax = a; bn = n; bd = den[a]; }
                }
                const bool pos = D[ax] > 0;
                int64_t before[3] = {X1[0] >> FXS, X1[1] >> FXS, X1[2] >> FXS};
                before[ax] -= pos ? 1 : -1;
                lin = before[0] >= 0 && before[0] < P.res[0] && before[1] >= 0 && before[1] < P.res[1] &&
                      before[2] >= 0 && before[2] < P.res[2];
                lf = 2u * ax + (pos ? 0u : 1u);   // entry face of the next segment
                if (SCATTER) {
                    const int b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
                    lu = face_bin(X0[b0], D[b0], before[b0], bn, bd, N, P.status);
                    lv = face_bin(X0[b1], D[b1], before[b1], bn, bd, N, P.status);
                    lA = A0 + floor_div((A1 - A0) * bn, bd);
                }
            }
            int incl = m;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULLM, incl, o);
                if (lane >= o) incl += y;
            }
            const int wtotal = __shfl_sync(FULLM, incl, 31);
            const int64_t first = ncross + (incl - m);          // index of my first crossing on the curve
            // the crossing before my first one: nearest lower lane with crossings, else the carry
            const unsigned has = __ballot_sync(FULLM, m > 0);
            const unsigned lower = has & ((1u << lane) - 1u);
            const int src = lower ? 31 - __clz(lower) : lane;
            uint32_t pf = __shfl_sync(FULLM, lf, src), pu = __shfl_sync(FULLM, lu, src),
                     pv = __shfl_sync(FULLM, lv, src);
            int64_t pA = __shfl_sync(FULLM, lA, src);
            const int src_incl = __shfl_sync(FULLM, incl, src);
            bool prev_stored = __shfl_sync(FULLM, lin ? 1 : 0, src) != 0;
            if (lower) {
                // the segment ending at src's last crossing exists iff that crossing is not the curve's first
                prev_stored = prev_stored && ncross + src_incl - 1 >= 1;
            } else {
                pf = cf; pu = cu; pv = cv; pA = cA;
                prev_stored = cstored;
            }
            // walk my crossings in order, emitting the segment that ends at each
            if (m > 0) {
                int64_t cur[3] = {X0[0] >> FXS, X0[1] >> FXS, X0[2] >> FXS};
                int64_t j = first;
                for (;;) {
                    int ax = -1;
                    int64_t bn = 0, bd = 1;
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        if (!act[a]) continue;
                        const int64_t n = D[a] > 0 ? nextp[a] * FX - X0[a] : X0[a] - nextp[a] * FX;
                        if (ax < 0 || n * bd < bn * den[a]) { ax = a; bn = n; bd = den[a]; }
                    }
                    if (ax < 0) break;
                    const int b0 = ax == 0 ? 1 : 0, b1 = ax == 2 ? 1 : 2;
                    const bool pos = D[ax] > 0;
                    const uint32_t hf = 2u * ax + (pos ? 1u : 0u);
                    uint32_t hu = 0, hv = 0;
                    int64_t hA = 0;
                    if (SCATTER) {
                        hu = face_bin(X0[b0], D[b0], cur[b0], bn, bd, N, P.status);
                        hv = face_bin(X0[b1], D[b1], cur[b1], bn, bd, N, P.status);
                        hA = A0 + floor_div((A1 - A0) * bn, bd);
                    }
                    bool st = false;
                    if (j >= 1) {
                        st = cur[0] >= 0 && cur[0] < P.res[0] && cur[1] >= 0 && cur[1] < P.res[1] && cur[2] >= 0 &&
                             cur[2] < P.res[2];
                        if (st) {
                            const uint32_t vox =
                                (uint32_t)(cur[0] + (int64_t)P.res[0] * (cur[1] + (int64_t)P.res[1] * cur[2]));
                            if (SCATTER) {
                                // with `pair`, cnt holds the cursors (the offsets to begin with)
                                const uint32_t at = pair ? atomicAdd(cnt + vox, 1u) : offset[vox] + atomicAdd(cnt + vox, 1u);
                                const uint32_t attr8 = (uint32_t)(((pA + hA) * 255 + 65535) / 131070);
                                const uint64_t r =
                                    rec_pack(pf, pu, pv, hf, hu, hv, attr8, prev_stored ? 1u : 0u, (uint32_t)c);
                                const uint64_t kk = ((uint64_t)c << 32) | (uint64_t)(j - 1);
                                if (pair) {
                                    store_slot(pair + at, r, kk);
                                } else {
                                    rec[at] = r;
                                    key[at] = kk;
                                }
                            } else {
                                atomicAdd(cnt + vox, 1u);
                            }
                            nstored_all++;
                        }
                    }
                    prev_stored = st;
                    cur[ax] += pos ? 1 : -1;
                    pf = 2u * ax + (pos ? 0u : 1u);
                    pu = hu;
                    pv = hv;
                    pA = hA;
                    j++;
                    if (pos) { nextp[ax]++; act[ax] = nextp[ax] <= lastp[ax]; }
                    else     { nextp[ax]--; act[ax] = nextp[ax] >= lastp[ax]; }
                }
            }
            // carry: the window's last crossing
            if (has) {
                const int top = 31 - __clz(has);
                cf = __shfl_sync(FULLM, lf, top);
                cu = __shfl_sync(FULLM, lu, top);
                cv = __shfl_sync(FULLM, lv, top);
                cA = __shfl_sync(FULLM, lA, top);
                const bool tl = __shfl_sync(FULLM, lin ? 1 : 0, top) != 0;
                cstored = tl && ncross + wtotal - 1 >= 1;
            } else {
                // no crossing in this window: keep the carry (the shuffles above kept every lane converged)
            }
            ncross += wtotal;
        }
        if (__any_sync(FULLM, bad_vertex) && lane == 0) atomicOr(P.status, ST_BAD_VERTEX);
    }
    if (!SCATTER) {
        for (int o = 16; o > 0; o >>= 1) nstored_all += __shfl_xor_sync(0xffffffffu, nstored_all, o);
        if (lane == 0 && nstored_all) atomicAdd(total, nstored_all);
    }
}

// ------------------------------------------------------------------ bounding box (fit mode)
__device__ __forceinline__ int f2ord(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__global__ void bbox_kernel(const float *__restrict__ xyz, int64_t nv, int *mn, int *mx,
                            uint32_t *status) {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            float v = xyz[3 * i + a];
            if (!isfinite(v)) bad = true;
            else { lo[a] = fminf(lo[a], v); hi[a] = fmaxf(hi[a], v); }
        }
    }
    if (bad) atomicOr(status, ST_BAD_VERTEX);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        for (int s = 16; s > 0; s >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], s));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], s));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(mn + a, f2ord(lo[a]));
            atomicMax(mx + a, f2ord(hi[a]));
        }
    }
}

// ------------------------------------------------------------------ exclusive scan
// Reduce-then-scan over tiles of 4096 counts (256 threads x 16): tile sums,
// a one-block scan of the tile sums, then a tile-local scan plus the prefix.
constexpr int SCAN_T = 256, SCAN_I = 16, SCAN_TILE = SCAN_T * SCAN_I;

__global__ void __launch_bounds__(SCAN_T)
scan_reduce_kernel(const uint32_t *__restrict__ cnt, int64_t n, unsigned long long *tile_sum) {
    const int64_t base = blockIdx.x * (int64_t)SCAN_TILE + threadIdx.x * SCAN_I;
    unsigned long long s = 0;
    if (base + SCAN_I <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(cnt + base);
#pragma unroll
        for (int q = 0; q < SCAN_I / 4; q++) {
            uint4 v = __ldg(p + q);
            s += (unsigned long long)v.x + v.y + v.z + v.w;
        }
    } else {
        for (int q = 0; q < SCAN_I; q++)
            if (base + q < n) s += cnt[base + q];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ unsigned long long ws[SCAN_T / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < SCAN_T / 32; w++) t += ws[w];
        tile_sum[blockIdx.x] = t;
    }
}

// One block: exclusive scan of the tile sums in chunks of 1024, total checked.
__global__ void __launch_bounds__(1024)
scan_tiles_kernel(unsigned long long *tile_sum, int64_t ntiles, uint32_t *offset_end, uint32_t *status) {
    __shared__ unsigned long long ws[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < ntiles; c0 += 1024) {
        const int64_t i = c0 + threadIdx.x;
        unsigned long long v = i < ntiles ? tile_sum[i] : 0ull, x = v;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long w = ws[threadIdx.x], z = w;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, z, o);
                if (threadIdx.x >= o) z += y;
            }
            ws[threadIdx.x] = z - w;            // exclusive warp prefix
        }
        __syncthreads();
        const unsigned long long excl = carry + ws[threadIdx.x >> 5] + x - v;
        if (i < ntiles) tile_sum[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (carry > 0xffffffffull) atomicOr(status, ST_OVERFLOW);
        *offset_end = (uint32_t)carry;
    }
}

__global__ void __launch_bounds__(SCAN_T)
scan_down_kernel(const uint32_t *__restrict__ cnt, int64_t n,
                 const unsigned long long *__restrict__ tile_prefix, uint32_t *__restrict__ offset) {
    const int64_t base = blockIdx.x * (int64_t)SCAN_TILE + threadIdx.x * SCAN_I;
    uint32_t v[SCAN_I];
    const bool full = base + SCAN_I <= n;
    if (full) {
        const uint4 *p = reinterpret_cast<const uint4 *>(cnt + base);
#pragma unroll
        for (int q = 0; q < SCAN_I / 4; q++) {
            uint4 w = __ldg(p + q);
            v[4 * q] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < SCAN_I; q++) v[q] = base + q < n ? cnt[base + q] : 0u;
    }
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_I; q++) s += v[q];
    uint32_t x = s;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) >= o) x += y;
    }
    __shared__ uint32_t ws[SCAN_T / 32];
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w = threadIdx.x < SCAN_T / 32 ? ws[threadIdx.x] : 0u, z = w;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (threadIdx.x >= o) z += y;
        }
        if (threadIdx.x < SCAN_T / 32) ws[threadIdx.x] = z - w;
    }
    __syncthreads();
    uint32_t run = (uint32_t)tile_prefix[blockIdx.x] + ws[threadIdx.x >> 5] + x - s;
    if (full) {
        uint4 *p = reinterpret_cast<uint4 *>(offset + base);
#pragma unroll
        for (int q = 0; q < SCAN_I / 4; q++) {
            uint4 w;
            w.x = run; run += v[4 * q];
            w.y = run; run += v[4 * q + 1];
            w.z = run; run += v[4 * q + 2];
            w.w = run; run += v[4 * q + 3];
            p[q] = w;
        }
    } else {
        for (int q = 0; q < SCAN_I; q++) {
            if (base + q < n) offset[base + q] = run;
            run += v[q];
        }
    }
}

// ------------------------------------------------------------------ canonical per-voxel order
// With `pair`, the scattered (record, key) pairs are read from there and
// every list is written to rec / key; without, lists are sorted in place.
__global__ void __launch_bounds__(256)
sort_small_kernel(const uint32_t *__restrict__ offset, int64_t nvox, uint64_t *rec, uint64_t *key,
                  const PairSlot *__restrict__ pair, uint32_t *long_list, uint32_t *long_count) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const uint32_t beg = offset[v], n = offset[v + 1] - beg;
    if (n == 0 || (n == 1 && !pair)) return;
    if (n > SMALL_LIST) {
        long_list[atomicAdd(long_count, 1u)] = (uint32_t)v;
        return;
    }
    uint64_t k[SMALL_LIST], r[SMALL_LIST];
    for (uint32_t i = 0; i < n; i++) {
        uint64_t kk, rr;
        if (pair) {
            rr = pair[beg + i].r;
            kk = pair[beg + i].k;
        } else {
            kk = key[beg + i];
            rr = rec[beg + i];
        }
        int j = (int)i - 1;
        while (j >= 0 && k[j] > kk) {
            k[j + 1] = k[j];
            r[j + 1] = r[j];
            j--;
        }
        k[j + 1] = kk;
        r[j + 1] = rr;
    }
    for (uint32_t i = 0; i < n; i++) {
        key[beg + i] = k[i];
        rec[beg + i] = r[i];
    }
}

// Ascending bitonic network in its "flip" form: every comparator puts the
// minimum at the lower index, so indices >= n act as +infinity padding and
// their comparators can be skipped.
template <class GetK, class Swap>
__device__ void bitonic_block(uint32_t n, GetK getk, Swap swp) {
    uint32_t P = 1;
    while (P < n) P <<= 1;
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
            const uint32_t half = k >> 1, blk = t / half, off = t % half;
            const uint32_t lo = blk * k + off, hi = blk * k + k - 1 - off;
            if (hi < n && getk(lo) > getk(hi)) swp(lo, hi);
        }
        __syncthreads();
        for (uint32_t j = k >> 2; j > 0; j >>= 1) {
            for (uint32_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const uint32_t blk = t / j, off = t % j;
                const uint32_t lo = blk * 2 * j + off, hi = lo + j;
                if (hi < n && getk(lo) > getk(hi)) swp(lo, hi);
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256)
sort_long_kernel(const uint32_t *__restrict__ offset, uint64_t *rec, uint64_t *key,
                 const PairSlot *__restrict__ pair, const uint32_t *__restrict__ long_list,
                 const uint32_t *__restrict__ long_count) {
    extern __shared__ uint64_t sm[];
    uint64_t *sk = sm, *sr = sm + SMEM_LIST;
    const uint32_t nl = *long_count;
    for (uint32_t li = blockIdx.x; li < nl; li += gridDim.x) {
        const uint32_t v = long_list[li];
        const uint32_t beg = offset[v], n = offset[v + 1] - beg;
        uint64_t *gk = key + beg, *gr = rec + beg;
        if (pair && n > SMEM_LIST) {   // sorted in place in the final arrays
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                gr[i] = pair[beg + i].r;
                gk[i] = pair[beg + i].k;
            }
            __syncthreads();
        }
        if (n <= SMEM_LIST) {
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                if (pair) {
                    sr[i] = pair[beg + i].r;
                    sk[i] = pair[beg + i].k;
                } else {
                    sk[i] = gk[i];
                    sr[i] = gr[i];
                }
            }
            __syncthreads();
            bitonic_block(n, [&](uint32_t i) { return sk[i]; },
                          [&](uint32_t a, uint32_t b) {
                              uint64_t t = sk[a]; sk[a] = sk[b]; sk[b] = t;
                              t = sr[a]; sr[a] = sr[b]; sr[b] = t;
                          });
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                gk[i] = sk[i];
                gr[i] = sr[i];
            }
        } else {
            bitonic_block(n, [&](uint32_t i) { return gk[i]; },
                          [&](uint32_t a, uint32_t b) {
                              uint64_t t = gk[a]; gk[a] = gk[b]; gk[b] = t;
                              t = gr[a]; gr[a] = gr[b]; gr[b] = t;
                          });
        }
        __syncthreads();
    }
}

bool valid_bins(int n) { return n >= 2 && n <= 128 && (n & (n - 1)) == 0; }

}  // namespace

int64_t scan_tile_count(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE; }

void scan_counts(cudaStream_t s, const uint32_t *cnt, int64_t n, unsigned long long *tiles, uint32_t *offset,
                 uint32_t *status) {
    const int64_t ntiles = scan_tile_count(n);
    scan_reduce_kernel<<<(unsigned)ntiles, SCAN_T, 0, s>>>(cnt, n, tiles);
    scan_tiles_kernel<<<1, 1024, 0, s>>>(tiles, ntiles, offset + n, status);
    scan_down_kernel<<<(unsigned)ntiles, SCAN_T, 0, s>>>(cnt, n, tiles, offset);
}

extern "C" lvr_status lvr_voxelize(lvr_ctx *ctx, const float *xyz, const float *attr,
                                   const int64_t *curve_offsets, int64_t n_curves,
                                   int64_t n_vertices, lvr_grid_desc *g, lvr_lineset **out) {
    if (!ctx) return LVR_EINVAL;
    if (!out || !g) return set_err(ctx, LVR_EINVAL, "lvr_voxelize: null argument");
    *out = nullptr;
    if (n_curves < 0 || n_vertices < 0) return set_err(ctx, LVR_EINVAL, "negative sizes");
    if (n_curves > 0xffffffffLL) return set_err(ctx, LVR_EINVAL, "more than 2^32 curves");
    if (n_vertices > 0 && !xyz) return set_err(ctx, LVR_EINVAL, "xyz is null");
    if (!curve_offsets) return set_err(ctx, LVR_EINVAL, "curve_offsets is null");
    if (n_curves == 0 && n_vertices != 0) return set_err(ctx, LVR_EINVAL, "vertices without curves");
    if (!valid_bins(g->bins)) return set_err(ctx, LVR_EINVAL, "bins must be a power of two in [2,128]");
    if (g->fit && (g->res[0] < 1 || g->res[0] > 4096))
        return set_err(ctx, LVR_EINVAL, "fit: res[0] must be in [1,4096]");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;

    // stage host inputs: xyz | attr | offsets, 256-byte aligned slots
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t bx = (size_t)n_vertices * 12, ba = attr ? (size_t)n_vertices * 4 : 0,
                 bo = (size_t)(n_curves + 1) * 8;
    lvr_status st = LVR_OK;
    const bool hx = n_vertices > 0 && !is_device_ptr(xyz), ha = attr && !is_device_ptr(attr),
               ho = !is_device_ptr(curve_offsets);
    if (hx || ha || ho) {
        st = ensure_stage_in(ctx, al(bx) + al(ba) + al(bo));
        if (st != LVR_OK) return st;
    }
    const void *dx = xyz, *da = attr, *dof = curve_offsets;
    if ((st = stage_input(ctx, xyz, bx, 0, &dx)) != LVR_OK) return st;
    if ((st = stage_input(ctx, attr, ba, al(bx), &da)) != LVR_OK) return st;
    if ((st = stage_input(ctx, curve_offsets, bo, al(bx) + al(ba), &dof)) != LVR_OK) return st;

    LVR_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, 4, s));
    uint32_t *h32 = (uint32_t *)ctx->h_pinned;
    unsigned long long *h64 = (unsigned long long *)((char *)ctx->h_pinned + 64);

    if (g->fit) {   // bounding box -> origin, scale, res keeping the aspect ratio (Sec. 3.1)
        if (n_vertices == 0) return set_err(ctx, LVR_EINVAL, "fit: no vertices");
        int init[6] = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000, (int)0x80000000};
        LVR_CUDA(ctx, cudaMemcpyAsync(ctx->d_u64, init, sizeof init, cudaMemcpyHostToDevice, s));
        int *mn = (int *)ctx->d_u64, *mx = mn + 3;
        bbox_kernel<<<grid1d(n_vertices, 256) > 1024 ? 1024 : grid1d(n_vertices, 256), 256, 0, s>>>(
            (const float *)dx, n_vertices, mn, mx, ctx->d_status);
        LVR_CUDA(ctx, cudaGetLastError());
        int hb[6];
        LVR_CUDA(ctx, cudaMemcpyAsync(hb, ctx->d_u64, sizeof hb, cudaMemcpyDeviceToHost, s));
        LVR_CUDA(ctx, cudaMemcpyAsync(h32, ctx->d_status, 4, cudaMemcpyDeviceToHost, s));
        LVR_CUDA(ctx, cudaStreamSynchronize(s));
        if (*h32) return set_err(ctx, LVR_EINVAL, "fit: vertex not finite");
        float lo[3], hi[3];
        double ext[3], emax = 0.0;
        for (int a = 0; a < 3; a++) {
            int l = hb[a], h = hb[3 + a];
            l = l >= 0 ? l : l ^ 0x7fffffff;
            h = h >= 0 ? h : h ^ 0x7fffffff;
            memcpy(&lo[a], &l, 4);
            memcpy(&hi[a], &h, 4);
            ext[a] = (double)hi[a] - (double)lo[a];
            emax = ext[a] > emax ? ext[a] : emax;
        }
        if (!(emax > 0.0)) return set_err(ctx, LVR_EINVAL, "fit: degenerate bounding box");
        const int rmax = g->res[0];
        for (int a = 0; a < 3; a++) {
            double r = ceil(ext[a] * (double)rmax / emax);
            g->res[a] = r < 1.0 ? 1 : (int32_t)r;
            g->origin[a] = lo[a];
        }
        g->scale = (float)((double)rmax / emax);
    }
    for (int a = 0; a < 3; a++)
        if (g->res[a] < 1 || g->res[a] > 4096) return set_err(ctx, LVR_EINVAL, "res out of [1,4096]");
    if (!(g->scale > 0.0f) || !isfinite(g->scale)) return set_err(ctx, LVR_EINVAL, "scale must be > 0");
    const int64_t nvox = (int64_t)g->res[0] * g->res[1] * g->res[2];
    if (nvox >= 0xffffffffLL) return set_err(ctx, LVR_EINVAL, "grid has 2^32 or more voxels");

    VoxParams P;
    P.xyz = (const float *)dx;
    P.offs = (const int64_t *)dof;
    P.nc = n_curves;
    P.nv = n_vertices;
    for (int a = 0; a < 3; a++) {
        P.o[a] = g->origin[a];
        P.res[a] = g->res[a];
    }
    P.s = g->scale;
    P.N = g->bins;
    P.amin = g->attr_min;
    P.aspan = g->attr_max - g->attr_min;          // float32 subtraction, as specified
    P.attr = (da && g->attr_max > g->attr_min) ? (const float *)da : nullptr;
    P.status = ctx->d_status;

    // scratch: counts / cursors [nvox], tile sums, long-list queue
    const int64_t ntiles = (nvox + SCAN_TILE - 1) / SCAN_TILE;
    const size_t b_cnt = al((size_t)nvox * 4), b_tiles = al((size_t)ntiles * 8);
    const size_t b_long = al((size_t)nvox * 4 + 16);
    if ((st = ensure_scratch(ctx, b_cnt + b_tiles + b_long)) != LVR_OK) return st;
    uint32_t *cnt = (uint32_t *)ctx->scratch;
    unsigned long long *tiles = (unsigned long long *)((char *)ctx->scratch + b_cnt);
    uint32_t *long_count = (uint32_t *)((char *)ctx->scratch + b_cnt + b_tiles);
    uint32_t *long_list = long_count + 4;
    unsigned long long *total = ctx->d_u64;

    LVR_CUDA(ctx, cudaMemsetAsync(cnt, 0, (size_t)nvox * 4, s));
    LVR_CUDA(ctx, cudaMemsetAsync(total, 0, 8, s));
    if (n_curves > 0) {
        vox_warp_kernel<false><<<grid1d(n_curves * 32, 256), 256, 0, s>>>(P, cnt, nullptr, nullptr, nullptr, nullptr, total);
        LVR_CUDA(ctx, cudaGetLastError());
    }
    LVR_CUDA(ctx, cudaMemcpyAsync(h32, ctx->d_status, 4, cudaMemcpyDeviceToHost, s));
    LVR_CUDA(ctx, cudaMemcpyAsync(h64, total, 8, cudaMemcpyDeviceToHost, s));
    LVR_CUDA(ctx, cudaStreamSynchronize(s));
    const uint32_t flags = *h32;
    if (flags & ST_BAD_OFFSETS) return set_err(ctx, LVR_EINVAL, "curve offsets must start at 0, not decrease and end at n_vertices");
    if (flags & ST_BAD_VERTEX) return set_err(ctx, LVR_EINVAL, "vertex not finite or outside +-2^14 voxels of the grid");
    if (flags & ST_BAD_ATTR) return set_err(ctx, LVR_EINVAL, "attribute not finite");
    if (flags & ST_INTERNAL) return set_err(ctx, LVR_ECUDA, "voxeliser internal check failed");
    const unsigned long long nseg = *h64;
    if (nseg > 0xffffffffull) return set_err(ctx, LVR_EOVERFLOW, "%llu segments exceed 2^32-1", nseg);

    lvr_lineset *ls = new lvr_lineset();
    ls->ctx = ctx;
    for (int a = 0; a < 3; a++) {
        ls->res[a] = g->res[a];
        ls->origin[a] = g->origin[a];
    }
    ls->bins = g->bins;
    ls->scale = g->scale;
    ls->nvox = nvox;
    ls->nseg = (int64_t)nseg;
    if ((st = dev_alloc(ctx, (void **)&ls->offset, (size_t)(nvox + 1) * 4)) != LVR_OK ||
        (st = dev_alloc(ctx, (void **)&ls->rec, (size_t)nseg * 8)) != LVR_OK ||
        (st = dev_alloc(ctx, (void **)&ls->key, (size_t)nseg * 8)) != LVR_OK) {
        lvr_free_lineset(ls);
        return st;
    }
    scan_reduce_kernel<<<(unsigned)ntiles, SCAN_T, 0, s>>>(cnt, nvox, tiles);
    scan_tiles_kernel<<<1, 1024, 0, s>>>(tiles, ntiles, ls->offset + nvox, ctx->d_status);
    scan_down_kernel<<<(unsigned)ntiles, SCAN_T, 0, s>>>(cnt, nvox, tiles, ls->offset);
    LVR_CUDA(ctx, cudaGetLastError());
    if (nseg > 0) {
        if ((size_t)nseg * sizeof(PairSlot) > ctx->vox_pair_bytes) {   // grow-only scatter target
            dev_free(ctx, ctx->vox_pair);
            ctx->vox_pair = nullptr;
            ctx->vox_pair_bytes = 0;
            const size_t b = (size_t)nseg * sizeof(PairSlot) + (size_t)nseg * 4 + 4096;
            if ((st = dev_alloc(ctx, &ctx->vox_pair, b)) != LVR_OK) {
                lvr_free_lineset(ls);
                return st;
            }
            ctx->vox_pair_bytes = b;
        }
        PairSlot *pair = (PairSlot *)ctx->vox_pair;
        // the scatter's cursors start at the offsets (one random atomic per segment)
        LVR_CUDA(ctx, cudaMemcpyAsync(cnt, ls->offset, (size_t)nvox * 4, cudaMemcpyDeviceToDevice, s));
        vox_warp_kernel<true><<<grid1d(n_curves * 32, 256), 256, 0, s>>>(P, cnt, ls->offset, ls->rec, ls->key, pair,
                                                                         total);
        LVR_CUDA(ctx, cudaMemsetAsync(long_count, 0, 4, s));
        sort_small_kernel<<<grid1d(nvox, 256), 256, 0, s>>>(ls->offset, nvox, ls->rec, ls->key, pair, long_list,
                                                            long_count);
        sort_long_kernel<<<304, 256, 2 * SMEM_LIST * sizeof(uint64_t), s>>>(ls->offset, ls->rec, ls->key, pair,
                                                                         long_list, long_count);
        LVR_CUDA(ctx, cudaGetLastError());
    }
    *out = ls;
    return LVR_OK;
}

// ------------------------------------------------------------------ allocation-free variant
// lvr_voxelize_static: the same voxeliser for callers that must not allocate
// device memory (see include/lvr.h). Its scratch lives in one file-scope
// device array, reserved on every device that loads the library until the
// process exits. Host code never uses the array's name as an address: the
// device address is looked up once per device with cudaGetSymbolAddress.
namespace {

constexpr uint32_t STATIC_MAX_VOXELS = LVR_STATIC_MAX_VOXELS;
constexpr size_t STATIC_TILES = (STATIC_MAX_VOXELS + SCAN_TILE - 1) / SCAN_TILE;
// layout (bytes): counts [MAXV] u32 | long list [MAXV] u32 | tile sums [TILES] u64 |
//                 total u64 | status u32 | long count u32
constexpr size_t ST_OFF_LONG = (size_t)STATIC_MAX_VOXELS * 4;
constexpr size_t ST_OFF_TILES = ST_OFF_LONG + (size_t)STATIC_MAX_VOXELS * 4;
constexpr size_t ST_OFF_TOTAL = ST_OFF_TILES + STATIC_TILES * 8;
constexpr size_t ST_OFF_STATUS = ST_OFF_TOTAL + 8;
constexpr size_t ST_OFF_LCOUNT = ST_OFF_STATUS + 4;
constexpr size_t STATIC_BYTES = ST_OFF_LCOUNT + 4;

__device__ __align__(256) unsigned char g_static_scratch[STATIC_BYTES];

constexpr int MAX_DEVICES = 64;
void *g_static_addr[MAX_DEVICES] = {};
std::mutex g_static_mu;

// Device address of the scratch array on the current device (looked up once).
cudaError_t static_scratch(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    }
    *out = (unsigned char *)g_static_addr[dev];
    return cudaSuccess;
}

}  // namespace

// True when p is device memory of device `dev`, or managed memory.
static bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

extern "C" lvr_status lvr_voxelize_static(const float *xyz, const float *attr, const int64_t *curve_offsets,
                                          int64_t n_curves, int64_t n_vertices, const lvr_grid_desc *g,
                                          uint32_t *offset, uint64_t *records, uint64_t *keys,
                                          int64_t capacity, int64_t *n_segments, void *cuda_stream) {
    if (!g || !curve_offsets || !offset || !n_segments || capacity < 0) return LVR_EINVAL;
    if ((capacity > 0 || n_curves > 0) && (!records || !keys)) return LVR_EINVAL;
    *n_segments = 0;
    if (n_curves < 0 || n_vertices < 0 || n_curves > 0xffffffffLL) return LVR_EINVAL;
    if (n_curves == 0 && n_vertices != 0) return LVR_EINVAL;
    if (n_vertices > 0 && !xyz) return LVR_EINVAL;
    if (g->fit || !valid_bins(g->bins)) return LVR_EINVAL;
    for (int a = 0; a < 3; a++)
        if (g->res[a] < 1 || g->res[a] > 4096) return LVR_EINVAL;
    if (!(g->scale > 0.0f) || !isfinite(g->scale)) return LVR_EINVAL;
    const int64_t nvox = (int64_t)g->res[0] * g->res[1] * g->res[2];
    if (nvox > (int64_t)STATIC_MAX_VOXELS) return LVR_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return LVR_EDEVICE;
    // every buffer must already be in the current device's memory: nothing is
    // staged, and the kernels run on this device
    const void *ptrs[6] = {xyz, attr, curve_offsets, offset, records, keys};
    for (const void *p : ptrs)
        if (p && !on_device(p, dev)) return LVR_EINVAL;
    unsigned char *base = nullptr;
    if (static_scratch(dev, &base) != cudaSuccess) return LVR_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t *cnt = (uint32_t *)base;
    uint32_t *long_list = (uint32_t *)(base + ST_OFF_LONG);
    unsigned long long *tiles = (unsigned long long *)(base + ST_OFF_TILES);
    unsigned long long *total = (unsigned long long *)(base + ST_OFF_TOTAL);
    uint32_t *status = (uint32_t *)(base + ST_OFF_STATUS);
    uint32_t *long_count = (uint32_t *)(base + ST_OFF_LCOUNT);

    VoxParams P;
    P.xyz = xyz;
    P.offs = curve_offsets;
    P.nc = n_curves;
    P.nv = n_vertices;
    for (int a = 0; a < 3; a++) {
        P.o[a] = g->origin[a];
        P.res[a] = g->res[a];
    }
    P.s = g->scale;
    P.N = g->bins;
    P.amin = g->attr_min;
    P.aspan = g->attr_max - g->attr_min;
    P.attr = (attr && g->attr_max > g->attr_min) ? attr : nullptr;
    P.status = status;

    // the array keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(cnt, 0, (size_t)nvox * 4, s) != cudaSuccess ||
        cudaMemsetAsync(total, 0, 16, s) != cudaSuccess)
        return LVR_ECUDA;
    if (n_curves > 0) vox_warp_kernel<false><<<grid1d(n_curves * 32, 256), 256, 0, s>>>(P, cnt, nullptr, nullptr, nullptr, nullptr, total);
    if (cudaGetLastError() != cudaSuccess) return LVR_ECUDA;
    unsigned long long h_total = 0;
    uint32_t h_status = 0;
    if (cudaMemcpyAsync(&h_total, total, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LVR_ECUDA;
    if (h_status & (ST_BAD_OFFSETS | ST_BAD_VERTEX | ST_BAD_ATTR)) return LVR_EINVAL;
    if (h_status & ST_INTERNAL) return LVR_ECUDA;
    if (h_total > 0xffffffffull) return LVR_EOVERFLOW;
    *n_segments = (int64_t)h_total;
    if ((int64_t)h_total > capacity) return LVR_EOVERFLOW;

    const int64_t ntiles = (nvox + SCAN_TILE - 1) / SCAN_TILE;
    scan_reduce_kernel<<<(unsigned)ntiles, SCAN_T, 0, s>>>(cnt, nvox, tiles);
    scan_tiles_kernel<<<1, 1024, 0, s>>>(tiles, ntiles, offset + nvox, status);
    scan_down_kernel<<<(unsigned)ntiles, SCAN_T, 0, s>>>(cnt, nvox, tiles, offset);
    if (h_total > 0) {
        if (cudaMemsetAsync(cnt, 0, (size_t)nvox * 4, s) != cudaSuccess ||
            cudaMemsetAsync(long_count, 0, 4, s) != cudaSuccess)
            return LVR_ECUDA;
        vox_warp_kernel<true><<<grid1d(n_curves * 32, 256), 256, 0, s>>>(P, cnt, offset, records, keys, nullptr,
                                                                         total);
        sort_small_kernel<<<grid1d(nvox, 256), 256, 0, s>>>(offset, nvox, records, keys, nullptr, long_list,
                                                            long_count);
        sort_long_kernel<<<304, 256, 2 * SMEM_LIST * sizeof(uint64_t), s>>>(offset, records, keys, nullptr,
                                                                           long_list, long_count);
    }
    if (cudaGetLastError() != cudaSuccess) return LVR_ECUDA;
    return LVR_OK;
}
