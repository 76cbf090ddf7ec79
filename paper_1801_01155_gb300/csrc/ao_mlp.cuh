// Learned ambient-occlusion surrogate: layout, bfloat16 helpers and the
// tensor-core (mma.sync m16n8k16, bf16 x bf16 -> f32) building blocks shared
// by the trainer (ao_mlp.cu) and the fused inference in the ray caster
// (render.cu). Not part of the paper: the surrogate stands in for the traced
// density AO of Sec. 5.3.
//
// Model: 400 inputs, three hidden layers of 64 with ReLU, sigmoid output.
// Per-hit inputs 0..14: the hit segment's unit direction with its first
// non-zero component made positive (3), the unit tube normal (3), and the
// hit point's offset inside the level-l cell of its voxel for l = 0, 1, 2,
// p / 2^l - floor(v / 2^l) - 1/2 (9); input 15 is zero. Per-voxel inputs
// 16..390: for l = 0, 1, 2 the 5^3 level-l cells around the voxel's cell
// (dz, dy, dx in -2..2, x fastest), log1p(8 rho) with rho = dens_l / 8^l
// (Eq. 1's density as the AO march samples it), zero outside the level;
// inputs 391..399 are zero. Parameters are float32 masters used as bfloat16
// (nearest even); bf16 enters every product (inputs, weights, hidden
// activations), sums are float32. The per-voxel part of layer 1 depends only
// on the hit voxel: it is evaluated once per voxel and stored as bf16 (the
// "voxel term"); the per-hit part and the bias are added per hit.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace aomlp {

constexpr int NIN = 400, NH = 64;
constexpr int NHIT = 15, VOFF = 16, NVIN = 375;   // per-hit inputs; first per-voxel input; per-voxel inputs
constexpr int VK = NIN - VOFF;                    // per-voxel K of layer 1 (24 mma k-steps)
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NH, NPARAM = OB4 + 1;

// Device-side model: bf16 weights (row-major [out][in]) and float biases.
struct Net {
    const __nv_bfloat16 *w1;   // [64][400]
    const __nv_bfloat16 *w2;   // [64][64]
    const __nv_bfloat16 *w3;   // [64][64]
    const float *b1, *b2, *b3; // [64]
    const float *w4;           // [64], values already rounded to bf16
    const float *b4;           // [1]
    // fragment-ordered copies for the renderer's shared-tile MLP: f1[n][lane]
    // = (b0, b1) of layer 1's per-hit k-step; f2 / f3 [n][lane][2] = the
    // (b0, b1) pairs of k-steps 0-1 and 2-3 of layers 2 / 3
    const uint2 *f1;
    const uint4 *f2, *f3;
};

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // .x = lo (low half)
    return *reinterpret_cast<const uint32_t *>(&v);
}

// D += A(16x16, row) * B(16x8, col); bf16 inputs, f32 accumulate.
// Fragments (g = lane/4, t = lane%4): a0 = A[g][2t..2t+1], a1 = A[g+8][2t..],
// a2 = A[g][2t+8..], a3 = A[g+8][2t+8..]; b0 = B[2t..2t+1][g], b1 = B[2t+8..][g];
// c0,c1 = C[g][2t..2t+1], c2,c3 = C[g+8][2t..2t+1].
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Unit vector d / |d| (zero stays zero), the ray caster's expression for the
// segment direction.
__device__ __forceinline__ void unit_direction(float dx, float dy, float dz, float u[3]) {
    const float L2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float s = L2 > 0.0f ? 1.0f / sqrtf(L2) : 0.0f;
    u[0] = dx * s;
    u[1] = dy * s;
    u[2] = dz * s;
}

// Per-hit inputs 0..14 from the unit segment direction u, the unit normal n,
// the hit point p (grid coordinates) and its voxel v, bf16-rounded.
__device__ __forceinline__ void hit_inputs(float ux, float uy, float uz, float nx, float ny, float nz, float px,
                                           float py, float pz, int vx, int vy, int vz, float h[NHIT]) {
    const float s = ux != 0.0f ? (ux > 0.0f ? 1.0f : -1.0f)
                  : (uy != 0.0f ? (uy > 0.0f ? 1.0f : -1.0f) : (uz > 0.0f ? 1.0f : -1.0f));
    h[0] = bf16_round(s * ux);
    h[1] = bf16_round(s * uy);
    h[2] = bf16_round(s * uz);
    h[3] = bf16_round(nx);
    h[4] = bf16_round(ny);
    h[5] = bf16_round(nz);
    const float p[3] = {px, py, pz};
    const int v[3] = {vx, vy, vz};
#pragma unroll
    for (int l = 0; l < 3; l++) {
        const float sc = l == 0 ? 1.0f : (l == 1 ? 0.5f : 0.25f);
#pragma unroll
        for (int c = 0; c < 3; c++) h[6 + 3 * l + c] = bf16_round(p[c] * sc - (float)(v[c] >> l) - 0.5f);
    }
}

// Row stride of a warp's per-hit input tile (16 hits x 16 inputs): 24
// elements keep the rows 16-byte aligned and the fragment loads free of bank
// conflicts.
constexpr int HIN_STRIDE = 24;

// Per-hit inputs of one hit as 16 bf16 (input 15 zero) into `row` (16-byte aligned).
__device__ __forceinline__ void store_hit_inputs(const float h[NHIT], __nv_bfloat16 *row) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 7; i++) w[i] = pack_bf16x2(h[2 * i], h[2 * i + 1]);
    w[7] = pack_bf16x2(h[14], 0.0f);
    uint4 *d = reinterpret_cast<uint4 *>(row);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// The output fragments of one m16n8 layer (8 n-tiles, 64 features) are, lane
// for lane, the A fragments of the next layer's 4 k-steps: k-step k takes
// n-tiles 2k (columns 0..7) and 2k+1 (columns 8..15). ReLU and bf16 here.
__device__ __forceinline__ void relu_to_a(const float acc[8][4], uint32_t a[4][4]) {
#pragma unroll
    for (int k = 0; k < 4; k++) {
        a[k][0] = pack_bf16x2(fmaxf(acc[2 * k][0], 0.0f), fmaxf(acc[2 * k][1], 0.0f));
        a[k][1] = pack_bf16x2(fmaxf(acc[2 * k][2], 0.0f), fmaxf(acc[2 * k][3], 0.0f));
        a[k][2] = pack_bf16x2(fmaxf(acc[2 * k + 1][0], 0.0f), fmaxf(acc[2 * k + 1][1], 0.0f));
        a[k][3] = pack_bf16x2(fmaxf(acc[2 * k + 1][2], 0.0f), fmaxf(acc[2 * k + 1][3], 0.0f));
    }
}

// acc = bias + A (16 x 64) x W^T for a 64 x 64 layer W (bf16 [out][in]).
__device__ __forceinline__ void dense64(const __nv_bfloat16 *W, const float *bias, const uint32_t a[4][4],
                                        float acc[8][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int n = 0; n < 8; n++) {
        acc[n][0] = acc[n][2] = __ldg(bias + n * 8 + 2 * t);
        acc[n][1] = acc[n][3] = __ldg(bias + n * 8 + 2 * t + 1);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
#pragma unroll
        for (int n = 0; n < 8; n++) {
            const uint32_t *wr = reinterpret_cast<const uint32_t *>(W + (n * 8 + g) * NH + k * 16);
            mma16816(acc[n], a[k], __ldg(wr + t), __ldg(wr + t + 4));
        }
    }
}

// The whole model for the 16 hits of one warp, on tensor cores, with the
// activations kept in registers. `hin` is the warp's per-hit input tile
// (row r = hit r, stride HIN_STRIDE); vt_lo / vt_hi point to the voxel
// terms of rows g = lane / 4 and g + 8 (null: zero). Layer 1 starts its
// accumulators at b1 + voxel term and adds the per-hit part in one k-step.
// Returns, in lanes with lane % 4 == 0, the AO of rows g (lo) and g + 8 (hi).
__device__ __forceinline__ void mlp_tile(const Net &net, const __nv_bfloat16 *vt_lo, const __nv_bfloat16 *vt_hi,
                                         const __nv_bfloat16 *hin, float &ao_lo, float &ao_hi) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[8][4];
    uint32_t a[4][4];
    {
        uint32_t x[4];
        const uint32_t *r0 = reinterpret_cast<const uint32_t *>(hin + g * HIN_STRIDE);
        const uint32_t *r1 = reinterpret_cast<const uint32_t *>(hin + (g + 8) * HIN_STRIDE);
        x[0] = r0[t];
        x[1] = r1[t];
        x[2] = r0[t + 4];
        x[3] = r1[t + 4];
#pragma unroll
        for (int n = 0; n < 8; n++) {
            const int f = n * 8 + 2 * t;
            const float b0 = __ldg(net.b1 + f), b1 = __ldg(net.b1 + f + 1);
            float lo0 = 0.0f, lo1 = 0.0f, hi0 = 0.0f, hi1 = 0.0f;
            if (vt_lo) {
                const uint32_t u = __ldg(reinterpret_cast<const unsigned int *>(vt_lo + f));
                const __nv_bfloat162 pr = *reinterpret_cast<const __nv_bfloat162 *>(&u);
                lo0 = __bfloat162float(pr.x);
                lo1 = __bfloat162float(pr.y);
            }
            if (vt_hi) {
                const uint32_t u = __ldg(reinterpret_cast<const unsigned int *>(vt_hi + f));
                const __nv_bfloat162 pr = *reinterpret_cast<const __nv_bfloat162 *>(&u);
                hi0 = __bfloat162float(pr.x);
                hi1 = __bfloat162float(pr.y);
            }
            acc[n][0] = b0 + lo0;
            acc[n][1] = b1 + lo1;
            acc[n][2] = b0 + hi0;
            acc[n][3] = b1 + hi1;
            const uint32_t *wr = reinterpret_cast<const uint32_t *>(net.w1 + (n * 8 + g) * NIN);
            mma16816(acc[n], x, __ldg(wr + t), __ldg(wr + t + 4));
        }
    }
    relu_to_a(acc, a);
    dense64(net.w2, net.b2, a, acc);
    relu_to_a(acc, a);
    dense64(net.w3, net.b3, a, acc);
    // layer 4 from the layer-3 fragments: bf16(ReLU(z3)) . w4, summed over the quad
    float lo = 0.0f, hi = 0.0f;
#pragma unroll
    for (int n = 0; n < 8; n++) {
        const float w0 = __ldg(net.w4 + n * 8 + 2 * t), w1 = __ldg(net.w4 + n * 8 + 2 * t + 1);
        lo = fmaf(bf16_round(fmaxf(acc[n][0], 0.0f)), w0, lo);
        lo = fmaf(bf16_round(fmaxf(acc[n][1], 0.0f)), w1, lo);
        hi = fmaf(bf16_round(fmaxf(acc[n][2], 0.0f)), w0, hi);
        hi = fmaf(bf16_round(fmaxf(acc[n][3], 0.0f)), w1, hi);
    }
    lo += __shfl_xor_sync(0xffffffffu, lo, 1);
    lo += __shfl_xor_sync(0xffffffffu, lo, 2);
    hi += __shfl_xor_sync(0xffffffffu, hi, 1);
    hi += __shfl_xor_sync(0xffffffffu, hi, 2);
    const float b4 = __ldg(net.b4);
    ao_lo = 1.0f / (1.0f + __expf(-(lo + b4)));
    ao_hi = 1.0f / (1.0f + __expf(-(hi + b4)));
}

// ---- the same model with short code: activations in shared memory
// A warp's 16 x 64 bf16 activation tile: rows of 128 bytes whose 16-byte
// chunks (8 features each) are XOR-swizzled by the row, so the ldmatrix row
// reads and the fragment stores both touch distinct banks.
constexpr int ACT_BYTES = 16 * 128;

__device__ __forceinline__ int act_off(int row, int chunk) { return row * 128 + ((chunk ^ (row & 7)) << 4); }

// Per-hit inputs of one hit (16 bf16, input 15 zero) into row `row` of the tile.
__device__ __forceinline__ void store_hit_inputs_act(const float h[NHIT], uint8_t *act, int row) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 7; i++) w[i] = pack_bf16x2(h[2 * i], h[2 * i + 1]);
    w[7] = pack_bf16x2(h[14], 0.0f);
    *reinterpret_cast<uint4 *>(act + act_off(row, 0)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(act + act_off(row, 1)) = make_uint4(w[4], w[5], w[6], w[7]);
}

// A fragments of k-step k (features 16k .. 16k + 15) of the tile: matrices
// (rows 0-7 | 8-15) x (features 16k .. 16k + 7 | 16k + 8 .. 16k + 15).
__device__ __forceinline__ void act_a(const uint8_t *act, int k, uint32_t a[4]) {
    const int lane = threadIdx.x & 31;
    const int row = (lane & 7) + ((lane >> 3) & 1) * 8, chunk = 2 * k + (lane >> 4);
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(act + act_off(row, chunk));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

// ReLU + bf16 of one n-tile's accumulators (features 8n .. 8n + 7) into the tile.
__device__ __forceinline__ void act_store(uint8_t *act, int n, const float acc[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    *reinterpret_cast<uint32_t *>(act + act_off(g, n) + 4 * t) =
        pack_bf16x2(fmaxf(acc[0], 0.0f), fmaxf(acc[1], 0.0f));
    *reinterpret_cast<uint32_t *>(act + act_off(g + 8, n) + 4 * t) =
        pack_bf16x2(fmaxf(acc[2], 0.0f), fmaxf(acc[3], 0.0f));
}

// The model for the 16 hits whose per-hit inputs are in rows 0..15 of the
// warp's tile (vt_lo / vt_hi and the result lanes as in mlp_tile). Each layer
// takes its input fragments into registers, then walks its 8 n-tiles in a
// loop that is not unrolled, writing each n-tile's activations back into the
// tile: the code stays small and few registers are live. Every mma, rounding
// and sum is the one mlp_tile performs, in the same order, so the results are
// identical.
__device__ __forceinline__ void mlp_tile_smem(const Net &net, const __nv_bfloat16 *vt_lo,
                                              const __nv_bfloat16 *vt_hi, uint8_t *act, float &ao_lo,
                                              float &ao_hi) {
    const int lane = threadIdx.x & 31, t = lane & 3;
    {   // layer 1: b1 + voxel term + the per-hit part (one k-step)
        uint32_t x[4];
        act_a(act, 0, x);
        __syncwarp();   // every lane holds its inputs before the tile is overwritten
#pragma unroll 2
        for (int n = 0; n < 8; n++) {
            const int f = n * 8 + 2 * t;
            const float2 bb = __ldg(reinterpret_cast<const float2 *>(net.b1 + f));
            const float b0 = bb.x, b1 = bb.y;
            float lo0 = 0.0f, lo1 = 0.0f, hi0 = 0.0f, hi1 = 0.0f;
            if (vt_lo) {
                const uint32_t u = __ldg(reinterpret_cast<const unsigned int *>(vt_lo + f));
                const __nv_bfloat162 pr = *reinterpret_cast<const __nv_bfloat162 *>(&u);
                lo0 = __bfloat162float(pr.x);
                lo1 = __bfloat162float(pr.y);
            }
            if (vt_hi) {
                const uint32_t u = __ldg(reinterpret_cast<const unsigned int *>(vt_hi + f));
                const __nv_bfloat162 pr = *reinterpret_cast<const __nv_bfloat162 *>(&u);
                hi0 = __bfloat162float(pr.x);
                hi1 = __bfloat162float(pr.y);
            }
            float acc[4] = {b0 + lo0, b1 + lo1, b0 + hi0, b1 + hi1};
            const uint2 w = __ldg(net.f1 + n * 32 + lane);
            mma16816(acc, x, w.x, w.y);
            act_store(act, n, acc);
        }
        __syncwarp();
    }
    uint32_t a[4][4];
    {   // layer 2
#pragma unroll
        for (int k = 0; k < 4; k++) act_a(act, k, a[k]);
        __syncwarp();
#pragma unroll 2
        for (int n = 0; n < 8; n++) {
            float acc[4];
            const float2 bb = __ldg(reinterpret_cast<const float2 *>(net.b2 + n * 8 + 2 * t));
            acc[0] = acc[2] = bb.x;
            acc[1] = acc[3] = bb.y;
            const uint4 w01 = __ldg(net.f2 + (n * 32 + lane) * 2), w23 = __ldg(net.f2 + (n * 32 + lane) * 2 + 1);
            mma16816(acc, a[0], w01.x, w01.y);
            mma16816(acc, a[1], w01.z, w01.w);
            mma16816(acc, a[2], w23.x, w23.y);
            mma16816(acc, a[3], w23.z, w23.w);
            act_store(act, n, acc);
        }
        __syncwarp();
    }
    // layer 3, and layer 4 from its fragments: bf16(ReLU(z3)) . w4, summed over the quad
#pragma unroll
    for (int k = 0; k < 4; k++) act_a(act, k, a[k]);
    __syncwarp();   // the tile's last reads are done before the caller reuses it
    float lo = 0.0f, hi = 0.0f;
#pragma unroll 2
    for (int n = 0; n < 8; n++) {
        float acc[4];
        const float2 bb = __ldg(reinterpret_cast<const float2 *>(net.b3 + n * 8 + 2 * t));
        acc[0] = acc[2] = bb.x;
        acc[1] = acc[3] = bb.y;
        const uint4 w01 = __ldg(net.f3 + (n * 32 + lane) * 2), w23 = __ldg(net.f3 + (n * 32 + lane) * 2 + 1);
        mma16816(acc, a[0], w01.x, w01.y);
        mma16816(acc, a[1], w01.z, w01.w);
        mma16816(acc, a[2], w23.x, w23.y);
        mma16816(acc, a[3], w23.z, w23.w);
        const float2 w4 = __ldg(reinterpret_cast<const float2 *>(net.w4 + n * 8 + 2 * t));
        const float w0 = w4.x, w1 = w4.y;
        lo = fmaf(bf16_round(fmaxf(acc[0], 0.0f)), w0, lo);
        lo = fmaf(bf16_round(fmaxf(acc[1], 0.0f)), w1, lo);
        hi = fmaf(bf16_round(fmaxf(acc[2], 0.0f)), w0, hi);
        hi = fmaf(bf16_round(fmaxf(acc[3], 0.0f)), w1, hi);
    }
    lo += __shfl_xor_sync(0xffffffffu, lo, 1);
    lo += __shfl_xor_sync(0xffffffffu, lo, 2);
    hi += __shfl_xor_sync(0xffffffffu, hi, 1);
    hi += __shfl_xor_sync(0xffffffffu, hi, 2);
    const float b4 = __ldg(net.b4);
    ao_lo = 1.0f / (1.0f + __expf(-(lo + b4)));
    ao_hi = 1.0f / (1.0f + __expf(-(hi + b4)));
}

}  // namespace aomlp

struct lvr_ao_model;
// Device view of a model's current parameters (ao_mlp.cu).
aomlp::Net ao_net(const lvr_ao_model *m);
