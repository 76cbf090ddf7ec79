// Learned ambient-occlusion surrogate: layout, bfloat16 helpers and the
// tensor-core (mma.sync m16n8k16, bf16 x bf16 -> f32) building blocks shared
// by the trainer (ao_mlp.cu) and the fused inference in the ray caster
// (render.cu). Not part of the paper: the surrogate stands in for the traced
// density AO of Sec. 5.3.
//
// Model (inputs 256 = 3 + 250 + 3 padding, three hidden layers of 64, ReLU,
// sigmoid output). Inputs: the hit segment's direction with its first
// non-zero component made positive (3), then for the 5^3 level-0 voxels
// around the hit voxel (dz, dy, dx in -2..2, x fastest) log1p(count) and
// log1p(summed length), zero outside the grid. Parameters are float32
// masters used as bfloat16 (nearest even); bf16 enters every product (inputs,
// weights, hidden activations), sums are float32. The neighbourhood part of
// layer 1 depends only on the hit voxel: it is evaluated once per voxel and
// stored as bf16 (the "voxel term"), and the direction part and bias are
// added per hit.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace aomlp {

constexpr int NIN = 256, NH = 64;
constexpr int OW1 = 0, OB1 = OW1 + NH * NIN, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NH, NPARAM = OB4 + 1;

// Device-side model: bf16 weights (row-major [out][in]) and float biases.
struct Net {
    const __nv_bfloat16 *w2;   // [64][64]
    const __nv_bfloat16 *w3;   // [64][64]
    const float *w1t;          // [64][4]: bf16(W1[f][0..2]) as float, b1[f]
    const float *b2, *b3;      // [64]
    const float *w4;           // [64], values already rounded to bf16
    const float *b4;           // [1]
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

// Direction feature: sign-normalised unit segment direction, bf16-rounded.
__device__ __forceinline__ void tangent_feature(float ux, float uy, float uz, float t[3]) {
    const float s = ux != 0.0f ? (ux > 0.0f ? 1.0f : -1.0f)
                  : (uy != 0.0f ? (uy > 0.0f ? 1.0f : -1.0f) : (uz > 0.0f ? 1.0f : -1.0f));
    t[0] = bf16_round(s * ux);
    t[1] = bf16_round(s * uy);
    t[2] = bf16_round(s * uz);
}

// Layers 2..4 for 16 hits of one warp. `h` is the warp's 16 x 64 bf16 layer-1
// activation tile in shared memory (row stride 64 elements); it is reused for
// the layer-2 activations. Returns, in lanes with t == 0 (lane % 4 == 0), the
// AO of rows g (lo) and g + 8 (hi).
__device__ __forceinline__ void layers234(const Net &net, __nv_bfloat16 *h, float &ao_lo, float &ao_hi) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    float acc[8][4];
    // layer 2 then layer 3: acc = h * W^T (+ b), ReLU, bf16 back into h
#pragma unroll 1
    for (int layer = 0; layer < 2; layer++) {
        const __nv_bfloat16 *W = layer == 0 ? net.w2 : net.w3;
        const float *bias = layer == 0 ? net.b2 : net.b3;
#pragma unroll
        for (int n = 0; n < 8; n++) {
            acc[n][0] = acc[n][2] = __ldg(bias + n * 8 + 2 * t);
            acc[n][1] = acc[n][3] = __ldg(bias + n * 8 + 2 * t + 1);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            uint32_t a[4];
            const uint32_t *hr0 = reinterpret_cast<const uint32_t *>(h + g * NH + k * 16);
            const uint32_t *hr1 = reinterpret_cast<const uint32_t *>(h + (g + 8) * NH + k * 16);
            a[0] = hr0[t];
            a[1] = hr1[t];
            a[2] = hr0[t + 4];
            a[3] = hr1[t + 4];
#pragma unroll
            for (int n = 0; n < 8; n++) {
                const uint32_t *wr = reinterpret_cast<const uint32_t *>(W + (n * 8 + g) * NH + k * 16);
                mma16816(acc[n], a, __ldg(wr + t), __ldg(wr + t + 4));
            }
        }
        __syncwarp();
        if (layer == 0) {
#pragma unroll
            for (int n = 0; n < 8; n++) {
                uint32_t *o0 = reinterpret_cast<uint32_t *>(h + g * NH + n * 8);
                uint32_t *o1 = reinterpret_cast<uint32_t *>(h + (g + 8) * NH + n * 8);
                o0[t] = pack_bf16x2(fmaxf(acc[n][0], 0.0f), fmaxf(acc[n][1], 0.0f));
                o1[t] = pack_bf16x2(fmaxf(acc[n][2], 0.0f), fmaxf(acc[n][3], 0.0f));
            }
            __syncwarp();
        }
    }
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

// Layer-1 activation of one hit for 32 consecutive features f0..f0+31:
// bf16(ReLU(voxel_term[f] + (b1[f] + W1[f][0..2] . t))) written to `row`.
__device__ __forceinline__ void layer1_half(const Net &net, const __nv_bfloat16 *vterm, const float t[3], int f0,
                                            __nv_bfloat16 *row) {
    const uint4 *vp = reinterpret_cast<const uint4 *>(vterm + f0);
    const float4 *wt = reinterpret_cast<const float4 *>(net.w1t);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const uint4 v = __ldg(vp + q);
        const uint32_t words[4] = {v.x, v.y, v.z, v.w};
        uint32_t out[4];
#pragma unroll
        for (int w = 0; w < 4; w++) {
            const __nv_bfloat162 pr = *reinterpret_cast<const __nv_bfloat162 *>(&words[w]);
            float z[2] = {__bfloat162float(pr.x), __bfloat162float(pr.y)};
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const float4 c = __ldg(wt + f0 + q * 8 + w * 2 + e);
                const float d = fmaf(c.x, t[0], fmaf(c.y, t[1], fmaf(c.z, t[2], c.w)));
                z[e] = fmaxf(z[e] + d, 0.0f);
            }
            out[w] = pack_bf16x2(z[0], z[1]);
        }
        *reinterpret_cast<uint4 *>(row + f0 + q * 8) = make_uint4(out[0], out[1], out[2], out[3]);
    }
}

}  // namespace aomlp

struct lvr_ao_model;
// Device view of a model's current parameters (ao_mlp.cu).
aomlp::Net ao_net(const lvr_ao_model *m);
