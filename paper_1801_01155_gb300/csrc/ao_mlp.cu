// Learned AO surrogate: model handle, per-voxel terms, batched inference,
// training samples and the trainer (forward / backward / Adam). Layout and
// arithmetic of the model: see ao_mlp.cuh. Tensor cores via mma.sync
// m16n8k16 (bf16 inputs, f32 accumulation) in every contraction.
#include <math.h>
#include <string.h>

#include <numeric>
#include <vector>

#include "ao_mlp.cuh"
#include "lvr_internal.cuh"

using namespace aomlp;
typedef __nv_bfloat16 bf16;

namespace {

// ------------------------------------------------------------------ parameter copies
// bf16 weight copies and bf16-rounded W4, refreshed after every change of
// the masters.
__global__ void refresh_kernel(const float *__restrict__ p, bf16 *w1b, bf16 *w2b, bf16 *w3b, float *w4b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NH * NIN; i += gridDim.x * blockDim.x) {
        w1b[i] = __float2bfloat16_rn(p[OW1 + i]);
        if (i < NH * NH) {
            w2b[i] = __float2bfloat16_rn(p[OW2 + i]);
            w3b[i] = __float2bfloat16_rn(p[OW3 + i]);
        }
        if (i < NH) w4b[i] = bf16_round(p[OW4 + i]);
    }
}

// The same bf16 weights as mma B fragments in the order the renderer's lanes
// read them (see Net): lane (g, t) of n-tile n takes rows n * 8 + g, columns
// k * 16 + 2t (+1) and k * 16 + 2t + 8 (+1).
__global__ void frag_kernel(const float *__restrict__ p, uint32_t *f) {
    for (int i = threadIdx.x; i < 8 * 32 * 18; i += blockDim.x) {
        const int n = i / (32 * 18), r = i % (32 * 18), lane = r / 18, e = r % 18;
        const int g = lane >> 2, t = lane & 3, row = n * 8 + g;
        float lo, hi;
        if (e < 2) {                                   // layer 1, per-hit k-step
            const int c = 2 * t + 8 * e;
            lo = p[OW1 + row * NIN + c];
            hi = p[OW1 + row * NIN + c + 1];
        } else {                                       // layers 2, 3: k-step, then b0 / b1
            const int L = (e - 2) / 8, j = (e - 2) % 8, k = j >> 1, c = k * 16 + 2 * t + 8 * (j & 1);
            const int off = L == 0 ? OW2 : OW3;
            lo = p[off + row * NH + c];
            hi = p[off + row * NH + c + 1];
        }
        const uint32_t v = pack_bf16x2(lo, hi);
        if (e < 2) f[(n * 32 + lane) * 2 + e] = v;
        else f[8 * 32 * 2 + ((e - 2) / 8) * (8 * 32 * 8) + (n * 32 + lane) * 8 + (e - 2) % 8] = v;
    }
}

// ------------------------------------------------------------------ inputs
// Per-voxel input values of one LoD level: bf16(log1p(8 dens_l / 8^l)),
// rows (x) of `pitch` elements.
__global__ void logd_kernel(const float *__restrict__ dens, int dx, int dy, int64_t n, int pitch, float inv8l,
                            bf16 *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / dx;
        out[row * pitch + (i - row * dx)] = __float2bfloat16_rn(log1pf(8.0f * (dens[i] * inv8l)));
    }
}

// The three levels' input values (rows padded to `pitch` elements, a
// multiple of 8: 16-byte rows, as the voxel term's tensor maps need) and
// dimensions.
struct Logd {
    const bf16 *d[3];
    int dims[3][3];
    int pitch[3];
};

// Per-voxel inputs 16..390 of voxel v into row[0..374]: for each level the
// 5^3 cells around v's cell, x fastest; `lane` / `nl` split the work.
__device__ __forceinline__ void gather_voxel_inputs(const Logd &L, int vx, int vy, int vz, bf16 *row, int lane,
                                                    int nl) {
    for (int i = lane; i < NVIN; i += nl) {
        const int l = i / 125, n = i - 125 * l;
        const int X = (vx >> l) + n % 5 - 2, Y = (vy >> l) + (n / 5) % 5 - 2, Z = (vz >> l) + n / 25 - 2;
        bf16 v = __float2bfloat16_rn(0.0f);
        if ((unsigned)X < (unsigned)L.dims[l][0] && (unsigned)Y < (unsigned)L.dims[l][1] &&
            (unsigned)Z < (unsigned)L.dims[l][2])
            v = L.d[l][X + (int64_t)L.pitch[l] * (Y + (int64_t)L.dims[l][1] * Z)];
        row[i] = v;
    }
}

// Per-hit inputs of sample i from its voxel id, raw direction, point and normal.
__device__ __forceinline__ void sample_hit_inputs(int dx, int dy, int32_t v, const float *dir, const float *pos,
                                                  const float *nrm, float h[NHIT]) {
    float u[3];
    unit_direction(dir[0], dir[1], dir[2], u);
    hit_inputs(u[0], u[1], u[2], nrm[0], nrm[1], nrm[2], pos[0], pos[1], pos[2], v % dx, (v / dx) % dy, v / (dx * dy),
               h);
}

// Training inputs: one warp per sample; an out-of-range voxel id gives an all-zero row.
__global__ void features_kernel(Logd L, int64_t n, const int32_t *__restrict__ vox, const float *__restrict__ dir,
                                const float *__restrict__ pos, const float *__restrict__ nrm, bf16 *X) {
    const int lane = threadIdx.x & 31;
    const int dx = L.dims[0][0], dy = L.dims[0][1];
    const int64_t nvox = (int64_t)dx * dy * L.dims[0][2];
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        bf16 *row = X + i * NIN;
        const int32_t v = vox[i];
        if (v < 0 || (int64_t)v >= nvox) {
            for (int k = lane; k < NIN; k += 32) row[k] = __float2bfloat16_rn(0.0f);
            continue;
        }
        if (lane == 0) {
            float h[NHIT];
            sample_hit_inputs(dx, dy, v, dir + 3 * i, pos + 3 * i, nrm + 3 * i, h);
            for (int k = 0; k < NHIT; k++) row[k] = __float2bfloat16_rn(h[k]);
            row[NHIT] = __float2bfloat16_rn(0.0f);
        }
        if (lane < NIN - VOFF - NVIN) row[VOFF + NVIN + lane] = __float2bfloat16_rn(0.0f);
        gather_voxel_inputs(L, v % dx, (v / dx) % dy, v / (dx * dy), row + VOFF, lane, 32);
    }
}

// Learned AO of n samples: the same device code as the ray caster's fused
// inference. One warp per 16 samples; out-of-range voxel ids give NaN.
__global__ void __launch_bounds__(128)
infer_kernel(Net net, const bf16 *__restrict__ vterm, int dx, int dy, int64_t nvox, int64_t n,
             const int32_t *__restrict__ vox, const float *__restrict__ dir, const float *__restrict__ pos,
             const float *__restrict__ nrm, float *ao) {
    __shared__ __align__(16) bf16 tile[4][16 * HIN_STRIDE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2;
    bf16 *hin = tile[warp];
    auto ok = [&](int64_t i) { return i < n && vox[i] >= 0 && vox[i] < nvox; };
    for (int64_t base = ((int64_t)blockIdx.x * 4 + warp) * 16; base < n; base += (int64_t)gridDim.x * 64) {
        if (lane < 16) {
            const int64_t i = base + lane;
            float hx[NHIT];
            if (ok(i)) sample_hit_inputs(dx, dy, vox[i], dir + 3 * i, pos + 3 * i, nrm + 3 * i, hx);
            else for (int k = 0; k < NHIT; k++) hx[k] = 0.0f;
            store_hit_inputs(hx, hin + lane * HIN_STRIDE);
        }
        __syncwarp();
        float lo, hi;
        mlp_tile(net, ok(base + g) ? vterm + (int64_t)vox[base + g] * NH : nullptr,
                 ok(base + g + 8) ? vterm + (int64_t)vox[base + g + 8] * NH : nullptr, hin, lo, hi);
        if ((lane & 3) == 0) {
            const int g = lane >> 2;
            if (base + g < n) ao[base + g] = vox[base + g] >= 0 && vox[base + g] < nvox ? lo : __int_as_float(0x7fc00000);
            if (base + g + 8 < n)
                ao[base + g + 8] = vox[base + g + 8] >= 0 && vox[base + g + 8] < nvox ? hi : __int_as_float(0x7fc00000);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ trainer
// C[z] = op(A) x op(B) over the k-range of split z (f32 partials).
// A_COL: op(A)[m][k] = A[k * lda + m], else A[m * lda + k].
// B_KN:  op(B)[k][n] = B[k * ldb + n], else B[n * ldb + k].
constexpr int GT = 64, GK = 32, GKP = GK + 8;
template <bool A_COL, bool B_KN>
__global__ void __launch_bounds__(128)
gemm_kernel(int M, int N, int K, const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B, int ldb, float *C,
            int kchunk) {
    __shared__ __align__(16) bf16 sa[GT][GKP];
    __shared__ __align__(16) bf16 sb[GT][GKP];
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT, z = blockIdx.z;
    const int kb = z * kchunk, ke = min(K, kb + kchunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    const bf16 zero = __float2bfloat16_rn(0.0f);
    float acc[8][4];
#pragma unroll
    for (int n = 0; n < 8; n++) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.0f;
    for (int k0 = kb; k0 < ke; k0 += GK) {
        for (int i = tid; i < GT * GK; i += 128) {
            int m, k;
            if (A_COL) { m = i % GT; k = i / GT; } else { k = i % GK; m = i / GK; }
            const int gm = m0 + m, gk = k0 + k;
            sa[m][k] = (gm < M && gk < ke) ? (A_COL ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk]) : zero;
            int nn, kk;
            if (B_KN) { nn = i % GT; kk = i / GT; } else { kk = i % GK; nn = i / GK; }
            const int gn = n0 + nn, gk2 = k0 + kk;
            sb[nn][kk] = (gn < N && gk2 < ke) ? (B_KN ? B[(int64_t)gk2 * ldb + gn] : B[(int64_t)gn * ldb + gk2]) : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GK; ks += 16) {
            uint32_t a[4];
            const uint32_t *r0 = reinterpret_cast<const uint32_t *>(&sa[warp * 16 + g][ks]);
            const uint32_t *r1 = reinterpret_cast<const uint32_t *>(&sa[warp * 16 + g + 8][ks]);
            a[0] = r0[t];
            a[1] = r1[t];
            a[2] = r0[t + 4];
            a[3] = r1[t + 4];
#pragma unroll
            for (int n = 0; n < 8; n++) {
                const uint32_t *br = reinterpret_cast<const uint32_t *>(&sb[n * 8 + g][ks]);
                mma16816(acc[n], a, br[t], br[t + 4]);
            }
        }
        __syncthreads();
    }
    float *Cz = C + (int64_t)z * M * N;
#pragma unroll
    for (int n = 0; n < 8; n++) {
        const int gm = m0 + warp * 16 + g, gn = n0 + n * 8 + 2 * t;
        if (gm < M && gn < N) { Cz[(int64_t)gm * N + gn] = acc[n][0]; if (gn + 1 < N) Cz[(int64_t)gm * N + gn + 1] = acc[n][1]; }
        if (gm + 8 < M && gn < N) { Cz[(int64_t)(gm + 8) * N + gn] = acc[n][2]; if (gn + 1 < N) Cz[(int64_t)(gm + 8) * N + gn + 1] = acc[n][3]; }
    }
}

// out[i] = sum_z part[z][i] (fixed order), i < n
__global__ void sum_splits_kernel(const float *__restrict__ part, int splits, int64_t n, float *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < splits; z++) s += part[(int64_t)z * n + i];
        out[i] = s;
    }
}

// Z [R][64] += bias, H = bf16(ReLU(Z)).
__global__ void act_kernel(float *Z, const float *__restrict__ bias, int64_t R, bf16 *H) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < R * NH; i += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[i] + bias[i % NH];
        Z[i] = z;
        H[i] = __float2bfloat16_rn(fmaxf(z, 0.0f));
    }
}

constexpr int EB = 256;   // rows per block of the row-wise kernels

// Output layer and MSE: y = sigmoid(H3 . w4 + b4), dz4 = 2 (y - t) / R * y (1 - y);
// per-block partial sums of (y - t)^2, dz4 and dz4 * H3[:, j] (for b4 and W4).
__global__ void __launch_bounds__(EB)
out_kernel(const bf16 *__restrict__ H3, const float *__restrict__ w4b, const float *__restrict__ b4,
           const float *__restrict__ target, int64_t R, float *dz4, float *part /*[blocks][66]*/, float *pred) {
    __shared__ float red[EB];
    const int64_t r = blockIdx.x * (int64_t)EB + threadIdx.x;
    float d = 0.0f, e2 = 0.0f;
    if (r < R) {
        float z = __ldg(b4);
        for (int j = 0; j < NH; j++) z = fmaf(__bfloat162float(H3[r * NH + j]), w4b[j], z);
        const float y = 1.0f / (1.0f + expf(-z));
        if (pred) pred[r] = y;
        const float e = y - (target ? target[r] : 0.0f);
        e2 = e * e;
        d = 2.0f * e / (float)R * y * (1.0f - y);
        dz4[r] = d;
    }
    // block sums: [0] loss, [1] dz4, [2 + j] dz4 * H3[:, j]
    for (int c = 0; c < 2 + NH; c++) {
        float v = c == 0 ? e2 : (c == 1 ? d : (r < R ? d * __bfloat162float(H3[r * NH + c - 2]) : 0.0f));
        red[threadIdx.x] = v;
        __syncthreads();
        for (int s = EB / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * (2 + NH) + c] = red[0];
        __syncthreads();
    }
}

// dZ = dH (f32) masked by Z > 0, as bf16; per-block column sums of the f32 dZ
// (bias gradient). For the last hidden layer dH = dz4 w4^T (outer product).
__global__ void __launch_bounds__(EB)
back_act_kernel(const float *__restrict__ dH, const float *__restrict__ dz4, const float *__restrict__ w4b,
                const float *__restrict__ Z, int64_t R, bf16 *dZb, float *part /*[blocks][64]*/) {
    __shared__ float red[EB / 64][NH + 1];
    const int j = threadIdx.x % NH, sub = threadIdx.x / NH;
    float s = 0.0f;
    for (int64_t r = blockIdx.x * (int64_t)(EB / 64) * 16 + sub; r < min(R, (int64_t)(blockIdx.x + 1) * (EB / 64) * 16);
         r += EB / 64) {
        const int64_t i = r * NH + j;
        const float dh = dH ? dH[i] : dz4[r] * w4b[j];
        const float d = Z[i] > 0.0f ? dh : 0.0f;
        dZb[i] = __float2bfloat16_rn(d);
        s += d;
    }
    red[sub][j] = s;
    __syncthreads();
    if (sub == 0) {
        float tsum = 0.0f;
        for (int q = 0; q < EB / 64; q++) tsum += red[q][j];
        part[blockIdx.x * NH + j] = tsum;
    }
}

// sum_b part[b][c] for c < ncols into out[c] (fixed order)
__global__ void colsum_kernel(const float *__restrict__ part, int nb, int ncols, int stride, float *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols) return;
    float s = 0.0f;
    for (int b = 0; b < nb; b++) s += part[(int64_t)b * stride + c];
    out[c] = s;
}

__global__ void adam_kernel(float *p, const float *__restrict__ gr, float *m, float *v, int n, float lr, float c1,
                            float c2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float g = gr[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g, vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// rows of the batch: X[b] = Xall[idx(b)], y[b] = yall[idx(b)], idx = (start + b) * P mod n
__global__ void gather_rows_kernel(const bf16 *__restrict__ Xall, const float *__restrict__ yall, int64_t n,
                                   int64_t start, int64_t P, int rows, bf16 *X, float *y) {
    const int b = blockIdx.x;
    if (b >= rows) return;
    const int64_t src = (int64_t)(((uint64_t)(start + b) * (uint64_t)P) % (uint64_t)n);   // < 2^63
    const uint4 *s = reinterpret_cast<const uint4 *>(Xall + src * NIN);
    uint4 *d = reinterpret_cast<uint4 *>(X + (int64_t)b * NIN);
    for (int q = threadIdx.x; q < NIN / 8; q += blockDim.x) d[q] = s[q];
    if (threadIdx.x == 0) y[b] = yall[src];
}

// deterministic compaction of first-hit samples (voxel >= 0), one block
__global__ void __launch_bounds__(1024)
compact_samples_kernel(const int32_t *__restrict__ vox, const float *__restrict__ dir, const float *__restrict__ ao,
                       const float *__restrict__ pos, const float *__restrict__ nrm, int64_t n, int64_t cap,
                       int32_t *ovox, float *odir, float *oao, float *opos, float *onrm, int32_t *oset, int set,
                       unsigned long long *count) {
    __shared__ int wsum[32];
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = *count;
    __syncthreads();
    for (int64_t c0 = 0; c0 < n; c0 += 1024) {
        const int64_t i = c0 + threadIdx.x;
        const int keep = i < n && vox[i] >= 0;
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) wsum[w] = __popc(ball);
        __syncthreads();
        int pre = 0, tot = 0;
        for (int q = 0; q < 32; q++) { if (q < w) pre += wsum[q]; tot += wsum[q]; }
        const unsigned long long at = base + pre + __popc(ball & ((1u << lane) - 1u));
        if (keep && at < (unsigned long long)cap) {
            ovox[at] = vox[i];
            odir[3 * at] = dir[3 * i];
            odir[3 * at + 1] = dir[3 * i + 1];
            odir[3 * at + 2] = dir[3 * i + 2];
            oao[at] = ao[i];
            for (int c = 0; c < 3; c++) {
                opos[3 * at + c] = pos[3 * i + c];
                onrm[3 * at + c] = nrm[3 * i + c];
            }
            oset[at] = set;
        }
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base < (unsigned long long)cap ? base : (unsigned long long)cap;
}

}  // namespace

Net ao_net(const lvr_ao_model *m) {
    Net n;
    n.w1 = (const bf16 *)m->w1b;
    n.w2 = (const bf16 *)m->w2b;
    n.w3 = (const bf16 *)m->w3b;
    n.b1 = m->params + OB1;
    n.b2 = m->params + OB2;
    n.b3 = m->params + OB3;
    n.w4 = m->w4b;
    n.b4 = m->params + OB4;
    const uint32_t *f = (const uint32_t *)m->wfrag;
    n.f1 = reinterpret_cast<const uint2 *>(f);
    n.f2 = reinterpret_cast<const uint4 *>(f + 8 * 32 * 2);
    n.f3 = reinterpret_cast<const uint4 *>(f + 8 * 32 * 2 + 8 * 32 * 8);
    return n;
}

namespace {

lvr_status refresh(lvr_ctx *ctx, lvr_ao_model *m) {
    refresh_kernel<<<64, 256, 0, ctx->stream>>>(m->params, (bf16 *)m->w1b, (bf16 *)m->w2b, (bf16 *)m->w3b, m->w4b);
    frag_kernel<<<1, 256, 0, ctx->stream>>>(m->params, (uint32_t *)m->wfrag);
    for (auto &b : m->bound) b.gen = 0;   // voxel terms depend on W1
    LVR_CUDA(ctx, cudaGetLastError());
    return LVR_OK;
}

lvr_status model_alloc(lvr_ctx *ctx, lvr_ao_model **out) {
    lvr_ao_model *m = new lvr_ao_model();
    m->ctx = ctx;
    lvr_status st;
    if ((st = dev_alloc(ctx, (void **)&m->params, NPARAM * 4)) != LVR_OK ||
        (st = dev_alloc(ctx, &m->w1b, NH * NIN * 2)) != LVR_OK || (st = dev_alloc(ctx, &m->w2b, NH * NH * 2)) != LVR_OK ||
        (st = dev_alloc(ctx, &m->w3b, NH * NH * 2)) != LVR_OK || (st = dev_alloc(ctx, (void **)&m->w4b, NH * 4)) != LVR_OK ||
        (st = dev_alloc(ctx, &m->wfrag, 8 * 32 * 18 * 4)) != LVR_OK) {
        lvr_free_ao_model(m);
        return st;
    }
    *out = m;
    return LVR_OK;
}

// Trainer scratch for one batch of R rows.
struct Work {
    bf16 *X, *H1, *H2, *H3, *dZ1, *dZ2, *dZ3;
    float *y, *Z1, *Z2, *Z3, *dH, *dz4, *part, *split, *pred;
    int splits;
};

lvr_status work_alloc(lvr_ctx *ctx, int R, Work &w, std::vector<void *> &keep) {
    w.splits = R >= 4096 ? 32 : (R >= 1024 ? 8 : 1);
    const size_t rb = (size_t)R;
    const size_t nblk = (rb + EB - 1) / EB + (rb + 63) / 64 + 8;
    struct { void **p; size_t b; } req[] = {
        {(void **)&w.X, rb * NIN * 2}, {(void **)&w.H1, rb * NH * 2}, {(void **)&w.H2, rb * NH * 2},
        {(void **)&w.H3, rb * NH * 2}, {(void **)&w.dZ1, rb * NH * 2}, {(void **)&w.dZ2, rb * NH * 2},
        {(void **)&w.dZ3, rb * NH * 2}, {(void **)&w.y, rb * 4}, {(void **)&w.Z1, rb * NH * 4},
        {(void **)&w.Z2, rb * NH * 4}, {(void **)&w.Z3, rb * NH * 4}, {(void **)&w.dH, rb * NH * 4},
        {(void **)&w.dz4, rb * 4}, {(void **)&w.part, nblk * (NH + 2) * 4},
        {(void **)&w.split, (size_t)w.splits * NH * NIN * 4}, {(void **)&w.pred, rb * 4}};
    for (auto &q : req) {
        lvr_status st = dev_alloc(ctx, q.p, q.b);
        if (st != LVR_OK) return st;
        keep.push_back(*q.p);
    }
    return LVR_OK;
}

void gemm(cudaStream_t s, bool acol, bool bkn, int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb,
          float *C, int splits, float *split_buf) {
    const int kchunk = ((K + splits - 1) / splits + GK - 1) / GK * GK;
    const int nz = (K + kchunk - 1) / kchunk;
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, nz);
    float *dst = nz > 1 ? split_buf : C;
    if (!acol && !bkn) gemm_kernel<false, false><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, dst, kchunk);
    else if (!acol && bkn) gemm_kernel<false, true><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, dst, kchunk);
    else if (acol && bkn) gemm_kernel<true, true><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, dst, kchunk);
    else gemm_kernel<true, false><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, dst, kchunk);
    if (nz > 1) sum_splits_kernel<<<grid1d((int64_t)M * N, 256), 256, 0, s>>>(split_buf, nz, (int64_t)M * N, C);
}

// One forward (and, if `grads`, backward) pass over the R rows in w.X / w.y.
// Returns per-block loss partial sums in w.part (column 0).
void pass(cudaStream_t s, const lvr_ao_model *m, int R, Work &w, float *grads) {
    const float *p = m->params;
    const bf16 *w1b = (const bf16 *)m->w1b, *w2b = (const bf16 *)m->w2b, *w3b = (const bf16 *)m->w3b;
    const unsigned ge = grid1d((int64_t)R * NH, 256) > 4096 ? 4096 : grid1d((int64_t)R * NH, 256);
    // forward: Z = H W^T + b, H' = bf16(ReLU(Z))
    gemm(s, false, false, R, NH, NIN, w.X, NIN, w1b, NIN, w.Z1, 1, nullptr);
    act_kernel<<<ge, 256, 0, s>>>(w.Z1, p + OB1, R, w.H1);
    gemm(s, false, false, R, NH, NH, w.H1, NH, w2b, NH, w.Z2, 1, nullptr);
    act_kernel<<<ge, 256, 0, s>>>(w.Z2, p + OB2, R, w.H2);
    gemm(s, false, false, R, NH, NH, w.H2, NH, w3b, NH, w.Z3, 1, nullptr);
    act_kernel<<<ge, 256, 0, s>>>(w.Z3, p + OB3, R, w.H3);
    const int nb = (R + EB - 1) / EB;
    out_kernel<<<nb, EB, 0, s>>>(w.H3, m->w4b, p + OB4, w.y, R, w.dz4, w.part, w.pred);
    if (!grads) return;
    // output layer gradients: db4, dW4
    colsum_kernel<<<1, 32, 0, s>>>(w.part + 1, nb, 1, 2 + NH, grads + OB4);    // db4 = sum dz4
    colsum_kernel<<<1, 64, 0, s>>>(w.part + 2, nb, NH, 2 + NH, grads + OW4);   // dW4 = H3^T dz4
    const int nb64 = (R + 63) / 64;
    float *bpart = w.part + (size_t)nb * (2 + NH);
    // layer 3: dZ3 = (dz4 w4) * [Z3 > 0]; dW3 = dZ3^T H2; db3
    back_act_kernel<<<nb64, EB, 0, s>>>(nullptr, w.dz4, m->w4b, w.Z3, R, w.dZ3, bpart);
    colsum_kernel<<<1, 64, 0, s>>>(bpart, nb64, NH, NH, grads + OB3);
    gemm(s, true, true, NH, NH, R, w.dZ3, NH, w.H2, NH, grads + OW3, w.splits, w.split);
    // layer 2: dH2 = dZ3 W3; dZ2 = dH2 * [Z2 > 0]; dW2 = dZ2^T H1
    gemm(s, false, true, R, NH, NH, w.dZ3, NH, w3b, NH, w.dH, 1, nullptr);
    back_act_kernel<<<nb64, EB, 0, s>>>(w.dH, nullptr, nullptr, w.Z2, R, w.dZ2, bpart);
    colsum_kernel<<<1, 64, 0, s>>>(bpart, nb64, NH, NH, grads + OB2);
    gemm(s, true, true, NH, NH, R, w.dZ2, NH, w.H1, NH, grads + OW2, w.splits, w.split);
    // layer 1: dH1 = dZ2 W2; dZ1; dW1 = dZ1^T X
    gemm(s, false, true, R, NH, NH, w.dZ2, NH, w2b, NH, w.dH, 1, nullptr);
    back_act_kernel<<<nb64, EB, 0, s>>>(w.dH, nullptr, nullptr, w.Z1, R, w.dZ1, bpart);
    colsum_kernel<<<1, 64, 0, s>>>(bpart, nb64, NH, NH, grads + OB1);
    gemm(s, true, true, NH, NIN, R, w.dZ1, NH, w.X, NIN, grads + OW1, w.splits, w.split);
}

lvr_status adam_step(lvr_ctx *ctx, lvr_ao_model *m, float lr) {
    if (!m->adam_m || !m->adam_v) {   // both moments, zeroed, or neither
        float *mm = nullptr, *vv = nullptr;
        lvr_status st = dev_alloc(ctx, (void **)&mm, NPARAM * 4);
        if (st == LVR_OK) st = dev_alloc(ctx, (void **)&vv, NPARAM * 4);
        cudaError_t e = cudaSuccess;
        if (st == LVR_OK) e = cudaMemsetAsync(mm, 0, NPARAM * 4, ctx->stream);
        if (st == LVR_OK && e == cudaSuccess) e = cudaMemsetAsync(vv, 0, NPARAM * 4, ctx->stream);
        if (st != LVR_OK || e != cudaSuccess) {
            dev_free(ctx, mm);
            dev_free(ctx, vv);
            return st != LVR_OK ? st : cuda_err(ctx, e, "adam moments");
        }
        dev_free(ctx, m->adam_m);
        dev_free(ctx, m->adam_v);
        m->adam_m = mm;
        m->adam_v = vv;
        m->adam_t = 0;
    }
    m->adam_t++;
    const float c1 = 1.0f - powf(0.9f, (float)m->adam_t), c2 = 1.0f - powf(0.999f, (float)m->adam_t);
    adam_kernel<<<64, 256, 0, ctx->stream>>>(m->params, m->grads, m->adam_m, m->adam_v, NPARAM, lr, c1, c2);
    return refresh(ctx, m);
}

// Mean squared error of the last forward pass over R rows (sum of the
// per-block partial sums in fixed order).
lvr_status host_loss(lvr_ctx *ctx, const Work &w, int R, double *mse) {
    const int nb = (R + EB - 1) / EB;
    std::vector<float> part((size_t)nb * (2 + NH));
    LVR_CUDA(ctx, cudaMemcpyAsync(part.data(), w.part, part.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += part[(size_t)b * (2 + NH)];
    *mse = s / R;
    return LVR_OK;
}

// splitmix64: counter-based generator for initial weights and sampling views
uint64_t mix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}
double unit(uint64_t seed, uint64_t i) { return (mix64(seed * 0x100000001b3ull + i) >> 11) * (1.0 / 9007199254740992.0); }

}  // namespace

// ------------------------------------------------------------------ binding the voxel term
// The three levels' input values of a LoD into `buf` (bf16, levels back to back).
static lvr_status make_logd(lvr_ctx *ctx, const lvr_lod *lod, void **buf, size_t *bytes, Logd &L) {
    if (lod->levels < 3) return set_err(ctx, LVR_EINVAL, "learned AO needs a LoD of >= 3 levels");
    size_t off[3], tot = 0;
    int64_t cnt[3];
    for (int l = 0; l < 3; l++) {
        cnt[l] = (int64_t)lod->dims[l][0] * lod->dims[l][1] * lod->dims[l][2];
        L.pitch[l] = (lod->dims[l][0] + 7) & ~7;
        off[l] = tot;
        tot += ((size_t)L.pitch[l] * lod->dims[l][1] * lod->dims[l][2] * 2 + 255) & ~(size_t)255;
        for (int a = 0; a < 3; a++) L.dims[l][a] = lod->dims[l][a];
    }
    if (*bytes < tot) {
        dev_free(ctx, *buf);
        *buf = nullptr;
        *bytes = 0;
        lvr_status st = dev_alloc(ctx, buf, tot);
        if (st != LVR_OK) return st;
        *bytes = tot;
    }
    for (int l = 0; l < 3; l++) {
        bf16 *d = (bf16 *)((char *)*buf + off[l]);
        L.d[l] = d;
        const unsigned g = grid1d(cnt[l], 256) > 8192 ? 8192 : grid1d(cnt[l], 256);
        logd_kernel<<<g, 256, 0, ctx->stream>>>(lod->dens[l], lod->dims[l][0], lod->dims[l][1], cnt[l], L.pitch[l],
                                                1.0f / (float)(1 << (3 * l)), d);
    }
    LVR_CUDA(ctx, cudaGetLastError());
    return LVR_OK;
}

lvr_status ao_bind(lvr_ctx *ctx, lvr_ao_model *m, const lvr_lod *lod, const void **vterm) {
    m->clock++;
    for (auto &b : m->bound)
        if (b.gen == lod->gen && b.vterm) {
            b.used = m->clock;
            *vterm = b.vterm;
            return LVR_OK;
        }
    // an empty entry (the one with the largest buffer), else the least recently used
    lvr_ao_model::Bound *slot = nullptr;
    for (auto &b : m->bound)
        if (b.gen == 0 && (!slot || b.bytes > slot->bytes)) slot = &b;
    if (!slot) {
        slot = &m->bound[0];
        for (auto &b : m->bound)
            if (b.used < slot->used) slot = &b;
    }
    Logd L;
    lvr_status st = make_logd(ctx, lod, &m->logd, &m->logd_bytes, L);
    if (st != LVR_OK) return st;
    const int64_t nvox = (int64_t)lod->dims[0][0] * lod->dims[0][1] * lod->dims[0][2];
    const size_t vb = (size_t)nvox * NH * 2;
    if (slot->bytes < vb) {
        dev_free(ctx, slot->vterm);
        slot->vterm = nullptr;
        slot->bytes = 0;
        slot->gen = 0;
        if ((st = dev_alloc(ctx, &slot->vterm, vb)) != LVR_OK) return st;
        slot->bytes = vb;
    }
    // the coarse levels' terms (fp32, one row of 64 per level-1 and level-2 cell)
    const size_t cb = (size_t)((int64_t)L.dims[1][0] * L.dims[1][1] * L.dims[1][2] +
                               (int64_t)L.dims[2][0] * L.dims[2][1] * L.dims[2][2]) * NH * 4;
    if (m->vcoarse_bytes < cb) {
        dev_free(ctx, m->vcoarse);
        m->vcoarse = nullptr;
        m->vcoarse_bytes = 0;
        if ((st = dev_alloc(ctx, (void **)&m->vcoarse, cb)) != LVR_OK) return st;
        m->vcoarse_bytes = cb;
    }
    const void *ld[3] = {L.d[0], L.d[1], L.d[2]};
    if ((st = ao_vterm_tc(ctx, ld, L.pitch, L.dims, m->vcoarse, m->w1b, slot->vterm)) != LVR_OK) return st;
    if ((st = ao_vterm_tc_status(ctx)) != LVR_OK) return st;
    slot->gen = lod->gen;
    slot->used = m->clock;
    *vterm = slot->vterm;
    return LVR_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" int lvr_ao_nparams(void) { return NPARAM; }

extern "C" lvr_status lvr_ao_model_create(lvr_ctx *ctx, const float *params, lvr_ao_model **out) {
    if (!ctx) return LVR_EINVAL;
    if (!params || !out) return set_err(ctx, LVR_EINVAL, "lvr_ao_model_create: null argument");
    *out = nullptr;
    for (int i = 0; i < NPARAM; i++)
        if (!isfinite(params[i])) return set_err(ctx, LVR_EINVAL, "parameters must be finite");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    lvr_ao_model *m;
    lvr_status st = model_alloc(ctx, &m);
    if (st != LVR_OK) return st;
    cudaError_t e = cudaMemcpyAsync(m->params, params, NPARAM * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
        lvr_free_ao_model(m);
        return cuda_err(ctx, e, "lvr_ao_model_create");
    }
    if ((st = refresh(ctx, m)) != LVR_OK) {
        lvr_free_ao_model(m);
        return st;
    }
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // params came from caller memory
    *out = m;
    return LVR_OK;
}

// Restore a model's training state (lvr_ao_model_set_state): parameters,
// Adam moments and step count; the bf16 copies are refreshed and the cached
// voxel terms dropped.
lvr_status ao_set_state(lvr_ctx *ctx, lvr_ao_model *m, const float *params, const float *am, const float *av,
                        int64_t step) {
    if (!m->adam_m || !m->adam_v) {
        float *mm = nullptr, *vv = nullptr;
        lvr_status st = dev_alloc(ctx, (void **)&mm, NPARAM * 4);
        if (st == LVR_OK) st = dev_alloc(ctx, (void **)&vv, NPARAM * 4);
        if (st != LVR_OK) {
            dev_free(ctx, mm);
            dev_free(ctx, vv);
            return st;
        }
        dev_free(ctx, m->adam_m);
        dev_free(ctx, m->adam_v);
        m->adam_m = mm;
        m->adam_v = vv;
    }
    LVR_CUDA(ctx, cudaMemcpyAsync(m->params, params, NPARAM * 4, cudaMemcpyDefault, ctx->stream));
    LVR_CUDA(ctx, cudaMemcpyAsync(m->adam_m, am, NPARAM * 4, cudaMemcpyDefault, ctx->stream));
    LVR_CUDA(ctx, cudaMemcpyAsync(m->adam_v, av, NPARAM * 4, cudaMemcpyDefault, ctx->stream));
    m->adam_t = step;
    lvr_status st = refresh(ctx, m);
    if (st != LVR_OK) return st;
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // inputs may be caller memory
    return LVR_OK;
}

extern "C" lvr_status lvr_ao_model_params(lvr_ctx *ctx, const lvr_ao_model *m, float *params) {
    if (!ctx) return LVR_EINVAL;
    if (!m || !params) return set_err(ctx, LVR_EINVAL, "lvr_ao_model_params: null argument");
    return copy_out(ctx, params, m->params, NPARAM * 4);
}

extern "C" void lvr_free_ao_model(lvr_ao_model *m) {
    if (!m) return;
    lvr_ctx *ctx = m->ctx;
    cudaSetDevice(ctx->device);
    void *ps[] = {m->params, m->grads, m->adam_m, m->adam_v, m->w1b, m->w2b, m->w3b, m->w4b, m->wfrag, m->logd, m->vcoarse};
    for (void *p : ps) dev_free(ctx, p);
    for (auto &b : m->bound) dev_free(ctx, b.vterm);
    delete m;
}

extern "C" lvr_status lvr_ao_infer(lvr_ctx *ctx, lvr_ao_model *m, const lvr_lod *lod, int64_t n,
                                   const int32_t *voxel, const float *dir, const float *pos, const float *normal,
                                   float *ao) {
    if (!ctx) return LVR_EINVAL;
    if (!m || !lod || n < 0 || (n > 0 && (!voxel || !dir || !pos || !normal || !ao)))
        return set_err(ctx, LVR_EINVAL, "lvr_ao_infer: bad argument");
    if (n == 0) return LVR_OK;
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    const int dx = lod->dims[0][0], dy = lod->dims[0][1];
    const int64_t nvox = (int64_t)dx * dy * lod->dims[0][2];
    const size_t bv = ((size_t)n * 4 + 255) & ~(size_t)255, b3 = ((size_t)n * 12 + 255) & ~(size_t)255;
    lvr_status st;
    if ((st = ensure_stage_in(ctx, bv + 3 * b3)) != LVR_OK) return st;
    const void *dv, *dd, *dp, *dn;
    if ((st = stage_input(ctx, voxel, (size_t)n * 4, 0, &dv)) != LVR_OK) return st;
    if ((st = stage_input(ctx, dir, (size_t)n * 12, bv, &dd)) != LVR_OK) return st;
    if ((st = stage_input(ctx, pos, (size_t)n * 12, bv + b3, &dp)) != LVR_OK) return st;
    if ((st = stage_input(ctx, normal, (size_t)n * 12, bv + 2 * b3, &dn)) != LVR_OK) return st;
    // voxel ids are checked on the host copy when host memory was given; on the
    // device an id out of range gives NaN
    if (!is_device_ptr(voxel))
        for (int64_t i = 0; i < n; i++)
            if (voxel[i] < 0 || voxel[i] >= nvox) return set_err(ctx, LVR_EINVAL, "voxel id out of range");
    const void *vt = nullptr;
    if ((st = ao_bind(ctx, m, lod, &vt)) != LVR_OK) return st;
    const bool host_out = !is_device_ptr(ao);
    float *dout = ao;
    if (host_out) {
        if ((st = ensure_stage_out(ctx, (size_t)n * 4)) != LVR_OK) return st;
        dout = (float *)ctx->stage_out;
    }
    const int64_t tiles = (n + 63) / 64;
    infer_kernel<<<(unsigned)(tiles > 65535 ? 65535 : tiles), 128, 0, ctx->stream>>>(
        ao_net(m), (const bf16 *)vt, dx, dy, nvox, n, (const int32_t *)dv, (const float *)dd,
        (const float *)dp, (const float *)dn, dout);
    LVR_CUDA(ctx, cudaGetLastError());
    if (host_out) return copy_out(ctx, ao, dout, (size_t)n * 4);
    return LVR_OK;
}

extern "C" lvr_status lvr_ao_features(lvr_ctx *ctx, const lvr_lod *lod, int64_t n, const int32_t *voxel,
                                      const float *dir, const float *pos, const float *normal, uint16_t *X) {
    if (!ctx) return LVR_EINVAL;
    if (!lod || n < 0 || (n > 0 && (!voxel || !dir || !pos || !normal || !X)))
        return set_err(ctx, LVR_EINVAL, "lvr_ao_features: bad argument");
    if (n == 0) return LVR_OK;
    if (!is_device_ptr(voxel) || !is_device_ptr(dir) || !is_device_ptr(pos) || !is_device_ptr(normal) ||
        !is_device_ptr(X))
        return set_err(ctx, LVR_EINVAL, "lvr_ao_features takes device buffers");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    void *buf = nullptr;
    size_t bytes = 0;
    Logd L;
    lvr_status st = make_logd(ctx, lod, &buf, &bytes, L);
    if (st == LVR_OK) {
        const unsigned g = grid1d(n * 32, 256) > 65535 ? 65535 : grid1d(n * 32, 256);
        features_kernel<<<g, 256, 0, ctx->stream>>>(L, n, voxel, dir, pos, normal, (bf16 *)X);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_err(ctx, e, "lvr_ao_features");
    }
    dev_free(ctx, buf);
    return st;
}

extern "C" lvr_status lvr_ao_train_step(lvr_ctx *ctx, lvr_ao_model *m, int64_t n, const uint16_t *X, const float *y,
                                        float lr, float *loss, float *grads) {
    if (!ctx) return LVR_EINVAL;
    if (!m || n < 1 || n > (1 << 20) || !X || !y) return set_err(ctx, LVR_EINVAL, "lvr_ao_train_step: bad argument");
    if (!is_device_ptr(X) || !is_device_ptr(y)) return set_err(ctx, LVR_EINVAL, "lvr_ao_train_step takes device X, y");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    lvr_status st;
    if (!m->grads && (st = dev_alloc(ctx, (void **)&m->grads, NPARAM * 4)) != LVR_OK) return st;
    Work w;
    std::vector<void *> keep;
    if ((st = work_alloc(ctx, (int)n, w, keep)) != LVR_OK) {
        for (void *p : keep) dev_free(ctx, p);
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(w.X, X, (size_t)n * NIN * 2, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w.y, y, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        pass(s, m, (int)n, w, m->grads);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) st = cuda_err(ctx, e, "lvr_ao_train_step");
    double mse = 0.0;
    if (st == LVR_OK && loss && (st = host_loss(ctx, w, (int)n, &mse)) == LVR_OK) *loss = (float)mse;
    if (st == LVR_OK && grads) st = copy_out(ctx, grads, m->grads, NPARAM * 4);
    if (st == LVR_OK && lr > 0.0f) st = adam_step(ctx, m, lr);
    for (void *p : keep) dev_free(ctx, p);
    return st;
}

// hit samples of one view with traced AO (render.cu)
lvr_status render_samples(lvr_ctx *ctx, const lvr_lineset *ls, const lvr_lod *lod, const lvr_view *view,
                          const lvr_render_desc *desc, int32_t depth, uint32_t seed, int32_t *vox, float *dir,
                          float *ao, float *pos, float *nrm);

extern "C" lvr_status lvr_train_ao(lvr_ctx *ctx, const lvr_lineset *const *sets, const lvr_lod *const *lods, int nsets,
                                   const lvr_ao_train_desc *td, lvr_ao_model **out, float *final_mse) {
    if (!ctx) return LVR_EINVAL;
    if (!sets || !lods || nsets < 1 || !td || !out) return set_err(ctx, LVR_EINVAL, "lvr_train_ao: null argument");
    *out = nullptr;
    if (td->n_samples < 64 || td->epochs < 1 || td->batch < 64 || td->batch % 64 || td->batch > (1 << 16) ||
        !(td->lr > 0.0f) || td->view_size < 8 || td->view_size > 4096 || !td->render || td->depth < 1)
        return set_err(ctx, LVR_EINVAL, "lvr_train_ao: bad training description");
    for (int i = 0; i < nsets; i++)
        if (!sets[i] || !lods[i]) return set_err(ctx, LVR_EINVAL, "null line set or LoD");
    LVR_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    lvr_status st;
    const int64_t N = td->n_samples;
    const int V = td->view_size;
    // sample buffers
    int32_t *svox = nullptr, *sset = nullptr, *pvox = nullptr;
    float *sdir = nullptr, *sao = nullptr, *spos = nullptr, *snrm = nullptr;
    float *pdir = nullptr, *pao = nullptr, *ppos = nullptr, *pnrm = nullptr;
    bf16 *Xall = nullptr;
    void *logd = nullptr;
    size_t logd_bytes = 0;
    unsigned long long *cnt = ctx->d_u64 + 4;
    std::vector<void *> keep;
    auto A = [&](void **p, size_t b) { st = dev_alloc(ctx, p, b); if (st == LVR_OK) keep.push_back(*p); return st == LVR_OK; };
    auto cleanup = [&]() {
        for (void *p : keep) dev_free(ctx, p);
        dev_free(ctx, logd);
    };
    const size_t VV = (size_t)V * V;
    if (!A((void **)&svox, N * 4) || !A((void **)&sset, N * 4) || !A((void **)&sdir, N * 12) || !A((void **)&sao, N * 4) ||
        !A((void **)&spos, N * 12) || !A((void **)&snrm, N * 12) || !A((void **)&pvox, VV * 4) ||
        !A((void **)&pdir, VV * 12) || !A((void **)&pao, VV * 4) || !A((void **)&ppos, VV * 12) ||
        !A((void **)&pnrm, VV * 12) || !A((void **)&Xall, (size_t)N * NIN * 2)) {
        cleanup();
        return st;
    }
    // 1. samples: hits at random depth with traced AO from seeded orbit views of every set
    const lvr_render_desc &rd = *td->render;
    LVR_CUDA(ctx, cudaMemsetAsync(cnt, 0, 8, s));
    for (int set = 0; set < nsets; set++) {
        const int64_t goal = N * (set + 1) / nsets;
        unsigned long long have = 0;
        for (int v = 0; v < 4096; v++) {
            LVR_CUDA(ctx, cudaMemcpyAsync(&have, cnt, 8, cudaMemcpyDeviceToHost, s));
            LVR_CUDA(ctx, cudaStreamSynchronize(s));
            if ((int64_t)have >= goal) break;
            const lvr_lineset *ls = sets[set];
            const double c[3] = {ls->res[0] / 2.0, ls->res[1] / 2.0, ls->res[2] / 2.0};
            const double half = 0.5 * sqrt((double)ls->res[0] * ls->res[0] + (double)ls->res[1] * ls->res[1] +
                                           (double)ls->res[2] * ls->res[2]);
            const uint64_t key = ((uint64_t)set << 20) | (uint64_t)v;
            const double az = 2.0 * M_PI * unit(td->seed, 2 * key), el = -0.6 + 1.5 * unit(td->seed, 2 * key + 1);
            lvr_view vw;
            memset(&vw, 0, sizeof vw);
            const double d[3] = {cos(el) * cos(az), sin(el), cos(el) * sin(az)};
            for (int a = 0; a < 3; a++) {
                vw.eye[a] = (float)(c[a] + 1.8 * half * d[a]);
                vw.at[a] = (float)c[a];
            }
            vw.up[1] = 1.0f;
            vw.fovy_deg = 40.0f;
            vw.width = vw.height = V;
            vw.light_dir[1] = -1.0f;
            const uint32_t vseed = (uint32_t)mix64(td->seed ^ (key * 0x2545f4914f6cdd1dull));
            if ((st = render_samples(ctx, ls, lods[set], &vw, &rd, td->depth, vseed, pvox, pdir, pao, ppos, pnrm)) != LVR_OK) {
                cleanup();
                return st;
            }
            compact_samples_kernel<<<1, 1024, 0, s>>>(pvox, pdir, pao, ppos, pnrm, (int64_t)VV, goal, svox, sdir, sao,
                                                      spos, snrm, sset, set, cnt);
            LVR_CUDA(ctx, cudaGetLastError());
        }
        if ((int64_t)have < goal) {
            cleanup();
            return set_err(ctx, LVR_EINVAL, "line set %d: too few hits to collect samples", set);
        }
        // 2. features of this set's samples (its own LoD)
        const int64_t lo = N * set / nsets;
        Logd L;
        if ((st = make_logd(ctx, lods[set], &logd, &logd_bytes, L)) != LVR_OK) { cleanup(); return st; }
        const int64_t ns = goal - lo;
        features_kernel<<<grid1d(ns * 32, 256) > 65535 ? 65535 : grid1d(ns * 32, 256), 256, 0, s>>>(
            L, ns, svox + lo, sdir + 3 * lo, spos + 3 * lo, snrm + 3 * lo, Xall + lo * NIN);
        LVR_CUDA(ctx, cudaGetLastError());
    }
    // 3. model: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases
    std::vector<float> p0(NPARAM);
    for (int i = 0; i < NPARAM; i++) {
        const int fan = i < OW2 ? NIN : NH;
        p0[i] = (float)((2.0 * unit(td->seed ^ 0x5eedull, (uint64_t)i) - 1.0) / sqrt((double)fan));
    }
    for (int f = 0; f < NH; f++) {   // padding inputs
        p0[OW1 + f * NIN + NHIT] = 0.0f;
        for (int k = VOFF + NVIN; k < NIN; k++) p0[OW1 + f * NIN + k] = 0.0f;
    }
    lvr_ao_model *m;
    if ((st = lvr_ao_model_create(ctx, p0.data(), &m)) != LVR_OK) { cleanup(); return st; }
    if ((st = dev_alloc(ctx, (void **)&m->grads, NPARAM * 4)) != LVR_OK) { lvr_free_ao_model(m); cleanup(); return st; }
    // 4. epochs of Adam over minibatches; rows in a stride permutation per epoch
    const int R = td->batch;
    Work w;
    if ((st = work_alloc(ctx, R, w, keep)) != LVR_OK) { lvr_free_ao_model(m); cleanup(); return st; }
    const int64_t steps = (N + R - 1) / R;
    static const int64_t primes[] = {1000003, 2000003, 3000017, 4000037, 5000011, 6000011, 7000003, 8000009};
    const double total = (double)steps * td->epochs;
    for (int ep = 0; ep < td->epochs; ep++) {
        int64_t P = primes[ep % 8];
        while (std::gcd(P, N) != 1) P += 2;
        for (int64_t it = 0; it < steps; it++) {
            // step size: cosine decay from lr to 0 over all steps
            const double k = (double)(ep * steps + it) / total;
            const float lr = (float)(td->lr * 0.5 * (1.0 + cos(M_PI * k)));
            gather_rows_kernel<<<R, 32, 0, s>>>(Xall, sao, N, it * R + ep * 7919, P, R, w.X, w.y);
            pass(s, m, R, w, m->grads);
            if ((st = adam_step(ctx, m, lr)) != LVR_OK) { lvr_free_ao_model(m); cleanup(); return st; }
        }
        LVR_CUDA(ctx, cudaGetLastError());
    }
    // 5. final mean squared error over all samples (forward only)
    double se = 0.0;
    for (int64_t b = 0; b < N; b += R) {
        const int rows = (int)(N - b < R ? N - b : R);
        gather_rows_kernel<<<rows, 32, 0, s>>>(Xall, sao, N, b, 1, rows, w.X, w.y);
        pass(s, m, rows, w, nullptr);
        double mse = 0.0;
        if ((st = host_loss(ctx, w, rows, &mse)) != LVR_OK) { lvr_free_ao_model(m); cleanup(); return st; }
        se += mse * rows;
    }
    if (final_mse) *final_mse = (float)(se / N);
    cleanup();
    LVR_CUDA(ctx, cudaStreamSynchronize(s));
    *out = m;
    return LVR_OK;
}
