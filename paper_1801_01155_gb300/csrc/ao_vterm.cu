// Learned AO: the per-voxel part of layer 1 (the "voxel term") on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// The voxel term of voxel v sums W1[f][k] x_v[k] over the 375 per-voxel
// inputs: for each LoD level l the 5^3 cells around v's level-l cell. It is
// a sum of three 5^3-tap convolutions with 64 outputs,
//   vterm[v] = bf16( T0[v] + T1[v >> 1] + T2[v >> 2] ),
//   T_l[c][f] = sum_{n in 5^3} W1[f][16 + 125 l + n] x_l[c + offset(n)],
// and T1, T2 depend only on the level-1 / level-2 cell, so they are computed
// once per coarse cell (fp32) and added where the level-0 term is finished.
//
// One persistent kernel per level, from the coarsest: level 2 stores T2,
// level 1 stores T1 + T2 of its parent, level 0 finishes the voxel term. A
// tile is 128 consecutive cells of one x-row (M = 128), N = 64 outputs, and
// the K dimension runs over the 25 (dz, dy) offsets (padded to 32) for each
// of the 5 dx offsets:
//  - TMA (cp.async.bulk.tensor.3d) loads the tile's halo, x0 - 8 .. x0 + 135
//    by y - 2 .. y + 2 by z - 2 .. z + 2, of a bf16 copy of the level whose
//    rows are padded to 16 bytes (cells outside the level read zero) into one
//    of two shared buffers; the next tile's halo is in flight meanwhile.
//  - The block rearranges the halo into R[g][r][j] = x(x0 - 2 + r, y + dy,
//    z + dz) for (dz, dy) = pair 8 g + j, r = 0 .. 135: K-major 16-byte rows
//    (8 pairs) at a 16-byte stride, which is the MMA operand layout without
//    swizzle with 8-row groups 128 bytes apart. The A operand of offset dx
//    is then R itself seen from row dx: its descriptor starts 16 dx bytes
//    further, so no tap is copied five times.
//  - One thread issues ten tcgen05.mma (5 dx offsets x 2 steps of K = 16;
//    M 128, N 64; bf16 in, fp32 accumulation in tensor memory) against the
//    weights, loaded once in the same layout, and commits them to an mbarrier.
//  - Each warp reads its 32 accumulator rows (tcgen05.ld), adds the coarser
//    levels' term of the parent cell and stores bf16 (level 0) or fp32.
// Every wait is bounded (2 s): a wait that runs out sets the status word,
// and the block waits (bounded) for its own copy and MMA in flight, frees
// its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "ao_mlp.cuh"
#include "lvr_internal.cuh"

namespace {

typedef __nv_bfloat16 bf16;
using aomlp::NH;
using aomlp::NIN;
using aomlp::VOFF;

constexpr int TM = 128;                   // cells per tile (MMA M)
constexpr int HX = TM + 16;               // halo row: x0 - 8 .. x0 + 135
constexpr int HALO = HX * 25;             // halo elements (y and z: 5 each)
constexpr int HALO_BYTES = HALO * 2;      // 7200, the TMA transaction size
constexpr int RROWS = TM + 8;             // rows of R: x0 - 2 .. x0 + 133 (132 used)
constexpr int RG = 4;                     // 16-byte groups of (dz, dy) pairs: 25 used of 32
constexpr int RG_BYTES = RROWS * 16;      // 2176
constexpr int OFF_R = 0;                                       // 8.5 KB
constexpr int OFF_B = OFF_R + RG * RG_BYTES;                   // 5 x 4 KB of weights
constexpr int B_DX_BYTES = RG * NH * 16;
constexpr int OFF_H = OFF_B + 5 * B_DX_BYTES;                  // 2 x halo
constexpr int HALO_STRIDE = (HALO_BYTES + 127) & ~127;
constexpr int OFF_BAR = OFF_H + 2 * HALO_STRIDE;               // 3 mbarriers
constexpr int OFF_TMEM = OFF_BAR + 32;
constexpr int SMEM_BYTES = OFF_TMEM + 16;
constexpr int BLOCKS_PER_SM = 5;
constexpr uint32_t TMEM_COLS = 64;        // the fp32 accumulator, 128 lanes x 64 columns
constexpr uint32_t VT_TIMEOUT = 1u << 4;  // status bit: a bounded wait ran out

struct ConvArgs {
    int dx, dy, dz;            // the level's cells
    int level;                 // 0, 1, 2: weight columns 16 + 125 level .. + 124
    const bf16 *w1b;           // bf16 W1, [64][400]
    float *tout;               // levels 1, 2: fp32 [cells][64]
    bf16 *vterm;               // level 0: bf16 [voxels][64]
    const float *tadd;         // levels 0, 1: the next level's term (fp32 [parent cells][64])
    int dp[3];                 // its cells
    uint32_t *status;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the mbarrier, at most 2 s.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    if (bar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (bar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
}

__device__ __forceinline__ void tma_halo(uint32_t dst, const CUtensorMap *tm, int x, int y, int z, uint32_t bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(HALO_BYTES) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle; lbo = byte step
// between the two 8-element K halves of an MMA's K = 16, sbo = byte step
// between 8-row groups; bits 46-47 = 1 (the tcgen05 descriptor version).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator (bits 4-5 = 1), bf16 A
// and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NH >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}


// 32 bytes to a 32-byte aligned global address in one store.
__device__ __forceinline__ void st_global_256(void *p, const uint32_t w[8]) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                 "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

template <bool FINAL>
__global__ void __launch_bounds__(128, BLOCKS_PER_SM) vterm_conv_kernel(const __grid_constant__ CUtensorMap tm, const ConvArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    bf16 *Rt = reinterpret_cast<bf16 *>(smem + OFF_R);
    bf16 *B = reinterpret_cast<bf16 *>(smem + OFF_B);
    const uint32_t bar_h[2] = {smem_addr(smem + OFF_BAR), smem_addr(smem + OFF_BAR + 8)};
    const uint32_t bar_mma = smem_addr(smem + OFF_BAR + 16);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + OFF_TMEM);
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (a.dx + TM - 1) / TM;
    const int64_t ntiles = (int64_t)ntx * a.dy * a.dz;

    if (tid == 0) {
        abort_flag = 0;
        for (int i = 0; i < 3; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(smem + OFF_BAR + 8 * i)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // weights of this level, per dx offset: B_dx[g][n][j] = W1[n][16 + 125 level + tap], tap = dx +
    // 5 dy + 25 dz for (dz, dy) = pair 8 g + j (zero beyond the 25 pairs)
    const bf16 *w = a.w1b + VOFF + 125 * a.level;
    for (int i = tid; i < 5 * RG * NH; i += blockDim.x) {
        const int n = i % NH, g = (i / NH) % RG, dx = i / (NH * RG);
        alignas(16) bf16 v[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const int p = 8 * g + j;
            v[j] = p < 25 ? w[n * NIN + dx + 5 * (p % 5) + 25 * (p / 5)] : __float2bfloat16_rn(0.0f);
        }
        *reinterpret_cast<uint4 *>(B + ((dx * RG + g) * NH + n) * 8) = *reinterpret_cast<const uint4 *>(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    auto tile_xyz = [&](int64_t t, int &x0, int &y, int &z) {
        x0 = (int)(t % ntx) * TM;
        y = (int)((t / ntx) % a.dy);
        z = (int)(t / ((int64_t)ntx * a.dy));
    };
    auto issue = [&](int64_t t, int buf) {
        int x0, y, z;
        tile_xyz(t, x0, y, z);
        tma_halo(smem_addr(smem + OFF_H + buf * HALO_STRIDE), &tm, x0 - 8, y - 2, z - 2, bar_h[buf]);
    };
    int64_t pending_tma = -1;   // the halo copy in flight (iteration index), for the abort path
    if (tid == 0 && blockIdx.x < ntiles) {
        issue(blockIdx.x, 0);
        pending_tma = 0;
    }
    int it = 0;
    bool mma_pending = false;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, it++) {
        const int buf = it & 1;
        if (tid == 0 && t + gridDim.x < ntiles) {
            issue(t + gridDim.x, buf ^ 1);   // its previous reader finished before the last barrier
            pending_tma = it + 1;
        }
        int x0, y, z;
        tile_xyz(t, x0, y, z);
        if (!bar_wait(bar_h[buf], (uint32_t)(it >> 1) & 1u)) abort_flag = 1;
        if (tid == 0 && pending_tma == it) pending_tma = -1;
        // R[g][r][j] = halo(x0 - 2 + r, pair 8 g + j), zero beyond the 25 pairs; rows 0 .. 131 (the
        // MMAs of offsets 0 .. 4 read rows dx .. dx + 127); x0 - 2 + r is halo column r + 6
        const bf16 *H = reinterpret_cast<const bf16 *>(smem + OFF_H + buf * HALO_STRIDE);
        for (int i = tid; i < RG * (TM + 4); i += blockDim.x) {
            const int r = i % (TM + 4), g = i / (TM + 4);
            alignas(16) bf16 v[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int p = 8 * g + j;
                v[j] = p < 25 ? H[p * HX + r + 6] : __float2bfloat16_rn(0.0f);
            }
            *reinterpret_cast<uint4 *>(Rt + (g * RROWS + r) * 8) = *reinterpret_cast<const uint4 *>(v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (abort_flag) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t r0 = smem_addr(Rt), b0 = smem_addr(B);
            // A of offset dx: R from row dx; K step s: pair groups 2 s, 2 s + 1 (lbo = group stride,
            // sbo = 128 bytes between 8-row groups); B of offset dx: its 4 KB block
#pragma unroll
            for (int dx = 0; dx < 5; dx++)
#pragma unroll
                for (int st = 0; st < 2; st++)
                    mma_bf16(tmem, smem_desc(r0 + (uint32_t)(2 * st * RG_BYTES + 16 * dx), RG_BYTES, 128),
                             smem_desc(b0 + (uint32_t)(dx * B_DX_BYTES + 2 * st * NH * 16), NH * 16, 128),
                             (dx | st) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_mma)
                         : "memory");
        }
        mma_pending = true;
        if (!bar_wait(bar_mma, (uint32_t)it & 1u)) abort_flag = 1;
        __syncthreads();
        if (abort_flag) break;
        mma_pending = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp w holds accumulator rows 32 w .. 32 w + 31 (tensor-memory lanes)
        const int m = warp * 32 + lane, x = x0 + m;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        const bool in = x < a.dx;
        const int64_t cell = x + (int64_t)a.dx * (y + (int64_t)a.dy * z);
        // the coarser levels' term of the parent cell, all 64 values requested before the first is used
        float4 add[NH / 4];
        const float4 *pa = (in && a.tadd)
                               ? reinterpret_cast<const float4 *>(
                                     a.tadd + ((x >> 1) + (int64_t)a.dp[0] * ((y >> 1) + (int64_t)a.dp[1] * (z >> 1))) * NH)
                               : nullptr;
#pragma unroll
        for (int q = 0; q < NH / 4; q++) add[q] = pa ? __ldg(pa + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < NH; c += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)c, v);
            if (!in) continue;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float4 u = add[c / 4 + q];
                v[4 * q] += u.x;
                v[4 * q + 1] += u.y;
                v[4 * q + 2] += u.z;
                v[4 * q + 3] += u.w;
            }
            // one 32-byte store per whole sector (a lane's row is 128 or 256 bytes, 32-byte aligned)
            if constexpr (FINAL) {
                uint32_t o[8];
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                    o[q] = *reinterpret_cast<const uint32_t *>(&h);
                }
                st_global_256(a.vterm + cell * NH + c, o);
            } else {
                st_global_256(a.tout + cell * NH + c, reinterpret_cast<const uint32_t *>(v));
                st_global_256(a.tout + cell * NH + c + 8, reinterpret_cast<const uint32_t *>(v + 8));
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (abort_flag) {
        // a wait ran out: let this block's own copy and MMA in flight land
        // (bounded) before its shared and tensor memory are given back
        if (tid == 0) {
            atomicOr(a.status, VT_TIMEOUT);
            if (pending_tma >= 0) bar_wait(bar_h[pending_tma & 1], (uint32_t)(pending_tma >> 1) & 1u);
            if (mma_pending) bar_wait(bar_mma, (uint32_t)it & 1u);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiled)p;
    }
    return fn;
}

}  // namespace

// The voxel term of every level-0 voxel (see the top of this file).
// logd[l]: bf16 log-density of level l, rows of pitch[l] elements (a multiple
// of 8, 16-byte aligned); dims[l]: its cells; coarse: fp32 scratch of
// (cells of level 1 + cells of level 2) x 64; w1b: bf16 W1 [64][400].
lvr_status ao_vterm_tc(lvr_ctx *ctx, const void *const logd[3], const int pitch[3], const int dims[3][3],
                       float *coarse, const void *w1b, void *vterm) {
    EncodeTiled enc = encoder();
    if (!enc) return set_err(ctx, LVR_ECUDA, "voxel term: cuTensorMapEncodeTiled is not available");
    static bool attr_set[64] = {};
    int dev = ctx->device, sms = 0;
    LVR_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        LVR_CUDA(ctx, cudaFuncSetAttribute(vterm_conv_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        LVR_CUDA(ctx, cudaFuncSetAttribute(vterm_conv_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr_set[dev] = true;
    }
    const int64_t c1 = (int64_t)dims[1][0] * dims[1][1] * dims[1][2];
    float *T[3] = {nullptr, coarse, coarse + c1 * NH};   // level 1 holds T1 + T2 of its parent
    uint32_t *status = ctx->d_status + 3;
    LVR_CUDA(ctx, cudaMemsetAsync(status, 0, 4, ctx->stream));
    for (int l = 2; l >= 0; l--) {
        CUtensorMap tm;
        const cuuint64_t gdim[3] = {(cuuint64_t)dims[l][0], (cuuint64_t)dims[l][1], (cuuint64_t)dims[l][2]};
        const cuuint64_t gstr[2] = {(cuuint64_t)pitch[l] * 2, (cuuint64_t)pitch[l] * dims[l][1] * 2};
        const cuuint32_t box[3] = {(cuuint32_t)HX, 5, 5}, est[3] = {1, 1, 1};
        const CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(logd[l]), gdim, gstr, box, est,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return set_err(ctx, LVR_ECUDA, "voxel term: tensor map of level %d refused (%d)", l, (int)r);
        ConvArgs a;
        a.dx = dims[l][0];
        a.dy = dims[l][1];
        a.dz = dims[l][2];
        a.level = l;
        a.w1b = (const bf16 *)w1b;
        a.tout = T[l];
        a.vterm = (bf16 *)vterm;
        a.tadd = l < 2 ? T[l + 1] : nullptr;
        for (int k = 0; k < 3; k++) a.dp[k] = l < 2 ? dims[l + 1][k] : 0;
        a.status = status;
        const int64_t ntiles = (int64_t)((a.dx + TM - 1) / TM) * a.dy * a.dz;
        const int64_t grid = ntiles < (int64_t)sms * BLOCKS_PER_SM ? ntiles : (int64_t)sms * BLOCKS_PER_SM;
        if (grid < 1) continue;
        if (l == 0) vterm_conv_kernel<true><<<(unsigned)grid, 128, SMEM_BYTES, ctx->stream>>>(tm, a);
        else vterm_conv_kernel<false><<<(unsigned)grid, 128, SMEM_BYTES, ctx->stream>>>(tm, a);
        LVR_CUDA(ctx, cudaGetLastError());
    }
    return LVR_OK;
}

// Status of the last ao_vterm_tc (synchronises the stream): LVR_ETIMEOUT when
// a bounded wait inside it ran out.
lvr_status ao_vterm_tc_status(lvr_ctx *ctx) {
    uint32_t *h = (uint32_t *)ctx->h_pinned;
    LVR_CUDA(ctx, cudaMemcpyAsync(h, ctx->d_status + 3, 4, cudaMemcpyDeviceToHost, ctx->stream));
    LVR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (h[0] & VT_TIMEOUT) return set_err(ctx, LVR_ETIMEOUT, "voxel term: a tensor-core pipeline wait ran out");
    return LVR_OK;
}
