// cnn.cu -- a10 learned clutter filter: a 4-layer 3D convolutional network
// (2 -> 32 -> 32 -> 32 -> 2 channels, 5 frames x 3 x 3 pixel kernels, zero
// "same" padding, ReLU between layers) applied to the normalised IQ
// ensemble, its training step (forward, backward, Adam) and the power
// Doppler of its output.  The paper proposes filters learned from simulated
// ensembles as future work (Sec. 1, Sec. 4); this is that filter's hot path.
//
// Layout: activations channels-last, [N][F][Z][X][32] BF16 (the 2-channel
// input and output are zero-padded to 32 channels, so every layer is one
// shape).  Forward convolution = implicit GEMM on the tcgen05 tensor cores:
// one CTA tile is 128 voxels (4 depth rows x 32 lateral pixels of one
// frame) x 32 output channels; K runs over 45 taps x 32 input channels.
// For each tap one TMA box load at the tap-shifted coordinates brings the
// 128 x 64-byte operand rows into shared memory (64-byte swizzle; the
// tensor map's zero fill outside the volume is the "same" padding; the
// innermost coordinate is always channel 0, so every load is aligned).  The
// 45 weight tiles (32 x 32 BF16 each, 90 KB) stay resident in shared memory
// for the CTA's lifetime.  Two MMAs of K = 16 per tap accumulate in FP32 in
// tensor memory; two accumulator buffers let the epilogue of one tile
// overlap the MMAs of the next.  Epilogues: bias + ReLU -> BF16, bias ->
// FP32 (last layer), or gradient x ReLU mask -> BF16 (backward).
//
// The data gradient of a layer is the same convolution with the kernel
// flipped in all three axes and its channel roles swapped; the weight
// gradient (a reduction over voxels) runs on the CUDA cores in FP32.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>

#include "fq_internal.cuh"
#include "tc.cuh"

using namespace fqtc;

namespace {

constexpr int C = 32;                 // channels of every activation tensor
constexpr int NTAP = 45;              // 5 x 3 x 3
constexpr int TILE_M = 128;           // voxels per tile: 4 depth rows x 32 lateral
constexpr int TILE_Z = 4, TILE_X = 32;
constexpr int ROWB = C * 2;           // 64 bytes per operand row
constexpr int A_BYTES = TILE_M * ROWB;        // 8 KB per tap stage
constexpr int W_TAP_BYTES = C * ROWB;         // 2 KB per tap
constexpr int W_BYTES = NTAP * W_TAP_BYTES;   // 90 KB
constexpr int STAGES = 6;
constexpr int CONV_THREADS = 192;     // warp 0 TMA, warp 1 MMA + TMEM owner, warps 2-5 epilogue
constexpr int TMEM_COLS = 64;         // two 32-column FP32 accumulators
constexpr int CONV_SMEM = W_BYTES + STAGES * A_BYTES + 1024;

// instruction descriptor: FP32 D, BF16 A and B, both K-major, N = 32, M = 128
constexpr uint32_t kConvIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(C >> 3) << 17) |
                                ((uint32_t)(TILE_M >> 4) << 24);

enum Epi { EPI_RELU_BF16 = 0, EPI_LINEAR_F32 = 1, EPI_MASK_BF16 = 2 };

__host__ __device__ constexpr int tap_dt(int t) { return t / 9 - 2; }
__host__ __device__ constexpr int tap_dz(int t) { return (t / 3) % 3 - 1; }
__host__ __device__ constexpr int tap_dx(int t) { return t % 3 - 1; }

struct ConvDims {
    int N, F, Z, X;
    int tiles;         // N F (Z / 4) (X / 32)
};

__device__ __forceinline__ void tile_coords(const ConvDims &d, int tile, int &n, int &f, int &z0, int &x0)
{
    const int xb = d.X / TILE_X, zb = d.Z / TILE_Z;
    int r = tile;
    const int bx = r % xb; r /= xb;
    const int bz = r % zb; r /= zb;
    f = r % d.F;
    n = r / d.F;
    z0 = bz * TILE_Z;
    x0 = bx * TILE_X;
}

__device__ __forceinline__ void mma_bf16_n32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kConvIdesc), "r"(accumulate)
        : "memory");
}

// Epilogue of one accumulator row (32 channels of voxel `vox`).
template <int EPI>
__device__ __forceinline__ void epilogue_store(const float (&v)[32], const float *s_bias, int64_t vox, void *out,
                                               const __nv_bfloat16 *mask)
{
    if (EPI == EPI_LINEAR_F32) {
        float4 *o = reinterpret_cast<float4 *>((float *)out + vox * C);
#pragma unroll
        for (int i = 0; i < 8; ++i)
            o[i] = make_float4(v[4 * i] + s_bias[4 * i], v[4 * i + 1] + s_bias[4 * i + 1],
                               v[4 * i + 2] + s_bias[4 * i + 2], v[4 * i + 3] + s_bias[4 * i + 3]);
    } else {
        float m[32];
        if (EPI == EPI_MASK_BF16) {
            const uint4 *mp = reinterpret_cast<const uint4 *>(mask + vox * C);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                uint4 u = mp[i];
                const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float2 fl = __bfloat1622float2(h[k]);
                    m[8 * i + 2 * k] = fl.x;
                    m[8 * i + 2 * k + 1] = fl.y;
                }
            }
        }
        uint4 packed[4];
        __nv_bfloat162 *pb = reinterpret_cast<__nv_bfloat162 *>(packed);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float a0 = v[2 * k], a1 = v[2 * k + 1];
            if (EPI == EPI_RELU_BF16) {
                a0 = fmaxf(a0 + s_bias[2 * k], 0.0f);
                a1 = fmaxf(a1 + s_bias[2 * k + 1], 0.0f);
            } else {
                a0 = m[2 * k] > 0.0f ? a0 : 0.0f;
                a1 = m[2 * k + 1] > 0.0f ? a1 : 0.0f;
            }
            pb[k] = __floats2bfloat162_rn(a0, a1);
        }
        uint4 *o = reinterpret_cast<uint4 *>((__nv_bfloat16 *)out + vox * C);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = packed[i];
    }
}

template <int EPI>
__global__ void __launch_bounds__(CONV_THREADS, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap in_map, const __grid_constant__ CUtensorMap w_map,
                   const ConvDims d, const float *__restrict__ bias, void *__restrict__ out,
                   const __nv_bfloat16 *__restrict__ mask, int *__restrict__ status)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *w_s = base;                 // 45 weight tiles
    unsigned char *a_s = base + W_BYTES;       // STAGES operand stages
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_full[2], acc_empty[2], w_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ float s_bias[C];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        mbar_init(&w_bar, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < C) s_bias[threadIdx.x] = bias ? bias[threadIdx.x] : 0.0f;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer: the weights once, then one stage per (tile, tap)
            mbar_expect_tx(&w_bar, W_BYTES);
            for (int t = 0; t < NTAP; ++t) tma_load_2d(w_s + t * W_TAP_BYTES, &w_map, &w_bar, 0, t * C);
            int it = 0;
            bool fail = false;
            for (int tile = blockIdx.x; tile < d.tiles && !fail; tile += gridDim.x) {
                int n, f, z0, x0;
                tile_coords(d, tile, n, f, z0, x0);
                for (int t = 0; t < NTAP; ++t, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!mbar_wait(&empty_bar[s], ph ^ 1u)) { fail = true; break; }
                    mbar_expect_tx(&full_bar[s], A_BYTES);
                    tma_load_5d(a_s + s * A_BYTES, &in_map, &full_bar[s], 0, x0 + tap_dx(t), z0 + tap_dz(t),
                                f + tap_dt(t), n);
                }
            }
            if (fail) {
                s_fail = 1;
                // let the copies already issued land before the CTA can exit
                for (int k = 1; k <= STAGES && it - k >= 0; ++k) {
                    const int j = it - k;
                    mbar_wait(&full_bar[j % STAGES], (uint32_t)(j / STAGES) & 1u);
                }
                mbar_wait(&w_bar, 0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer
            bool fail = !mbar_wait(&w_bar, 0);
            tc_fence_after();
            int it = 0, j = 0;
            for (int tile = blockIdx.x; tile < d.tiles && !fail; tile += gridDim.x, ++j) {
                const int buf = j & 1;
                if (!mbar_wait(&acc_empty[buf], (((uint32_t)j >> 1) & 1u) ^ 1u)) { fail = true; break; }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(buf * C);
                for (int t = 0; t < NTAP; ++t, ++it) {
                    const int s = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!mbar_wait(&full_bar[s], ph)) { fail = true; break; }
                    tc_fence_after();
                    const uint64_t ad = sw64_desc(smem_u32(a_s + s * A_BYTES));
                    const uint64_t bd = sw64_desc(smem_u32(w_s + t * W_TAP_BYTES));
                    mma_bf16_n32(acc, ad, bd, t > 0 ? 1u : 0u);
                    mma_bf16_n32(acc, ad + 2, bd + 2, 1u);  // second 16 channels: +32 bytes
                    mma_commit(&empty_bar[s]);
                }
                if (fail) break;
                mma_commit(&acc_full[buf]);
            }
            if (fail) s_fail = 1;
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = depth row w % 4 of the tile
        const int q = warp & 3;
        int j = 0;
        for (int tile = blockIdx.x; tile < d.tiles; tile += gridDim.x, ++j) {
            const int buf = j & 1;
            if (!warp_wait(&acc_full[buf], ((uint32_t)j >> 1) & 1u)) {
                if (lane == 0) s_fail = 1;
                break;
            }
            tc_fence_after();
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * C), v);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
            int n, f, z0, x0;
            tile_coords(d, tile, n, f, z0, x0);
            const int64_t vox = (((int64_t)n * d.F + f) * d.Z + (z0 + q)) * d.X + x0 + lane;
            epilogue_store<EPI>(v, s_bias, vox, out, mask);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(status, (int)FQ_ERR_TIMEOUT);
}

// ------------------------------------------------- frame-ring convolution --
// For volumes whose width X is a multiple of 128: a tile is 128 pixels of
// one depth row of one frame.  A CTA takes work units (n, depth row z,
// 128-pixel block, run of up to RING_FCH frames) and walks the frames of a
// unit in order.  Input frames live in a ring of 5 shared-memory slots; one
// slot holds rows z - 1 .. z + 1 x pixels x0 - 1 .. x0 + 128 of one frame
// in 4 chunks of 8 channels, each chunk a [3][130] array of 16-byte rows
// (one TMA box per chunk; zero fill outside the volume).  In this
// no-swizzle K-major layout rows sit 16 bytes apart, so the operand of tap
// (dt, dz, dx) is the slot of frame f + dt at row offset (1 + dz) 130 +
// 1 + dx: each tap is a descriptor, and each output frame loads one new
// input frame (25 KB) instead of 45 shifted tiles.  The MMA thread issues
// the dt = -2 taps first and then frees that frame's slot, so the next
// frame's load overlaps the remaining 36 taps.
constexpr int RING_X = 128;
constexpr int RING_W = RING_X + 2;                  // with the lateral halo
constexpr int RING_BOX = 3 * RING_W * 16;          // 6240 bytes: one TMA box (3 rows x 130 pixels x 8 channels)
constexpr int RING_CHUNK = 6272;                    // the box's stride in a slot, padded to a multiple of 128
constexpr int RING_SLOT = 4 * RING_CHUNK;           // 25088 bytes
constexpr int RING_SLOTS = 5;
constexpr int RING_FCH = 32;                        // frames per work unit
constexpr int RING_SMEM = W_BYTES + RING_SLOTS * RING_SLOT + 1024;

// K-major shared-memory matrix descriptor without swizzle: 8-row core
// matrices of 16-byte rows; `lbo` = bytes between core matrices along K,
// `sbo` = bytes between 8-row groups.
__device__ __forceinline__ uint64_t nosw_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; layout type 0 = no swizzle
    return d;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

struct RingUnit {
    int n, z, x0, fa, fb;
};

__device__ __forceinline__ RingUnit ring_unit(const ConvDims &d, int u)
{
    const int nfc = (d.F + RING_FCH - 1) / RING_FCH, nxb = d.X / RING_X;
    RingUnit r;
    const int fc = u % nfc;
    u /= nfc;
    r.x0 = (u % nxb) * RING_X;
    u /= nxb;
    r.z = u % d.Z;
    r.n = u / d.Z;
    r.fa = fc * RING_FCH;
    r.fb = min(d.F, r.fa + RING_FCH);
    return r;
}

__device__ __forceinline__ int ring_slot(int g) { return (g + 10) % RING_SLOTS; }  // g >= -2

template <int EPI>
__global__ void __launch_bounds__(CONV_THREADS, 1)
    conv_ring_kernel(const __grid_constant__ CUtensorMap in_map, const __nv_bfloat16 *__restrict__ wchunk,
                     const ConvDims d, int units, const float *__restrict__ bias, void *__restrict__ out,
                     const __nv_bfloat16 *__restrict__ mask, int *__restrict__ status)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *w_s = base;
    unsigned char *ring = base + W_BYTES;
    __shared__ __align__(8) uint64_t slot_full[RING_SLOTS], slot_free[RING_SLOTS], acc_full[2], acc_empty[2], w_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ float s_bias[C];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < RING_SLOTS; ++s) {
            mbar_init(&slot_full[s], 1);
            mbar_init(&slot_free[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        mbar_init(&w_bar, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < C) s_bias[threadIdx.x] = bias ? bias[threadIdx.x] : 0.0f;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            // ---- producer: weights once, then the frames of each unit in order.
            // Per slot: bit s of `loaded` = the slot has been filled before,
            // bit s of `par` = parity of its fill count.
            mbar_expect_tx(&w_bar, W_BYTES);
            bulk_load(w_s, wchunk, W_BYTES, &w_bar);
            uint32_t loaded = 0, par = 0;
            bool fail = false;
            for (int u = blockIdx.x; u < units && !fail; u += gridDim.x) {
                const RingUnit r = ring_unit(d, u);
                for (int g = r.fa - 2; g <= r.fb + 1; ++g) {
                    const int s = ring_slot(g);
                    // the previous fill of this slot has count parity par ^ 1 ... its release phase
                    if (((loaded >> s) & 1u) && !mbar_wait(&slot_free[s], ((par >> s) & 1u) ^ 1u)) {
                        fail = true;
                        break;
                    }
                    mbar_expect_tx(&slot_full[s], 4 * RING_BOX);
                    unsigned char *dst = ring + s * RING_SLOT;
                    for (int k = 0; k < 4; ++k)
                        tma_load_5d(dst + k * RING_CHUNK, &in_map, &slot_full[s], 8 * k, r.x0 - 1, r.z - 1, g, r.n);
                    loaded |= 1u << s;
                    par ^= 1u << s;
                }
            }
            if (fail) {
                s_fail = 1;
                for (int s = 0; s < RING_SLOTS; ++s)  // let issued copies land
                    if ((loaded >> s) & 1u) mbar_wait(&slot_full[s], ((par >> s) & 1u) ^ 1u);
                mbar_wait(&w_bar, 0);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer.  Descriptors: one base per operand array; a tap's
            // operand is the base plus its byte offset / 16 in the start-address
            // field (addresses stay below 256 KB, so the field never carries).
            bool fail = !mbar_wait(&w_bar, 0);
            tc_fence_after();
            uint32_t wpar = 0;  // bit s: parity of the waits on slot s so far
            int j = 0;
            const uint64_t ring_d = nosw_desc(smem_u32(ring), RING_CHUNK, 128);
            const uint64_t w_d = nosw_desc(smem_u32(w_s), C * 16, 128);
            for (int u = blockIdx.x; u < units && !fail; u += gridDim.x) {
                const RingUnit r = ring_unit(d, u);
                for (int f = r.fa; f < r.fb && !fail; ++f, ++j) {
                    const int buf = j & 1;
                    if (!mbar_wait(&acc_empty[buf], (((uint32_t)j >> 1) & 1u) ^ 1u)) { fail = true; break; }
                    tc_fence_after();
                    const uint32_t acc = tmem + (uint32_t)(buf * C);
#pragma unroll
                    for (int dt = -2; dt <= 2; ++dt) {
                        const int s = ring_slot(f + dt);
                        if (f == r.fa || dt == 2) {  // first use of frame f + dt in this unit
                            if (!mbar_wait(&slot_full[s], (wpar >> s) & 1u)) { fail = true; break; }
                            wpar ^= 1u << s;
                            tc_fence_after();
                        }
                        const uint64_t a0 = ring_d + (uint64_t)((s * RING_SLOT) >> 4);
#pragma unroll
                        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                            for (int dx = -1; dx <= 1; ++dx) {
                                const int t = (dt + 2) * 9 + (dz + 1) * 3 + (dx + 1);
                                const uint64_t ad = a0 + (uint64_t)((((1 + dz) * RING_W + 1 + dx) * 16) >> 4);
                                const uint64_t bd = w_d + (uint64_t)((t * W_TAP_BYTES) >> 4);
                                mma_bf16_n32(acc, ad, bd, t > 0 ? 1u : 0u);
                                mma_bf16_n32(acc, ad + (uint64_t)((2 * RING_CHUNK) >> 4),
                                             bd + (uint64_t)((2 * C * 16) >> 4), 1u);
                            }
                        if (dt == -2) mma_commit(&slot_free[ring_slot(f - 2)]);  // its last use
                    }
                    if (fail) break;
                    mma_commit(&acc_full[buf]);
                }
                if (fail) break;
                for (int g = r.fb - 2; g <= r.fb + 1; ++g) mma_commit(&slot_free[ring_slot(g)]);
            }
            if (fail) s_fail = 1;
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = pixels x0 + 32 (w % 4) + lane
        const int q = warp & 3;
        int j = 0;
        bool stop = false;
        for (int u = blockIdx.x; u < units && !stop; u += gridDim.x) {
            const RingUnit r = ring_unit(d, u);
            for (int f = r.fa; f < r.fb; ++f, ++j) {
                const int buf = j & 1;
                if (!warp_wait(&acc_full[buf], ((uint32_t)j >> 1) & 1u)) {
                    if (lane == 0) s_fail = 1;
                    stop = true;
                    break;
                }
                tc_fence_after();
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * C), v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[buf]);
                const int64_t vox = (((int64_t)r.n * d.F + f) * d.Z + r.z) * d.X + r.x0 + q * 32 + lane;
                epilogue_store<EPI>(v, s_bias, vox, out, mask);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(status, (int)FQ_ERR_TIMEOUT);
}

// ------------------------------------------------------------ small kernels --
// Master FP32 weights [45][32 in][32 out] -> BF16 tap tiles for the forward
// pass (rows = out channel, 32 in channels each) and for the data gradient
// (kernel flipped in all three axes: tap 44 - t; rows = in channel).
// The chunked images hold the same tiles as [tap][K chunk of 8][row][8]
// (16-byte core-matrix rows) for the frame-ring kernel.
__global__ void pack_weights_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wf,
                                    __nv_bfloat16 *__restrict__ wb, __nv_bfloat16 *__restrict__ wfc,
                                    __nv_bfloat16 *__restrict__ wbc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NTAP * C * C) return;
    const int t = i / (C * C), ci = (i / C) % C, co = i % C;
    const __nv_bfloat16 v = __float2bfloat16_rn(w[i]);
    const int tb = NTAP - 1 - t;
    wf[((size_t)t * C + co) * C + ci] = v;
    wb[((size_t)tb * C + ci) * C + co] = v;
    wfc[(((size_t)t * 4 + ci / 8) * C + co) * 8 + ci % 8] = v;
    wbc[(((size_t)tb * 4 + co / 8) * C + ci) * 8 + co % 8] = v;
}

// Packing of a Casorati ensemble [P][F][2] (pixel p = x + X z) for the
// network.  Pass 1 (one thread per pixel): the pixel's temporal mean (when
// removing it) and its sum of squared deviations, accumulated per CTA.
__global__ void casorati_stats_kernel(const float *__restrict__ iq, int F, int64_t P, int remove_mean,
                                      float2 *__restrict__ mean, double *__restrict__ part)
{
    __shared__ double red[8];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double ss = 0.0;
    if (p < P) {
        const float2 *s = reinterpret_cast<const float2 *>(iq) + p * F;
        float mr = 0.0f, mi = 0.0f;
        if (remove_mean) {
            for (int f = 0; f < F; ++f) {
                mr += s[f].x;
                mi += s[f].y;
            }
            mr /= (float)F;
            mi /= (float)F;
        }
        mean[p] = make_float2(mr, mi);
        for (int f = 0; f < F; ++f) {
            const float a = s[f].x - mr, b = s[f].y - mi;
            ss += (double)a * a + (double)b * b;
        }
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// scale = 1 / RMS of the deviations over the whole ensemble (real and
// imaginary parts counted separately), into *scale.
__global__ void casorati_scale_kernel(const double *__restrict__ part, int n, int64_t count, float *__restrict__ scale)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *scale = s > 0.0 ? (float)(1.0 / sqrt(s / (double)count)) : 1.0f;
}

// Pass 2 (one thread per pixel, frames in turn): (s - mean) * scale * gain
// into the BF16 volume [F][Z][X][32] (channels 0, 1; the rest 0) and / or
// the FP32 target [F][Z][X][2].
__global__ void casorati_pack_kernel(const float *__restrict__ iq, int F, int64_t P, const float2 *__restrict__ mean,
                                     const float *__restrict__ scale, float gain, __nv_bfloat16 *__restrict__ vol,
                                     float *__restrict__ tgt)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const float g = *scale * gain;
    const float2 m = mean[p];
    const float2 *s = reinterpret_cast<const float2 *>(iq) + p * F;
    for (int f = 0; f < F; ++f) {
        const float a = (s[f].x - m.x) * g, b = (s[f].y - m.y) * g;
        const int64_t i = (int64_t)f * P + p;
        if (vol) {
            uint4 out[4] = {};
            reinterpret_cast<__nv_bfloat162 *>(out)[0] = __floats2bfloat162_rn(a, b);
            uint4 *o = reinterpret_cast<uint4 *>(vol + i * C);
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = out[k];
        }
        if (tgt) reinterpret_cast<float2 *>(tgt)[i] = make_float2(a, b);
    }
}

// MSE loss of channels 0, 1 of y [V][32] against t [V][2]: gradient
// 2 (y - t) / (2 V) into dy [V][32] BF16 (other channels 0) and per-block
// partial sums of the squared error.
__global__ void mse_grad_kernel(const float *__restrict__ y, const float *__restrict__ t, int64_t V,
                                __nv_bfloat16 *__restrict__ dy, double *__restrict__ part)
{
    __shared__ double red[8];
    const float inv = 1.0f / (float)(2 * V);
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const float e0 = y[v * C] - t[2 * v], e1 = y[v * C + 1] - t[2 * v + 1];
        acc += (double)e0 * e0 + (double)e1 * e1;
        uint4 out[4] = {};
        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(out);
        h[0] = __floats2bfloat162_rn(2.0f * e0 * inv, 2.0f * e1 * inv);
        uint4 *o = reinterpret_cast<uint4 *>(dy + v * C);
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = out[k];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void sum_parts_kernel(const double *__restrict__ part, int n, int64_t count, float *__restrict__ loss)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *loss = (float)(s / (double)count);
}

// Weight gradient partials: dW[t][ci][co] = sum_v x[v + d_t][ci] dy[v][co]
// over one chunk of voxels per CTA (256 threads, 4 outputs each), FP32.
constexpr int kWgChunk = 4096;  // voxels per CTA
constexpr int kWgSub = 64;      // voxels per shared-memory step

__global__ void __launch_bounds__(256) wgrad_kernel(const __nv_bfloat16 *__restrict__ x,
                                                    const __nv_bfloat16 *__restrict__ dy, ConvDims d,
                                                    float *__restrict__ part)
{
    __shared__ float xs[kWgSub][C + 1], gs[kWgSub][C + 1];
    const int t = blockIdx.y;
    const int dt = tap_dt(t), dz = tap_dz(t), dx = tap_dx(t);
    const int64_t V = (int64_t)d.N * d.F * d.Z * d.X;
    const int64_t v0 = (int64_t)blockIdx.x * kWgChunk;
    const int ci = threadIdx.x >> 3, co0 = (threadIdx.x & 7) * 4;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t vb = v0; vb < v0 + kWgChunk && vb < V; vb += kWgSub) {
        for (int i = threadIdx.x; i < kWgSub * C; i += 256) {
            const int r = i / C, c = i % C;
            const int64_t v = vb + r;
            float xv = 0.0f, gv = 0.0f;
            if (v < V) {
                gv = __bfloat162float(dy[v * C + c]);
                const int xx = (int)(v % d.X), zz = (int)((v / d.X) % d.Z), ff = (int)((v / ((int64_t)d.X * d.Z)) % d.F);
                const int64_t nn = v / ((int64_t)d.X * d.Z * d.F);
                const int sx = xx + dx, sz = zz + dz, sf = ff + dt;
                if (sx >= 0 && sx < d.X && sz >= 0 && sz < d.Z && sf >= 0 && sf < d.F)
                    xv = __bfloat162float(x[((((int64_t)nn * d.F + sf) * d.Z + sz) * d.X + sx) * C + c]);
            }
            xs[r][c] = xv;
            gs[r][c] = gv;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < kWgSub; ++r) {
            const float a = xs[r][ci];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = fmaf(a, gs[r][co0 + k], acc[k]);
        }
        __syncthreads();
    }
    float *o = part + ((size_t)blockIdx.x * NTAP + t) * C * C + ci * C + co0;
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = acc[k];
}

// Sum the chunk partials into dW [45][32][32]; block NTAP also forms
// db[co] = sum_v dy[v][co].
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int n_chunks, const __nv_bfloat16 *__restrict__ dy,
                                    int64_t V, float *__restrict__ dw, float *__restrict__ db)
{
    if (blockIdx.x < NTAP) {
        const int t = blockIdx.x;
        for (int i = threadIdx.x; i < C * C; i += blockDim.x) {
            float s = 0.0f;
            for (int c = 0; c < n_chunks; ++c) s += part[((size_t)c * NTAP + t) * C * C + i];
            dw[(size_t)t * C * C + i] = s;
        }
        return;
    }
    __shared__ float red[8][C + 1];
    float acc = 0.0f;
    const int co = threadIdx.x % C, lane_v = threadIdx.x / C;  // 8 voxel lanes per channel
    for (int64_t v = lane_v; v < V; v += blockDim.x / C) acc += __bfloat162float(dy[v * C + co]);
    red[lane_v][co] = acc;
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0.0f;
        for (int k = 0; k < (int)(blockDim.x / C); ++k) s += red[k][threadIdx.x];
        db[threadIdx.x] = s;
    }
}

// Adam on a flat FP32 parameter array.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// PD of the network output y [F][Z][X][32] (channels 0, 1): mean over
// frames of |y|^2, divided by scale^2 (undoing the input normalisation).
__global__ void cnn_pd_kernel(const float *__restrict__ y, int F, int Z, int X, float inv_scale2, float *__restrict__ pd)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)Z * X) return;
    float s = 0.0f;
    for (int f = 0; f < F; ++f) {
        const float *q = y + ((int64_t)f * Z * X + p) * C;
        s += q[0] * q[0] + q[1] * q[1];
    }
    pd[p] = s / (float)F * inv_scale2;
}

// ------------------------------------------------------------------- host --
struct ParamLayout {   // offsets in floats inside the parameter block
    size_t w[4], b[4], m, v, n_train;  // master weights/biases, then Adam m and v over the same span
    size_t wf_bytes_off, wb_bytes_off;   // 64-byte-row tap tiles (per-tap kernel)
    size_t wfc_bytes_off, wbc_bytes_off; // 16-byte-chunk tap tiles (frame-ring kernel)
    size_t total_bytes;
};

ParamLayout param_layout()
{
    ParamLayout L;
    size_t o = 0;
    for (int l = 0; l < 4; ++l) { L.w[l] = o; o += (size_t)NTAP * C * C; }
    for (int l = 0; l < 4; ++l) { L.b[l] = o; o += C; }
    L.n_train = o;
    L.m = o; o += L.n_train;
    L.v = o; o += L.n_train;
    size_t bytes = (o * 4 + 255) & ~(size_t)255;
    L.wf_bytes_off = bytes; bytes += (size_t)4 * NTAP * C * C * 2;
    L.wb_bytes_off = bytes; bytes += (size_t)4 * NTAP * C * C * 2;
    L.wfc_bytes_off = bytes; bytes += (size_t)4 * NTAP * C * C * 2;
    L.wbc_bytes_off = bytes; bytes += (size_t)4 * NTAP * C * C * 2;
    L.total_bytes = bytes;
    return L;
}

struct ActLayout {
    size_t act[3], out, dy[2], part, loss_part, total;
    int wg_chunks;
};

ActLayout act_layout(int N, int F, int Z, int X)
{
    ActLayout L;
    const size_t V = (size_t)N * F * Z * X;
    size_t o = 0;
    for (int i = 0; i < 3; ++i) { L.act[i] = o; o += (V * C * 2 + 255) & ~(size_t)255; }
    L.out = o; o += (V * C * 4 + 255) & ~(size_t)255;
    for (int i = 0; i < 2; ++i) { L.dy[i] = o; o += (V * C * 2 + 255) & ~(size_t)255; }
    L.wg_chunks = (int)((V + kWgChunk - 1) / kWgChunk);
    L.part = o; o += ((size_t)L.wg_chunks * NTAP * C * C * 4 + 255) & ~(size_t)255;
    L.loss_part = o; o += 1024 * 8;
    L.total = o;
    return L;
}

fq_status encode_act_map(CUtensorMap *map, const void *p, int N, int F, int Z, int X, bool ring)
{
    auto enc = (PFN_cuTensorMapEncodeTiled_v12000)fqi::tensor_map_encoder_ptr();
    FQ_REQUIRE(enc, FQ_ERR_CUDA, "cnn: cuTensorMapEncodeTiled unavailable");
    std::memset(map, 0, sizeof *map);
    cuuint64_t dims[5] = {(cuuint64_t)C, (cuuint64_t)X, (cuuint64_t)Z, (cuuint64_t)F, (cuuint64_t)N};
    cuuint64_t strides[4] = {(cuuint64_t)C * 2, (cuuint64_t)X * C * 2, (cuuint64_t)Z * X * C * 2,
                             (cuuint64_t)F * Z * X * C * 2};
    // per-tap kernel: 32 channels x 32 pixels x 4 rows, 64-byte swizzle;
    // frame-ring kernel: 8 channels x 130 pixels x 3 rows, no swizzle
    cuuint32_t box_tap[5] = {(cuuint32_t)C, (cuuint32_t)TILE_X, (cuuint32_t)TILE_Z, 1, 1};
    cuuint32_t box_ring[5] = {8, (cuuint32_t)RING_W, 3, 1, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(p), dims, strides,
                     ring ? box_ring : box_tap, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     ring ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    FQ_REQUIRE(r == CUDA_SUCCESS, FQ_ERR_CUDA, "cnn: activation tensor map (%d)", (int)r);
    return FQ_OK;
}

fq_status encode_w_map(CUtensorMap *map, const void *p)
{
    auto enc = (PFN_cuTensorMapEncodeTiled_v12000)fqi::tensor_map_encoder_ptr();
    FQ_REQUIRE(enc, FQ_ERR_CUDA, "cnn: cuTensorMapEncodeTiled unavailable");
    std::memset(map, 0, sizeof *map);
    cuuint64_t dims[2] = {(cuuint64_t)C, (cuuint64_t)NTAP * C};
    cuuint64_t strides[1] = {(cuuint64_t)C * 2};
    cuuint32_t box[2] = {(cuuint32_t)C, (cuuint32_t)C};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(p), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    FQ_REQUIRE(r == CUDA_SUCCESS, FQ_ERR_CUDA, "cnn: weight tensor map (%d)", (int)r);
    return FQ_OK;
}

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    return sms;
}

// One convolution of layer `layer` (forward or data-gradient kernel): the
// frame-ring kernel when the width is a multiple of 128, else the per-tap one.
fq_status conv(int epi, const void *in, const void *params, int layer, bool backward, const float *bias, void *out,
               const __nv_bfloat16 *mask, const ConvDims &d, int *status, cudaStream_t st)
{
    const ParamLayout L = param_layout();
    const char *pb = (const char *)params;
    const size_t lo = (size_t)layer * NTAP * C * C * 2;
    const bool ring = d.X % RING_X == 0;
    CUtensorMap in_map;
    fq_status s = encode_act_map(&in_map, in, d.N, d.F, d.Z, d.X, ring);
    if (s) return s;
    if (ring) {
        const __nv_bfloat16 *wc = (const __nv_bfloat16 *)(pb + (backward ? L.wbc_bytes_off : L.wfc_bytes_off) + lo);
        const int units = d.N * d.Z * (d.X / RING_X) * ((d.F + RING_FCH - 1) / RING_FCH);
        const int grid = units < num_sms() ? units : num_sms();
        auto launch = [&](auto kern) -> fq_status {
            fq_status r = fqi::cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               RING_SMEM), "cnn: smem attribute");
            if (r) return r;
            kern<<<grid, CONV_THREADS, RING_SMEM, st>>>(in_map, wc, d, units, bias, out, mask, status);
            return fqi::launch_check("cnn: conv (frame ring)");
        };
        if (epi == EPI_RELU_BF16) return launch(conv_ring_kernel<EPI_RELU_BF16>);
        if (epi == EPI_LINEAR_F32) return launch(conv_ring_kernel<EPI_LINEAR_F32>);
        return launch(conv_ring_kernel<EPI_MASK_BF16>);
    }
    CUtensorMap w_map;
    s = encode_w_map(&w_map, pb + (backward ? L.wb_bytes_off : L.wf_bytes_off) + lo);
    if (s) return s;
    const int grid = d.tiles < num_sms() ? d.tiles : num_sms();
    auto launch = [&](auto kern) -> fq_status {
        fq_status r = fqi::cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           CONV_SMEM), "cnn: smem attribute");
        if (r) return r;
        kern<<<grid, CONV_THREADS, CONV_SMEM, st>>>(in_map, w_map, d, bias, out, mask, status);
        return fqi::launch_check("cnn: conv");
    };
    if (epi == EPI_RELU_BF16) return launch(conv_tc_kernel<EPI_RELU_BF16>);
    if (epi == EPI_LINEAR_F32) return launch(conv_tc_kernel<EPI_LINEAR_F32>);
    return launch(conv_tc_kernel<EPI_MASK_BF16>);
}

fq_status check_dims(int N, int F, int Z, int X, const char *who)
{
    FQ_REQUIRE(N >= 1 && F >= 1 && Z >= 1 && X >= TILE_X, FQ_ERR_SHAPE, "%s: bad volume size", who);
    FQ_REQUIRE(X % RING_X == 0 || (Z % TILE_Z == 0 && X % TILE_X == 0), FQ_ERR_SHAPE,
               "%s: X must be a multiple of 128, or of 32 with Z a multiple of 4 (got Z %d, X %d)", who, Z, X);
    FQ_REQUIRE((int64_t)N * F * (Z / TILE_Z) * (X / TILE_X) < ((int64_t)1 << 31), FQ_ERR_SHAPE, "%s: too many tiles",
               who);
    return FQ_OK;
}

ConvDims make_dims(int N, int F, int Z, int X)
{
    ConvDims d;
    d.N = N; d.F = F; d.Z = Z; d.X = X;
    d.tiles = N * F * (Z / TILE_Z) * (X / TILE_X);
    return d;
}

}  // namespace

extern "C" {

size_t fq_cnn_param_bytes(void) { return param_layout().total_bytes; }

size_t fq_cnn_prep_bytes(int32_t Z, int32_t X)
{
    const int64_t P = (int64_t)Z * X;
    const int64_t blocks = (P + 255) / 256;
    return (((size_t)P * 8 + 255) & ~(size_t)255) + (size_t)blocks * 8 + 256;
}

size_t fq_cnn_act_bytes(int32_t n_vol, int32_t F, int32_t Z, int32_t X)
{
    if (n_vol < 1 || F < 1 || Z < 1 || X < 1) return 0;
    return act_layout(n_vol, F, Z, X).total;
}

fq_status fq_cnn_pack(void *params, void *stream)
{
    FQ_REQUIRE(params && fqi::aligned(params, 256), FQ_ERR_INVALID_ARG, "fq_cnn_pack: null or unaligned params");
    const ParamLayout L = param_layout();
    cudaStream_t st = (cudaStream_t)stream;
    float *pf = (float *)params;
    char *pb = (char *)params;
    for (int l = 0; l < 4; ++l) {
        __nv_bfloat16 *wf = (__nv_bfloat16 *)(pb + L.wf_bytes_off) + (size_t)l * NTAP * C * C;
        __nv_bfloat16 *wb = (__nv_bfloat16 *)(pb + L.wb_bytes_off) + (size_t)l * NTAP * C * C;
        __nv_bfloat16 *wfc = (__nv_bfloat16 *)(pb + L.wfc_bytes_off) + (size_t)l * NTAP * C * C;
        __nv_bfloat16 *wbc = (__nv_bfloat16 *)(pb + L.wbc_bytes_off) + (size_t)l * NTAP * C * C;
        pack_weights_kernel<<<(NTAP * C * C + 255) / 256, 256, 0, st>>>(pf + L.w[l], wf, wb, wfc, wbc);
    }
    return fqi::launch_check("fq_cnn_pack");
}

fq_status fq_cnn_from_casorati(const float *iq, int32_t F, int32_t Z, int32_t X, int32_t remove_mean,
                               const float *scale_in, float *scale_out, float gain, void *vol, float *target,
                               void *workspace, size_t workspace_bytes, void *stream)
{
    FQ_REQUIRE(iq && (vol || target) && F >= 1 && Z >= 1 && X >= 1 && workspace, FQ_ERR_INVALID_ARG,
               "fq_cnn_from_casorati: bad arguments");
    FQ_REQUIRE(scale_in || scale_out, FQ_ERR_INVALID_ARG, "fq_cnn_from_casorati: needs scale_in or scale_out");
    FQ_REQUIRE(fqi::aligned(iq, 8) && fqi::aligned(vol, 16) && fqi::aligned(target, 8) &&
                   fqi::aligned(workspace, 256),
               FQ_ERR_ALIGN, "fq_cnn_from_casorati: alignment");
    const int64_t P = (int64_t)Z * X;
    const int blocks = (int)((P + 255) / 256);
    const size_t need = fq_cnn_prep_bytes(Z, X);
    FQ_REQUIRE(workspace_bytes >= need, FQ_ERR_WORKSPACE, "fq_cnn_from_casorati: workspace needs %zu bytes", need);
    float2 *mean = (float2 *)workspace;
    double *part = (double *)((char *)workspace + (((size_t)P * 8 + 255) & ~(size_t)255));
    cudaStream_t st = (cudaStream_t)stream;
    casorati_stats_kernel<<<blocks, 256, 0, st>>>(iq, F, P, remove_mean, mean, part);
    const float *scale = scale_in;
    if (!scale_in) {
        casorati_scale_kernel<<<1, 32, 0, st>>>(part, blocks, 2 * P * F, scale_out);
        scale = scale_out;
    }
    casorati_pack_kernel<<<blocks, 256, 0, st>>>(iq, F, P, mean, scale, gain, (__nv_bfloat16 *)vol, target);
    return fqi::launch_check("fq_cnn_from_casorati");
}

fq_status fq_cnn_conv(int32_t mode, const void *in, const void *params, int32_t layer, int32_t backward,
                      void *out, const void *mask, int32_t n_vol, int32_t F, int32_t Z, int32_t X, int32_t *status,
                      void *stream)
{
    fq_status s = check_dims(n_vol, F, Z, X, "fq_cnn_conv");
    if (s) return s;
    FQ_REQUIRE(in && params && out && status && layer >= 0 && layer < 4 && mode >= 0 && mode <= 2 &&
                   (mode != EPI_MASK_BF16 || mask),
               FQ_ERR_INVALID_ARG, "fq_cnn_conv: bad arguments");
    FQ_REQUIRE(fqi::aligned(in, 16) && fqi::aligned(out, 16) && fqi::aligned(mask, 16) && fqi::aligned(params, 256),
               FQ_ERR_ALIGN, "fq_cnn_conv: alignment");
    const ParamLayout L = param_layout();
    const float *bias = backward ? nullptr : (const float *)params + L.b[layer];
    return conv(mode, in, params, layer, backward != 0, bias, out, (const __nv_bfloat16 *)mask,
                make_dims(n_vol, F, Z, X), (int *)status, (cudaStream_t)stream);
}

fq_status fq_cnn_forward(const void *params, const void *vol, int32_t n_vol, int32_t F, int32_t Z, int32_t X,
                         void *acts, size_t act_bytes, int32_t *status, void *stream)
{
    fq_status s = check_dims(n_vol, F, Z, X, "fq_cnn_forward");
    if (s) return s;
    const ActLayout A = act_layout(n_vol, F, Z, X);
    FQ_REQUIRE(params && vol && acts && status, FQ_ERR_INVALID_ARG, "fq_cnn_forward: null argument");
    FQ_REQUIRE(act_bytes >= A.total, FQ_ERR_WORKSPACE, "fq_cnn_forward: activations need %zu bytes", A.total);
    FQ_REQUIRE(fqi::aligned(acts, 256) && fqi::aligned(vol, 16) && fqi::aligned(params, 256), FQ_ERR_ALIGN,
               "fq_cnn_forward: alignment");
    const ParamLayout L = param_layout();
    char *ab = (char *)acts;
    const ConvDims d = make_dims(n_vol, F, Z, X);
    cudaStream_t st = (cudaStream_t)stream;
    const void *in = vol;
    for (int l = 0; l < 4; ++l) {
        const float *bias = (const float *)params + L.b[l];
        void *out = l < 3 ? (void *)(ab + A.act[l]) : (void *)(ab + A.out);
        s = conv(l < 3 ? EPI_RELU_BF16 : EPI_LINEAR_F32, in, params, l, false, bias, out, nullptr, d, (int *)status,
                 st);
        if (s) return s;
        in = out;
    }
    return FQ_OK;
}

fq_status fq_cnn_backward(const void *params, const void *vol, const float *target, int32_t n_vol, int32_t F,
                          int32_t Z, int32_t X, void *acts, size_t act_bytes, float *grads, float *loss,
                          int32_t *status, void *stream)
{
    fq_status s = check_dims(n_vol, F, Z, X, "fq_cnn_backward");
    if (s) return s;
    const ActLayout A = act_layout(n_vol, F, Z, X);
    FQ_REQUIRE(params && vol && target && acts && grads && loss && status, FQ_ERR_INVALID_ARG,
               "fq_cnn_backward: null argument");
    FQ_REQUIRE(act_bytes >= A.total, FQ_ERR_WORKSPACE, "fq_cnn_backward: activations need %zu bytes", A.total);
    const ParamLayout L = param_layout();
    char *ab = (char *)acts;
    const ConvDims d = make_dims(n_vol, F, Z, X);
    const int64_t V = (int64_t)n_vol * F * Z * X;
    cudaStream_t st = (cudaStream_t)stream;
    const __nv_bfloat16 *act_in[4] = {(const __nv_bfloat16 *)vol, (const __nv_bfloat16 *)(ab + A.act[0]),
                                      (const __nv_bfloat16 *)(ab + A.act[1]), (const __nv_bfloat16 *)(ab + A.act[2])};
    __nv_bfloat16 *dy[2] = {(__nv_bfloat16 *)(ab + A.dy[0]), (__nv_bfloat16 *)(ab + A.dy[1])};
    double *lp = (double *)(ab + A.loss_part);
    int lb = (int)((V + 255) / 256);
    if (lb > 1024) lb = 1024;
    mse_grad_kernel<<<lb, 256, 0, st>>>((const float *)(ab + A.out), target, V, dy[0], lp);
    sum_parts_kernel<<<1, 32, 0, st>>>(lp, lb, 2 * V, loss);
    s = fqi::launch_check("fq_cnn_backward: loss");
    if (s) return s;
    int cur = 0;
    for (int l = 3; l >= 0; --l) {
        // weight and bias gradients of layer l from its input and output gradient
        dim3 g((unsigned)A.wg_chunks, NTAP);
        float *part = (float *)(ab + A.part);
        wgrad_kernel<<<g, 256, 0, st>>>(act_in[l], dy[cur], d, part);
        wgrad_reduce_kernel<<<NTAP + 1, 256, 0, st>>>(part, A.wg_chunks, dy[cur], V, grads + L.w[l], grads + L.b[l]);
        s = fqi::launch_check("fq_cnn_backward: weight gradient");
        if (s) return s;
        if (l == 0) break;
        // data gradient through layer l, masked by the ReLU of layer l - 1
        s = conv(EPI_MASK_BF16, dy[cur], params, l, true, nullptr, dy[cur ^ 1], act_in[l], d, (int *)status, st);
        if (s) return s;
        cur ^= 1;
    }
    return FQ_OK;
}

fq_status fq_cnn_adam(void *params, const float *grads, float lr, int32_t step, void *stream)
{
    FQ_REQUIRE(params && grads && step >= 1 && lr > 0.0f, FQ_ERR_INVALID_ARG, "fq_cnn_adam: bad arguments");
    const ParamLayout L = param_layout();
    float *pf = (float *)params;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, step)));
    cudaStream_t st = (cudaStream_t)stream;
    adam_kernel<<<152 * 4, 256, 0, st>>>(pf, grads, pf + L.m, pf + L.v, (int64_t)L.n_train, lr, b1, b2, eps, c1, c2);
    fq_status s = fqi::launch_check("fq_cnn_adam");
    if (s) return s;
    return fq_cnn_pack(params, stream);
}

fq_status fq_cnn_power_doppler(const float *out, int32_t F, int32_t Z, int32_t X, float scale, float *pd,
                               void *stream)
{
    FQ_REQUIRE(out && pd && F >= 1 && Z >= 1 && X >= 1 && scale > 0.0f, FQ_ERR_INVALID_ARG,
               "fq_cnn_power_doppler: bad arguments");
    const int64_t P = (int64_t)Z * X;
    cnn_pd_kernel<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(out, F, Z, X,
                                                                                 1.0f / (scale * scale), pd);
    return fqi::launch_check("fq_cnn_power_doppler");
}

size_t fq_cnn_act_offset(int32_t which, int32_t n_vol, int32_t F, int32_t Z, int32_t X)
{
    if (n_vol < 1 || F < 1 || Z < 1 || X < 1 || which < 0 || which > 3) return (size_t)-1;
    const ActLayout A = act_layout(n_vol, F, Z, X);
    return which < 3 ? A.act[which] : A.out;
}

size_t fq_cnn_param_offset(int32_t what, int32_t layer)
{
    const ParamLayout L = param_layout();
    if (layer < 0 || layer > 3) return (size_t)-1;
    switch (what) {
    case 0: return L.w[layer] * 4;
    case 1: return L.b[layer] * 4;
    case 2: return L.m * 4;
    case 3: return L.v * 4;
    case 4: return L.n_train * 4;
    default: return (size_t)-1;
    }
}

}  // extern "C"
