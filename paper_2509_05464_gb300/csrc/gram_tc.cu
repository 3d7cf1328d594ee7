// gram_tc.cu -- a6 Casorati Gram on the tcgen05 tensor cores (BF16 or TF32
// operands, FP32 accumulation in tensor memory).
//
// G = S^H S for the complex Casorati matrix S (P x F) is the real product
// Gr = X^T X of X = S viewed as a real P x 2F matrix (interleaved re, im
// columns): Re G_ij = Gr[2i][2j] + Gr[2i+1][2j+1] and
// Im G_ij = Gr[2i][2j+1] - Gr[2i+1][2j].
//
// Steps: (1) transpose X into a K-major copy Xt[2F][Pp] of the operand type
// (pixels contiguous, zero-padded to a multiple of 64; FP32 inputs are
// rounded to BF16 or to TF32 here); (2) one CTA per (128 x 256 output tile,
// pixel chunk), upper tiles only: a TMA producer thread streams one
// 128-byte swizzle row per operand row (64 BF16 or 32 TF32 pixels) through
// a 4-stage mbarrier ring, one thread issues tcgen05.mma (M = 128, N = 256,
// 32 bytes of K per instruction) into a 256-column TMEM accumulator, and
// four warps read the accumulator back with tcgen05.ld into FP32 partial
// tiles; (3) a reduction over pixel chunks that also forms the complex G,
// the lower triangle from the upper one by Hermitian symmetry.  Every
// mbarrier wait is bounded (about 2 s of global time); on expiry the CTA
// records FQ_ERR_TIMEOUT in the status word, stops issuing, releases its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "fq_internal.cuh"
#include "tc.cuh"

namespace {

using namespace fqtc;

constexpr int BM = 128;           // output rows per CTA (TMEM lanes)
constexpr int BN = 256;           // output columns per CTA (TMEM columns, FP32)
constexpr int ROW_BYTES = 128;    // K bytes per stage = one 128-byte swizzle row
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * ROW_BYTES;       // 16 KB
constexpr int B_BYTES = BN * ROW_BYTES;       // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int TC_THREADS = 128;
constexpr int TMEM_COLS = 256;
constexpr int PIX_PAD = 64;       // Xt row length is a multiple of this
constexpr int MAX_TILES = 64;     // upper tiles for 2F <= 1024

struct TileList {
    int n;
    unsigned short m0[MAX_TILES], n0[MAX_TILES];
};

// Instruction descriptor: FP32 accumulator, A and B of one type (BF16 = 1
// under kind::f16, TF32 = 2 under kind::tf32), both K-major, M = 128, N = 256.
template <int ESZ>
constexpr uint32_t idesc()
{
    return (1u << 4) | ((ESZ == 2 ? 1u : 2u) << 7) | ((ESZ == 2 ? 1u : 2u) << 10) | ((uint32_t)(BN >> 3) << 17) |
           ((uint32_t)(BM >> 4) << 24);
}

template <int ESZ>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    if constexpr (ESZ == 2) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc<2>()), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc<4>()), "r"(accumulate)
            : "memory");
    }
}
// ---------------------------------------------------------------- kernels --
__device__ __forceinline__ void store_op(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void store_op(float *p, float v)
{
    uint32_t t;  // TF32: round to nearest, ties away, 10 explicit mantissa bits
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
    *p = __uint_as_float(t);
}

// Xt[2i][p] = Re S[p][i], Xt[2i+1][p] = Im S[p][i], zero for p >= P.
template <typename T, typename OpT>
__global__ void transpose_kernel(const T *__restrict__ S, int64_t P, int F, int64_t Pp, OpT *__restrict__ Xt)
{
    __shared__ float tile[32][33];
    const int C = 2 * F;
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t p = p0 + r;
        const int c = c0 + threadIdx.x;
        float v = 0.0f;
        if (p < P && c < C) v = fqi::load_f(S, p * C + c);
        tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r;
        const int64_t p = p0 + threadIdx.x;
        if (c < C && p < Pp) store_op(Xt + (int64_t)c * Pp + p, tile[threadIdx.x][r]);
    }
}

template <int ESZ>
__global__ void __launch_bounds__(TC_THREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TileList tiles,
                   int ksteps_total, int ksteps_per_chunk, int Mp, int Np, float *__restrict__ part,
                   int *__restrict__ status, int skip_loads)
{
    constexpr int BK = ROW_BYTES / ESZ;   // pixels per stage
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned operand ring (128-byte swizzle atoms)
    unsigned char *ring = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // consecutive CTAs share a pixel chunk (one per output tile), so the
    // operand rows they stream are re-read from L2 rather than DRAM
    const int chunk = blockIdx.y;
    const int m0 = tiles.m0[blockIdx.x];
    const int n0 = tiles.n0[blockIdx.x];
    const int kbeg = chunk * ksteps_per_chunk;
    const int kend = min(ksteps_total, kbeg + ksteps_per_chunk);
    const int nk = max(0, kend - kbeg);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer (skip_loads: the test hook that lets every wait run out)
        for (int it = 0; it < nk && !skip_loads; ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            if (!mbar_wait(&empty_bar[s], ph ^ 1u)) { s_fail = 1; break; }
            unsigned char *a = ring + s * STAGE_BYTES;
            unsigned char *b = a + A_BYTES;
            const int kx = (kbeg + it) * BK;
            mbar_expect_tx(&full_bar[s], STAGE_BYTES);
            tma_load_2d(a, &tmap, &full_bar[s], kx, m0);
            tma_load_2d(b, &tmap, &full_bar[s], kx, n0);
            tma_load_2d(b + (BN / 2) * ROW_BYTES, &tmap, &full_bar[s], kx, n0 + BN / 2);
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: 4 instructions of 32 K-bytes per stage
        for (int it = 0; it < nk; ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
            if (!mbar_wait(&full_bar[s], ph)) { s_fail = 1; break; }
            tc_fence_after();
            const uint32_t a = smem_u32(ring + s * STAGE_BYTES);
            const uint32_t b = a + A_BYTES;
            const uint64_t ad = sw128_desc(a), bd = sw128_desc(b);
#pragma unroll
            for (int kk = 0; kk < ROW_BYTES / 32; ++kk)  // +32 bytes = +2 in the encoded start address
                mma_issue<ESZ>(tmem, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), (it > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&empty_bar[s]);
        }
        mma_commit(&done_bar);
    }
    __syncwarp();

    // ---- epilogue: TMEM -> FP32 partial tile (warp w owns rows 32w .. 32w + 31)
    bool ok = nk > 0;
    if (ok) ok = warp_wait(&done_bar, 0);
    tc_fence_after();
    if (!ok && nk > 0 && lane == 0) s_fail = 1;
    float *dst = part + (size_t)chunk * Mp * Np;
    const int row = m0 + warp * 32 + lane;
    for (int c = 0; c < BN; c += 32) {
        float v[32];
        if (ok) {
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 0.0f;
        }
        float4 *o = reinterpret_cast<float4 *>(dst + (size_t)row * Np + n0 + c);
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(status, (int)FQ_ERR_TIMEOUT);
}

// Sum the chunks and form the complex G from the real 2F x 2F product; the
// upper triangle (i <= j) is read, the lower one is its conjugate.
__global__ void gram_tc_reduce_kernel(const float *__restrict__ part, int n_chunks, int Mp, int Np, int F,
                                      float2 *__restrict__ G)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F * F) return;
    const int i0 = idx / F, j0 = idx % F;
    const int i = min(i0, j0), j = max(i0, j0);
    float re = 0.0f, im = 0.0f;
    for (int c = 0; c < n_chunks; ++c) {
        const float *d = part + (size_t)c * Mp * Np;
        re += d[(size_t)(2 * i) * Np + 2 * j] + d[(size_t)(2 * i + 1) * Np + 2 * j + 1];
        im += d[(size_t)(2 * i) * Np + 2 * j + 1] - d[(size_t)(2 * i + 1) * Np + 2 * j];
    }
    G[idx] = make_float2(re, i0 <= j0 ? im : -im);
}

// ------------------------------------------------------------------- host --
int g_skip_loads = 0;  // fq_debug_set(FQ_DEBUG_SKIP_TC_LOADS, ...)

struct TcPlan {
    int64_t Pp;
    int esz, bk, C, Mp, Np, ksteps, chunks, per_chunk;
    TileList tiles;
    size_t xt_off, part_off, total;
};

TcPlan tc_plan(int64_t P, int F, int esz)
{
    TcPlan t;
    t.esz = esz;
    t.bk = ROW_BYTES / esz;
    t.Pp = (P + PIX_PAD - 1) / PIX_PAD * PIX_PAD;
    t.C = 2 * F;
    const int m_tiles = (t.C + BM - 1) / BM;
    const int n_tiles = (t.C + BN - 1) / BN;
    t.Mp = m_tiles * BM;
    t.Np = n_tiles * BN;
    // tiles holding some entry (r, c) with r <= c: m0 <= n0 + BN - 1
    t.tiles.n = 0;
    for (int mt = 0; mt < m_tiles; ++mt)
        for (int nt = 0; nt < n_tiles; ++nt)
            if (mt * BM <= nt * BN + BN - 1) {
                t.tiles.m0[t.tiles.n] = (unsigned short)(mt * BM);
                t.tiles.n0[t.tiles.n] = (unsigned short)(nt * BN);
                ++t.tiles.n;
            }
    t.ksteps = (int)(t.Pp / t.bk);
    // about four waves of one CTA per SM: the tail of the last wave is a
    // quarter of the run instead of half (one CTA per SM fits its ring)
    int want = (4 * 152 + t.tiles.n - 1) / t.tiles.n;
    want = want < 1 ? 1 : (want > t.ksteps ? t.ksteps : want);
    t.per_chunk = (t.ksteps + want - 1) / want;
    t.chunks = (t.ksteps + t.per_chunk - 1) / t.per_chunk;
    size_t o = 0;
    t.xt_off = o;
    o += ((size_t)t.C * t.Pp * esz + 255) & ~(size_t)255;
    t.part_off = o;
    o += ((size_t)t.chunks * t.Mp * t.Np * 4 + 255) & ~(size_t)255;
    t.total = o;
    return t;
}

template <int ESZ>
fq_status launch_tc(const TcPlan &t, const CUtensorMap &map, float *part, int *status, cudaStream_t st)
{
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024;
    fq_status s = fqi::cuda_check(
        cudaFuncSetAttribute(gram_tc_kernel<ESZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
        "tensor-core Gram: smem attribute");
    if (s) return s;
    dim3 grid((unsigned)t.tiles.n, (unsigned)t.chunks);
    gram_tc_kernel<ESZ><<<grid, TC_THREADS, smem, st>>>(map, t.tiles, t.ksteps, t.per_chunk, t.Mp, t.Np, part,
                                                        status, g_skip_loads);
    return fqi::launch_check("tensor-core Gram: mma");
}

}  // namespace

namespace fqi {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

void *tensor_map_encoder_ptr() { return (void *)tensor_map_encoder(); }

size_t gram_tc_workspace_bytes(int64_t P, int F, int esz) { return tc_plan(P, F, esz).total; }

// Tensor-core Gram into G (device float2 [F][F]).  esz = 2: BF16 operands,
// esz = 4: TF32 operands.  `ws` is the 256-byte aligned scratch of
// gram_tc_workspace_bytes; a timed-out wait sets *status to FQ_ERR_TIMEOUT.
fq_status gram_tc(const void *S, int dtype, int64_t P, int F, int esz, float2 *G, char *ws, int *status,
                  cudaStream_t st)
{
    FQ_REQUIRE(esz == 2 || esz == 4, FQ_ERR_INVALID_ARG, "tensor-core Gram: operand size %d", esz);
    FQ_REQUIRE(2 * F <= 1024 && P >= 1, FQ_ERR_SHAPE, "tensor-core Gram: F = %d", F);
    const TcPlan t = tc_plan(P, F, esz);
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    FQ_REQUIRE(enc, FQ_ERR_CUDA, "tensor-core Gram: cuTensorMapEncodeTiled unavailable");
    void *Xt = ws + t.xt_off;
    float *part = (float *)(ws + t.part_off);
    dim3 tb(32, 8), tg((unsigned)(t.Pp / 32), (unsigned)((t.C + 31) / 32));
    if (esz == 2) {
        if (dtype == FQ_F32)
            transpose_kernel<float, __nv_bfloat16><<<tg, tb, 0, st>>>((const float *)S, P, F, t.Pp,
                                                                      (__nv_bfloat16 *)Xt);
        else
            transpose_kernel<__nv_bfloat16, __nv_bfloat16><<<tg, tb, 0, st>>>((const __nv_bfloat16 *)S, P, F, t.Pp,
                                                                              (__nv_bfloat16 *)Xt);
    } else {
        if (dtype == FQ_F32)
            transpose_kernel<float, float><<<tg, tb, 0, st>>>((const float *)S, P, F, t.Pp, (float *)Xt);
        else
            transpose_kernel<__nv_bfloat16, float><<<tg, tb, 0, st>>>((const __nv_bfloat16 *)S, P, F, t.Pp,
                                                                      (float *)Xt);
    }
    fq_status s = launch_check("tensor-core Gram: transpose");
    if (s) return s;

    CUtensorMap map;
    std::memset(&map, 0, sizeof map);
    cuuint64_t dims[2] = {(cuuint64_t)t.Pp, (cuuint64_t)t.C};
    cuuint64_t strides[1] = {(cuuint64_t)t.Pp * (cuuint64_t)esz};
    cuuint32_t box[2] = {(cuuint32_t)t.bk, (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult cr = enc(&map, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Xt,
                      dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    FQ_REQUIRE(cr == CUDA_SUCCESS, FQ_ERR_CUDA, "tensor-core Gram: cuTensorMapEncodeTiled failed (%d)", (int)cr);

    s = esz == 2 ? launch_tc<2>(t, map, part, status, st) : launch_tc<4>(t, map, part, status, st);
    if (s) return s;
    gram_tc_reduce_kernel<<<(F * F + 255) / 256, 256, 0, st>>>(part, t.chunks, t.Mp, t.Np, F, G);
    return launch_check("tensor-core Gram: reduce");
}

}  // namespace fqi

extern "C" fq_status fq_debug_set(int32_t what, int32_t value)
{
    FQ_REQUIRE(what == FQ_DEBUG_SKIP_TC_LOADS, FQ_ERR_INVALID_ARG, "fq_debug_set: unknown setting %d", what);
    g_skip_loads = value != 0;
    return FQ_OK;
}
