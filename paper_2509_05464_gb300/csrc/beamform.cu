// beamform.cu -- a4 rf2iq and a5 plane-wave delay-and-sum compounding
// (Sec. 2.4.1, Alg. 3).
//
// Layout: rf2iq writes the channel IQ frames-innermost, [A*M][Ns][F_pad]
// complex, so that the DAS kernel, which computes each (pixel, transmit,
// element) delay once and applies it to a chunk of 16 frames, reads the two
// interpolation samples of those frames as contiguous 16-byte vectors.
// Alg. 3 (steps 2.2-2.3) builds each transmit's delays once and applies
// them to every frame through a stored sparse matrix; here the delays live
// in registers for the duration of a frame chunk instead.
//
// Precision: delays, interpolation index and carrier phase are float-float;
// the aperture decision is binary32 on coordinates rounded from IEEE double;
// FP32 channel data interpolate in FP32, 16-bit data in their own precision;
// accumulation is FP32.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "batch.cuh"
#include "fq_internal.cuh"
#include "rf_poly.cuh"

namespace {

using fqi::ff;

constexpr int kMaxHalfTaps = 32;
constexpr int kFrameChunk = 16;  // frames per DAS tile and per rf2iq CTA (F_pad multiple)

// ------------------------------------------------------------------ rf2iq --
struct Rf2iqParams {
    int L, F, Fp, ns, J;
    fqi::df2 f0_over_fs;
    float h[2 * kMaxHalfTaps + 1];
};

constexpr int kRfTile = 128;  // output samples per CTA

static_assert(kRfTile == fqb::kIqTile && kFrameChunk == fqb::kFrameChunkB, "batched item shapes");

// One tile: output samples bx * 64 .. + 63 of channel line l, frames
// 16 bz .. 16 bz + 15.  `mix` is the dynamic shared memory.
template <typename InT, typename OutT>
__device__ __forceinline__ void rf2iq_tile(const Rf2iqParams &p, int bx, int l, int bz, const InT *__restrict__ rf,
                                           OutT *__restrict__ iq, float2 *mix)
{
    const int k0 = bx * kRfTile;
    const int f0 = bz * kFrameChunk;
    const int J = p.J;
    const int W = kRfTile + 2 * J;      // window samples
    const int WS = W | 1;               // odd row stride: the 16 frame rows fall in distinct banks
    float2 *rot = mix + kFrameChunk * WS;  // [W]: exp(-i 2 pi f0 n / fs)
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        int n = k0 - J + i;
        // fractional carrier cycles (f0/fs) n in float-float, then sincospi
        ff cyc = fqi::ff_mul_f(fqi::ff_load(p.f0_over_fs), (float)n);
        float fr = fqi::ff_frac(cyc);
        float sn, cs;
        sincospif(2.0f * fr, &sn, &cs);
        rot[i] = make_float2(cs, -sn);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kFrameChunk * W; i += blockDim.x) {
        int fl = i / W, w = i - fl * W;
        int n = k0 - J + w;
        int f = f0 + fl;
        float v = 0.0f;
        if (n >= 0 && n < p.ns && f < p.F) v = fqi::load_f(rf, ((int64_t)f * p.L + l) * p.ns + n);
        float2 r = rot[w];
        mix[fl * WS + w] = make_float2(v * r.x, v * r.y);
    }
    __syncthreads();
    // thread -> (frame fl = t % 16, sample kk = t / 16 + 16 q)
    const int fl = threadIdx.x % kFrameChunk;
    for (int kk = threadIdx.x / kFrameChunk; kk < kRfTile; kk += blockDim.x / kFrameChunk) {
        int k = k0 + kk;
        if (k >= p.ns) break;
        // IQ[k] = 2 sum_{j=-J..J} h_j mix[k - j]; sample n sits at window index n - (k0 - J),
        // so sample k - j is at kk + J - j
        const float2 *src = mix + fl * WS + kk + J;
        float re = 0.0f, im = 0.0f;
        for (int j = -J; j <= J; ++j) {
            float2 m = src[-j];
            float hj = p.h[j + J];
            re = fmaf(hj, m.x, re);
            im = fmaf(hj, m.y, im);
        }
        int f = f0 + fl;
        if (f < p.Fp) fqi::store_c(iq, ((int64_t)l * p.ns + k) * p.Fp + f, make_float2(2.0f * re, 2.0f * im));
    }
}

// The 8 outputs k .. k + 7 of frame f from the 24 demodulated samples
// k - 8 .. k + 15 of that frame (taps from the parameters).
template <typename OutT>
__device__ __forceinline__ void fir_j8_store(const Rf2iqParams &p, const float2 (&m)[24], int l, int k, int f,
                                             OutT *__restrict__ iq)
{
    constexpr int J = 8, G = 8;
#pragma unroll
    for (int o = 0; o < G; ++o) {
        float re = 0.0f, im = 0.0f;
#pragma unroll
        for (int j = -J; j <= J; ++j) {
            re = fmaf(p.h[j + J], m[o + J - j].x, re);
            im = fmaf(p.h[j + J], m[o + J - j].y, im);
        }
        if (k + o < p.ns && f < p.Fp)
            fqi::store_c(iq, ((int64_t)l * p.ns + k + o) * p.Fp + f, make_float2(2.0f * re, 2.0f * im));
    }
}

// The same tile for the common half-length J = 8 (fs / f0 near 4): the
// window size is a compile-time constant and each thread filters 8
// consecutive samples of one frame from a 24-value register window (24
// shared-memory reads instead of 8 x 17), with the taps in registers.
template <typename InT, typename OutT>
__device__ __forceinline__ void rf2iq_tile_j8(const Rf2iqParams &p, int bx, int l, int bz, const InT *__restrict__ rf,
                                              OutT *__restrict__ iq, float2 *mix)
{
    constexpr int J = 8, W = kRfTile + 2 * J, WS = W | 1, G = 8;
    static_assert(kRfTile == 16 * G, "256 threads = 16 frames x 16 groups of 8 samples");
    const int k0 = bx * kRfTile;
    const int f0 = bz * kFrameChunk;
    float2 *rot = mix + kFrameChunk * WS;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        int n = k0 - J + i;
        ff cyc = fqi::ff_mul_f(fqi::ff_load(p.f0_over_fs), (float)n);
        float fr = fqi::ff_frac(cyc);
        float sn, cs;
        sincospif(2.0f * fr, &sn, &cs);
        rot[i] = make_float2(cs, -sn);
    }
    __syncthreads();
    // two samples per thread: windows start at even samples (k0 - J, J even)
    // and rows hold an even number of samples when Ns is even
    const bool pairs = (p.ns & 1) == 0;
    for (int i = threadIdx.x; i < kFrameChunk * (W / 2); i += blockDim.x) {
        const int fl = i / (W / 2), w = 2 * (i - fl * (W / 2));
        const int n = k0 - J + w;
        const int f = f0 + fl;
        float v0 = 0.0f, v1 = 0.0f;
        if (f < p.F) {
            const int64_t base = ((int64_t)f * p.L + l) * p.ns;
            if (pairs && n >= 0 && n + 1 < p.ns) {
                const float2 vv = fqi::load_f2(rf, base + n);
                v0 = vv.x;
                v1 = vv.y;
            } else {
                if (n >= 0 && n < p.ns) v0 = fqi::load_f(rf, base + n);
                if (n + 1 >= 0 && n + 1 < p.ns) v1 = fqi::load_f(rf, base + n + 1);
            }
        }
        const float2 r0 = rot[w], r1 = rot[w + 1];
        mix[fl * WS + w] = make_float2(v0 * r0.x, v0 * r0.y);
        mix[fl * WS + w + 1] = make_float2(v1 * r1.x, v1 * r1.y);
    }
    __syncthreads();
    const int fl = threadIdx.x % kFrameChunk, g = threadIdx.x / kFrameChunk;
    // window index of sample n is n - (k0 - J); output k0 + G g + o reads
    // window indices G g + o + J - j, j = -J .. J
    const float2 *src = mix + fl * WS + G * g;
    float2 m[G + 2 * J];
#pragma unroll
    for (int t = 0; t < G + 2 * J; ++t) m[t] = src[t];
    fir_j8_store(p, m, l, k0 + G * g, f0 + fl, iq);
}

template <typename InT, typename OutT>
__device__ __forceinline__ void rf2iq_any(const Rf2iqParams &p, int bx, int l, int bz, const InT *__restrict__ rf,
                                          OutT *__restrict__ iq, float2 *mix)
{
    if (p.J == 8) rf2iq_tile_j8<InT, OutT>(p, bx, l, bz, rf, iq, mix);
    else rf2iq_tile<InT, OutT>(p, bx, l, bz, rf, iq, mix);
}

template <typename InT, typename OutT>
__global__ void __launch_bounds__(256) rf2iq_kernel(const Rf2iqParams p, const InT *__restrict__ rf,
                                                    OutT *__restrict__ iq)
{
    extern __shared__ float2 mix[];  // [kFrameChunk][W | 1] then the rotation row [W]
    rf2iq_any<InT, OutT>(p, blockIdx.x, blockIdx.y, blockIdx.z, rf, iq, mix);
}

// RF with J = 8 and Ns a multiple of the samples per 16 bytes: one CTA per
// (128-sample tile, channel line) walks every frame chunk, with the next
// chunk's raw samples in flight (cp.async into the other half of a double
// buffer) while the current one is filtered, so that the loads of a CTA
// overlap its filter and stores instead of alternating with them.  Same
// products and sums as rf2iq_tile_j8, so the results are identical.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename InT>
struct StreamShape {
    static constexpr int J = 8, W = kRfTile + 2 * J;
    static constexpr int VE = 16 / (int)sizeof(InT);  // samples per 16-byte vector
    static constexpr int NV = W / VE;                 // vectors per frame row
    static constexpr int ROW = NV + 1;                // odd row stride: 128-bit reads of 8 rows do not conflict
    static constexpr size_t smem = sizeof(float4) * 2 * kFrameChunk * ROW + sizeof(float2) * W;
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

template <typename InT, typename OutT>
__global__ void __launch_bounds__(256, 3) rf2iq_stream_kernel(const Rf2iqParams p, const InT *__restrict__ rf,
                                                              OutT *__restrict__ iq)
{
    using SS = StreamShape<InT>;
    constexpr int J = SS::J, W = SS::W, G = 8, VE = SS::VE, NV = SS::NV, ROW = SS::ROW;
    static_assert(W % VE == 0 && (G * sizeof(InT)) % 16 == 0 && kRfTile == 16 * G, "tile shape");
    extern __shared__ float4 raw[];  // [2][kFrameChunk][ROW] raw sample vectors, then the rotation row [W]
    float2 *rot = reinterpret_cast<float2 *>(raw + 2 * kFrameChunk * ROW);
    const int l = blockIdx.y, k0 = blockIdx.x * kRfTile;
    const int nch = p.Fp / kFrameChunk;
    const InT *line = rf + (int64_t)l * p.ns;
    const int64_t fstride = (int64_t)p.L * p.ns;
    auto issue = [&](int c) {
        float4 *dst = raw + (c & 1) * kFrameChunk * ROW;
        for (int i = threadIdx.x; i < kFrameChunk * NV; i += blockDim.x) {
            const int fl = i / NV, v = i - fl * NV;
            const int n = k0 - J + VE * v, f = c * kFrameChunk + fl;
            const bool ok = f < p.F && n >= 0 && n < p.ns;  // Ns % VE == 0: a vector is wholly in or out
            cp_async16(dst + fl * ROW + v, ok ? line + f * fstride + n : rf, ok ? 16 : 0);
        }
        cp_async_commit();
    };
    issue(0);
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        const int n = k0 - J + i;
        ff cyc = fqi::ff_mul_f(fqi::ff_load(p.f0_over_fs), (float)n);
        float fr = fqi::ff_frac(cyc);
        float sn, cs;
        sincospif(2.0f * fr, &sn, &cs);
        rot[i] = make_float2(cs, -sn);
    }
    const int fl = threadIdx.x % kFrameChunk, g = threadIdx.x / kFrameChunk;
    for (int c = 0; c < nch; ++c) {
        if (c + 1 < nch) {
            issue(c + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float4 *row = raw + ((c & 1) * kFrameChunk + fl) * ROW + G * g / VE;
        float2 m[G + 2 * J];
#pragma unroll
        for (int q = 0; q < (G + 2 * J) / VE; ++q) {
            const float4 v4 = row[q];
            const InT *vv = reinterpret_cast<const InT *>(&v4);
#pragma unroll
            for (int t = 0; t < VE; ++t) {
                const float v = to_f(vv[t]);
                const float2 r = rot[G * g + VE * q + t];
                m[VE * q + t] = make_float2(v * r.x, v * r.y);
            }
        }
        fir_j8_store(p, m, l, k0 + G * g, c * kFrameChunk + fl, iq);
        __syncthreads();  // the buffer is refilled by the next issue
    }
}

constexpr int kIqParamBytes = (sizeof(Rf2iqParams) + 15) & ~15;

template <typename InT, typename OutT>
__global__ void __launch_bounds__(256) rf2iq_batched_kernel(const fqb::EnsDev *__restrict__ ens,
                                                            const fqb::StageQueue q)
{
    extern __shared__ float2 mix[];
    __shared__ __align__(16) unsigned char s_par[kIqParamBytes];
    __shared__ int s_buf[2];
    int cur = -1;
    fqb::Item it;
    while (fqb::next_item(q, ens, fqb::ST_RF2IQ, s_buf, it)) {
        const fqb::EnsDev &e = ens[it.e];
        if (it.e != cur) {
            fqb::copy_block(s_par, e.iq_params, kIqParamBytes);
            cur = it.e;
            __syncthreads();
        }
        rf2iq_any<InT, OutT>(*reinterpret_cast<const Rf2iqParams *>(s_par), it.x, it.y, it.z,
                              (const InT *)e.rf, (OutT *)e.ch, mix);
    }
}

bool make_rf2iq_params(const fq_probe *probe, int L, int F, Rf2iqParams &p)
{
    std::memset(&p, 0, sizeof p);
    p.L = L;
    p.F = F;
    p.Fp = fq_frame_pad(F);
    p.ns = probe->n_samples;
    int J = 2 * (int)std::lround(probe->fs / probe->f0);
    if (J > kMaxHalfTaps || J < 0) return false;
    p.J = J;
    p.f0_over_fs = fqi::split_double(probe->f0 / probe->fs);
    // Hann-windowed ideal low-pass, cutoff f0, normalised to unit DC gain
    double h[2 * kMaxHalfTaps + 1];
    double sum = 0.0;
    const double fc = 2.0 * probe->f0 / probe->fs;  // cutoff in units of fs/2
    for (int j = -J; j <= J; ++j) {
        double ideal = (j == 0) ? fc : std::sin(M_PI * fc * j) / (M_PI * j);
        double w = 0.5 * (1.0 + std::cos(M_PI * j / (J + 1.0)));
        h[j + J] = w * ideal;
        sum += h[j + J];
    }
    for (int j = 0; j < 2 * J + 1; ++j) p.h[j] = (float)(h[j] / sum);
    return true;
}

template <typename InT, typename OutT>
fq_status launch_rf2iq(const Rf2iqParams &p, const void *rf, void *iq, cudaStream_t st)
{
    if (p.J == 8 && p.ns % StreamShape<InT>::VE == 0 && fqi::aligned(rf, 16)) {
        dim3 grid((p.ns + kRfTile - 1) / kRfTile, p.L);
        rf2iq_stream_kernel<InT, OutT><<<grid, 256, StreamShape<InT>::smem, st>>>(p, (const InT *)rf, (OutT *)iq);
        return fqi::launch_check("fq_rf2iq");
    }
    int W = kRfTile + 2 * p.J;
    size_t smem = sizeof(float2) * ((size_t)kFrameChunk * (W | 1) + W);
    dim3 grid((p.ns + kRfTile - 1) / kRfTile, p.L, p.Fp / kFrameChunk);
    rf2iq_kernel<InT, OutT><<<grid, 256, smem, st>>>(p, (const InT *)rf, (OutT *)iq);
    return fqi::launch_check("fq_rf2iq");
}

fq_status run_rf2iq(const fq_probe *probe, int L, int F, const void *rf, int rf_dtype, int iq_dtype, void *iq,
                    cudaStream_t st)
{
    Rf2iqParams p;
    FQ_REQUIRE(make_rf2iq_params(probe, L, F, p), FQ_ERR_SHAPE, "fq_rf2iq: 2 round(fs/f0) must be <= %d",
               kMaxHalfTaps);
    return fqi::with_storage(rf_dtype, "fq_rf2iq (rf)", [&](auto *in) {
        return fqi::with_storage(iq_dtype, "fq_rf2iq (iq)", [&](auto *out) {
            return launch_rf2iq<fqi::storage_t<decltype(in)>, fqi::storage_t<decltype(out)>>(p, rf, iq, st);
        });
    });
}

// -------------------------------------------------------------------- DAS --
struct DasParams {
    fqi::ProbeFF pr;
    double pitch_x, pitch_y;  // exact, for the binary32 aperture decision
    int A, F, Fp;
    int gx, gy, gz;
    int64_t P;
    double x0, y0, z0, dx, dy, dz;
    float half_per_z;   // 1 / (2 f#)
    float inv_A;
    int rot_tab;        // carrier phase from a per-sample table (see das_smem_bytes)
    float pi_f0_fs;     // pi f0 / fs
    fqi::AngleFF ang[FQ_MAX_ANGLES];
};

constexpr int kDasThreads = 128;
constexpr int kDasTPP = fqb::kDasThreadsPerPixel;  // threads per pixel

// (sin x, cos x) for |x| <= 0.8 from the fitted polynomials of rf_poly.cuh
// (binary32 evaluation error below 6e-8)
__device__ __forceinline__ void das_sincos_poly(float x, float &s, float &c)
{
    using namespace fqpoly;
    const float t = x * x;
    s = x * fmaf(fmaf(fmaf(kSinPoly3, t, kSinPoly2), t, kSinPoly1), t, kSinPoly0);
    c = fmaf(fmaf(fmaf(fmaf(kCosPoly4, t, kCosPoly3), t, kCosPoly2), t, kCosPoly1), t, kCosPoly0);
}

// Tiles and their order.  A CTA of W = blockDim.x / TPP pixel columns
// takes W consecutive voxels along x of one (y, z) row, and CTAs are
// numbered x-block fastest, then y, then z: the CTAs resident at one time
// cover a thin slab of depths over the whole lateral extent.  A channel
// line is then needed only over the band of samples that the slab's
// delays reach (for the 3D workload about a tenth of the record), which
// stays in L2 while the slab is beamformed, instead of every sample of
// every line (ordering by x, then z, then y made every resident set span
// all depths: the 3D DAS read its channel data from DRAM ~50 times).
__host__ __device__ inline int64_t das_ctas(int gx, int gy, int gz, int W)
{
    return (int64_t)((gx + W - 1) / W) * gy * gz;
}

// Dynamic shared memory of a DAS tile of T threads (W = T / TPP pixels):
// element abscissae per column and ordinates per row (3 floats each, nx + ny
// <= M + 1), each pixel's transmit path per angle (A W float pairs) and the
// per-sample carrier table (rot_ns float pairs).
// Offsets in floats, each a multiple of 4 (16 bytes), so that the float2
// tables stay aligned.
__host__ __device__ inline int das_off_ptx(int M) { return (3 * (M + 1) + 3) & ~3; }
__host__ __device__ inline int das_off_acc(int M, int A, int W) { return das_off_ptx(M) + ((2 * A * W + 3) & ~3); }
__host__ __device__ inline int das_off_rot(int M, int A, int W) { return das_off_acc(M, A, W); }
// rot_ns: samples of the per-sample carrier table (0 = no table)
__host__ __device__ inline size_t das_smem_bytes(int M, int A, int T, int TPP, int rot_ns)
{
    const int W = T / TPP;
    return sizeof(float) * (size_t)das_off_rot(M, A, W) + sizeof(float2) * (size_t)rot_ns;
}
// The carrier phase e^{i 2 pi f0 tau} = e^{i 2 pi (f0/fs) i} e^{i 2 pi (f0/fs) phi}
// (u = tau fs = i + phi) comes from a per-sample table and a short
// polynomial when the table fits (ns <= kRotTabMax) and the second angle's
// half stays inside the polynomial's range (pi f0 / fs <= 0.8, i.e. at least
// ~3.93 samples per carrier period: every workload here samples at ~4 f0).
constexpr int kRotTabMax = 2048;
inline bool das_rot_tab(const fq_probe *probe)
{
    return probe->n_samples <= kRotTabMax && M_PI * probe->f0 / probe->fs <= (double)fqpoly::kTapXMax;
}

// Running sums of one thread's FPT frames of the chunk, read as FPT / FL
// 16-byte groups of FL frames (FL = 4 for 16-bit data, 2 for FP32) GS groups
// apart, interpolated at i + phi and rotated by (cs, sn).
//
// SepAcc (FP32 data): the interpolation in f32x2 on (re, im) pairs, then sum
// v cos and sum v sin per frame (rotated at the end: (C.re - S.im,
// C.im + S.re)), two f32x2 operations per frame each.
template <int FPT, int GS>
struct SepAcc {
    fqi::f2 C[FPT], S[FPT];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int k = 0; k < FPT; ++k) C[k] = S[k] = fqi::f2_dup(0.0f);
    }
    __device__ __forceinline__ void add(const float *b0, int64_t stride, float phi, float cs, float sn)
    {
        const ulonglong2 *q0 = reinterpret_cast<const ulonglong2 *>(b0);
        const ulonglong2 *q1 = reinterpret_cast<const ulonglong2 *>(b0 + stride);
        ulonglong2 t0[FPT / 2], t1[FPT / 2];
#pragma unroll
        for (int g = 0; g < FPT / 2; ++g) {
            t0[g] = __ldg(q0 + g * GS);
            t1[g] = __ldg(q1 + g * GS);
        }
        const fqi::f2 PHI = fqi::f2_dup(phi), CS = fqi::f2_dup(cs), SN = fqi::f2_dup(sn);
#pragma unroll
        for (int g = 0; g < FPT / 2; ++g) {
            const fqi::f2 v0 = fqi::f2_fma(PHI, fqi::f2_sub(fqi::f2{t1[g].x}, fqi::f2{t0[g].x}), fqi::f2{t0[g].x});
            const fqi::f2 v1 = fqi::f2_fma(PHI, fqi::f2_sub(fqi::f2{t1[g].y}, fqi::f2{t0[g].y}), fqi::f2{t0[g].y});
            C[2 * g] = fqi::f2_fma(v0, CS, C[2 * g]);
            S[2 * g] = fqi::f2_fma(v0, SN, S[2 * g]);
            C[2 * g + 1] = fqi::f2_fma(v1, CS, C[2 * g + 1]);
            S[2 * g + 1] = fqi::f2_fma(v1, SN, S[2 * g + 1]);
        }
    }
    __device__ __forceinline__ float2 get(int k) const
    {
        float cr, ci, sr, si;
        fqi::f2_split(C[k], cr, ci);
        fqi::f2_split(S[k], sr, si);
        return make_float2(cr - si, ci + sr);
    }
};

// the real parts (lo) and imaginary parts (hi) of two packed 16-bit (re, im)
// words as binary32 pairs
__device__ __forceinline__ void widen_pair(uint32_t a, uint32_t b, fqi::f2 &re, fqi::f2 &im, __nv_bfloat16 *)
{
    asm("{ .reg .b32 r0, r1, i0, i1;\n\t shl.b32 r0, %2, 16;\n\t shl.b32 r1, %3, 16;\n\t"
        " and.b32 i0, %2, 0xffff0000;\n\t and.b32 i1, %3, 0xffff0000;\n\t"
        " mov.b64 %0, {r0, r1};\n\t mov.b64 %1, {i0, i1}; }"
        : "=l"(re.v), "=l"(im.v) : "r"(a), "r"(b));
}
__device__ __forceinline__ void widen_pair(uint32_t a, uint32_t b, fqi::f2 &re, fqi::f2 &im, __half *)
{
    const float2 x = __half22float2(*reinterpret_cast<const __half2 *>(&a));
    const float2 y = __half22float2(*reinterpret_cast<const __half2 *>(&b));
    re = fqi::f2_make(x.x, y.x);
    im = fqi::f2_make(x.y, y.y);
}

// RotAcc (BF16 / FP16 data): the interpolation as packed 16-bit (re, im)
// pairs (phi rounded to the storage type, as the storage itself), then the
// rotated sums of two frames per pair of registers, (re_k, re_k+1) and
// (im_k, im_k+1): four f32x2 operations per two frames, and half the
// registers of SepAcc's form.
template <int FPT, int GS, typename H>
struct RotAcc {
    using H2 = typename std::conditional<std::is_same<H, __half>::value, __half2, __nv_bfloat162>::type;
    fqi::f2 R[FPT / 2], I[FPT / 2];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int m = 0; m < FPT / 2; ++m) R[m] = I[m] = fqi::f2_dup(0.0f);
    }
    __device__ __forceinline__ void add(const H *b0, int64_t stride, float phi, float cs, float sn)
    {
        const uint4 *q0 = reinterpret_cast<const uint4 *>(b0);
        const uint4 *q1 = reinterpret_cast<const uint4 *>(b0 + stride);
        uint4 t0[FPT / 4], t1[FPT / 4];
#pragma unroll
        for (int g = 0; g < FPT / 4; ++g) {
            t0[g] = __ldg(q0 + g * GS);
            t1[g] = __ldg(q1 + g * GS);
        }
        H2 ph;
        if constexpr (std::is_same<H, __half>::value) ph = __float2half2_rn(phi);
        else ph = __float2bfloat162_rn(phi);
        const fqi::f2 CS = fqi::f2_dup(cs), SN = fqi::f2_dup(sn), NSN = fqi::f2_dup(-sn);
#pragma unroll
        for (int g = 0; g < FPT / 4; ++g) {
            const H2 *a = reinterpret_cast<const H2 *>(&t0[g]);
            const H2 *b = reinterpret_cast<const H2 *>(&t1[g]);
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const H2 x = __hfma2(ph, __hsub2(b[k], a[k]), a[k]);
                w[k] = *reinterpret_cast<const uint32_t *>(&x);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                fqi::f2 RE, IM;
                widen_pair(w[2 * h], w[2 * h + 1], RE, IM, (H *)nullptr);
                const int m = 2 * g + h;
                R[m] = fqi::f2_fma(RE, CS, R[m]);
                R[m] = fqi::f2_fma(IM, NSN, R[m]);
                I[m] = fqi::f2_fma(RE, SN, I[m]);
                I[m] = fqi::f2_fma(IM, CS, I[m]);
            }
        }
    }
    __device__ __forceinline__ float2 get(int k) const
    {
        float r0, r1, i0, i1;
        fqi::f2_split(R[k / 2], r0, r1);
        fqi::f2_split(I[k / 2], i0, i1);
        return (k & 1) ? make_float2(r1, i1) : make_float2(r0, i0);
    }
};

// One DAS tile of FP32 channel data.  A CTA of W = blockDim.x / 4 pixel
// columns (four threads per pixel) takes W consecutive voxels along x of one
// (y, z) row, frames 16 by .. 16 by + 15 (das_ctas gives the order of the
// CTAs).  The pixels of a CTA share y and z, so the rows of a matrix probe
// inside the receive aperture are the same for all of them; a warp walks
// those rows and, in each, the columns that the aperture of any of its
// pixels can reach, in groups of four elements.  Each thread of a pixel
// evaluates the float-float receive distance of one element of a group
// (g0 + sub) once for every transmit (the transmit paths of the pixel sit in
// shared memory) and, per transmit, its delay and carrier rotation; the
// four threads then take every element of the group (delays shared by
// shuffles), thread q over frames 2 (4 g + q) .. + 1 for g = 0, 1 (16-byte
// groups interleaved, so that a load instruction of a pixel's threads reads
// 64 adjacent bytes).  Sums: element groups in order (rows, then columns),
// transmits, the group's elements in order.  With 8 frames of FP32 per
// thread (two threads per element) the 2D workload's DAS measured 7.0 ms
// against 5.0 ms, and one warp per pixel (as das_tile_w) 5.4 ms: the 16-byte
// groups of FP32 data hold two frames, and the extra frames per delay do
// not pay for the wider loads.  `etab` is the dynamic shared memory
// (das_smem_bytes).
template <typename ChT, typename OutT>
__device__ __forceinline__ void das_tile(const DasParams &p, int64_t bx, int by, const ChT *__restrict__ ch,
                                            OutT *__restrict__ iq, float *etab)
{
    static_assert(sizeof(ChT) == 4, "das_tile takes FP32 channel data");
    constexpr int TPP = kDasTPP, FS = kDasTPP;  // four threads per pixel, each a frame slot
    constexpr int FPT = kFrameChunk / FS;
    constexpr int FL = 2;  // FP32 frames per 16 bytes
    const int M = p.pr.M, nxe = p.pr.nx, nye = p.pr.ny;
    const int W = blockDim.x / TPP;
    float *exf = etab, *exh = etab + nxe, *exl = etab + 2 * nxe;
    float *eyf = etab + 3 * nxe, *eyh = eyf + nye, *eyl = eyf + 2 * nye;
    float2 *ptx_s = reinterpret_cast<float2 *>(etab + das_off_ptx(M));
    float2 *rot_s = reinterpret_cast<float2 *>(etab + das_off_rot(M, p.A, W));
    for (int c = threadIdx.x; c < nxe + nye; c += blockDim.x) {
        const bool isx = c < nxe;
        const int i = isx ? c : c - nxe, n = isx ? nxe : nye;
        const double e = __dmul_rn(__dsub_rn((double)i, __dmul_rn(0.5, (double)(n - 1))), isx ? p.pitch_x : p.pitch_y);
        const fqi::df2 sp = fqi::split_double(e);
        if (isx) {
            exf[i] = (float)e; exh[i] = sp.hi; exl[i] = sp.lo;
        } else {
            eyf[i] = (float)e; eyh[i] = sp.hi; eyl[i] = sp.lo;
        }
    }

    const int sub = threadIdx.x % TPP;  // the element of a group whose delay this thread evaluates, and the frame slot
    const int col = threadIdx.x / TPP;
    const int nxb = (p.gx + W - 1) / W;
    const int xb = (int)(bx % nxb);
    const int64_t t = bx / nxb;
    const int iy = (int)(t % p.gy);
    const int iz = (int)(t / p.gy);
    const int ix = xb * W + col;
    const bool live = ix < p.gx && iz < p.gz;
    const int64_t pix = ((int64_t)iy * p.gz + iz) * p.gx + ix;
    const int fbase = by * kFrameChunk;
    const double xd = __dadd_rn(p.x0, __dmul_rn((double)(live ? ix : 0), p.dx));
    const double yd = __dadd_rn(p.y0, __dmul_rn((double)iy, p.dy));
    const double zd = __dadd_rn(p.z0, __dmul_rn((double)iz, p.dz));
    const float xf = (float)xd, yf = (float)yd, zf = (float)zd;
    const fqi::df2 xs = fqi::split_double(xd), ys = fqi::split_double(yd), zs = fqi::split_double(zd);
    const ff X = {xs.hi, xs.lo}, Y = {ys.hi, ys.lo}, Z = {zs.hi, zs.lo};
    const ff zz = fqi::ff_sqr(Z);
    const float half = __fmul_rn(zf, p.half_per_z);
    const bool matrix = nye > 1;
    const ff fs_c = fqi::ff_load(p.pr.fs_over_c);
    const ff f0_fs = fqi::ff_load(p.pr.f0_over_fs);
    const int ns = p.pr.ns;
    const int64_t row_stride = (int64_t)p.Fp * 2;
    const int64_t line_stride = (int64_t)ns * row_stride;

    if (p.rot_tab) {
        for (int n = threadIdx.x; n < ns; n += blockDim.x) {
            float sn, cs;
            sincospif(2.0f * fqi::ff_frac(fqi::ff_mul(f0_fs, ff{(float)n, 0.0f})), &sn, &cs);
            rot_s[n] = make_float2(cs, sn);
        }
    }
    if (sub == 0) {
        for (int a = 0; a < p.A; ++a) {
            const fqi::AngleFF an = p.ang[a];
            ff ptx = fqi::ff_add(fqi::ff_mul(fqi::ff_load(an.ux), X), fqi::ff_mul(fqi::ff_load(an.uy), Y));
            ptx = fqi::ff_add(ptx, fqi::ff_mul(fqi::ff_load(an.uz), Z));
            ptx = fqi::ff_add(ptx, fqi::ff_neg(fqi::ff_load(an.origin)));
            ptx_s[a * W + col] = make_float2(ptx.hi, ptx.lo);
        }
    }
    __syncthreads();

    int row_lo = 0, row_hi = nye - 1;
    if (matrix) {
        row_lo = nye;
        row_hi = -1;
        for (int r = 0; r < nye; ++r) {
            if (fabsf(__fsub_rn(yf, eyf[r])) <= half) {
                row_lo = min(row_lo, r);
                row_hi = r;
            }
        }
    }
    int c_lo = nxe, c_hi = -1;
    if (live) {
        if (nxe > 1 && p.pitch_x > 0.0) {
            const float c0f = 0.5f * (float)(nxe - 1);
            const float ip = (float)(1.0 / p.pitch_x);
            const float lo = fminf(fmaxf(floorf((xf - half) * ip + c0f), -2.0f), (float)nxe + 1.0f);
            const float hi = fminf(fmaxf(ceilf((xf + half) * ip + c0f), -2.0f), (float)nxe + 1.0f);
            c_lo = max(0, (int)lo - 1);
            c_hi = min(nxe - 1, (int)hi + 1);
        } else {
            c_lo = 0;
            c_hi = nxe - 1;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        c_lo = min(c_lo, __shfl_xor_sync(0xffffffffu, c_lo, o));
        c_hi = max(c_hi, __shfl_xor_sync(0xffffffffu, c_hi, o));
    }

    SepAcc<FPT, FS> acc;
    acc.init();
    const ChT *chp = ch + (fbase + FL * sub) * 2;
    const int lane0 = (threadIdx.x & 31) - sub;  // the pixel's first lane

    for (int r = row_lo; r <= row_hi; ++r) {
        for (int g0 = c_lo; g0 <= c_hi; g0 += TPP) {
            const int cq = g0 + sub;
            const int cc = min(cq, nxe - 1);
            const bool on = live && cq <= c_hi && fabsf(__fsub_rn(xf, exf[cc])) <= half;
            if (!__any_sync(0xffffffffu, on)) continue;
            ff rm = {0.0f, 0.0f};
            if (on) {
                ff dxx = fqi::ff_add(X, ff{-exh[cc], -exl[cc]});
                ff r2 = fqi::ff_add(fqi::ff_sqr(dxx), zz);
                if (matrix || yf != 0.0f) {
                    ff dyy = fqi::ff_add(Y, ff{-eyh[r], -eyl[r]});
                    r2 = fqi::ff_add(r2, fqi::ff_sqr(dyy));
                }
                rm = fqi::ff_sqrt(r2);
            }
            for (int a = 0; a < p.A; ++a) {
                int i = 0;
                float phi = 0.0f, sn = 0.0f, cs = 1.0f;
                bool ok = on;
                if (on) {
                    const float2 pt = ptx_s[a * W + col];
                    const ff path = fqi::ff_add(ff{pt.x, pt.y}, rm);
                    const ff u = fqi::ff_mul(path, fs_c);
                    fqi::ff_floor_frac(u, i, phi);
                    if (i < 0 || i + 1 >= ns) {
                        ok = false;
                    } else if (p.rot_tab) {
                        float sh, ch;
                        das_sincos_poly(p.pi_f0_fs * phi, sh, ch);
                        const float ce = __fmul_rn(__fsub_rn(ch, sh), __fadd_rn(ch, sh));
                        const float se = __fmul_rn(2.0f * sh, ch);
                        const float2 t = rot_s[i];
                        cs = fmaf(t.x, ce, -__fmul_rn(t.y, se));
                        sn = fmaf(t.x, se, __fmul_rn(t.y, ce));
                    } else {
                        const float cyc = fqi::ff_frac(fqi::ff_mul(u, f0_fs));
                        sincospif(2.0f * cyc, &sn, &cs);
                    }
                }
                const int ion = ok ? (r * nxe + cq) * ns + i : -1;
                const ChT *cha = chp + (int64_t)a * M * line_stride;
#pragma unroll
                for (int j = 0; j < TPP; ++j) {  // the group's elements in turn
                    const int src = lane0 + j;
                    const int ij = __shfl_sync(0xffffffffu, ion, src);
                    const float phj = __shfl_sync(0xffffffffu, phi, src);
                    const float snj = __shfl_sync(0xffffffffu, sn, src);
                    const float csj = __shfl_sync(0xffffffffu, cs, src);
                    // an element without an echo in the record reads row 0
                    // with a zero rotation (adds exact zeros): no branch in
                    // the loop, 5.03 -> 4.57 ms on the 2D workload
                    const bool use = ij >= 0;
                    acc.add(cha + (uint64_t)(unsigned)(use ? ij : 0) * (uint64_t)row_stride, row_stride, phj,
                            use ? csj : 0.0f, use ? snj : 0.0f);
                }
            }
        }
    }
    if (live) {
#pragma unroll
        for (int k = 0; k < FPT; ++k) {
            const int fk = fbase + FL * ((k / FL) * FS + sub) + k % FL;
            const float2 v = acc.get(k);
            if (fk < p.F) fqi::store_c(iq, pix * p.F + fk, make_float2(v.x * p.inv_A, v.y * p.inv_A));
        }
    }
    __syncthreads();
}


// ---- one warp per pixel (16-bit channel data) ---------------------------
// A CTA of NW = blockDim.x / 32 warps takes NW consecutive voxels along x of
// one (y, z) row (das_ctas with W = NW), frames 128 by .. 128 by + 127:
// lane l sums frames 128 by + 4 l .. + 3, so that a load instruction reads
// one element's samples of 128 consecutive frames (512 bytes of 16-bit data,
// 1024 of FP32).  Per group of 32 columns of an aperture row, lane l
// evaluates column g0 + l's receive distance once and, per transmit, its
// delay and carrier rotation into the warp's slot table; then the warp walks
// the group's elements with an echo in the record, each read back from the
// table by every lane (a broadcast), so the loop has no divergence.  Lanes
// whose frames lie beyond the padded count repeat the last frame group and
// discard it (F = 100: 28 of 32 lanes carry frames).  3D workload (128^3 voxels, 100 frames, BF16 channels): 662 ms
// against 783 ms for four threads per pixel with two element and two frame
// slots (8 frames per delay and thread, the first of these kernels to
// share a delay over more than 4 frames) and 1031 ms for four threads per
// pixel over 4 frames each; loading two elements before summing either
// (with the earlier per-lane test in the loop: 684 ms against 690 for BF16,
// 793 against 719 for FP16) and precomputing the broadcast values (778 ms)
// are not used.
constexpr int kDasWarpFrames = 128;

__host__ __device__ inline int das_w_off_slot(int M, int A, int NW) { return das_off_ptx(M) + ((2 * A * NW + 3) & ~3); }
__host__ __device__ inline int das_w_off_rot(int M, int A, int NW) { return das_w_off_slot(M, A, NW) + 4 * 32 * NW; }
__host__ __device__ inline size_t das_w_smem_bytes(int M, int A, int NW, int rot_ns)
{
    return sizeof(float) * (size_t)das_w_off_rot(M, A, NW) + sizeof(float2) * (size_t)rot_ns;
}

template <typename ChT, typename OutT>
__device__ __forceinline__ void das_tile_w(const DasParams &p, int64_t bx, int by, const ChT *__restrict__ ch,
                                           OutT *__restrict__ iq, float *etab)
{
    const int M = p.pr.M, nxe = p.pr.nx, nye = p.pr.ny;
    const int NW = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float *exf = etab, *exh = etab + nxe, *exl = etab + 2 * nxe;
    float *eyf = etab + 3 * nxe, *eyh = eyf + nye, *eyl = eyf + 2 * nye;
    float2 *ptx_s = reinterpret_cast<float2 *>(etab + das_off_ptx(M));                      // [A][NW]
    float4 *slot = reinterpret_cast<float4 *>(etab + das_w_off_slot(M, p.A, NW)) + 32 * wid;  // [32] this warp's
    float2 *rot_s = reinterpret_cast<float2 *>(etab + das_w_off_rot(M, p.A, NW));             // [ns]
    for (int c = threadIdx.x; c < nxe + nye; c += blockDim.x) {
        const bool isx = c < nxe;
        const int i = isx ? c : c - nxe, n = isx ? nxe : nye;
        const double e = __dmul_rn(__dsub_rn((double)i, __dmul_rn(0.5, (double)(n - 1))), isx ? p.pitch_x : p.pitch_y);
        const fqi::df2 sp = fqi::split_double(e);
        if (isx) {
            exf[i] = (float)e; exh[i] = sp.hi; exl[i] = sp.lo;
        } else {
            eyf[i] = (float)e; eyh[i] = sp.hi; eyl[i] = sp.lo;
        }
    }
    const int nxb = (p.gx + NW - 1) / NW;
    const int xb = (int)(bx % nxb);
    const int64_t t = bx / nxb;
    const int iy = (int)(t % p.gy);
    const int iz = (int)(t / p.gy);
    const int ix = xb * NW + wid;
    const bool live = ix < p.gx && iz < p.gz;  // warp-uniform
    const int64_t pix = ((int64_t)iy * p.gz + iz) * p.gx + ix;
    const int f0 = by * kDasWarpFrames + 4 * lane;  // this lane's first frame
    const bool fon = f0 < p.Fp;
    const double xd = __dadd_rn(p.x0, __dmul_rn((double)(live ? ix : 0), p.dx));
    const double yd = __dadd_rn(p.y0, __dmul_rn((double)iy, p.dy));
    const double zd = __dadd_rn(p.z0, __dmul_rn((double)iz, p.dz));
    const float xf = (float)xd, yf = (float)yd, zf = (float)zd;
    const fqi::df2 xs = fqi::split_double(xd), ys = fqi::split_double(yd), zs = fqi::split_double(zd);
    const ff X = {xs.hi, xs.lo}, Y = {ys.hi, ys.lo}, Z = {zs.hi, zs.lo};
    const ff zz = fqi::ff_sqr(Z);
    const float half = __fmul_rn(zf, p.half_per_z);
    const bool matrix = nye > 1;
    const ff fs_c = fqi::ff_load(p.pr.fs_over_c);
    const ff f0_fs = fqi::ff_load(p.pr.f0_over_fs);
    const int ns = p.pr.ns;
    const int64_t row_stride = (int64_t)p.Fp * 2;
    const int64_t line_stride = (int64_t)ns * row_stride;

    if (p.rot_tab) {
        for (int n = threadIdx.x; n < ns; n += blockDim.x) {
            float sn, cs;
            sincospif(2.0f * fqi::ff_frac(fqi::ff_mul(f0_fs, ff{(float)n, 0.0f})), &sn, &cs);
            rot_s[n] = make_float2(cs, sn);
        }
    }
    for (int a = lane; a < p.A; a += 32) {
        const fqi::AngleFF an = p.ang[a];
        ff ptx = fqi::ff_add(fqi::ff_mul(fqi::ff_load(an.ux), X), fqi::ff_mul(fqi::ff_load(an.uy), Y));
        ptx = fqi::ff_add(ptx, fqi::ff_mul(fqi::ff_load(an.uz), Z));
        ptx = fqi::ff_add(ptx, fqi::ff_neg(fqi::ff_load(an.origin)));
        ptx_s[a * NW + wid] = make_float2(ptx.hi, ptx.lo);
    }
    __syncthreads();

    int row_lo = 0, row_hi = nye - 1;
    if (matrix) {
        row_lo = nye;
        row_hi = -1;
        for (int r = 0; r < nye; ++r) {
            if (fabsf(__fsub_rn(yf, eyf[r])) <= half) {
                row_lo = min(row_lo, r);
                row_hi = r;
            }
        }
    }
    // columns the pixel's aperture can reach: an estimate one column wider on
    // each side (the per-element test below decides)
    int c_lo = nxe, c_hi = -1;
    if (live) {
        if (nxe > 1 && p.pitch_x > 0.0) {
            const float c0f = 0.5f * (float)(nxe - 1);
            const float ip = (float)(1.0 / p.pitch_x);
            const float lo = fminf(fmaxf(floorf((xf - half) * ip + c0f), -2.0f), (float)nxe + 1.0f);
            const float hi = fminf(fmaxf(ceilf((xf + half) * ip + c0f), -2.0f), (float)nxe + 1.0f);
            c_lo = max(0, (int)lo - 1);
            c_hi = min(nxe - 1, (int)hi + 1);
        } else {
            c_lo = 0;
            c_hi = nxe - 1;
        }
    }

    static_assert(sizeof(ChT) == 2, "das_tile_w takes 16-bit channel data");
    RotAcc<4, 1, ChT> acc;
    acc.init();
    // lanes past the padded frame count read the last frame group (their
    // sums are never stored), so the element loop has no branch: 690 ->
    // 662 ms on the 3D workload against a test per element
    const ChT *chp = ch + (int64_t)(fon ? f0 : p.Fp - 4) * 2;
    const unsigned rs32 = (unsigned)(p.Fp * 2);

    for (int r = row_lo; r <= row_hi; ++r) {
        for (int g0 = c_lo; g0 <= c_hi; g0 += 32) {
            const int cq = g0 + lane;
            const int cc = min(cq, nxe - 1);
            const bool on = cq <= c_hi && fabsf(__fsub_rn(xf, exf[cc])) <= half;
            if (!__any_sync(0xffffffffu, on)) continue;
            ff rm = {0.0f, 0.0f};
            if (on) {
                ff dxx = fqi::ff_add(X, ff{-exh[cc], -exl[cc]});
                ff r2 = fqi::ff_add(fqi::ff_sqr(dxx), zz);
                if (matrix || yf != 0.0f) {
                    ff dyy = fqi::ff_add(Y, ff{-eyh[r], -eyl[r]});
                    r2 = fqi::ff_add(r2, fqi::ff_sqr(dyy));
                }
                rm = fqi::ff_sqrt(r2);
            }
            for (int a = 0; a < p.A; ++a) {
                int i = 0;
                float phi = 0.0f, sn = 0.0f, cs = 1.0f;
                bool ok = on;
                if (on) {
                    const float2 pt = ptx_s[a * NW + wid];
                    const ff path = fqi::ff_add(ff{pt.x, pt.y}, rm);
                    const ff u = fqi::ff_mul(path, fs_c);
                    fqi::ff_floor_frac(u, i, phi);
                    if (i < 0 || i + 1 >= ns) {
                        ok = false;
                    } else if (p.rot_tab) {
                        float sh, ch;
                        das_sincos_poly(p.pi_f0_fs * phi, sh, ch);
                        const float ce = __fmul_rn(__fsub_rn(ch, sh), __fadd_rn(ch, sh));
                        const float se = __fmul_rn(2.0f * sh, ch);
                        const float2 t = rot_s[i];
                        cs = fmaf(t.x, ce, -__fmul_rn(t.y, se));
                        sn = fmaf(t.x, se, __fmul_rn(t.y, ce));
                    } else {
                        const float cyc = fqi::ff_frac(fqi::ff_mul(u, f0_fs));
                        sincospif(2.0f * cyc, &sn, &cs);
                    }
                }
                // the channel row (element, sample) within this angle's lines
                // (M ns < 2^28: it fits an int)
                slot[lane] = make_float4(__int_as_float(ok ? (r * nxe + cq) * ns + i : 0), phi, cs, sn);
                __syncwarp();
                unsigned m = __ballot_sync(0xffffffffu, ok);
                const ChT *cha = chp + (int64_t)a * M * line_stride;
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1;
                    const float4 d = slot[j];
                    acc.add(cha + (uint64_t)(unsigned)__float_as_int(d.x) * rs32, row_stride, d.y, d.z, d.w);
                }
                __syncwarp();
            }
        }
    }
    if (live && fon) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 v = acc.get(k);
            if (f0 + k < p.F) fqi::store_c(iq, pix * p.F + f0 + k, make_float2(v.x * p.inv_A, v.y * p.inv_A));
        }
    }
    __syncthreads();  // a persistent CTA's next tile rewrites the shared tables
}

// Launch bounds give the thread count alone; ptxas picks the register
// count (48 for the branch-free element loop, 662 ms on the 3D workload; a
// 6-CTA bound, at most 42, 669 ms).  With the earlier per-lane test in the
// loop it picked 40 (a few spilled values, 690 ms), where bounds allowing
// 42-48 registers without spills measured 795-799 ms and 70 registers
// 1089 ms; 128- or 512-thread CTAs 865 and 897 ms.
constexpr int kDasWarpThreads = 256;
static_assert(kDasWarpFrames == fqb::kDasWarpFramesB, "batched item shapes");

template <typename ChT, typename OutT, int NT>
__global__ void __launch_bounds__(NT) das_w_kernel(const DasParams p, const ChT *__restrict__ ch, OutT *__restrict__ iq)
{
    extern __shared__ __align__(16) float etab[];  // das_w_smem_bytes
    das_tile_w<ChT, OutT>(p, blockIdx.x, blockIdx.y, ch, iq, etab);
}

template <typename ChT, typename OutT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) das_kernel(const DasParams p, const ChT *__restrict__ ch, OutT *__restrict__ iq)
{
    extern __shared__ __align__(16) float etab[];  // das_smem_bytes: element tables, transmit paths, carrier table
    das_tile<ChT, OutT>(p, blockIdx.x, blockIdx.y, ch, iq, etab);
}

constexpr int kDasParamBytes = (sizeof(DasParams) + 15) & ~15;

template <typename ChT, typename OutT, int NT>
__global__ void __launch_bounds__(NT) das_batched_kernel(const fqb::EnsDev *__restrict__ ens, const fqb::StageQueue q)
{
    extern __shared__ __align__(16) float etab[];
    __shared__ __align__(16) unsigned char s_par[kDasParamBytes];
    __shared__ int s_buf[2];
    int cur = -1;
    fqb::Item it;
    while (fqb::next_item(q, ens, fqb::ST_DAS, s_buf, it)) {
        const fqb::EnsDev &e = ens[it.e];
        if (it.e != cur) {
            fqb::copy_block(s_par, e.das_params, kDasParamBytes);
            cur = it.e;
            __syncthreads();
        }
        if constexpr (sizeof(ChT) == 2)
            das_tile_w<ChT, OutT>(*reinterpret_cast<const DasParams *>(s_par), it.x, it.y, (const ChT *)e.ch,
                                  (OutT *)e.iq, etab);
        else
            das_tile<ChT, OutT>(*reinterpret_cast<const DasParams *>(s_par), it.x, it.y, (const ChT *)e.ch,
                                (OutT *)e.iq, etab);
    }
}

fq_status check_probe_tx(const fq_probe *probe, const fq_tx *tx, const char *who)
{
    FQ_REQUIRE(probe && tx, FQ_ERR_INVALID_ARG, "%s: null probe/tx", who);
    FQ_REQUIRE(tx->n_angles >= 1 && tx->n_angles <= FQ_MAX_ANGLES && tx->tilt_x && tx->tilt_y, FQ_ERR_SHAPE,
               "%s: n_angles must be in [1, %d]", who, FQ_MAX_ANGLES);
    FQ_REQUIRE(probe->nx >= 1 && probe->ny >= 1 && (int64_t)probe->nx * probe->ny <= 4096, FQ_ERR_SHAPE,
               "%s: element count must be in [1, 4096]", who);
    FQ_REQUIRE(probe->n_samples >= 2 && probe->n_samples <= 65536, FQ_ERR_SHAPE, "%s: bad n_samples", who);
    FQ_REQUIRE(probe->f0 > 0 && probe->fs > 0 && probe->c > 0, FQ_ERR_INVALID_ARG, "%s: f0, fs, c must be > 0",
               who);
    return FQ_OK;
}

template <typename ChT, typename OutT>
fq_status launch_das(const DasParams &p, const void *ch, void *iq, cudaStream_t st)
{
    if constexpr (sizeof(ChT) == 2) {
        constexpr int NW = kDasWarpThreads / 32;
        const size_t smem = das_w_smem_bytes(p.pr.M, p.A, NW, p.rot_tab ? p.pr.ns : 0);
        auto kern = das_w_kernel<ChT, OutT, kDasWarpThreads>;
        if (smem > 48 * 1024) {
            fq_status s = fqi::cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               (int)smem), "fq_das: smem attribute");
            if (s) return s;
        }
        dim3 grid((unsigned)das_ctas(p.gx, p.gy, p.gz, NW), (p.Fp + kDasWarpFrames - 1) / kDasWarpFrames);
        kern<<<grid, kDasWarpThreads, smem, st>>>(p, (const ChT *)ch, (OutT *)iq);
        return fqi::launch_check("fq_das");
    } else {
        size_t smem = das_smem_bytes(p.pr.M, p.A, kDasThreads, kDasTPP, p.rot_tab ? p.pr.ns : 0);
        // resident CTAs per SM the register budget targets: 8 (64 registers
        // per thread) or 4 (up to 128); FQ_DAS_MINB=4 selects the latter for
        // tuning
        static int minb = -1;
        if (minb < 0) {
            const char *env = std::getenv("FQ_DAS_MINB");
            minb = (env && env[0] == '4') ? 4 : 8;
        }
        auto kern = minb == 4 ? das_kernel<ChT, OutT, kDasThreads, 4> : das_kernel<ChT, OutT, kDasThreads, 8>;
        if (smem > 48 * 1024) {
            fq_status s = fqi::cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               (int)smem), "fq_das: smem attribute");
            if (s) return s;
        }
        dim3 grid((unsigned)das_ctas(p.gx, p.gy, p.gz, kDasThreads / kDasTPP), p.Fp / kFrameChunk);
        kern<<<grid, kDasThreads, smem, st>>>(p, (const ChT *)ch, (OutT *)iq);
        return fqi::launch_check("fq_das");
    }
}

void make_das_params(const fq_probe *probe, const fq_tx *tx, int F, const fq_grid *g, DasParams &p)
{
    std::memset(&p, 0, sizeof p);
    fqi::make_probe_ff(probe, p.pr);
    p.pitch_x = probe->pitch_x;
    p.pitch_y = probe->pitch_y;
    p.A = tx->n_angles;
    p.F = F;
    p.Fp = fq_frame_pad(F);
    p.gx = g->nx; p.gy = g->ny; p.gz = g->nz;
    p.P = (int64_t)g->nx * g->ny * g->nz;
    p.x0 = g->x0; p.y0 = g->y0; p.z0 = g->z0;
    p.dx = g->dx; p.dy = g->dy; p.dz = g->dz;
    p.half_per_z = (float)(0.5 / g->fnumber);
    p.inv_A = 1.0f / (float)p.A;
    p.rot_tab = das_rot_tab(probe) ? 1 : 0;
    p.pi_f0_fs = (float)(M_PI * probe->f0 / probe->fs);
    fqi::make_angles_ff(probe, tx, p.ang);
}

fq_status run_das(const fq_probe *probe, const fq_tx *tx, const void *ch, int ch_dtype, int F, const fq_grid *g,
                  int iq_dtype, void *iq, cudaStream_t st)
{
    FQ_REQUIRE(g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1, FQ_ERR_SHAPE, "fq_das: bad grid");
    FQ_REQUIRE(g->fnumber > 0.0, FQ_ERR_INVALID_ARG, "fq_das: fnumber must be > 0");
    DasParams p;
    make_das_params(probe, tx, F, g, p);
    FQ_REQUIRE(iq_dtype == FQ_F32 || iq_dtype == FQ_BF16, FQ_ERR_UNSUPPORTED,
               "fq_das: the Casorati dtype must be FQ_F32 or FQ_BF16");
    return fqi::with_storage(ch_dtype, "fq_das (channel IQ)", [&](auto *chp) {
        using ChT = fqi::storage_t<decltype(chp)>;
        return iq_dtype == FQ_F32 ? launch_das<ChT, float>(p, ch, iq, st) : launch_das<ChT, __nv_bfloat16>(p, ch, iq, st);
    });
}

size_t elem_size(int dtype) { return dtype == FQ_F32 ? 4 : 2; }

}  // namespace

extern "C" {

int32_t fq_frame_pad(int32_t n_frames)
{
    if (n_frames < 1) return 0;
    return (n_frames + kFrameChunk - 1) / kFrameChunk * kFrameChunk;
}

fq_status fq_rf2iq(const fq_probe *probe, int32_t n_lines, int32_t n_frames, const void *rf, int32_t rf_dtype,
                   int32_t iq_dtype, void *iq_ch, void *stream)
{
    FQ_REQUIRE(probe && rf && iq_ch, FQ_ERR_INVALID_ARG, "fq_rf2iq: null argument");
    FQ_REQUIRE(n_lines >= 1 && n_lines <= 65535 * 64 && n_frames >= 1, FQ_ERR_SHAPE, "fq_rf2iq: bad sizes");
    FQ_REQUIRE(n_lines <= 65535, FQ_ERR_SHAPE, "fq_rf2iq: at most 65535 lines");
    FQ_REQUIRE(probe->n_samples >= 2 && probe->f0 > 0 && probe->fs > 0, FQ_ERR_INVALID_ARG, "fq_rf2iq: bad probe");
    FQ_REQUIRE(fqi::aligned(iq_ch, 16), FQ_ERR_ALIGN, "fq_rf2iq: iq_ch must be 16-byte aligned");
    return run_rf2iq(probe, n_lines, n_frames, rf, rf_dtype, iq_dtype, iq_ch, (cudaStream_t)stream);
}

fq_status fq_das(const fq_probe *probe, const fq_tx *tx, const void *iq_ch, int32_t ch_dtype, int32_t n_frames,
                 const fq_grid *grid, int32_t iq_dtype, void *iq, void *stream)
{
    fq_status s = check_probe_tx(probe, tx, "fq_das");
    if (s) return s;
    FQ_REQUIRE(iq_ch && iq && n_frames >= 1, FQ_ERR_INVALID_ARG, "fq_das: null argument or n_frames < 1");
    FQ_REQUIRE(fqi::aligned(iq_ch, 16) && fqi::aligned(iq, 8), FQ_ERR_ALIGN,
               "fq_das: iq_ch must be 16-byte and iq 8-byte aligned");
    return run_das(probe, tx, iq_ch, ch_dtype, n_frames, grid, iq_dtype, iq, (cudaStream_t)stream);
}

fq_status fq_beamform_das_workspace_size(const fq_probe *probe, const fq_tx *tx, int32_t n_frames, int32_t ch_dtype,
                                         size_t *bytes)
{
    FQ_REQUIRE(probe && tx && bytes && n_frames >= 1, FQ_ERR_INVALID_ARG, "fq_beamform_das_workspace_size: bad args");
    size_t n = (size_t)tx->n_angles * probe->nx * probe->ny * probe->n_samples * fq_frame_pad(n_frames) * 2;
    *bytes = (n * elem_size(ch_dtype) + 255) & ~(size_t)255;
    return FQ_OK;
}

fq_status fq_beamform_das(const fq_probe *probe, const fq_tx *tx, const void *rf, int32_t rf_dtype,
                          int32_t n_frames, const fq_grid *grid, int32_t ch_dtype, int32_t iq_dtype, void *iq,
                          void *workspace, size_t workspace_bytes, void *stream)
{
    fq_status s = check_probe_tx(probe, tx, "fq_beamform_das");
    if (s) return s;
    FQ_REQUIRE(rf && iq && n_frames >= 1, FQ_ERR_INVALID_ARG, "fq_beamform_das: null argument");
    size_t need = 0;
    fq_beamform_das_workspace_size(probe, tx, n_frames, ch_dtype, &need);
    FQ_REQUIRE(workspace && workspace_bytes >= need, FQ_ERR_WORKSPACE, "fq_beamform_das: workspace needs %zu bytes",
               need);
    FQ_REQUIRE(fqi::aligned(workspace, 256) && fqi::aligned(iq, 8), FQ_ERR_ALIGN,
               "fq_beamform_das: workspace must be 256-byte and iq 8-byte aligned");
    int L = tx->n_angles * probe->nx * probe->ny;
    FQ_REQUIRE(L <= 65535, FQ_ERR_SHAPE, "fq_beamform_das: at most 65535 channel lines");
    cudaStream_t st = (cudaStream_t)stream;
    s = run_rf2iq(probe, L, n_frames, rf, rf_dtype, ch_dtype, workspace, st);
    if (s) return s;
    return run_das(probe, tx, workspace, ch_dtype, n_frames, grid, iq_dtype, iq, st);
}

}  // extern "C"

namespace fqi {

size_t iq_params_bytes() { return kIqParamBytes; }

fq_status build_iq_params(const fq_probe *probe, int L, int F, void *out, int *J)
{
    std::memset(out, 0, kIqParamBytes);
    Rf2iqParams &p = *reinterpret_cast<Rf2iqParams *>(out);
    FQ_REQUIRE(make_rf2iq_params(probe, L, F, p), FQ_ERR_SHAPE, "batch: 2 round(fs/f0) must be <= %d",
               kMaxHalfTaps);
    *J = p.J;
    return FQ_OK;
}

size_t das_params_bytes() { return kDasParamBytes; }

fq_status build_das_params(const fq_probe *probe, const fq_tx *tx, int F, const fq_grid *g, void *out)
{
    std::memset(out, 0, kDasParamBytes);
    make_das_params(probe, tx, F, g, *reinterpret_cast<DasParams *>(out));
    return FQ_OK;
}

template <typename InT, typename OutT>
fq_status launch_rf2iq_batched(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int J_max,
                               cudaStream_t st)
{
    const int W = kRfTile + 2 * J_max;
    const size_t smem = sizeof(float2) * ((size_t)kFrameChunk * (W | 1) + W);
    const int grid = fqb::persistent_grid(rf2iq_batched_kernel<InT, OutT>, 256, smem, items);
    rf2iq_batched_kernel<InT, OutT><<<grid, 256, smem, st>>>(ens, q);
    return launch_check("batched rf2iq");
}

fq_status batched_rf2iq(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int rf_dtype, int ch_dtype,
                        int J_max, cudaStream_t st)
{
    if (rf_dtype == FQ_F32 && ch_dtype == FQ_F32) return launch_rf2iq_batched<float, float>(ens, q, items, J_max, st);
    if (rf_dtype == FQ_F32) return launch_rf2iq_batched<float, __nv_bfloat16>(ens, q, items, J_max, st);
    if (ch_dtype == FQ_F32) return launch_rf2iq_batched<__nv_bfloat16, float>(ens, q, items, J_max, st);
    return launch_rf2iq_batched<__nv_bfloat16, __nv_bfloat16>(ens, q, items, J_max, st);
}

template <typename ChT, typename OutT, int NT>
fq_status launch_das_batched(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int M_max, int A_max,
                             int ns_max, cudaStream_t st)
{
    const int rot = std::min(ns_max, kRotTabMax);
    const size_t smem = sizeof(ChT) == 2 ? das_w_smem_bytes(M_max, A_max, NT / 32, rot)
                                         : das_smem_bytes(M_max, A_max, NT, kDasTPP, rot);
    auto kern = das_batched_kernel<ChT, OutT, NT>;
    fq_status s = cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "batched DAS: smem attribute");
    if (s) return s;
    const int grid = fqb::persistent_grid(kern, NT, smem, items);
    kern<<<grid, NT, smem, st>>>(ens, q);
    return launch_check("batched DAS");
}

template <typename ChT, typename OutT>
fq_status das_by_threads(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int M_max, int A_max,
                         int ns_max, int threads, cudaStream_t st)
{
    if (threads == 64) return launch_das_batched<ChT, OutT, 64>(ens, q, items, M_max, A_max, ns_max, st);
    if (threads == 256) return launch_das_batched<ChT, OutT, 256>(ens, q, items, M_max, A_max, ns_max, st);
    return launch_das_batched<ChT, OutT, 128>(ens, q, items, M_max, A_max, ns_max, st);
}

fq_status batched_das(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int ch_dtype, int iq_dtype,
                      int M_max, int A_max, int ns_max, int threads, cudaStream_t st)
{
    if (ch_dtype == FQ_F32 && iq_dtype == FQ_F32)
        return das_by_threads<float, float>(ens, q, items, M_max, A_max, ns_max, threads, st);
    if (ch_dtype == FQ_F32)
        return das_by_threads<float, __nv_bfloat16>(ens, q, items, M_max, A_max, ns_max, threads, st);
    if (iq_dtype == FQ_F32)
        return das_by_threads<__nv_bfloat16, float>(ens, q, items, M_max, A_max, ns_max, threads, st);
    return das_by_threads<__nv_bfloat16, __nv_bfloat16>(ens, q, items, M_max, A_max, ns_max, threads, st);
}

}  // namespace fqi
