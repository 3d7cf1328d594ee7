// rf_freq.cu -- RF synthesis in the frequency domain: Eq. 1 evaluated per
// frequency as Alg. 2 step 2.6 does (wavenumber, attenuation and
// directivity at each frequency, spectral weights, then the inverse
// transform), with the geometry of the time-domain kernels (ideal plane-wave
// transmit, receive at the element centre).  It closes the narrowband
// approximation of the time-domain model (attenuation and directivity at
// f0) and measures what the paper's frequency loop costs on GB300.
//
//   RF[n] = df sum_s sum_{j < N/2} w_j Re{ S(f_j) A_j e^{i 2 pi f_j (n/fs - tau)} },
//   A_j = R D_j exp(-alpha f_j c tau) / r,  D_j = sinc(k_j b sin theta).
//
// Spectrum kernel: one CTA per (frame, transmit, element), one thread per
// 16 consecutive bins.  Per chunk of 256 scatterers the CTA first evaluates
// each scatterer's float-float delay (in cycles per bin, df tau), the
// attenuation exponent per bin, R / r and the directivity step b k_1 sin
// theta into shared memory; then every thread walks the chunk, anchors the
// phase e^{-i 2 pi j0 df tau}, the attenuation and the directivity sine at
// its first bin with accurate functions and advances them over its 16 bins
// by recurrences (complex rotation, ratio, Chebyshev), adding the terms into
// binary32 chunk sums that are folded into float-pair accumulators after
// each chunk.  Inverse-transform kernel: one CTA per line, an in-place
// radix-2 complex FFT of length N in shared memory of
// df w_j S(f_j) P_j, the real part of the first Ns samples is the RF.
#include <cmath>
#include <cstring>
#include <vector>

#include "fq_internal.cuh"

namespace {

using fqi::ff;

constexpr int kBinsPerThread = 16;
constexpr int kChunk = 256;
constexpr int kMaxFft = 8192;

struct FreqParams {
    fqi::ProbeFF pr;
    int A, J, N;
    int64_t S;
    fqi::df2 dfc;        // df / c (cycles per bin per metre of path)
    float atn_per_m;     // alpha (Np / (m Hz)) x df: attenuation exponent per bin per metre
    float bkx, bky;      // b k_1 per unit sin(theta): (width / 2) 2 pi df / c
    fqi::AngleFF ang[FQ_MAX_ANGLES];
};

__global__ void __launch_bounds__(kChunk) spectrum_kernel(const FreqParams p, const float *__restrict__ pos,
                                                          const float *__restrict__ amp, float2 *__restrict__ spec)
{
    __shared__ float s_ch[kChunk], s_cl[kChunk], s_atn[kChunk], s_rr[kChunk], s_bx[kChunk], s_by[kChunk];
    const int m = blockIdx.x, a = blockIdx.y, f = blockIdx.z;
    const int M = p.pr.M;
    const int64_t S = p.S;
    const float *X = pos + (int64_t)f * 3 * S, *Y = X + S, *Z = Y + S;
    const bool matrix = p.pr.ny > 1;
    const ff ex = fqi::elem_coord(m % p.pr.nx, p.pr.nx, p.pr.pitch_x);
    const ff ey = fqi::elem_coord(m / p.pr.nx, p.pr.ny, p.pr.pitch_y);
    const fqi::AngleFF an = p.ang[a];
    const ff dfc = fqi::ff_load(p.dfc);
    const int j0 = threadIdx.x * kBinsPerThread;
    const bool live = j0 < p.J;
    float accH[kBinsPerThread][2], accL[kBinsPerThread][2];
#pragma unroll
    for (int b = 0; b < kBinsPerThread; ++b) accH[b][0] = accH[b][1] = accL[b][0] = accL[b][1] = 0.0f;

    for (int64_t c0 = 0; c0 < S; c0 += kChunk) {
        const int n = (int)min((int64_t)kChunk, S - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int64_t s = c0 + t;
            const float x = X[s], y = Y[s], z = Z[s];
            const ff ptx = fqi::ff_dot3_minus(an.ux, an.uy, an.uz, an.origin, x, y, z);
            const ff dx = fqi::ff_add(ff{x, 0.0f}, fqi::ff_neg(ex));
            ff r2 = fqi::ff_add(fqi::ff_sqr(dx), fqi::ff_two_prod(z, z));
            ff dy = ff{0.0f, 0.0f};
            if (matrix || y != 0.0f) {
                dy = fqi::ff_add(ff{y, 0.0f}, fqi::ff_neg(ey));
                r2 = fqi::ff_add(r2, fqi::ff_sqr(dy));
            }
            const bool ok = r2.hi > 0.0f;
            const ff r = ok ? fqi::ff_sqrt(r2) : ff{1.0f, 0.0f};
            const ff L = fqi::ff_add(ptx, r);              // two-way path (m)
            const ff cyc = fqi::ff_mul(L, dfc);            // df tau
            s_ch[t] = cyc.hi;
            s_cl[t] = cyc.lo;
            s_atn[t] = p.atn_per_m * L.hi;
            const float rinv = 1.0f / r.hi;
            s_rr[t] = ok ? amp[s] * rinv : 0.0f;
            s_bx[t] = p.bkx * (dx.hi * rinv);
            s_by[t] = matrix ? p.bky * (dy.hi * rinv) : 0.0f;
        }
        __syncthreads();
        if (!live) continue;
        float fa[kBinsPerThread][2];
#pragma unroll
        for (int b = 0; b < kBinsPerThread; ++b) fa[b][0] = fa[b][1] = 0.0f;
        for (int t = 0; t < n; ++t) {
            const float rr = s_rr[t];
            if (rr == 0.0f) continue;
            const ff cyc = {s_ch[t], s_cl[t]};
            // phase e^{-i 2 pi j df tau} at the first bin and its step
            float sn, cs, ws, wc;
            sincospif(-2.0f * fqi::ff_frac(fqi::ff_mul_f(cyc, (float)j0)), &sn, &cs);
            sincospif(-2.0f * fqi::ff_frac(cyc), &ws, &wc);
            float zr = cs, zi = sn;
            // attenuation exp(-alpha f_j L) and its ratio per bin
            const float atn = s_atn[t];
            float att = expf(-atn * (float)j0);
            const float q = expf(-atn);
            // directivity sinc(j beta): sine by the Chebyshev recurrence
            const float bx = s_bx[t], by = s_by[t];
            float sbx, cbx, sx0, cx0;
            sincosf(bx, &sbx, &cbx);
            sincosf(bx * (float)j0, &sx0, &cx0);
            float sx_prev = fmaf(sx0, cbx, -cx0 * sbx), sx = sx0;  // sin((j0 - 1) bx), sin(j0 bx)
            const float tcx = 2.0f * cbx;
            float sy_prev = 0.0f, sy = 0.0f, tcy = 0.0f;
            if (matrix) {
                float sby, cby, sy0, cy0;
                sincosf(by, &sby, &cby);
                sincosf(by * (float)j0, &sy0, &cy0);
                sy_prev = fmaf(sy0, cby, -cy0 * sby);
                sy = sy0;
                tcy = 2.0f * cby;
            }
#pragma unroll
            for (int b = 0; b < kBinsPerThread; ++b) {
                const float jj = (float)(j0 + b);
                const float xb = jj * bx;
                float D = (xb == 0.0f) ? 1.0f : __fdividef(sx, xb);
                if (matrix) {
                    const float yb = jj * by;
                    D *= (yb == 0.0f) ? 1.0f : __fdividef(sy, yb);
                    const float syn = fmaf(tcy, sy, -sy_prev);
                    sy_prev = sy;
                    sy = syn;
                }
                const float A = rr * att * D;
                fa[b][0] = fmaf(A, zr, fa[b][0]);
                fa[b][1] = fmaf(A, zi, fa[b][1]);
                const float nzr = fmaf(zr, wc, -zi * ws), nzi = fmaf(zr, ws, zi * wc);
                zr = nzr;
                zi = nzi;
                att *= q;
                const float sxn = fmaf(tcx, sx, -sx_prev);
                sx_prev = sx;
                sx = sxn;
            }
        }
        // fold the chunk's binary32 sums into the float-pair accumulators
#pragma unroll
        for (int b = 0; b < kBinsPerThread; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float h = accH[b][c], d = fa[b][c];
                const float s = h + d, bb = s - h;
                const float e = (h - (s - bb)) + (d - bb);
                const float l = accL[b][c] + e;
                accH[b][c] = s + l;
                accL[b][c] = l - (accH[b][c] - s);
            }
    }
    if (!live) return;
    float2 *out = spec + (((int64_t)f * p.A + a) * M + m) * p.J;
#pragma unroll
    for (int b = 0; b < kBinsPerThread; ++b)
        if (j0 + b < p.J) out[j0 + b] = make_float2(accH[b][0] + accL[b][0], accH[b][1] + accL[b][1]);
}

// x[n] = sum_j Z[j] e^{+i 2 pi j n / N}, Z[j] = wS[j] P[j] (j < N/2, else 0);
// RF[n] = Re x[n] for n < Ns
template <typename OutT>
__global__ void __launch_bounds__(512) ifft_kernel(const float2 *__restrict__ spec, const float *__restrict__ wS,
                                                   int J, int N, int logN, int ns, OutT *__restrict__ rf)
{
    extern __shared__ float2 buf[];
    const int64_t line = blockIdx.x;
    const float2 *P = spec + line * J;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        float2 v = make_float2(0.0f, 0.0f);
        if (j < J) {
            const float2 q = P[j];
            v = make_float2(wS[j] * q.x, wS[j] * q.y);
        }
        buf[__brev((unsigned)j) >> (32 - logN)] = v;  // bit-reversed order for the in-place DIT
    }
    __syncthreads();
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len >> 1;
        for (int k = threadIdx.x; k < N / 2; k += blockDim.x) {
            const int grp = k / half, pos = k - grp * half;
            const int i0 = grp * len + pos, i1 = i0 + half;
            float sn, cs;
            sincospif(2.0f * (float)pos / (float)len, &sn, &cs);  // e^{+i 2 pi pos / len}
            const float2 u = buf[i0], t = buf[i1];
            const float2 v = make_float2(fmaf(t.x, cs, -t.y * sn), fmaf(t.x, sn, t.y * cs));
            buf[i0] = make_float2(u.x + v.x, u.y + v.y);
            buf[i1] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
    OutT *o = rf + line * ns;
    for (int n = threadIdx.x; n < ns; n += blockDim.x) fqi::store_f(o, n, buf[n].x);
}

double pulse_spectrum(double f, double f0, double T)
{
    const double g[3] = {f0, f0 + 1.0 / T, f0 - 1.0 / T}, c[3] = {0.5, 0.25, 0.25};
    auto sinc = [](double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; };
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += c[k] * (sinc(M_PI * (f - g[k]) * T) + sinc(M_PI * (f + g[k]) * T));
    return 0.5 * T * s;
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

size_t spec_bytes(const fq_probe *probe, const fq_tx *tx, int F, int N)
{
    return (((size_t)F * tx->n_angles * probe->nx * probe->ny * (N / 2) * sizeof(float2)) + 255) & ~(size_t)255;
}

}  // namespace

extern "C" fq_status fq_simulate_rf_freq_workspace_size(const fq_probe *probe, const fq_tx *tx, int32_t n_frames,
                                                        int32_t n_fft, size_t *bytes)
{
    FQ_REQUIRE(probe && tx && bytes && n_frames >= 1 && pow2(n_fft), FQ_ERR_INVALID_ARG,
               "fq_simulate_rf_freq_workspace_size: bad arguments (n_fft must be a power of two)");
    *bytes = spec_bytes(probe, tx, n_frames, n_fft) + (((size_t)(n_fft / 2) * 4 + 255) & ~(size_t)255);
    return FQ_OK;
}

extern "C" fq_status fq_simulate_rf_freq(const fq_probe *probe, const fq_tx *tx, const float *pos, const float *amp,
                                         int64_t S, int32_t n_frames, int32_t n_fft, int32_t out_dtype, void *rf,
                                         void *workspace, size_t workspace_bytes, void *stream)
{
    FQ_REQUIRE(probe && tx && rf && workspace, FQ_ERR_INVALID_ARG, "fq_simulate_rf_freq: null argument");
    FQ_REQUIRE(S >= 0 && n_frames >= 1 && (S == 0 || (pos && amp)), FQ_ERR_INVALID_ARG,
               "fq_simulate_rf_freq: bad scatterer arguments");
    FQ_REQUIRE(tx->n_angles >= 1 && tx->n_angles <= FQ_MAX_ANGLES && tx->tilt_x && tx->tilt_y, FQ_ERR_SHAPE,
               "fq_simulate_rf_freq: n_angles must be in [1, %d]", FQ_MAX_ANGLES);
    FQ_REQUIRE(probe->nx >= 1 && probe->ny >= 1 && probe->nx * probe->ny <= 65535 && probe->n_samples >= 2,
               FQ_ERR_SHAPE, "fq_simulate_rf_freq: bad probe sizes");
    FQ_REQUIRE(pow2(n_fft) && n_fft >= probe->n_samples && n_fft <= kMaxFft, FQ_ERR_SHAPE,
               "fq_simulate_rf_freq: n_fft must be a power of two in [n_samples, %d]", kMaxFft);
    FQ_REQUIRE(out_dtype == FQ_F32 || out_dtype == FQ_BF16, FQ_ERR_UNSUPPORTED,
               "fq_simulate_rf_freq: out_dtype must be FQ_F32 or FQ_BF16");
    size_t need = 0;
    fq_simulate_rf_freq_workspace_size(probe, tx, n_frames, n_fft, &need);
    FQ_REQUIRE(workspace_bytes >= need, FQ_ERR_WORKSPACE, "fq_simulate_rf_freq: workspace needs %zu bytes", need);
    FQ_REQUIRE(fqi::aligned(workspace, 256), FQ_ERR_ALIGN, "fq_simulate_rf_freq: workspace not 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    FreqParams p;
    std::memset(&p, 0, sizeof p);
    fqi::make_probe_ff(probe, p.pr);
    p.A = tx->n_angles;
    p.N = n_fft;
    p.J = n_fft / 2;
    p.S = S;
    const double df = probe->fs / n_fft;
    p.dfc = fqi::split_double(df / probe->c);
    p.atn_per_m = (float)(probe->alpha_db_cm_mhz * 100.0 / (20.0 / std::log(10.0)) * 1e-6 * df);
    p.bkx = (float)(0.5 * probe->width_x * 2.0 * M_PI * df / probe->c);
    p.bky = (float)(0.5 * probe->width_y * 2.0 * M_PI * df / probe->c);
    fqi::make_angles_ff(probe, tx, p.ang);
    const int M = probe->nx * probe->ny;
    float2 *spec = reinterpret_cast<float2 *>(workspace);
    float *wS = reinterpret_cast<float *>(static_cast<char *>(workspace) + spec_bytes(probe, tx, n_frames, n_fft));
    // spectral weights df w_j S(f_j)
    std::vector<float> h(p.J);
    const double T = probe->n_cycles / probe->f0;
    for (int j = 0; j < p.J; ++j) h[j] = (float)(df * (j == 0 ? 1.0 : 2.0) * pulse_spectrum(j * df, probe->f0, T));
    fq_status s = fqi::cuda_check(cudaMemcpyAsync(wS, h.data(), sizeof(float) * p.J, cudaMemcpyHostToDevice, st),
                                  "fq_simulate_rf_freq: weights");
    if (s) return s;
    const int threads = ((p.J + kBinsPerThread - 1) / kBinsPerThread + 31) / 32 * 32;
    FQ_REQUIRE(threads <= kChunk, FQ_ERR_SHAPE, "fq_simulate_rf_freq: too many bins");
    dim3 grid((unsigned)M, (unsigned)p.A, (unsigned)n_frames);
    spectrum_kernel<<<grid, threads, 0, st>>>(p, pos, amp, spec);
    int logN = 0;
    while ((1 << logN) < n_fft) ++logN;
    const size_t smem = sizeof(float2) * (size_t)n_fft;
    const unsigned lines = (unsigned)((int64_t)n_frames * p.A * M);
    if (out_dtype == FQ_F32) {
        s = fqi::cuda_check(cudaFuncSetAttribute(ifft_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem), "fq_simulate_rf_freq: smem");
        if (s) return s;
        ifft_kernel<float><<<lines, 512, smem, st>>>(spec, wS, p.J, n_fft, logN, probe->n_samples, (float *)rf);
    } else {
        s = fqi::cuda_check(cudaFuncSetAttribute(ifft_kernel<__nv_bfloat16>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                            "fq_simulate_rf_freq: smem");
        if (s) return s;
        ifft_kernel<__nv_bfloat16><<<lines, 512, smem, st>>>(spec, wS, p.J, n_fft, logN, probe->n_samples,
                                                             (__nv_bfloat16 *)rf);
    }
    return fqi::launch_check("fq_simulate_rf_freq");
}

// ---------------------------------------------------------------------------
// Eq. 1 with its transmit sum over elements and Eq. 2's sub-elements (App.
// D; Alg. 2 steps 2.2, 2.6): every element e transmits with weight W_e and
// the plane-wave steering delay dtau_{a,e} = (u_a . e - min u_a . e') / c;
// every element is v sub-elements along x; a sub-element q at distance d
// contributes g_q(f) = D_q(f) exp(-alpha f d) e^{-i 2 pi f d / c} / d, with
// the sub-element's directivity (half-width w_x / 2v in x, w_y / 2 in y).
//   T_{a,s}(f) = sum_e W_e e^{-i 2 pi f dtau_{a,e}} (1/v) sum_mu g_{e mu}(f)
//   P_{a,m}(f) = sum_s R_s T_{a,s}(f) (1/v) sum_mu g_{m mu}(f)
// Per (frame, transmit): tx_field_kernel writes T for every scatterer and
// frequency bin into the workspace (one CTA per 4 scatterers, one thread per
// 16 bins, the (element, sub-element) terms of a scatterer first evaluated
// into shared memory: float-float cycles per bin of c dtau + d, the
// attenuation exponent, weight / d and the directivity steps); then
// pfield_spectrum_kernel (one CTA per receive element) multiplies each
// scatterer's transmit field by its receive sub-element sum, with the same
// per-bin recurrences and float-pair accumulation as spectrum_kernel; the
// inverse transform is ifft_kernel.
// ---------------------------------------------------------------------------
namespace {

constexpr int kTxScat = 4;  // scatterers per CTA of tx_field_kernel

struct PfieldParams {
    FreqParams fp;
    int v;              // sub-elements per element
    float bkx_sub;      // b_sub k_1 per unit sin(theta): (width_x / 2v) 2 pi df / c
};

// The 16 bins j0 .. j0 + 15 of one term sum_t amp_t e^{-i 2 pi j cyc_t}
// exp(-atn_t j) sinc(j bx_t) [sinc(j by_t)] added to acc (binary32), with the
// anchors at j0 from accurate functions and recurrences over the bins.
__device__ __forceinline__ void bins_term(float ch, float cl, float atn, float rr, float bx, float by, bool matrix,
                                          int j0, float (&acc)[kBinsPerThread][2])
{
    const ff cyc = {ch, cl};
    float sn, cs, ws, wc;
    sincospif(-2.0f * fqi::ff_frac(fqi::ff_mul_f(cyc, (float)j0)), &sn, &cs);
    sincospif(-2.0f * fqi::ff_frac(cyc), &ws, &wc);
    float zr = cs, zi = sn;
    float att = expf(-atn * (float)j0);
    const float q = expf(-atn);
    float sbx, cbx, sx0, cx0;
    sincosf(bx, &sbx, &cbx);
    sincosf(bx * (float)j0, &sx0, &cx0);
    float sx_prev = fmaf(sx0, cbx, -cx0 * sbx), sx = sx0;
    const float tcx = 2.0f * cbx;
    float sy_prev = 0.0f, sy = 0.0f, tcy = 0.0f;
    if (matrix) {
        float sby, cby, sy0, cy0;
        sincosf(by, &sby, &cby);
        sincosf(by * (float)j0, &sy0, &cy0);
        sy_prev = fmaf(sy0, cby, -cy0 * sby);
        sy = sy0;
        tcy = 2.0f * cby;
    }
#pragma unroll
    for (int b = 0; b < kBinsPerThread; ++b) {
        const float jj = (float)(j0 + b);
        const float xb = jj * bx;
        float D = (xb == 0.0f) ? 1.0f : __fdividef(sx, xb);
        if (matrix) {
            const float yb = jj * by;
            D *= (yb == 0.0f) ? 1.0f : __fdividef(sy, yb);
            const float syn = fmaf(tcy, sy, -sy_prev);
            sy_prev = sy;
            sy = syn;
        }
        const float A = rr * att * D;
        acc[b][0] = fmaf(A, zr, acc[b][0]);
        acc[b][1] = fmaf(A, zi, acc[b][1]);
        const float nzr = fmaf(zr, wc, -zi * ws), nzi = fmaf(zr, ws, zi * wc);
        zr = nzr;
        zi = nzi;
        att *= q;
        const float sxn = fmaf(tcx, sx, -sx_prev);
        sx_prev = sx;
        sx = sxn;
    }
}

// sub-element q's term for a scatterer at (x, y, z): float-float distance
// d, then (cycles per bin of path + d, attenuation exponent per bin, weight
// / d, directivity steps)
__device__ __forceinline__ void sub_term(const PfieldParams &p, float x, float y, float z, float4 qpos, ff path0,
                                         float w, float *out6)
{
    const bool matrix = p.fp.pr.ny > 1;
    const ff dx = fqi::ff_add(ff{x, 0.0f}, ff{-qpos.x, -qpos.y});
    ff r2 = fqi::ff_add(fqi::ff_sqr(dx), fqi::ff_two_prod(z, z));
    ff dy = ff{0.0f, 0.0f};
    if (matrix || y != 0.0f) {
        dy = fqi::ff_add(ff{y, 0.0f}, ff{-qpos.z, -qpos.w});
        r2 = fqi::ff_add(r2, fqi::ff_sqr(dy));
    }
    const bool ok = r2.hi > 0.0f && w != 0.0f;
    const ff d = ok ? fqi::ff_sqrt(r2) : ff{1.0f, 0.0f};
    const ff cyc = fqi::ff_mul(fqi::ff_add(path0, d), fqi::ff_load(p.fp.dfc));
    const float rinv = 1.0f / d.hi;
    out6[0] = cyc.hi;
    out6[1] = cyc.lo;
    out6[2] = p.fp.atn_per_m * d.hi;
    out6[3] = ok ? w * rinv : 0.0f;
    out6[4] = p.bkx_sub * (dx.hi * rinv);
    out6[5] = matrix ? p.fp.bky * (dy.hi * rinv) : 0.0f;
}

__global__ void __launch_bounds__(kChunk) tx_field_kernel(const PfieldParams p, int f, int a,
                                                          const float *__restrict__ pos, const float4 *__restrict__ subpos,
                                                          const float2 *__restrict__ steer, const float *__restrict__ apod,
                                                          float2 *__restrict__ T)
{
    extern __shared__ float ent[];  // [n_ent][6]
    const int M = p.fp.pr.M, v = p.v, n_ent = M * v;
    const int64_t S = p.fp.S;
    const float *X = pos + (int64_t)f * 3 * S, *Y = X + S, *Z = Y + S;
    const bool matrix = p.fp.pr.ny > 1;
    const int j0 = threadIdx.x * kBinsPerThread;
    const bool live = j0 < p.fp.J;
    for (int si = 0; si < kTxScat; ++si) {
        const int64_t s = (int64_t)blockIdx.x * kTxScat + si;
        if (s >= S) break;
        const float x = X[s], y = Y[s], z = Z[s];
        __syncthreads();
        for (int t = threadIdx.x; t < n_ent; t += blockDim.x) {
            const int e = t / v;
            const float2 st = steer[(int64_t)a * M + e];
            sub_term(p, x, y, z, subpos[t], ff{st.x, st.y}, apod[e] / (float)v, ent + 6 * t);
        }
        __syncthreads();
        if (!live) continue;
        float acc[kBinsPerThread][2];
#pragma unroll
        for (int b = 0; b < kBinsPerThread; ++b) acc[b][0] = acc[b][1] = 0.0f;
        for (int t = 0; t < n_ent; ++t) {
            const float *q = ent + 6 * t;
            if (q[3] == 0.0f) continue;
            bins_term(q[0], q[1], q[2], q[3], q[4], q[5], matrix, j0, acc);
        }
        float2 *o = T + s * p.fp.J;
#pragma unroll
        for (int b = 0; b < kBinsPerThread; ++b)
            if (j0 + b < p.fp.J) o[j0 + b] = make_float2(acc[b][0], acc[b][1]);
    }
}

__global__ void __launch_bounds__(kChunk) pfield_spectrum_kernel(const PfieldParams p, int f, int a,
                                                                 const float *__restrict__ pos,
                                                                 const float *__restrict__ amp,
                                                                 const float4 *__restrict__ subpos,
                                                                 const float2 *__restrict__ T,
                                                                 float2 *__restrict__ spec)
{
    constexpr int kCh = 64;  // scatterers per chunk
    __shared__ float ent[kCh * 8 * 6];  // [scatterer][sub-element < 8][6]
    const int m = blockIdx.x;
    const int M = p.fp.pr.M, v = p.v;
    const int64_t S = p.fp.S;
    const float *X = pos + (int64_t)f * 3 * S, *Y = X + S, *Z = Y + S;
    const bool matrix = p.fp.pr.ny > 1;
    const int j0 = threadIdx.x * kBinsPerThread;
    const bool live = j0 < p.fp.J;
    float accH[kBinsPerThread][2], accL[kBinsPerThread][2];
#pragma unroll
    for (int b = 0; b < kBinsPerThread; ++b) accH[b][0] = accH[b][1] = accL[b][0] = accL[b][1] = 0.0f;
    for (int64_t c0 = 0; c0 < S; c0 += kCh) {
        const int n = (int)min((int64_t)kCh, S - c0);
        __syncthreads();
        for (int t = threadIdx.x; t < n * v; t += blockDim.x) {
            const int64_t s = c0 + t / v;
            const int mu = t % v;
            sub_term(p, X[s], Y[s], Z[s], subpos[(int64_t)m * v + mu], ff{0.0f, 0.0f}, amp[s] / (float)v,
                     ent + 6 * ((t / v) * 8 + mu));
        }
        __syncthreads();
        if (!live) continue;
        float fa[kBinsPerThread][2];
#pragma unroll
        for (int b = 0; b < kBinsPerThread; ++b) fa[b][0] = fa[b][1] = 0.0f;
        for (int t = 0; t < n; ++t) {
            float g[kBinsPerThread][2];
#pragma unroll
            for (int b = 0; b < kBinsPerThread; ++b) g[b][0] = g[b][1] = 0.0f;
            bool any = false;
            for (int mu = 0; mu < v; ++mu) {
                const float *q = ent + 6 * (t * 8 + mu);
                if (q[3] == 0.0f) continue;
                any = true;
                bins_term(q[0], q[1], q[2], q[3], q[4], q[5], matrix, j0, g);
            }
            if (!any) continue;
            const float2 *Ts = T + (c0 + t) * p.fp.J + j0;
#pragma unroll
            for (int b = 0; b < kBinsPerThread; ++b) {
                const float2 tv = j0 + b < p.fp.J ? Ts[b] : make_float2(0.0f, 0.0f);
                fa[b][0] = fmaf(tv.x, g[b][0], fmaf(-tv.y, g[b][1], fa[b][0]));
                fa[b][1] = fmaf(tv.x, g[b][1], fmaf(tv.y, g[b][0], fa[b][1]));
            }
        }
#pragma unroll
        for (int b = 0; b < kBinsPerThread; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float h = accH[b][c], d = fa[b][c];
                const float s = h + d, bb = s - h;
                const float e = (h - (s - bb)) + (d - bb);
                const float l = accL[b][c] + e;
                accH[b][c] = s + l;
                accL[b][c] = l - (accH[b][c] - s);
            }
    }
    if (!live) return;
    float2 *out = spec + (((int64_t)f * p.fp.A + a) * M + m) * p.fp.J;
#pragma unroll
    for (int b = 0; b < kBinsPerThread; ++b)
        if (j0 + b < p.fp.J) out[j0 + b] = make_float2(accH[b][0] + accL[b][0], accH[b][1] + accL[b][1]);
}

constexpr int kMaxSub = 8;

struct PfieldLayout {
    size_t spec, wS, T, subpos, steer, apod, total;
};

PfieldLayout pfield_layout(const fq_probe *probe, const fq_tx *tx, int64_t S, int F, int N, int v)
{
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t M = (size_t)probe->nx * probe->ny, J = N / 2;
    PfieldLayout L;
    size_t o = 0;
    L.spec = o; o += al((size_t)F * tx->n_angles * M * J * sizeof(float2));
    L.wS = o; o += al(J * sizeof(float));
    L.T = o; o += al((size_t)(S > 0 ? S : 1) * J * sizeof(float2));
    L.subpos = o; o += al(M * v * sizeof(float4));
    L.steer = o; o += al((size_t)tx->n_angles * M * sizeof(float2));
    L.apod = o; o += al(M * sizeof(float));
    L.total = o;
    return L;
}

}  // namespace

extern "C" fq_status fq_simulate_rf_pfield_workspace_size(const fq_probe *probe, const fq_tx *tx, int64_t S,
                                                          int32_t n_frames, int32_t n_fft, int32_t n_sub,
                                                          size_t *bytes)
{
    FQ_REQUIRE(probe && tx && bytes && S >= 0 && n_frames >= 1 && pow2(n_fft) && n_sub >= 1 && n_sub <= kMaxSub,
               FQ_ERR_INVALID_ARG, "fq_simulate_rf_pfield_workspace_size: bad arguments");
    *bytes = pfield_layout(probe, tx, S, n_frames, n_fft, n_sub).total;
    return FQ_OK;
}

extern "C" fq_status fq_simulate_rf_pfield(const fq_probe *probe, const fq_tx *tx, const double *apod, int32_t n_sub,
                                           const float *pos, const float *amp, int64_t S, int32_t n_frames,
                                           int32_t n_fft, int32_t out_dtype, void *rf, void *workspace,
                                           size_t workspace_bytes, void *stream)
{
    FQ_REQUIRE(probe && tx && rf && workspace, FQ_ERR_INVALID_ARG, "fq_simulate_rf_pfield: null argument");
    FQ_REQUIRE(S >= 0 && n_frames >= 1 && (S == 0 || (pos && amp)), FQ_ERR_INVALID_ARG,
               "fq_simulate_rf_pfield: bad scatterer arguments");
    FQ_REQUIRE(n_sub >= 1 && n_sub <= kMaxSub, FQ_ERR_INVALID_ARG, "fq_simulate_rf_pfield: n_sub must be in [1, %d]",
               kMaxSub);
    FQ_REQUIRE(tx->n_angles >= 1 && tx->n_angles <= FQ_MAX_ANGLES && tx->tilt_x && tx->tilt_y, FQ_ERR_SHAPE,
               "fq_simulate_rf_pfield: n_angles must be in [1, %d]", FQ_MAX_ANGLES);
    const int M = probe->nx * probe->ny;
    FQ_REQUIRE(probe->nx >= 1 && probe->ny >= 1 && M * n_sub <= 4096 && probe->n_samples >= 2, FQ_ERR_SHAPE,
               "fq_simulate_rf_pfield: elements x sub-elements must be at most 4096");
    FQ_REQUIRE(pow2(n_fft) && n_fft >= probe->n_samples && n_fft <= kMaxFft, FQ_ERR_SHAPE,
               "fq_simulate_rf_pfield: n_fft must be a power of two in [n_samples, %d]", kMaxFft);
    FQ_REQUIRE(out_dtype == FQ_F32 || out_dtype == FQ_BF16, FQ_ERR_UNSUPPORTED,
               "fq_simulate_rf_pfield: out_dtype must be FQ_F32 or FQ_BF16");
    const PfieldLayout L = pfield_layout(probe, tx, S, n_frames, n_fft, n_sub);
    FQ_REQUIRE(workspace_bytes >= L.total, FQ_ERR_WORKSPACE, "fq_simulate_rf_pfield: workspace needs %zu bytes",
               L.total);
    FQ_REQUIRE(fqi::aligned(workspace, 256), FQ_ERR_ALIGN, "fq_simulate_rf_pfield: workspace not 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = static_cast<char *>(workspace);
    PfieldParams p;
    std::memset(&p, 0, sizeof p);
    fqi::make_probe_ff(probe, p.fp.pr);
    p.fp.A = tx->n_angles;
    p.fp.N = n_fft;
    p.fp.J = n_fft / 2;
    p.fp.S = S;
    const double df = probe->fs / n_fft;
    p.fp.dfc = fqi::split_double(df / probe->c);
    p.fp.atn_per_m = (float)(probe->alpha_db_cm_mhz * 100.0 / (20.0 / std::log(10.0)) * 1e-6 * df);
    p.fp.bky = (float)(0.5 * probe->width_y * 2.0 * M_PI * df / probe->c);
    p.bkx_sub = (float)(0.5 * probe->width_x / n_sub * 2.0 * M_PI * df / probe->c);
    p.v = n_sub;
    // host tables: spectral weights, sub-element centres, steering paths c dtau, weights
    std::vector<float> h(p.fp.J);
    const double T = probe->n_cycles / probe->f0;
    for (int j = 0; j < p.fp.J; ++j) h[j] = (float)(df * (j == 0 ? 1.0 : 2.0) * pulse_spectrum(j * df, probe->f0, T));
    std::vector<float4> sub((size_t)M * n_sub);
    std::vector<float2> steer((size_t)tx->n_angles * M);
    std::vector<float> w(M);
    for (int e = 0; e < M; ++e) {
        const int ix = e % probe->nx, iy = e / probe->nx;
        const double ex = ((double)ix - 0.5 * (probe->nx - 1)) * probe->pitch_x;
        const double ey = ((double)iy - 0.5 * (probe->ny - 1)) * probe->pitch_y;
        for (int mu = 0; mu < n_sub; ++mu) {
            const double qx = ex + ((double)mu - 0.5 * (n_sub - 1)) * probe->width_x / n_sub;
            const fqi::df2 a = fqi::split_double(qx), b = fqi::split_double(ey);
            sub[(size_t)e * n_sub + mu] = make_float4(a.hi, a.lo, b.hi, b.lo);
        }
        w[e] = apod ? (float)apod[e] : 1.0f;
    }
    for (int a = 0; a < tx->n_angles; ++a) {
        const double ux = std::sin(tx->tilt_x[a]), uy = std::sin(tx->tilt_y[a]);
        double best = 1e300;
        for (int e = 0; e < M; ++e) {
            const double ex = ((double)(e % probe->nx) - 0.5 * (probe->nx - 1)) * probe->pitch_x;
            const double ey = ((double)(e / probe->nx) - 0.5 * (probe->ny - 1)) * probe->pitch_y;
            best = std::min(best, ux * ex + uy * ey);
        }
        for (int e = 0; e < M; ++e) {
            const double ex = ((double)(e % probe->nx) - 0.5 * (probe->nx - 1)) * probe->pitch_x;
            const double ey = ((double)(e / probe->nx) - 0.5 * (probe->ny - 1)) * probe->pitch_y;
            const fqi::df2 d = fqi::split_double(ux * ex + uy * ey - best);
            steer[(size_t)a * M + e] = make_float2(d.hi, d.lo);
        }
    }
    float2 *spec = reinterpret_cast<float2 *>(ws + L.spec);
    float *wS = reinterpret_cast<float *>(ws + L.wS);
    float2 *Tf = reinterpret_cast<float2 *>(ws + L.T);
    float4 *dsub = reinterpret_cast<float4 *>(ws + L.subpos);
    float2 *dsteer = reinterpret_cast<float2 *>(ws + L.steer);
    float *dapod = reinterpret_cast<float *>(ws + L.apod);
    fq_status s = fqi::cuda_check(cudaMemcpyAsync(wS, h.data(), sizeof(float) * p.fp.J, cudaMemcpyHostToDevice, st),
                                  "fq_simulate_rf_pfield: weights");
    if (!s) s = fqi::cuda_check(cudaMemcpyAsync(dsub, sub.data(), sizeof(float4) * sub.size(), cudaMemcpyHostToDevice, st),
                                "fq_simulate_rf_pfield: sub-elements");
    if (!s) s = fqi::cuda_check(cudaMemcpyAsync(dsteer, steer.data(), sizeof(float2) * steer.size(),
                                                cudaMemcpyHostToDevice, st), "fq_simulate_rf_pfield: steering");
    if (!s) s = fqi::cuda_check(cudaMemcpyAsync(dapod, w.data(), sizeof(float) * M, cudaMemcpyHostToDevice, st),
                                "fq_simulate_rf_pfield: weights");
    if (!s) s = fqi::cuda_check(cudaStreamSynchronize(st), "fq_simulate_rf_pfield: tables");  // host vectors end here
    if (s) return s;
    const int threads = ((p.fp.J + kBinsPerThread - 1) / kBinsPerThread + 31) / 32 * 32;
    FQ_REQUIRE(threads <= kChunk, FQ_ERR_SHAPE, "fq_simulate_rf_pfield: too many bins");
    const size_t tx_smem = sizeof(float) * 6 * (size_t)M * n_sub;
    s = fqi::cuda_check(cudaFuncSetAttribute(tx_field_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tx_smem),
                        "fq_simulate_rf_pfield: smem");
    if (s) return s;
    for (int f = 0; f < n_frames; ++f)
        for (int a = 0; a < tx->n_angles; ++a) {
            if (S > 0) {
                tx_field_kernel<<<(unsigned)((S + kTxScat - 1) / kTxScat), threads, tx_smem, st>>>(p, f, a, pos, dsub,
                                                                                                     dsteer, dapod, Tf);
                s = fqi::launch_check("fq_simulate_rf_pfield: transmit field");
                if (s) return s;
            }
            pfield_spectrum_kernel<<<(unsigned)M, threads, 0, st>>>(p, f, a, pos, amp, dsub, Tf, spec);
            s = fqi::launch_check("fq_simulate_rf_pfield: spectrum");
            if (s) return s;
        }
    int logN = 0;
    while ((1 << logN) < n_fft) ++logN;
    const size_t smem = sizeof(float2) * (size_t)n_fft;
    const unsigned lines = (unsigned)((int64_t)n_frames * p.fp.A * M);
    if (out_dtype == FQ_F32) {
        s = fqi::cuda_check(cudaFuncSetAttribute(ifft_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem), "fq_simulate_rf_pfield: smem");
        if (s) return s;
        ifft_kernel<float><<<lines, 512, smem, st>>>(spec, wS, p.fp.J, n_fft, logN, probe->n_samples, (float *)rf);
    } else {
        s = fqi::cuda_check(cudaFuncSetAttribute(ifft_kernel<__nv_bfloat16>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                            "fq_simulate_rf_pfield: smem");
        if (s) return s;
        ifft_kernel<__nv_bfloat16><<<lines, 512, smem, st>>>(spec, wS, p.fp.J, n_fft, logN, probe->n_samples,
                                                             (__nv_bfloat16 *)rf);
    }
    return fqi::launch_check("fq_simulate_rf_pfield");
}
