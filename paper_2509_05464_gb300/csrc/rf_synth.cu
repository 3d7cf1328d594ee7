// rf_synth.cu -- a3 pulse-echo RF synthesis (Eq. 1 restated as a
// narrowband time-domain sum; App. D; Sec. 2.3).
//
// Design (GB300): one CTA owns the complete RF record of E consecutive
// receive elements for one (frame, transmit) pair and keeps it in shared
// memory (E x Ns FP32).  Its threads stream every scatterer of the frame
// once (coalesced structure-of-arrays loads, each thread one scatterer), and
// for each of the E elements evaluate the delay, amplitude and the few
// pulse taps that land in the record, accumulating them into the shared
// record with shared-memory atomics.  Nothing is atomically added in global
// memory: the record is written out once, coalesced, after the last
// scatterer.  The per-scatterer transmit path and its loads are shared by
// the E elements.
//
// Precision: the delay u = tau fs (hundreds to thousands of samples) must
// be known to ~1e-6 sample for the carrier phase, so the geometry
// (distance, transmit path, u) runs in float-float; the pulse itself is
// evaluated at the small offset j - frac(u), where binary32 suffices.  The
// pulse taps come from two complex rotors (carrier and Hann window) advanced
// by a fixed angle per sample.
#include <cmath>
#include <cstring>

#include "fq_internal.cuh"

namespace {

using fqi::ff;

struct RfParams {
    fqi::ProbeFF pr;
    int A;
    int64_t S;
    float kbx, kby;     // k0 * width / 2
    float att;          // attenuation per metre of two-way path (Np / m)
    float half_w;       // pulse half-support in samples: n_cycles fs / (2 f0)
    float w_c, w_h;     // carrier / Hann phase per sample (rad)
    float cwc, swc, cwh, swh;  // rotor steps
    int ntap;           // taps that can overlap the support
    fqi::AngleFF ang[FQ_MAX_ANGLES];
};

__device__ __forceinline__ float sinc_f(float u)
{
    return fabsf(u) < 1e-4f ? 1.0f - u * u * (1.0f / 6.0f) : sinf(u) / u;
}

template <int E, int NT, typename OutT>
__global__ void __launch_bounds__(NT) rf_synth_kernel(const RfParams p, const float *__restrict__ pos,
                                                      const float *__restrict__ amp,
                                                      const float *__restrict__ rf_base,
                                                      OutT *__restrict__ rf)
{
    extern __shared__ float tile[];  // [E][Ns]
    __shared__ float ex_hi[E], ex_lo[E], ey_hi[E], ey_lo[E];
    const int ns = p.pr.ns;
    const int M = p.pr.M;
    const int m0 = blockIdx.x * E;
    const int a = blockIdx.y;
    const int f = blockIdx.z;
    const int ne = min(E, M - m0);

    if (threadIdx.x < E) {
        int m = min(m0 + (int)threadIdx.x, M - 1);
        ff ex = fqi::elem_coord(m % p.pr.nx, p.pr.nx, p.pr.pitch_x);
        ff ey = fqi::elem_coord(m / p.pr.nx, p.pr.ny, p.pr.pitch_y);
        ex_hi[threadIdx.x] = ex.hi;
        ex_lo[threadIdx.x] = ex.lo;
        ey_hi[threadIdx.x] = ey.hi;
        ey_lo[threadIdx.x] = ey.lo;
    }
    for (int i = threadIdx.x; i < E * ns; i += NT) {
        int e = i / ns, k = i - e * ns;
        float v = 0.0f;
        if (rf_base && e < ne) v = rf_base[((int64_t)a * M + m0 + e) * ns + k];
        tile[i] = v;
    }
    __syncthreads();

    const fqi::AngleFF an = p.ang[a];
    const ff ux = fqi::ff_load(an.ux), uy = fqi::ff_load(an.uy), uz = fqi::ff_load(an.uz);
    const ff org = fqi::ff_load(an.origin);
    const ff fs_c = fqi::ff_load(p.pr.fs_over_c);
    const bool matrix = p.pr.ny > 1;
    const int64_t S = p.S;
    const float *X = pos + (int64_t)f * 3 * S;
    const float *Y = X + S;
    const float *Z = Y + S;

    for (int64_t s = threadIdx.x; s < S; s += NT) {
        const float R = amp[s];
        if (R == 0.0f) continue;
        const float x = X[s], y = Y[s], z = Z[s];
        // transmit path u . r - min u . e (float-float)
        ff ptx = fqi::ff_add(fqi::ff_mul_f(ux, x), fqi::ff_mul_f(uy, y));
        ptx = fqi::ff_add(ptx, fqi::ff_mul_f(uz, z));
        ptx = fqi::ff_add(ptx, fqi::ff_neg(org));
        const ff zz = fqi::ff_two_prod(z, z);
#pragma unroll 1
        for (int e = 0; e < ne; ++e) {
            ff dx = fqi::ff_add_f(ff{-ex_hi[e], -ex_lo[e]}, x);
            ff r2 = fqi::ff_add(fqi::ff_sqr(dx), zz);
            ff dy = {0.0f, 0.0f};
            if (matrix || y != 0.0f) {  // 2D workloads keep every scatterer at y = 0
                dy = fqi::ff_add_f(ff{-ey_hi[e], -ey_lo[e]}, y);
                r2 = fqi::ff_add(r2, fqi::ff_sqr(dy));
            }
            if (r2.hi <= 0.0f) continue;
            const ff r = fqi::ff_sqrt(r2);
            const ff path = fqi::ff_add(ptx, r);
            const ff u = fqi::ff_mul(path, fs_c);
            int k0;
            float frac;
            fqi::ff_floor_frac(u, k0, frac);
            const float inv_r = 1.0f / r.hi;
            float D = sinc_f(p.kbx * dx.hi * inv_r);
            if (matrix) D *= sinc_f(p.kby * dy.hi * inv_r);
            const float Aa = R * D * __expf(-p.att * path.hi) * inv_r;
            const int jlo = (int)ceilf(frac - p.half_w);
            const float t0 = (float)jlo - frac;
            float sc, cc, sh, ch;
            sincosf(p.w_c * t0, &sc, &cc);
            sincosf(p.w_h * t0, &sh, &ch);
            float *line = tile + e * ns;
            int k = k0 + jlo;
#pragma unroll 4
            for (int j = 0; j < p.ntap; ++j, ++k) {
                const float t = t0 + (float)j;
                if (fabsf(t) < p.half_w && k >= 0 && k < ns)
                    atomicAdd(line + k, Aa * (0.5f + 0.5f * ch) * cc);
                float nc = cc * p.cwc - sc * p.swc;
                sc = sc * p.cwc + cc * p.swc;
                cc = nc;
                float nh = ch * p.cwh - sh * p.swh;
                sh = sh * p.cwh + ch * p.swh;
                ch = nh;
            }
        }
    }
    __syncthreads();
    OutT *out = rf + (((int64_t)f * p.A + a) * M + m0) * ns;
    for (int i = threadIdx.x; i < ne * ns; i += NT) fqi::store_f(out, i, tile[i]);
}

template <int E, typename OutT>
fq_status launch_rf(const RfParams &p, int F, const float *pos, const float *amp, const float *base,
                    OutT *rf, cudaStream_t st)
{
    constexpr int NT = 256;
    size_t smem = sizeof(float) * (size_t)E * p.pr.ns;
    auto kern = rf_synth_kernel<E, NT, OutT>;
    fq_status s = fqi::cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                  "fq_simulate_rf: smem attribute");
    if (s) return s;
    dim3 grid((p.pr.M + E - 1) / E, p.A, F);
    kern<<<grid, NT, smem, st>>>(p, pos, amp, base, rf);
    return fqi::launch_check("fq_simulate_rf");
}

template <typename OutT>
fq_status dispatch_rf(const RfParams &p, int F, const float *pos, const float *amp, const float *base,
                      OutT *rf, cudaStream_t st)
{
    const size_t line = sizeof(float) * (size_t)p.pr.ns;
    const size_t budget = 200 * 1024;
    if (8 * line <= budget) return launch_rf<8>(p, F, pos, amp, base, rf, st);
    if (4 * line <= budget) return launch_rf<4>(p, F, pos, amp, base, rf, st);
    return launch_rf<2>(p, F, pos, amp, base, rf, st);
}

}  // namespace

extern "C" fq_status fq_simulate_rf(const fq_probe *probe, const fq_tx *tx, const float *pos,
                                    const float *amp, int64_t S, int32_t n_frames, const float *rf_base,
                                    int32_t out_dtype, void *rf, void *stream)
{
    FQ_REQUIRE(probe && tx && rf, FQ_ERR_INVALID_ARG, "fq_simulate_rf: null argument");
    FQ_REQUIRE(S >= 0 && n_frames >= 1, FQ_ERR_INVALID_ARG, "fq_simulate_rf: S=%lld n_frames=%d",
               (long long)S, n_frames);
    FQ_REQUIRE(S == 0 || (pos && amp), FQ_ERR_INVALID_ARG, "fq_simulate_rf: null pos/amp");
    FQ_REQUIRE(tx->n_angles >= 1 && tx->n_angles <= FQ_MAX_ANGLES && tx->tilt_x && tx->tilt_y, FQ_ERR_SHAPE,
               "fq_simulate_rf: n_angles must be in [1, %d]", FQ_MAX_ANGLES);
    FQ_REQUIRE(probe->nx >= 1 && probe->ny >= 1 && (int64_t)probe->nx * probe->ny <= 65536, FQ_ERR_SHAPE,
               "fq_simulate_rf: bad element count");
    FQ_REQUIRE(probe->n_samples >= 1 && probe->n_samples <= 8192, FQ_ERR_SHAPE,
               "fq_simulate_rf: n_samples must be in [1, 8192]");
    FQ_REQUIRE(probe->f0 > 0 && probe->fs > 0 && probe->c > 0 && probe->n_cycles >= 1, FQ_ERR_INVALID_ARG,
               "fq_simulate_rf: f0, fs, c, n_cycles must be positive");
    FQ_REQUIRE(out_dtype == FQ_F32 || out_dtype == FQ_BF16, FQ_ERR_UNSUPPORTED,
               "fq_simulate_rf: out_dtype must be FQ_F32 or FQ_BF16");
    FQ_REQUIRE(fqi::aligned(rf, 4), FQ_ERR_ALIGN, "fq_simulate_rf: rf must be 4-byte aligned");

    RfParams p;
    std::memset(&p, 0, sizeof p);
    fqi::make_probe_ff(probe, p.pr);
    p.A = tx->n_angles;
    p.S = S;
    const double k0 = 2.0 * M_PI * probe->f0 / probe->c;
    p.kbx = (float)(k0 * 0.5 * probe->width_x);
    p.kby = (float)(k0 * 0.5 * probe->width_y);
    p.att = (float)(probe->alpha_db_cm_mhz * 100.0 / (20.0 / std::log(10.0)) * probe->f0 * 1e-6);
    const double hw = probe->n_cycles * probe->fs / (2.0 * probe->f0);
    p.half_w = (float)hw;
    p.ntap = (int)std::floor(2.0 * hw) + 1;
    const double wc = 2.0 * M_PI * probe->f0 / probe->fs;
    const double wh = wc / probe->n_cycles;
    p.w_c = (float)wc;
    p.w_h = (float)wh;
    p.cwc = (float)std::cos(wc);
    p.swc = (float)std::sin(wc);
    p.cwh = (float)std::cos(wh);
    p.swh = (float)std::sin(wh);
    fqi::make_angles_ff(probe, tx, p.ang);
    cudaStream_t st = (cudaStream_t)stream;
    if (out_dtype == FQ_F32) return dispatch_rf(p, n_frames, pos, amp, rf_base, (float *)rf, st);
    return dispatch_rf(p, n_frames, pos, amp, rf_base, (__nv_bfloat16 *)rf, st);
}
