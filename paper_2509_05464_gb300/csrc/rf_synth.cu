// rf_synth.cu -- a3 pulse-echo RF synthesis (Eq. 1 restated as a
// narrowband time-domain sum; App. D; Sec. 2.3).
//
// Design (GB300): one CTA owns the complete RF records of E consecutive
// receive elements for one frame (and one transmit, or a group of transmits
// in the 4-element kernel) and keeps them in shared memory.  Its threads
// stream every scatterer of the frame (coalesced structure-of-arrays loads,
// one scatterer per thread), and for each element evaluate the delay,
// amplitude and the pulse taps that land in the record.  Taps are
// accumulated in fixed point with native shared-memory int32 atomics: on this
// GPU shared-memory FP32 atomic adds run as compare-and-swap loops and
// sustain ~3.7x fewer adds per second than int32 ones.  The 4-element kernel
// adds one int32 per tap with a per-record quantum that provably keeps the
// record in range (see rf_quad_tile); the 2-element and general kernels add
// a hi/lo pair (see add_fixed).  Nothing is atomically added in global
// memory: the records are converted back and written out once, coalesced,
// after the last scatterer.  Integer sums make the RF bit-reproducible.
//
// Precision: the delay u = tau fs (hundreds to thousands of samples) must
// be known to ~1e-6 sample for the carrier phase, so the geometry
// (distance, transmit path, u) runs in float-float; the pulse itself is
// evaluated at the small offset j - frac(u), where binary32 suffices: the
// taps' Hann-phase cosines follow the Chebyshev recurrence
// C_{j+1} = 2 cos(w) C_j - C_{j-1} from the first tap, and for the
// two-cycle pulse the carrier is cos(2 theta) = 2 C^2 - 1 of the Hann phase.
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "batch.cuh"
#include "fq_internal.cuh"
#include "rf_poly.cuh"

namespace {

using fqi::ff;

constexpr int kMaxTaps = 64;  // pulse taps per (scatterer, element) pair the kernel supports
// quad kernel: shared-memory records per CTA (angles x 4 elements x Ns int32)
// up to kQuadSmemMax (below QuadShared): the more angles a CTA holds, the
// more of the receive geometry, the scatterer loads and the bound pass it
// shares (2D compounded workload: 5 angles per CTA 6% faster than 3; 3D
// workload: all 9 angles, 216 KB of records at 1536 samples, 1686 ms against
// 1821 ms for groups of 5 and 4).  The CTAs that fit per SM by shared memory
// split 32 resident warps (64 registers per thread): on the 2D workload 32
// warps ran 9.4% faster than 16 (128 registers), 24 warps 7.8%.
inline int quad_ctas_per_sm(size_t smem) { return smem <= 52 * 1024 ? 4 : (smem <= 110 * 1024 ? 2 : 1); }

struct RfParams {
    fqi::ProbeFF pr;
    int A;
    int64_t S;
    float kbx, kby;     // k0 * width / 2
    float att;          // attenuation per metre of two-way path (Np / m)
    float half_w;       // pulse half-support in samples: n_cycles fs / (2 f0)
    float w_h;          // Hann phase per sample (rad): 2 pi f0 / (n_cycles fs)
    float w_c;          // carrier phase per sample (rad): 2 pi f0 / fs
    float two_cos_h, two_cos_c;  // Chebyshev recurrence factors 2 cos(w)
    float cos_h, sin_h, cos_c, sin_c;
    int jmin;           // smallest first-tap offset ceil(frac - half_w) over frac in [0, 1)
    int ntap_max;       // floor(2 half_w) + 1
    float tab_h[2][2];  // (cos, sin)(w_h * j) for j = jmin, jmin + 1
    float tab_c[2][2];  // (cos, sin)(w_c * j) for j = jmin, jmin + 1
    int two_cycle;      // n_cycles == 2: carrier = 2 C^2 - 1 of the Hann phase
    // first-tap thresholds on frac for the fast kernels: jlo = jmin + (frac > theta),
    // floor(frac + half_w) = floor(half_w) + (frac >= theta2)
    float theta, theta2, jmin_f;
    float att_l2;       // -att log2(e): exp(-att path) = 2^(att_l2 path)
    // quad kernel: transmit angles per CTA (ag), angle groups (n_ag), the
    // half-width of the tap-bound window (ceil(half_w) + 1 samples) and the
    // factor by which an echo's taps may exceed |amp| |D| / r (attenuation
    // gain before t = 0, binary32 rounding)
    int ag, n_ag, win;
    // quad kernel: scatterer groups, each accumulated into the records with
    // its own quantum and added to the FP32 output in turn (1 for 16-bit
    // outputs, whose storage rounding is far coarser than the records')
    int n_sg;
    float bound_margin;
    float dbx_far;      // the directivity bound at its largest argument, k0 width_x / 2
    float dc_corr;      // quad kernel, FP32 outputs: added to tap 4 of every echo, times its amplitude
    fqi::AngleFF ang[FQ_MAX_ANGLES];
};

constexpr float kPi = 3.14159265358979f;

// sin(u) / u for |u| < 2 pi: one conditional turn brings the argument into
// [-pi, pi] where the hardware sine is accurate to ~4e-7 absolute.
__device__ __forceinline__ float sinc_f(float u)
{
    const float v = fmaf(-2.0f * kPi, rintf(u * (0.5f / kPi)), u);  // u less whole turns, in [-pi, pi]
    const float small = fmaf(-u * u, 1.0f / 6.0f, 1.0f);
    const float big = __fdividef(__sinf(v), u);
    return fabsf(u) < 1e-3f ? small : big;
}

// Fitted polynomials (rf_poly.cuh, written by rf_poly_fit.py; Chebyshev
// interpolants rounded to binary32).  The hardware sin/cos approximations
// carry an absolute error near 4e-7 that does not average out over
// fractional delays, and delay-and-sum adds such a bias coherently over the
// elements: with them the compounded image error was 3.7x the RF error.

// (sin x, cos x) for |x| <= 0.8 (binary32 evaluation error below 6e-8)
__device__ __forceinline__ void sincos_poly(float x, float &s, float &c)
{
    using namespace fqpoly;
    const float t = x * x;
    float ps = fmaf(kSinPoly3, t, kSinPoly2);
    ps = fmaf(ps, t, kSinPoly1);
    ps = fmaf(ps, t, kSinPoly0);
    s = x * ps;
    float pc = fmaf(kCosPoly4, t, kCosPoly3);
    pc = fmaf(pc, t, kCosPoly2);
    pc = fmaf(pc, t, kCosPoly1);
    c = fmaf(pc, t, kCosPoly0);
}

// the same for two arguments in packed f32x2 (the same operations per lane)
__device__ __forceinline__ void sincos_poly2(fqi::f2 x, fqi::f2 &s, fqi::f2 &c)
{
    using namespace fqpoly;
    using fqi::f2_dup;
    using fqi::f2_fma;
    const fqi::f2 t = fqi::f2_mul(x, x);
    fqi::f2 ps = f2_fma(f2_dup(kSinPoly3), t, f2_dup(kSinPoly2));
    ps = f2_fma(ps, t, f2_dup(kSinPoly1));
    ps = f2_fma(ps, t, f2_dup(kSinPoly0));
    s = fqi::f2_mul(x, ps);
    fqi::f2 pc = f2_fma(f2_dup(kCosPoly4), t, f2_dup(kCosPoly3));
    pc = f2_fma(pc, t, f2_dup(kCosPoly2));
    pc = f2_fma(pc, t, f2_dup(kCosPoly1));
    c = f2_fma(pc, t, f2_dup(kCosPoly0));
}

// sin(u) / u for two arguments in packed f32x2 (the same operations per lane)
__device__ __forceinline__ fqi::f2 sinc_poly2(fqi::f2 u)
{
    using namespace fqpoly;
    using fqi::f2_dup;
    using fqi::f2_fma;
    const fqi::f2 v = f2_fma(u, u, f2_dup(-kSincCentre));
    fqi::f2 r = f2_fma(f2_dup(kSincPoly7), v, f2_dup(kSincPoly6));
    r = f2_fma(r, v, f2_dup(kSincPoly5));
    r = f2_fma(r, v, f2_dup(kSincPoly4));
    r = f2_fma(r, v, f2_dup(kSincPoly3));
    r = f2_fma(r, v, f2_dup(kSincPoly2));
    r = f2_fma(r, v, f2_dup(kSincPoly1));
    return f2_fma(r, v, f2_dup(kSincPoly0));
}

// sin(u) / u for |u| <= 5 (binary32 evaluation error below 2e-7)
__device__ __forceinline__ float sinc_poly(float u)
{
    using namespace fqpoly;
    const float v = fmaf(u, u, -kSincCentre);
    float r = fmaf(kSincPoly7, v, kSincPoly6);
    r = fmaf(r, v, kSincPoly5);
    r = fmaf(r, v, kSincPoly4);
    r = fmaf(r, v, kSincPoly3);
    r = fmaf(r, v, kSincPoly2);
    r = fmaf(r, v, kSincPoly1);
    return fmaf(r, v, kSincPoly0);
}

// 2^x (ex2.approx: relative error near 2^-22)
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// (cos, sin) of w * (jlo - frac) as exp(i w jlo) exp(-i w frac), with
// |w frac| < w: the series for w <= 0.8, the accurate library sincos
// otherwise.  SMALL: the caller guarantees w <= 0.8 (the paired and quad
// kernels serve pulses of 8 to 9 samples per Hann period, w < pi / 4).
template <bool SMALL = false>
__device__ __forceinline__ void first_tap(float w, float frac, float tc0, float ts0, float tc1, float ts1, bool sel1,
                                          float &c, float &s)
{
    float sf, cf;
    if (SMALL || w <= fqpoly::kTapXMax)
        sincos_poly(w * frac, sf, cf);
    else
        sincosf(w * frac, &sf, &cf);
    const float tc = sel1 ? tc1 : tc0, ts = sel1 ? ts1 : ts0;
    c = fmaf(cf, tc, sf * ts);
    s = fmaf(ts, cf, -tc * sf);
}

// one pulse tap of the two-cycle pulse from the Hann-phase cosine C:
// A (1 + C)/2 (2 C^2 - 1) = ((A C + A) C - A/2) C - A/2
__device__ __forceinline__ float tap2(float A, float hA, float C)
{
    return fmaf(fmaf(fmaf(A, C, A), C, -hA), C, -hA);
}

// Fixed-point accumulation.  A tap value v (in units of the largest
// |amplitude|, i.e. scaled by g = 2^-ceil(log2 max|amp|)) is held as
// V = v g 2^20 split into hi = rint(V / 2^16) and lo = V - 2^16 hi
// (|lo| <= 2^15), each added with a native shared-memory int32 atomic.  The
// sums are exact integers (order-independent, so the RF is bit-reproducible)
// and the split keeps 47 bits of range: |sum| < 2^27 in scaled units,
// resolution 2^-20.  Rounding to integers uses the 1.5 * 2^23 magic-number
// trick (exact for |x| < 2^22).
constexpr float kFixScale = 1048576.0f;          // 2^20
constexpr float kMagic = 12582912.0f;            // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;
constexpr float kTapClamp = 137438953472.0f;     // 2^37: |v g| <= 2^17 per tap

__device__ __forceinline__ void add_fixed(int *hi, int *lo, int k, float V)
{
    V = fminf(fmaxf(V, -kTapClamp), kTapClamp);
    const float ht = fmaf(V, 1.0f / 65536.0f, kMagic);
    const float hb = ht - kMagic;                 // rint(V / 2^16) as a float
    const float lf = fmaf(-hb, 65536.0f, V);      // exact remainder, |lf| <= 2^15
    const float lt = lf + kMagic;
    atomicAdd(hi + k, __float_as_int(ht) - kMagicBits);
    atomicAdd(lo + k, __float_as_int(lt) - kMagicBits);
}

template <int E, int NT, typename OutT>
__global__ void __launch_bounds__(NT, 2) rf_synth_kernel(const RfParams p, const float *__restrict__ pos,
                                                         const float *__restrict__ amp,
                                                         const float *__restrict__ rf_base,
                                                         OutT *__restrict__ rf)
{
    extern __shared__ int tile[];  // hi [E][Ns] then lo [E][Ns]
    __shared__ float ex_hi[E], ex_lo[E], ey_hi[E], ey_lo[E];
    __shared__ float s_red[NT / 32];
    const int ns = p.pr.ns;
    const int M = p.pr.M;
    const int m0 = blockIdx.x * E;
    const int a = blockIdx.y;
    const int f = blockIdx.z;
    const int ne = min(E, M - m0);
    const int64_t S = p.S;
    int *thi = tile, *tlo = tile + E * ns;

    // the amplitude scale g (identical in every CTA): largest |amp| -> [0.5, 1)
    float amax = 0.0f;
    for (int64_t s = threadIdx.x; s < S; s += NT) amax = fmaxf(amax, fabsf(amp[s]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = amax;
    if (threadIdx.x < E) {
        int m = min(m0 + (int)threadIdx.x, M - 1);
        ff ex = fqi::elem_coord(m % p.pr.nx, p.pr.nx, p.pr.pitch_x);
        ff ey = fqi::elem_coord(m / p.pr.nx, p.pr.ny, p.pr.pitch_y);
        ex_hi[threadIdx.x] = ex.hi;
        ex_lo[threadIdx.x] = ex.lo;
        ey_hi[threadIdx.x] = ey.hi;
        ey_lo[threadIdx.x] = ey.lo;
    }
    __syncthreads();
    amax = 0.0f;
    for (int w = 0; w < NT / 32; ++w) amax = fmaxf(amax, s_red[w]);
    int gexp = 0;
    if (amax > 0.0f) frexpf(amax, &gexp);                 // amax = mant * 2^gexp, mant in [0.5, 1)
    const float g = ldexpf(1.0f, -gexp);                  // exact power of two
    const float to_fix = g * kFixScale;

    for (int i = threadIdx.x; i < E * ns; i += NT) {
        int e = i / ns, k = i - e * ns;
        float v = 0.0f;
        if (rf_base && e < ne) v = rf_base[((int64_t)a * M + m0 + e) * ns + k];
        float V = fminf(fmaxf(v * to_fix, -kTapClamp), kTapClamp);
        const float ht = fmaf(V, 1.0f / 65536.0f, kMagic);
        const float hb = ht - kMagic;
        const float lt = fmaf(-hb, 65536.0f, V) + kMagic;
        thi[i] = __float_as_int(ht) - kMagicBits;
        tlo[i] = __float_as_int(lt) - kMagicBits;
    }
    __syncthreads();

    const fqi::AngleFF an = p.ang[a];
    const ff ux = fqi::ff_load(an.ux), uy = fqi::ff_load(an.uy), uz = fqi::ff_load(an.uz);
    const ff org = fqi::ff_load(an.origin);
    const float Kh = p.pr.fs_over_c.hi, Kl = p.pr.fs_over_c.lo;
    const bool matrix = p.pr.ny > 1;
    const float *X = pos + (int64_t)f * 3 * S;
    const float *Y = X + S;
    const float *Z = Y + S;
    const float half_w = p.half_w;
    const int ntap_max = p.ntap_max;
    const bool fast8 = p.two_cycle && ntap_max <= 9;  // the common pulse: at most 9 taps
    const float thc0 = p.tab_h[0][0], ths0 = p.tab_h[0][1], thc1 = p.tab_h[1][0], ths1 = p.tab_h[1][1];

    for (int64_t s = threadIdx.x; s < S; s += NT) {
        const float R = amp[s];
        if (R == 0.0f) continue;
        const float x = X[s], y = Y[s], z = Z[s];
        // transmit path u . r - min u . e, float-float (once per scatterer)
        const ff ptx = fqi::ff_dot3_minus(an.ux, an.uy, an.uz, an.origin, x, y, z);
        const ff zz = fqi::ff_two_prod(z, z);
        const bool use_y = matrix || y != 0.0f;  // 2D workloads keep every scatterer at y = 0
        const float Rfix = R * to_fix;
#pragma unroll 1
        for (int e = 0; e < ne; ++e) {
            // dx = x - ex as an unnormalised pair (TwoSum of x and -ex_hi, plus -ex_lo)
            const float exh = ex_hi[e];
            const float dxh = __fsub_rn(x, exh);
            const float bb = __fsub_rn(dxh, x);
            const float dxl = __fsub_rn(__fadd_rn(__fsub_rn(x, __fsub_rn(dxh, bb)), __fsub_rn(-exh, bb)), ex_lo[e]);
            // r^2 = dx^2 + z^2 (+ dy^2)
            const float p2 = __fmul_rn(dxh, dxh);
            float lo = __fmaf_rn(2.0f * dxh, dxl, __fmaf_rn(dxh, dxh, -p2));
            ff r2 = fqi::ff_two_sum(p2, zz.hi);
            lo = __fadd_rn(lo, zz.lo);
            float dyh = 0.0f;
            if (use_y) {
                const float eyh = ey_hi[e];
                dyh = __fsub_rn(y, eyh);
                const float cc = __fsub_rn(dyh, y);
                const float dyl = __fsub_rn(__fadd_rn(__fsub_rn(y, __fsub_rn(dyh, cc)), __fsub_rn(-eyh, cc)), ey_lo[e]);
                const float q2 = __fmul_rn(dyh, dyh);
                lo = __fadd_rn(lo, __fmaf_rn(2.0f * dyh, dyl, __fmaf_rn(dyh, dyh, -q2)));
                ff t2 = fqi::ff_two_sum(r2.hi, q2);
                r2.hi = t2.hi;
                lo = __fadd_rn(lo, t2.lo);
            }
            lo = __fadd_rn(lo, r2.lo);
            r2 = fqi::ff_fast_two_sum(r2.hi, lo);
            if (r2.hi <= 0.0f) continue;
            // r = sqrt(r^2) and 1/r from one reciprocal square root, plus a
            // Newton correction to float-float accuracy
            const float rs = rsqrtf(r2.hi);
            const float r0 = __fmul_rn(r2.hi, rs);
            const float rl = __fmul_rn(__fadd_rn(__fmaf_rn(-r0, r0, r2.hi), r2.lo), 0.5f * rs);
            // path = ptx + r, u = path * fs / c = k0 + frac
            ff path = fqi::ff_two_sum(ptx.hi, r0);
            path.lo = __fadd_rn(path.lo, __fadd_rn(ptx.lo, rl));
            const float uh = __fmul_rn(path.hi, Kh);
            const float ul = __fmaf_rn(path.hi, Kl, __fmaf_rn(path.lo, Kh, __fmaf_rn(path.hi, Kh, -uh)));
            float fl = floorf(uh);
            float frac = __fadd_rn(__fsub_rn(uh, fl), ul);
            if (frac < 0.0f) { frac += 1.0f; fl -= 1.0f; }
            else if (frac >= 1.0f) { frac -= 1.0f; fl += 1.0f; }
            // amplitude (fixed-point units): reflectivity x directivity x attenuation / r
            float D = sinc_f(p.kbx * dxh * rs);
            if (matrix) D *= sinc_f(p.kby * dyh * rs);
            const float Aa = Rfix * D * __expf(-p.att * path.hi) * rs;
            // taps j = jlo .. jlo + ntap - 1 with |j - frac| < half_w
            const int jlo = (int)ceilf(frac - half_w);
            const int ntap = (int)floorf(frac + half_w) - jlo + 1;
            const int kst = (int)fl + jlo;
            float ch, sh;
            first_tap(p.w_h, frac, thc0, ths0, thc1, ths1, jlo != p.jmin, ch, sh);
            int *lhi = thi + e * ns, *llo = tlo + e * ns;
            const bool inside = kst >= 0 && kst + ntap <= ns;
            if (fast8 && inside) {
                // C_j = cos(w_h (jlo + j - frac)) by the Chebyshev recurrence
                const float hA = 0.5f * Aa;
                float c0 = ch, c1 = fmaf(ch, p.cos_h, -sh * p.sin_h);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    add_fixed(lhi, llo, kst + j, tap2(Aa, hA, c0));
                    const float c2 = fmaf(p.two_cos_h, c1, -c0);
                    c0 = c1;
                    c1 = c2;
                }
                if (ntap > 8) add_fixed(lhi, llo, kst + 8, tap2(Aa, hA, c0));
            } else if (p.two_cycle) {
                const float hA = 0.5f * Aa;
                float c0 = ch, c1 = fmaf(ch, p.cos_h, -sh * p.sin_h);
                for (int j = 0; j < ntap; ++j) {
                    const int k = kst + j;
                    if (k >= 0 && k < ns) add_fixed(lhi, llo, k, tap2(Aa, hA, c0));
                    const float c2 = fmaf(p.two_cos_h, c1, -c0);
                    c0 = c1;
                    c1 = c2;
                }
            } else {
                float cc, sc;
                first_tap(p.w_c, frac, p.tab_c[0][0], p.tab_c[0][1], p.tab_c[1][0], p.tab_c[1][1], jlo != p.jmin, cc,
                          sc);
                float h0 = ch, h1 = fmaf(ch, p.cos_h, -sh * p.sin_h);
                float q0 = cc, q1 = fmaf(cc, p.cos_c, -sc * p.sin_c);
                for (int j = 0; j < ntap; ++j) {
                    const int k = kst + j;
                    if (k >= 0 && k < ns) add_fixed(lhi, llo, k, Aa * fmaf(0.5f, h0, 0.5f) * q0);
                    const float h2 = fmaf(p.two_cos_h, h1, -h0);
                    h0 = h1;
                    h1 = h2;
                    const float q2 = fmaf(p.two_cos_c, q1, -q0);
                    q0 = q1;
                    q1 = q2;
                }
            }
        }
    }
    __syncthreads();
    const float from_fix = 1.0f / to_fix;  // exact power of two
    OutT *out = rf + (((int64_t)f * p.A + a) * M + m0) * ns;
    for (int i = threadIdx.x; i < ne * ns; i += NT)
        fqi::store_f(out, i, fmaf((float)thi[i], 65536.0f, (float)tlo[i]) * from_fix);
}

// ---------------------------------------------------------------------------
// Paired-element kernel for the two-cycle pulse (at most 9 taps): each thread
// evaluates one scatterer for the CTA's two elements at once in packed
// f32x2 arithmetic (float-float geometry, amplitude products, Chebyshev taps,
// fixed-point split); hardware-function calls (rsqrt, sin, exp, sincos) stay
// scalar.  Same results as rf_synth_kernel up to rounding of the FP32 parts.
// ---------------------------------------------------------------------------
using fqi::f2;

// (hi, lo) = (rint(V / 2^16), V - 2^16 hi) of both lanes, as int32 pairs
__device__ __forceinline__ void split_fixed2(f2 V, int &h0, int &h1, int &l0, int &l1)
{
    const f2 ht = fqi::f2_fma(V, fqi::f2_dup(1.0f / 65536.0f), fqi::f2_dup(kMagic));
    const f2 hb = fqi::f2_sub(ht, fqi::f2_dup(kMagic));
    const f2 lt = fqi::f2_add(fqi::f2_fma(hb, fqi::f2_dup(-65536.0f), V), fqi::f2_dup(kMagic));
    float a, b, c, d;
    fqi::f2_split(ht, a, b);
    fqi::f2_split(lt, c, d);
    h0 = __float_as_int(a) - kMagicBits;
    h1 = __float_as_int(b) - kMagicBits;
    l0 = __float_as_int(c) - kMagicBits;
    l1 = __float_as_int(d) - kMagicBits;
}

__device__ __forceinline__ void add_fixed2(int *hi0, int *lo0, int *hi1, int *lo1, int k0, int k1, f2 V, bool on0,
                                           bool on1)
{
    int h0, h1, l0, l1;
    split_fixed2(V, h0, h1, l0, l1);
    if (on0) {
        atomicAdd(hi0 + k0, h0);
        atomicAdd(lo0 + k0, l0);
    }
    if (on1) {
        atomicAdd(hi1 + k1, h1);
        atomicAdd(lo1 + k1, l1);
    }
}

// Unpredicated form for taps known to lie in both records (a lane without
// an echo carries V = 0 and a valid index).
__device__ __forceinline__ void add_fixed2_all(int *hi0, int *lo0, int *hi1, int *lo1, int k0, int k1, f2 V)
{
    int h0, h1, l0, l1;
    split_fixed2(V, h0, h1, l0, l1);
    atomicAdd(hi0 + k0, h0);
    atomicAdd(lo0 + k0, l0);
    atomicAdd(hi1 + k1, h1);
    atomicAdd(lo1 + k1, l1);
}

// the two-cycle tap value for the pair: ((A C + A) C - A/2) C - A/2
__device__ __forceinline__ f2 tap2x2(f2 A, f2 hA, f2 C)
{
    const f2 nhA = fqi::f2_neg(hA);
    return fqi::f2_fma(fqi::f2_fma(fqi::f2_fma(A, C, A), C, nhA), C, nhA);
}

// One tile: elements 2 bx, 2 bx + 1 of transmit a, frame f.  `tile` is the
// dynamic shared memory (4 Ns ints), `s_red` NT / 32 floats.
template <int NT, typename OutT>
__device__ __forceinline__ void rf_pair_tile(const RfParams &p, int bx, int a, int f, const float *__restrict__ pos,
                                             const float *__restrict__ amp, const float *__restrict__ rf_base,
                                             OutT *__restrict__ rf, int *tile, float *s_red)
{
    constexpr int E = 2;
    const int ns = p.pr.ns;
    const int M = p.pr.M;
    const int m0 = bx * E;
    const int ne = min(E, M - m0);
    const int64_t S = p.S;
    int *hi0 = tile, *hi1 = tile + ns, *lo0 = tile + 2 * ns, *lo1 = tile + 3 * ns;

    float amax = 0.0f;
    for (int64_t s = threadIdx.x; s < S; s += NT) amax = fmaxf(amax, fabsf(amp[s]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = amax;
    __syncthreads();
    amax = 0.0f;
    for (int w = 0; w < NT / 32; ++w) amax = fmaxf(amax, s_red[w]);
    int gexp = 0;
    if (amax > 0.0f) frexpf(amax, &gexp);
    const float g = ldexpf(1.0f, -gexp);
    const float to_fix = g * kFixScale;

    for (int i = threadIdx.x; i < E * ns; i += NT) {
        int e = i / ns, k = i - e * ns;
        float v = 0.0f;
        if (rf_base && e < ne) v = rf_base[((int64_t)a * M + m0 + e) * ns + k];
        float V = fminf(fmaxf(v * to_fix, -kTapClamp), kTapClamp);
        const float ht = fmaf(V, 1.0f / 65536.0f, kMagic);
        const float hb = ht - kMagic;
        const float lt = fmaf(-hb, 65536.0f, V) + kMagic;
        tile[e * ns + k] = __float_as_int(ht) - kMagicBits;
        tile[(2 + e) * ns + k] = __float_as_int(lt) - kMagicBits;
    }
    __syncthreads();

    // element centres (float-float) of the pair
    const int m1c = min(m0 + 1, M - 1);
    const ff ex0 = fqi::elem_coord(m0 % p.pr.nx, p.pr.nx, p.pr.pitch_x);
    const ff ex1 = fqi::elem_coord(m1c % p.pr.nx, p.pr.nx, p.pr.pitch_x);
    const ff ey0 = fqi::elem_coord(m0 / p.pr.nx, p.pr.ny, p.pr.pitch_y);
    const ff ey1 = fqi::elem_coord(m1c / p.pr.nx, p.pr.ny, p.pr.pitch_y);
    const f2 EXH = fqi::f2_make(ex0.hi, ex1.hi), EXL = fqi::f2_make(ex0.lo, ex1.lo);
    const f2 EYH = fqi::f2_make(ey0.hi, ey1.hi), EYL = fqi::f2_make(ey0.lo, ey1.lo);
    const f2 NEXH = fqi::f2_neg(EXH), NEYH = fqi::f2_neg(EYH);
    const bool valid1 = ne > 1;

    const fqi::AngleFF an = p.ang[a];
    const ff ux = fqi::ff_load(an.ux), uy = fqi::ff_load(an.uy), uz = fqi::ff_load(an.uz);
    const ff org = fqi::ff_load(an.origin);
    const f2 KH = fqi::f2_dup(p.pr.fs_over_c.hi), KL = fqi::f2_dup(p.pr.fs_over_c.lo);
    const f2 HALF = fqi::f2_dup(0.5f);
    const bool matrix = p.pr.ny > 1;
    const float *X = pos + (int64_t)f * 3 * S;
    const float *Y = X + S;
    const float *Z = Y + S;
    const float half_w = p.half_w;
    const float thc0 = p.tab_h[0][0], ths0 = p.tab_h[0][1], thc1 = p.tab_h[1][0], ths1 = p.tab_h[1][1];
    const f2 COSH = fqi::f2_dup(p.cos_h), SINH = fqi::f2_dup(p.sin_h), TWOCOS = fqi::f2_dup(p.two_cos_h);

    for (int64_t s = threadIdx.x; s < S; s += NT) {
        const float R = amp[s];
        if (R == 0.0f) continue;
        const float x = X[s], y = Y[s], z = Z[s];
        const ff ptx = fqi::ff_dot3_minus(an.ux, an.uy, an.uz, an.origin, x, y, z);
        const ff zz = fqi::ff_two_prod(z, z);
        // dx = x - ex for both elements (TwoSum plus the low word)
        const f2 Xd = fqi::f2_dup(x);
        const f2 dxh = fqi::f2_sub(Xd, EXH);
        const f2 bb = fqi::f2_sub(dxh, Xd);
        const f2 dxl = fqi::f2_sub(fqi::f2_add(fqi::f2_sub(Xd, fqi::f2_sub(dxh, bb)), fqi::f2_sub(NEXH, bb)), EXL);
        // r^2 = dx^2 + z^2 (+ dy^2), float-float
        const f2 p2 = fqi::f2_mul(dxh, dxh);
        f2 lo = fqi::f2_fma(fqi::f2_add(dxh, dxh), dxl, fqi::f2_fma(dxh, dxh, fqi::f2_neg(p2)));
        const f2 ZZH = fqi::f2_dup(zz.hi);
        f2 sh2 = fqi::f2_add(p2, ZZH);
        f2 b2 = fqi::f2_sub(sh2, p2);
        f2 err = fqi::f2_add(fqi::f2_sub(p2, fqi::f2_sub(sh2, b2)), fqi::f2_sub(ZZH, b2));
        lo = fqi::f2_add(lo, fqi::f2_dup(zz.lo));
        f2 dyh = fqi::f2_dup(0.0f);
        if (matrix || y != 0.0f) {
            const f2 Yd = fqi::f2_dup(y);
            dyh = fqi::f2_sub(Yd, EYH);
            const f2 cy = fqi::f2_sub(dyh, Yd);
            const f2 dyl = fqi::f2_sub(fqi::f2_add(fqi::f2_sub(Yd, fqi::f2_sub(dyh, cy)), fqi::f2_sub(NEYH, cy)), EYL);
            const f2 q2 = fqi::f2_mul(dyh, dyh);
            lo = fqi::f2_add(lo, fqi::f2_fma(fqi::f2_add(dyh, dyh), dyl, fqi::f2_fma(dyh, dyh, fqi::f2_neg(q2))));
            const f2 t2 = fqi::f2_add(sh2, q2);
            const f2 b3 = fqi::f2_sub(t2, sh2);
            lo = fqi::f2_add(lo, fqi::f2_add(fqi::f2_sub(sh2, fqi::f2_sub(t2, b3)), fqi::f2_sub(q2, b3)));
            sh2 = t2;
        }
        lo = fqi::f2_add(lo, err);
        const f2 r2h = fqi::f2_add(sh2, lo);
        const f2 r2l = fqi::f2_sub(lo, fqi::f2_sub(r2h, sh2));
        float q0, q1;
        fqi::f2_split(r2h, q0, q1);
        const bool live0 = q0 > 0.0f;
        const bool live1 = valid1 && q1 > 0.0f;
        const f2 R2 = fqi::f2_make(live0 ? q0 : 1.0f, live1 ? q1 : 1.0f);
        const f2 RS = fqi::f2_make(rsqrtf(fqi::f2_lo(R2)), rsqrtf(fqi::f2_hi(R2)));
        // r = r0 + rl and 1/r from one reciprocal square root per element
        const f2 r0 = fqi::f2_mul(R2, RS);
        const f2 rl = fqi::f2_mul(fqi::f2_add(fqi::f2_fma(fqi::f2_neg(r0), r0, R2), r2l), fqi::f2_mul(HALF, RS));
        // path = ptx + r, u = path fs / c
        const f2 PH = fqi::f2_dup(ptx.hi);
        const f2 sp = fqi::f2_add(PH, r0);
        const f2 b4 = fqi::f2_sub(sp, PH);
        const f2 pl = fqi::f2_add(fqi::f2_add(fqi::f2_sub(PH, fqi::f2_sub(sp, b4)), fqi::f2_sub(r0, b4)),
                                  fqi::f2_add(fqi::f2_dup(ptx.lo), rl));
        const f2 uh = fqi::f2_mul(sp, KH);
        const f2 ul = fqi::f2_fma(sp, KL, fqi::f2_fma(pl, KH, fqi::f2_fma(sp, KH, fqi::f2_neg(uh))));
        float uh0, uh1, ul0, ul1;
        fqi::f2_split(uh, uh0, uh1);
        fqi::f2_split(ul, ul0, ul1);
        float fl0 = floorf(uh0), fl1 = floorf(uh1);
        const f2 FR = fqi::f2_add(fqi::f2_sub(uh, fqi::f2_make(fl0, fl1)), ul);
        float fr0, fr1;
        fqi::f2_split(FR, fr0, fr1);
        {  // bring frac into [0, 1) (it is within one of it): move whole samples into fl
            const float c0 = floorf(fr0), c1 = floorf(fr1);
            fr0 -= c0;
            fl0 += c0;
            fr1 -= c1;
            fl1 += c1;
        }
        // amplitude in fixed-point units
        float dxh0, dxh1, rs0, rs1, sp0, sp1;
        fqi::f2_split(dxh, dxh0, dxh1);
        fqi::f2_split(RS, rs0, rs1);
        fqi::f2_split(sp, sp0, sp1);
        float D0 = sinc_poly(p.kbx * dxh0 * rs0), D1 = sinc_poly(p.kbx * dxh1 * rs1);
        if (matrix) {
            float dy0, dy1;
            fqi::f2_split(dyh, dy0, dy1);
            D0 *= sinc_poly(p.kby * dy0 * rs0);
            D1 *= sinc_poly(p.kby * dy1 * rs1);
        }
        const float Rfix = R * to_fix;
        f2 A2 = fqi::f2_mul(fqi::f2_mul(fqi::f2_dup(Rfix), fqi::f2_make(D0, D1)),
                            fqi::f2_mul(fqi::f2_make(__expf(-p.att * sp0), __expf(-p.att * sp1)), RS));
        {  // one clamp per pair bounds every tap (|p| <= 1)
            float a0_, a1_;
            fqi::f2_split(A2, a0_, a1_);
            a0_ = live0 ? fminf(fmaxf(a0_, -kTapClamp), kTapClamp) : 0.0f;
            a1_ = live1 ? fminf(fmaxf(a1_, -kTapClamp), kTapClamp) : 0.0f;
            A2 = fqi::f2_make(a0_, a1_);
        }
        const int jlo0 = (int)ceilf(fr0 - half_w), jlo1 = (int)ceilf(fr1 - half_w);
        const int nt0 = (int)floorf(fr0 + half_w) - jlo0 + 1, nt1 = (int)floorf(fr1 + half_w) - jlo1 + 1;
        const int k0 = (int)fl0 + jlo0, k1 = (int)fl1 + jlo1;
        float ch0, sh0, ch1, sh1;
        first_tap<true>(p.w_h, fr0, thc0, ths0, thc1, ths1, jlo0 != p.jmin, ch0, sh0);
        first_tap<true>(p.w_h, fr1, thc0, ths0, thc1, ths1, jlo1 != p.jmin, ch1, sh1);
        const f2 CH = fqi::f2_make(ch0, ch1), SH = fqi::f2_make(sh0, sh1);
        f2 C0 = CH;
        f2 C1 = fqi::f2_fma(CH, COSH, fqi::f2_neg(fqi::f2_mul(SH, SINH)));
        const f2 hA = fqi::f2_mul(HALF, A2);
        const bool in0 = live0 && k0 >= 0 && k0 + nt0 <= ns;
        const bool in1 = live1 && k1 >= 0 && k1 + nt1 <= ns;
        if (ns >= 8 && (in0 || !live0) && (in1 || !live1)) {
            const int q0 = live0 ? k0 : 0, q1 = live1 ? k1 : 0;  // dead lanes: A = 0 at samples 0-7
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                add_fixed2_all(hi0, lo0, hi1, lo1, q0 + j, q1 + j, tap2x2(A2, hA, C0));
                const f2 C2 = fqi::f2_fma(TWOCOS, C1, fqi::f2_neg(C0));
                C0 = C1;
                C1 = C2;
            }
            if (nt0 > 8 || nt1 > 8)
                add_fixed2(hi0, lo0, hi1, lo1, k0 + 8, k1 + 8, tap2x2(A2, hA, C0), live0 && nt0 > 8,
                           live1 && nt1 > 8);
        } else {
            // an echo straddles a record end: per-tap bounds
            for (int j = 0; j < 9; ++j) {
                const int ka = k0 + j, kb = k1 + j;
                const bool oa = live0 && j < nt0 && ka >= 0 && ka < ns;
                const bool ob = live1 && j < nt1 && kb >= 0 && kb < ns;
                add_fixed2(hi0, lo0, hi1, lo1, oa ? ka : 0, ob ? kb : 0, tap2x2(A2, hA, C0), oa, ob);
                const f2 C2 = fqi::f2_fma(TWOCOS, C1, fqi::f2_neg(C0));
                C0 = C1;
                C1 = C2;
            }
        }
    }
    __syncthreads();
    const float from_fix = 1.0f / to_fix;
    OutT *out = rf + (((int64_t)f * p.A + a) * M + m0) * ns;
    for (int i = threadIdx.x; i < ne * ns; i += NT)
        fqi::store_f(out, i, fmaf((float)tile[i], 65536.0f, (float)tile[2 * ns + i]) * from_fix);
}

template <int NT, int MINB, typename OutT>
__global__ void __launch_bounds__(NT, MINB) rf_synth_pair_kernel(const RfParams p, const float *__restrict__ pos,
                                                              const float *__restrict__ amp,
                                                              const float *__restrict__ rf_base,
                                                              OutT *__restrict__ rf)
{
    extern __shared__ int tile[];  // hi [2][Ns] then lo [2][Ns]
    __shared__ float s_red[NT / 32];
    rf_pair_tile<NT, OutT>(p, blockIdx.x, blockIdx.y, blockIdx.z, pos, amp, rf_base, rf, tile, s_red);
}

// Persistent form over the RF items of many ensembles (no static-tissue base).
constexpr int kRfParamBytes = (sizeof(RfParams) + 15) & ~15;

template <int NT, int MINB, typename OutT>
__global__ void __launch_bounds__(NT, MINB) rf_pair_batched_kernel(const fqb::EnsDev *__restrict__ ens,
                                                                const fqb::StageQueue q)
{
    extern __shared__ int tile[];
    __shared__ float s_red[NT / 32];
    __shared__ __align__(16) unsigned char s_par[kRfParamBytes];
    __shared__ int s_buf[2];
    int cur = -1;
    fqb::Item it;
    while (fqb::next_item(q, ens, fqb::ST_RF, s_buf, it)) {
        const fqb::EnsDev &e = ens[it.e];
        if (it.e != cur) {
            fqb::copy_block(s_par, e.rf_params, kRfParamBytes);
            cur = it.e;
            __syncthreads();
        }
        rf_pair_tile<NT, OutT>(*reinterpret_cast<const RfParams *>(s_par), it.x, it.y, it.z, e.pos, e.amp_eff,
                               nullptr, (OutT *)e.rf, tile, s_red);
    }
}

// ---------------------------------------------------------------------------
// Quad-element kernel: 4 consecutive elements of one array row and a group of
// transmit angles per CTA.
//
// Geometry.  The float-float delay is evaluated for the quad's first element
// only; the other three follow from the exact identity
//     r_e - r_0 = (x_0 - x_e) (2 x - x_0 - x_e) / (r_e + r_0)
// evaluated in binary32: |r_e - r_0| is at most 3 pitches (a dozen samples),
// so its rounding error stays near 1e-6 sample.  The receive side (the four
// distances, directivities and 1/r) does not depend on the transmit, so it is
// evaluated once per scatterer and reused by every angle of the group; the
// transmit path, delays, attenuation and taps are per angle.  The taps of
// elements (0, 1) and (2, 3) run as packed f32x2 pairs.
//
// Accumulation: one int32 per sample, one shared-memory atomic per tap.
// Integer sums are exact modulo 2^32 in any order, so a record is exact (and
// bit-reproducible) as long as its final values fit in int32.  Each record
// gets the finest quantum q for which that is guaranteed:
//   pass 0  b_max = largest |amp| / (distance to the quad) sets the integer
//           units of pass 1;
//   pass 1  every (scatterer, element pair, angle) adds an upper bound of the
//           pair's taps, |amp| D_b / r_s in those units (r_s = distance to the
//           segment between the two elements, D_b >= |directivity|), at the
//           sample nearest to its binary32 mid-pair delay; both elements'
//           delays are within half a pitch of it, and the binary32 delay is
//           within 0.51 sample of the exact one, so a window of
//           2 floor(half_w + pitch fs / 2c + 0.52) + 1 samples around a sample
//           bounds the sum of |taps| that land on it in either record;
//   scale   1/q = the largest value that keeps (window maximum x margin +
//           largest |static base|) / q + half a quantum per scatterer (tap
//           rounding) below 2^31.
// The margin covers the attenuation gain of echoes that start just before
// t = 0 and binary32 rounding of the amplitudes.
// ---------------------------------------------------------------------------
constexpr float kInvRCap = 131072.0f;               // 1/r <= 2^17 per metre (r >= 7.6 um)
constexpr float kTapMax = 2147483520.0f;            // largest binary32 below 2^31: |tap| bound in quanta
constexpr float kUnitMax = 2097152.0f;              // 2^21: largest pass-1 bound in units
constexpr float kTwo31 = 2147483648.0f;

struct QuadShared {
    float red[32];                     // one per warp
    float invq[4 * FQ_MAX_ANGLES];     // 1 / q per record (angle in group, element)
    float q[4 * FQ_MAX_ANGLES];
    unsigned wmax[4 * FQ_MAX_ANGLES];  // window maximum of the pass-1 bounds (units)
    unsigned bmax[4 * FQ_MAX_ANGLES];  // largest |static base| (float bits, >= 0)
    float4 angK[FQ_MAX_ANGLES + 1];    // pass 1: fs / c, then per angle (u, -origin) fs / c
    float4 angFF[2 * FQ_MAX_ANGLES];   // pass 2: per angle (ux, uy) and (uz, origin) as float pairs
};

// Largest record (or bound-bin) area of a quad CTA: a block holds at most
// 227 KB (232,448 bytes) of shared memory on this GPU, less the kernels'
// static QuadShared and, in the batched kernel, the parameter block.
constexpr size_t kQuadSmemMax = 232448 - sizeof(QuadShared) - (size_t)kRfParamBytes - 64;

// an upper bound of |sin(u) / u| for |u| <= 5 (the fitted directivity's
// range): 1 - u^2/6 + u^4/120 bounds sin(u)/u from above for every u (the
// alternating series), is at least 0.16 on [pi, 5] where |sin(u)/u| < 0.22,
// and is exact to O(u^6) where the directivity is near 1
__device__ __forceinline__ float sinc_bound(float u)
{
    const float t = u * u;
    return fmaf(fmaf(t, 1.0f / 120.0f, -1.0f / 6.0f), t, 1.0f);
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = red[0];
    for (int w = 1; w < NT / 32; ++w) v = fmaxf(v, red[w]);
    __syncthreads();
    return v;
}

// a non-negative float below 2^22 rounded to the nearest integer
__device__ __forceinline__ int rint_small(float v) { return __float_as_int(v + kMagic) - kMagicBits; }

// one tap of two records: V = (V0, V1) in quanta (|V| < 2^31) rounded to the
// nearest integers and added
__device__ __forceinline__ void add_tap2(int *r0, int *r1, int k0, int k1, f2 V)
{
    float a, b;
    fqi::f2_split(V, a, b);
    atomicAdd(r0 + k0, __float2int_rn(a));
    atomicAdd(r1 + k1, __float2int_rn(b));
}

__device__ __forceinline__ void add_tap2_if(int *r0, int *r1, int k0, int k1, f2 V, bool on0, bool on1)
{
    float a, b;
    fqi::f2_split(V, a, b);
    if (on0) atomicAdd(r0 + k0, __float2int_rn(a));
    if (on1) atomicAdd(r1 + k1, __float2int_rn(b));
}

// the two-cycle tap from the Hann-phase cosine C with nhA = -A/2:
// ((A C + A) C - A/2) C - A/2
__device__ __forceinline__ f2 tap2n(f2 A, f2 nhA, f2 C)
{
    return fqi::f2_fma(fqi::f2_fma(fqi::f2_fma(A, C, A), C, nhA), C, nhA);
}

// (C_j, C_{j+1}, -C_j, -C_{j+1}) -> (C_{j+1}, C_{j+2}, -C_{j+1}, -C_{j+2})
__device__ __forceinline__ void cheb_step(f2 &C0, f2 &C1, f2 &N0, f2 &N1, f2 T, f2 NT)
{
    const f2 C2 = fqi::f2_fma(T, C1, N0);
    const f2 N2 = fqi::f2_fma(NT, C1, C0);
    C0 = C1;
    C1 = C2;
    N0 = N1;
    N1 = N2;
}

// One tile: elements 4 bx .. 4 bx + 3, angles ag * p.ag .. (of the group),
// frame f.  `tile` is the dynamic shared memory (p.ag * 4 * Ns ints).
// Delays: float-float (~48 bits) for FP32 outputs; for 16-bit outputs the
// binary32 delay (error ~1e-4 sample, a carrier-phase error ~2e-4 rad, below
// the BF16 / FP16 storage rounding of 2^-9 / 2^-11) saves the error-free
// transforms of the receive distance and the transmit path.
template <int NT, typename OutT, bool FFD = (sizeof(OutT) == 4)>
__device__ __forceinline__ void rf_quad_tile(const RfParams &p, int bx, int ag, int f, const float *__restrict__ pos,
                                             const float *__restrict__ amp, const float *__restrict__ rf_base,
                                             OutT *__restrict__ rf, int *tile, QuadShared &sh)
{
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps, at most 1024 threads");
    constexpr int E = 4;
    const int ns = p.pr.ns;
    const int M = p.pr.M;
    const int m0 = bx * E;
    const int ne = min(E, M - m0);
    const int64_t S = p.S;
    const int a0 = ag * p.ag;
    const int na = min(p.ag, p.A - a0);
    const int nrec = na * E;
    const bool matrix = p.pr.ny > 1;
    const float *X = pos + (int64_t)f * 3 * S;
    const float *Y = X + S;
    const float *Z = Y + S;

    // element abscissae: the first as a float pair, the others as binary32
    // offsets x_0 - x_e and sums x_0 + x_e (all in one row: nx % 4 == 0)
    const int row = m0 / p.pr.nx, col0 = m0 % p.pr.nx;
    const ff ex0 = fqi::elem_coord(col0, p.pr.nx, p.pr.pitch_x);
    const ff ey = fqi::elem_coord(row, p.pr.ny, p.pr.pitch_y);
    float cd[E], csh[E], csl[E], exf[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const ff xe = fqi::elem_coord(min(col0 + e, p.pr.nx - 1), p.pr.nx, p.pr.pitch_x);
        exf[e] = xe.hi + xe.lo;
        cd[e] = (ex0.hi - xe.hi) + (ex0.lo - xe.lo);
        const ff sum = fqi::ff_add(ex0, xe);  // x_0 + x_e as a float pair: 2 x - sum cancels exactly
        csh[e] = sum.hi;
        csl[e] = sum.lo;
    }
    bool live_e[E];
#pragma unroll
    for (int e = 0; e < E; ++e) live_e[e] = e < ne;
    const float eyf = ey.hi + ey.lo;
    // the quad's abscissae span [xlo, xhi] (dead lanes repeat the last element)
    const float xlo = fminf(fminf(exf[0], exf[1]), fminf(exf[2], exf[3]));
    const float xhi = fmaxf(fmaxf(exf[0], exf[1]), fmaxf(exf[2], exf[3]));

    // the previous item of a persistent CTA may still read the tile
    __syncthreads();
    if ((int)threadIdx.x <= na) {  // [0].w = fs / c; [1 + al] = the transmit direction and origin x fs / c
        const float K = p.pr.fs_over_c.hi;
        float4 g = make_float4(0.0f, 0.0f, 0.0f, K);
        if (threadIdx.x > 0) {
            const fqi::AngleFF &an = p.ang[a0 + threadIdx.x - 1];
            g = make_float4(an.ux.hi * K, an.uy.hi * K, an.uz.hi * K, -an.origin.hi * K);
            sh.angFF[2 * threadIdx.x - 2] = make_float4(an.ux.hi, an.ux.lo, an.uy.hi, an.uy.lo);
            sh.angFF[2 * threadIdx.x - 1] = make_float4(an.uz.hi, an.uz.lo, an.origin.hi, an.origin.lo);
        }
        sh.angK[threadIdx.x] = g;
    }

    // Scatterer groups [sb, se): the rounding error of a record grows with
    // the number of scatterers that share its quantum (the quantum follows
    // the sum of |taps|, which grows linearly, while the echo grows as its
    // square root), so FP32 outputs of large media take several groups,
    // each with its own quanta, summed into the output in FP32.
    for (int sg = 0; sg < p.n_sg; ++sg) {
    const int64_t sb = S * sg / p.n_sg, se = S * (sg + 1) / p.n_sg, Sg = se - sb;
    const bool with_base = rf_base != nullptr && sg == 0;
    __syncthreads();  // the previous group's store still reads the tile
    for (int i = threadIdx.x; i < na * 2 * (ns + 2 * p.win); i += NT) tile[i] = 0;
    if ((int)threadIdx.x < nrec) {
        sh.wmax[threadIdx.x] = 0u;
        sh.bmax[threadIdx.x] = 0u;
    }
    __syncthreads();

    // ---- pass 0: the largest possible tap, and the largest |base| per record
    float bm = 0.0f;
    for (int64_t s = sb + threadIdx.x; s < se; s += NT) {
        const float R = amp[s];
        if (R == 0.0f) continue;
        const float x = X[s], y = Y[s], z = Z[s];
        const float dx = x - fminf(fmaxf(x, xlo), xhi);  // distance to the quad's segment <= to any element
        const float dy = y - eyf;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, z * z));
        bm = fmaxf(bm, fabsf(R) * fminf(rsqrtf(r2), kInvRCap));
    }
    if (with_base) {
        for (int rec = 0; rec < nrec; ++rec) {
            const int al = rec >> 2, e = rec & 3;
            if (e >= ne) continue;
            const float *b = rf_base + ((int64_t)(a0 + al) * M + m0 + e) * ns;
            float v = 0.0f;
            for (int k = threadIdx.x; k < ns; k += NT) v = fmaxf(v, fabsf(b[k]));
            for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
            if ((threadIdx.x & 31) == 0) atomicMax(&sh.bmax[rec], __float_as_uint(v));
        }
    }
    bm = block_max<NT>(bm, sh.red);

    // ---- pass 1: tap bounds per element pair (0, 1), (2, 3).  The segment
    // between a pair's elements is at distance r_s <= r_e <= r_s + pitch from
    // the scatterer, so both elements' delays lie within pitch fs / (2 c) of
    // (ptx + r_s) fs / c + pitch fs / (2 c); the bound |amp| D / r_s is added
    // at the nearest sample of that binary32 delay, in records of ns + 2 win
    // bins (bin i holds sample i - win; win covers half_w + half a pitch +
    // 0.51 sample of rounding)
    const int win = p.win;
    const int wstride = ns + 2 * win;
    const float margin = p.bound_margin;
    // units: the sum over every scatterer stays below 2^30 and one bound below 2^21
    const float unit = fminf(1073741824.0f / ((float)Sg * bm * 1.0078125f), kUnitMax / (bm * 1.0078125f));
    unsigned *bins = reinterpret_cast<unsigned *>(tile);
    if (bm > 0.0f) {
        const float K = sh.angK[0].w;
        const float hpK0 = 0.5f * (exf[1] - exf[0]) * K, hpK1 = 0.5f * (exf[3] - exf[2]) * K;
        float nR = 0.0f, nx = 0.0f, ny = 0.0f, nz = 0.0f;  // one scatterer ahead
        if (sb + threadIdx.x < se) {
            nR = amp[sb + threadIdx.x];
            nx = X[sb + threadIdx.x];
            ny = Y[sb + threadIdx.x];
            nz = Z[sb + threadIdx.x];
        }
        for (int64_t s = sb + threadIdx.x; s < se; s += NT) {
            const float R = nR, x = nx, y = ny, z = nz;
            if (s + NT < se) {
                nR = amp[s + NT];
                nx = X[s + NT];
                ny = Y[s + NT];
                nz = Z[s + NT];
            }
            if (R == 0.0f) continue;
            const float dy = y - eyf;
            const float zy2 = fmaf(dy, dy, z * z);
            const float aR = fabsf(R) * unit;
            float reK[2];
            int ub[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float dxs = x - fminf(fmaxf(x, exf[2 * h]), exf[2 * h + 1]);
                const float r2 = fmaf(dxs, dxs, zy2);
                const float rs = rsqrtf(r2);
                reK[h] = fmaf(r2 > 0.0f ? r2 * rs : 0.0f, K, h ? hpK1 : hpK0);
                // |D| of either element: the bound at the pair's smallest
                // |argument| or at its largest possible one (k0 w / 2); 1 for
                // scatterers closer than the 1/r cap; the matrix probe's
                // y-directivity bounded by 1
                const float D = rs > kInvRCap ? 1.0f : fmaxf(sinc_bound(p.kbx * dxs * rs), p.dbx_far);
                ub[h] = (live_e[2 * h] || live_e[2 * h + 1]) ? rint_small(aR * fminf(rs, kInvRCap) * D) + 1 : 0;
            }
            for (int al = 0; al < na; ++al) {
                const float4 g = sh.angK[al + 1];  // (ux, uy, uz, -origin) fs / c
                const float ptxK = fmaf(g.x, x, fmaf(g.y, y, fmaf(g.z, z, g.w)));
                unsigned *rb = bins + al * 2 * wstride;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // nearest sample of the binary32 delay (within 0.51 of the exact
                    // one) as a bin index; any other value (huge or NaN delays)
                    // fails the test
                    const int kb = __float_as_int((ptxK + reK[h]) + kMagic) - (kMagicBits - win);
                    if (ub[h] && (unsigned)kb < (unsigned)wstride) atomicAdd(rb + h * wstride + kb, (unsigned)ub[h]);
                }
            }
        }
    }
    __syncthreads();
    {
        const int nch = (ns + 15) >> 4;
        for (int c = threadIdx.x; c < na * 2 * nch; c += NT) {
            const int rec = c / nch;
            const int t0 = (c - rec * nch) << 4;
            const unsigned *b = bins + rec * wstride + t0;  // sample t0 - win .. : the window of sample t0
            unsigned sum = 0u;
            for (int i = 0; i <= 2 * win; ++i) sum += b[i];
            unsigned m = sum;
            const int t1 = min(16, ns - t0);
            for (int t = 1; t < t1; ++t) {
                sum += b[t + 2 * win] - b[t - 1];
                m = max(m, sum);
            }
            atomicMax(&sh.wmax[rec], m);
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < nrec) {
        const int rec = threadIdx.x;
        const float B = bm > 0.0f ? (float)sh.wmax[rec >> 1] / unit : 0.0f;  // bound of sum |taps| (amplitude units)
        const float den = B * margin + __uint_as_float(sh.bmax[rec]) * 1.0009765625f;
        float iq = (kTwo31 - (0.5f * (float)Sg + 64.0f)) / den;
        if (!(iq > 0.0f && iq < 1e30f)) iq = 1.0f;
        sh.invq[rec] = iq;
        sh.q[rec] = 1.0f / iq;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nrec * ns; i += NT) {
        const int rec = i / ns, k = i - rec * ns;
        const int e = rec & 3;
        int v = 0;
        if (with_base && e < ne)
            v = __float2int_rn(rf_base[((int64_t)(a0 + (rec >> 2)) * M + m0 + e) * ns + k] * sh.invq[rec]);
        tile[i] = v;
    }
    __syncthreads();

    // ---- pass 2: the taps
    const float Kh = p.pr.fs_over_c.hi, Kl = p.pr.fs_over_c.lo;
    const float att_l2K = p.att_l2 / Kh;  // per sample of delay
    const float theta = p.theta, theta2 = p.theta2, jmin_f = p.jmin_f, att_l2 = p.att_l2;
    const int kfast = ns - 9;  // records k .. k + 8 inside [0, ns): 0 <= k <= kfast
    const float thc0 = p.tab_h[0][0], ths0 = p.tab_h[0][1], thc1 = p.tab_h[1][0], ths1 = p.tab_h[1][1];
    const f2 COSH = fqi::f2_dup(p.cos_h), SINH = fqi::f2_dup(p.sin_h), TWOCOS = fqi::f2_dup(p.two_cos_h);
    const f2 NCOSH = fqi::f2_dup(-p.cos_h), NSINH = fqi::f2_dup(-p.sin_h), NTWOCOS = fqi::f2_dup(-p.two_cos_h);
    const f2 NHALF = fqi::f2_dup(-0.5f);
    const f2 DCC = fqi::f2_dup(p.dc_corr);

    // the next scatterer's inputs are loaded one iteration ahead
    float nR = 0.0f, nx = 0.0f, ny = 0.0f, nz = 0.0f;
    if (bm > 0.0f && sb + threadIdx.x < se) {
        nR = amp[sb + threadIdx.x];
        nx = X[sb + threadIdx.x];
        ny = Y[sb + threadIdx.x];
        nz = Z[sb + threadIdx.x];
    }
    for (int64_t s = sb + threadIdx.x; bm > 0.0f && s < se; s += NT) {
        const float R = nR, x = nx, y = ny, z = nz;
        if (s + NT < se) {
            nR = amp[s + NT];
            nx = X[s + NT];
            ny = Y[s + NT];
            nz = Z[s + NT];
        }
        if (R == 0.0f) continue;
        const bool use_y = matrix || y != 0.0f;
        float dxh, dyh = 0.0f, q2 = 0.0f, zzh, rs0, r0, rl;
        bool pos0;
        if constexpr (FFD) {
            const ff zz = fqi::ff_two_prod(z, z);
            zzh = zz.hi;
            // ---- receive side, element 0: float-float distance
            dxh = __fsub_rn(x, ex0.hi);
            const float bb = __fsub_rn(dxh, x);
            const float dxl = __fsub_rn(__fadd_rn(__fsub_rn(x, __fsub_rn(dxh, bb)), __fsub_rn(-ex0.hi, bb)), ex0.lo);
            const float p2 = __fmul_rn(dxh, dxh);
            float lo = __fmaf_rn(2.0f * dxh, dxl, __fmaf_rn(dxh, dxh, -p2));
            ff r2 = fqi::ff_two_sum(p2, zz.hi);
            lo = __fadd_rn(lo, zz.lo);
            if (use_y) {
                dyh = __fsub_rn(y, ey.hi);
                const float cc = __fsub_rn(dyh, y);
                const float dyl = __fsub_rn(__fadd_rn(__fsub_rn(y, __fsub_rn(dyh, cc)), __fsub_rn(-ey.hi, cc)), ey.lo);
                q2 = __fmul_rn(dyh, dyh);
                lo = __fadd_rn(lo, __fmaf_rn(2.0f * dyh, dyl, __fmaf_rn(dyh, dyh, -q2)));
                ff t2 = fqi::ff_two_sum(r2.hi, q2);
                r2.hi = t2.hi;
                lo = __fadd_rn(lo, t2.lo);
            }
            lo = __fadd_rn(lo, r2.lo);
            r2 = fqi::ff_fast_two_sum(r2.hi, lo);
            pos0 = r2.hi > 0.0f;
            rs0 = pos0 ? rsqrtf(r2.hi) : 0.0f;
            r0 = __fmul_rn(r2.hi, rs0);
            rl = pos0 ? __fmul_rn(__fadd_rn(__fmaf_rn(-r0, r0, r2.hi), r2.lo), 0.5f * rs0) : 0.0f;
        } else {
            // ---- receive side, element 0: binary32 distance with one Newton
            // correction (explicitly rounded operations: the same results in
            // every kernel that inlines this tile)
            zzh = __fmul_rn(z, z);
            dxh = __fsub_rn(x, exf[0]);
            if (use_y) {
                dyh = __fsub_rn(y, eyf);
                q2 = __fmul_rn(dyh, dyh);
            }
            const float r2h = fmaf(dxh, dxh, __fadd_rn(zzh, q2));
            pos0 = r2h > 0.0f;
            rs0 = pos0 ? rsqrtf(r2h) : 0.0f;
            r0 = __fmul_rn(r2h, rs0);
            rl = pos0 ? __fmul_rn(fmaf(-r0, r0, r2h), __fmul_rn(0.5f, rs0)) : 0.0f;
        }
        // ---- receive side, every element: delay offset, directivity, R D / r
        const float zy2 = __fadd_rn(zzh, q2);  // z^2 (+ dy^2), binary32
        const float r0f = __fadd_rn(r0, rl);
        const float r0K = FFD ? 0.0f : __fmul_rn(r0f, Kh);
        float dxa[E], rsa[E], dee[E];
        bool liv[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            float dxe, rse;
            bool ok;
            if (e == 0) {
                dxe = dxh;
                rse = rs0;
                dee[e] = 0.0f;
                ok = pos0;
            } else {
                dxe = __fsub_rn(x, exf[e]);
                const float re2 = fmaf(dxe, dxe, zy2);
                rse = rsqrtf(re2);
                const float re = __fmul_rn(re2, rse);
                dee[e] = __fdividef(__fmul_rn(cd[e], __fsub_rn(fmaf(2.0f, x, -csh[e]), csl[e])),
                                    __fadd_rn(re, r0f));  // r_e - r_0
                ok = re2 > 0.0f;
            }
            dxa[e] = dxe;
            rsa[e] = fminf(rse, kInvRCap);
            liv[e] = live_e[e] && ok;
        }
        // R D / r per element pair, D = sinc(k0 w/2 dx / r) (x sinc(k0 h/2 dy / r))
        f2 RD2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const f2 RS = fqi::f2_make(rsa[2 * h], rsa[2 * h + 1]);
            f2 D = sinc_poly2(fqi::f2_mul(fqi::f2_mul(fqi::f2_dup(p.kbx), fqi::f2_make(dxa[2 * h], dxa[2 * h + 1])), RS));
            if (matrix) D = fqi::f2_mul(D, sinc_poly2(fqi::f2_mul(fqi::f2_dup(p.kby * dyh), RS)));
            RD2[h] = fqi::f2_mul(fqi::f2_mul(fqi::f2_dup(R), D), RS);
        }
        // the attenuation exp(-att (path_0 + r_e - r_0)) as the per-transmit
        // factor of element 0 times a per-element factor that does not depend
        // on the transmit (1 for element 0)
        RD2[0] = fqi::f2_mul(RD2[0], fqi::f2_make(1.0f, ex2_approx(att_l2 * dee[1])));
        RD2[1] = fqi::f2_mul(RD2[1], fqi::f2_make(ex2_approx(att_l2 * dee[2]), ex2_approx(att_l2 * dee[3])));
        const f2 DE2[2] = {fqi::f2_make(0.0f, dee[1]), fqi::f2_make(dee[2], dee[3])};
        for (int al = 0; al < na; ++al) {
            float fl0, fr0, path_hi;
            if constexpr (FFD) {
                const float4 g0 = sh.angFF[2 * al], g1 = sh.angFF[2 * al + 1];
                const ff ptx = fqi::ff_dot3_minus({g0.x, g0.y}, {g0.z, g0.w}, {g1.x, g1.y}, {g1.z, g1.w}, x, y, z);
                ff path = fqi::ff_two_sum(ptx.hi, r0);
                path.lo = __fadd_rn(path.lo, __fadd_rn(ptx.lo, rl));
                const float uh = __fmul_rn(path.hi, Kh);
                const float ul = __fmaf_rn(path.hi, Kl, __fmaf_rn(path.lo, Kh, __fmaf_rn(path.hi, Kh, -uh)));
                fl0 = floorf(uh);
                fr0 = __fadd_rn(__fsub_rn(uh, fl0), ul);
                const float c = floorf(fr0);
                fr0 -= c;
                fl0 += c;
                path_hi = path.hi;
            } else {
                // binary32: (u . r - origin) fs / c + r fs / c in samples
                const float4 g = sh.angK[al + 1];
                const float u = __fadd_rn(r0K, fmaf(g.x, x, fmaf(g.y, y, fmaf(g.z, z, g.w))));
                fl0 = floorf(u);
                fr0 = __fsub_rn(u, fl0);
                path_hi = u;  // the attenuation exponent takes samples here
            }
            // per element pair (0, 1), (2, 3), two lanes of packed f32x2 (element
            // 0's offset from itself is 0); FRND, MUFU, conversions and
            // selects stay scalar
            const ulonglong2 iqv = *reinterpret_cast<const ulonglong2 *>(&sh.invq[al * E]);
            const f2 IQ2[2] = {f2{iqv.x}, f2{iqv.y}};
            const f2 FR0 = fqi::f2_dup(fr0), FL0 = fqi::f2_dup(fl0);
            const f2 ATT0 = fqi::f2_dup(ex2_approx((FFD ? att_l2 : att_l2K) * path_hi));
            f2 A2[2], CH2[2], SH2[2];
            int ke[E];
            bool ine[E], nine[E];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const f2 T = fqi::f2_fma(DE2[h], fqi::f2_dup(Kh), FR0);
                float t0, t1;
                fqi::f2_split(T, t0, t1);
                const f2 C = fqi::f2_make(floorf(t0), floorf(t1));
                const f2 FR = fqi::f2_sub(T, C);
                const f2 FL = fqi::f2_add(FL0, C);
                float a0, a1;
                fqi::f2_split(fqi::f2_mul(fqi::f2_mul(RD2[h], IQ2[h]), ATT0), a0, a1);
                // one clamp bounds every tap (|p| <= 1)
                a0 = liv[2 * h] ? fminf(fmaxf(a0, -kTapMax), kTapMax) : 0.0f;
                a1 = liv[2 * h + 1] ? fminf(fmaxf(a1, -kTapMax), kTapMax) : 0.0f;
                A2[h] = fqi::f2_make(a0, a1);
                // taps j = jlo .. jlo + nt - 1 with |j - frac| < half_w: jlo is jmin
                // or jmin + 1, nt is 8 or 9
                float fr_0, fr_1;
                fqi::f2_split(FR, fr_0, fr_1);
                const bool lo0 = fr_0 <= theta, lo1 = fr_1 <= theta;
                float k0f, k1f;
                fqi::f2_split(fqi::f2_add(FL, fqi::f2_make(lo0 ? jmin_f : jmin_f + 1.0f, lo1 ? jmin_f : jmin_f + 1.0f)),
                              k0f, k1f);
                ke[2 * h] = (int)k0f;
                ke[2 * h + 1] = (int)k1f;
                // first tap (cos, sin)(w (jlo - frac)) = e^{i w jlo} e^{-i w frac}
                f2 SF, CF;
                sincos_poly2(fqi::f2_mul(fqi::f2_dup(p.w_h), FR), SF, CF);
                const f2 TC = fqi::f2_make(lo0 ? thc0 : thc1, lo1 ? thc0 : thc1);
                const f2 TS = fqi::f2_make(lo0 ? ths0 : ths1, lo1 ? ths0 : ths1);
                const f2 NTC = fqi::f2_make(lo0 ? -thc0 : -thc1, lo1 ? -thc0 : -thc1);
                CH2[h] = fqi::f2_fma(CF, TC, fqi::f2_mul(SF, TS));
                SH2[h] = fqi::f2_fma(TS, CF, fqi::f2_mul(NTC, SF));
                nine[2 * h] = lo0 || fr_0 >= theta2;
                nine[2 * h + 1] = lo1 || fr_1 >= theta2;
                ine[2 * h] = liv[2 * h] && (unsigned)ke[2 * h] <= (unsigned)kfast;
                ine[2 * h + 1] = liv[2 * h + 1] && (unsigned)ke[2 * h + 1] <= (unsigned)kfast;
            }
            int *rec = tile + al * E * ns;
            int *r0p = rec, *r1p = rec + ns, *r2p = rec + 2 * ns, *r3p = rec + 3 * ns;
            const f2 A01 = A2[0], A23 = A2[1];
            const f2 nhA01 = fqi::f2_mul(NHALF, A01), nhA23 = fqi::f2_mul(NHALF, A23);
            const f2 CH01 = CH2[0], SH01 = SH2[0];
            const f2 CH23 = CH2[1], SH23 = SH2[1];
            // Hann-phase cosines C_j and their negatives N_j = -C_j (exactly:
            // fma is symmetric in sign), so that C_{j+1} = 2 cos(w) C_j - C_{j-1}
            // needs no separate negation
            f2 Ca0 = CH01, Ca1 = fqi::f2_fma(CH01, COSH, fqi::f2_mul(SH01, NSINH));
            f2 Cb0 = CH23, Cb1 = fqi::f2_fma(CH23, COSH, fqi::f2_mul(SH23, NSINH));
            f2 Na0 = fqi::f2_neg(CH01), Na1 = fqi::f2_fma(CH01, NCOSH, fqi::f2_mul(SH01, SINH));
            f2 Nb0 = fqi::f2_neg(CH23), Nb1 = fqi::f2_fma(CH23, NCOSH, fqi::f2_mul(SH23, SINH));
            const bool fast = (ine[0] || !liv[0]) && (ine[1] || !liv[1]) && (ine[2] || !liv[2]) && (ine[3] || !liv[3]);
            if (fast) {
                const int q0 = liv[0] ? ke[0] : 0, q1 = liv[1] ? ke[1] : 0;  // dead lanes: A = 0 at samples 0-7
                const int q2i = liv[2] ? ke[2] : 0, q3 = liv[3] ? ke[3] : 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    f2 ta = tap2n(A01, nhA01, Ca0), tb = tap2n(A23, nhA23, Cb0);
                    if constexpr (FFD) {
                        if (j == 4) {  // the mean error of the recurrence's taps, taken out (see pulse_dc_bias)
                            ta = fqi::f2_fma(DCC, A01, ta);
                            tb = fqi::f2_fma(DCC, A23, tb);
                        }
                    }
                    add_tap2(r0p, r1p, q0 + j, q1 + j, ta);
                    add_tap2(r2p, r3p, q2i + j, q3 + j, tb);
                    cheb_step(Ca0, Ca1, Na0, Na1, TWOCOS, NTWOCOS);
                    cheb_step(Cb0, Cb1, Nb0, Nb1, TWOCOS, NTWOCOS);
                }
                if (nine[0] || nine[1])
                    add_tap2_if(r0p, r1p, ke[0] + 8, ke[1] + 8, tap2n(A01, nhA01, Ca0),
                                liv[0] && nine[0], liv[1] && nine[1]);
                if (nine[2] || nine[3])
                    add_tap2_if(r2p, r3p, ke[2] + 8, ke[3] + 8, tap2n(A23, nhA23, Cb0),
                                liv[2] && nine[2], liv[3] && nine[3]);
            } else {
                // an echo straddles a record end: per-tap bounds
                for (int j = 0; j < 9; ++j) {
                    int kk[E];
                    bool on[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        kk[e] = ke[e] + j;
                        on[e] = liv[e] && j < (nine[e] ? 9 : 8) && kk[e] >= 0 && kk[e] < ns;
                        if (!on[e]) kk[e] = 0;
                    }
                    add_tap2_if(r0p, r1p, kk[0], kk[1], tap2n(A01, nhA01, Ca0), on[0], on[1]);
                    add_tap2_if(r2p, r3p, kk[2], kk[3], tap2n(A23, nhA23, Cb0), on[2], on[3]);
                    cheb_step(Ca0, Ca1, Na0, Na1, TWOCOS, NTWOCOS);
                    cheb_step(Cb0, Cb1, Nb0, Nb1, TWOCOS, NTWOCOS);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nrec * ns; i += NT) {
        const int rec = i / ns, k = i - rec * ns;
        const int e = rec & 3;
        if (e >= ne) continue;
        OutT *out = rf + (((int64_t)f * p.A + a0 + (rec >> 2)) * M + m0 + e) * ns;
        const float v = __fmul_rn((float)tile[i], sh.q[rec]);
        fqi::store_f(out, k, sg == 0 ? v : __fadd_rn(fqi::load_f(out, k), v));  // this CTA owns these samples
    }
    }  // scatterer groups
}

template <int NT, int MINB, typename OutT>
__global__ void __launch_bounds__(NT, MINB) rf_synth_quad_kernel(const RfParams p, const float *__restrict__ pos,
                                                              const float *__restrict__ amp,
                                                              const float *__restrict__ rf_base,
                                                              OutT *__restrict__ rf)
{
    extern __shared__ int tile[];  // [angles in group][4][Ns]
    __shared__ __align__(16) QuadShared sh;
    rf_quad_tile<NT, OutT>(p, blockIdx.x, blockIdx.y, blockIdx.z, pos, amp, rf_base, rf, tile, sh);
}

size_t quad_smem(const RfParams &p)
{
    // the records (4 x Ns per angle) and, before them, the pass-1 bins (2 x (Ns + 2 win))
    return (size_t)p.ag * sizeof(int) * std::max<size_t>(4 * (size_t)p.pr.ns, 2 * (size_t)(p.pr.ns + 2 * p.win));
}

template <typename OutT>
fq_status launch_rf_quad(const RfParams &p, int F, const float *pos, const float *amp, const float *base, OutT *rf,
                         cudaStream_t st)
{
    const size_t smem = quad_smem(p);
    const int ctas = quad_ctas_per_sm(smem);  // x (1024 / ctas) threads = 32 warps per SM
    auto kern = ctas == 4 ? rf_synth_quad_kernel<256, 4, OutT>
                          : (ctas == 2 ? rf_synth_quad_kernel<512, 2, OutT> : rf_synth_quad_kernel<1024, 1, OutT>);
    fq_status s = fqi::cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                  "fq_simulate_rf: smem attribute");
    if (s) return s;
    dim3 grid((p.pr.M + 3) / 4, p.n_ag, F);
    kern<<<grid, 1024 / ctas, smem, st>>>(p, pos, amp, base, rf);
    return fqi::launch_check("fq_simulate_rf");
}

template <int NT, int MINB, typename OutT>
__global__ void __launch_bounds__(NT, MINB) rf_quad_batched_kernel(const fqb::EnsDev *__restrict__ ens,
                                                                const fqb::StageQueue q)
{
    extern __shared__ int tile[];
    __shared__ __align__(16) QuadShared sh;
    __shared__ __align__(16) unsigned char s_par[kRfParamBytes];
    __shared__ int s_buf[2];
    int cur = -1;
    fqb::Item it;
    while (fqb::next_item(q, ens, fqb::ST_RF, s_buf, it)) {
        const fqb::EnsDev &e = ens[it.e];
        if (it.e != cur) {
            fqb::copy_block(s_par, e.rf_params, kRfParamBytes);
            cur = it.e;
            __syncthreads();
        }
        rf_quad_tile<NT, OutT>(*reinterpret_cast<const RfParams *>(s_par), it.x, it.y, it.z, e.pos, e.amp_eff,
                               nullptr, (OutT *)e.rf, tile, sh);
    }
}

template <typename OutT>
fq_status launch_rf_pair(const RfParams &p, int F, const float *pos, const float *amp, const float *base, OutT *rf,
                         cudaStream_t st)
{
    constexpr int NT = 256;
    size_t smem = 4 * sizeof(int) * (size_t)p.pr.ns;
    static int minb = -1;
    if (minb < 0) {
        const char *env = std::getenv("FQ_RF_MINB");
        minb = (env && env[0] == '2') ? 2 : 3;
    }
    auto kern = minb == 3 ? rf_synth_pair_kernel<NT, 3, OutT> : rf_synth_pair_kernel<NT, 2, OutT>;
    fq_status s = fqi::cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                  "fq_simulate_rf: smem attribute");
    if (s) return s;
    dim3 grid((p.pr.M + 1) / 2, p.A, F);
    kern<<<grid, NT, smem, st>>>(p, pos, amp, base, rf);
    return fqi::launch_check("fq_simulate_rf");
}

template <int E, typename OutT>
fq_status launch_rf(const RfParams &p, int F, const float *pos, const float *amp, const float *base,
                    OutT *rf, cudaStream_t st)
{
    constexpr int NT = 256;
    size_t smem = 2 * sizeof(int) * (size_t)E * p.pr.ns;
    auto kern = rf_synth_kernel<E, NT, OutT>;
    fq_status s = fqi::cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                                  "fq_simulate_rf: smem attribute");
    if (s) return s;
    dim3 grid((p.pr.M + E - 1) / E, p.A, F);
    kern<<<grid, NT, smem, st>>>(p, pos, amp, base, rf);
    return fqi::launch_check("fq_simulate_rf");
}

// Elements per CTA (2); FQ_RF_ELEMS (2, 4, 8 or 16) overrides it for tuning.
int rf_elems(int ns)
{
    static int forced = -1;
    if (forced < 0) {
        const char *env = std::getenv("FQ_RF_ELEMS");
        int v = env ? std::atoi(env) : 0;
        forced = (v == 2 || v == 4 || v == 8 || v == 16) ? v : 0;
    }
    const size_t line = 2 * sizeof(int) * (size_t)ns;  // hi and lo accumulators
    if (forced && forced * line <= 200 * 1024) return forced;
    // 2 elements (32 KB at Ns = 2048) keep 4 CTAs per SM resident, which
    // hides the latency of the accumulation better than more reuse of the
    // per-scatterer work (measured on the 2D compounded workload: 115 ms
    // for 2 elements, 121 ms for 4)
    return 2;
}

// The paired and quad kernels serve the common pulse (two cycles,
// 8 <= n_cycles fs / f0 < 9, so every echo has 8 or 9 taps and the Hann
// phase per sample is below pi / 4) with element widths of at most
// 5 / pi wavelengths (directivity argument |u| <= 5 for the fitted sinc).
bool rf_fast_ok(const RfParams &p)
{
    return p.two_cycle && p.ntap_max == 9 && p.kbx <= fqpoly::kSincUMax && p.kby <= fqpoly::kSincUMax &&
           p.pr.ns >= 9;
}

// the quad kernel's records fit in shared memory and its rounding slack
// (half a quantum per scatterer) stays far below the int32 range
bool quad_ok(const RfParams &p) { return quad_smem(p) <= kQuadSmemMax && p.S < (int64_t(1) << 30); }

template <typename OutT>
fq_status dispatch_rf(const RfParams &p, int F, const float *pos, const float *amp, const float *base,
                      OutT *rf, cudaStream_t st)
{
    static int scalar_only = -1;
    if (scalar_only < 0) {
        const char *env = std::getenv("FQ_RF_SCALAR");
        scalar_only = env && env[0] == '1';
    }
    // the common pulse (two cycles, 8 <= n_cycles fs / f0 < 9, so every echo
    // has 8 or 9 taps) runs on the quad kernel when the array rows hold
    // whole quads, else on the packed-pair kernel
    if (!scalar_only && fqi::use_rf_quad(p.pr.nx) && rf_fast_ok(p) && quad_ok(p))
        return launch_rf_quad(p, F, pos, amp, base, rf, st);
    if (!scalar_only && rf_fast_ok(p) && 4 * sizeof(int) * (size_t)p.pr.ns <= 200 * 1024)
        return launch_rf_pair(p, F, pos, amp, base, rf, st);
    switch (rf_elems(p.pr.ns)) {
    case 16: return launch_rf<16>(p, F, pos, amp, base, rf, st);
    case 8: return launch_rf<8>(p, F, pos, amp, base, rf, st);
    case 4: return launch_rf<4>(p, F, pos, amp, base, rf, st);
    default: return launch_rf<2>(p, F, pos, amp, base, rf, st);
    }
}

// The quad kernel's pulse taps come from a binary32 Chebyshev recurrence
// started at the first tap; its rounded constants (the recurrence factor
// 2 cos w, the table entries e^{i w j}) give every echo the same small error
// pattern, whose sum over the taps (the echo's DC content) does not average
// out: ~-2.3e-7 of the echo amplitude for the two-cycle pulse at ~4 samples
// per carrier period.  rf2iq passes DC to baseband at -f0 with about half
// gain, and delay-and-sum adds that component coherently over every
// (transmit, element) term of a voxel while the echoes themselves add with
// random phases, so it grew to ~1.2e-5 of the beamformed image of the 3D
// workload.  This host routine runs the same binary32 operations lane by
// lane (the kernel's f32x2 instructions round each lane like these scalar
// ones) over 4096 fractional delays spread uniformly over [0, 1), against
// the pulse evaluated in double, and returns the mean error per unit
// amplitude; the kernel subtracts it at one tap of every echo (FP32
// outputs).
float pulse_dc_bias(const RfParams &p, double f0, double fs, int n_cycles)
{
    using namespace fqpoly;
    const double hw = n_cycles * fs / (2.0 * f0);
    const double wh = 2.0 * M_PI * f0 / (n_cycles * fs), wc = 2.0 * M_PI * f0 / fs;
    const int N = 4096;
    double err = 0.0;
    for (int i = 0; i < N; ++i) {
        const float fr = ((float)i + 0.5f) / (float)N;
        const bool lo = fr <= p.theta;
        const int jlo = p.jmin + (lo ? 0 : 1);
        const bool nine = lo || fr >= p.theta2;
        const float x = p.w_h * fr;
        const float t = x * x;
        float ps = std::fmaf(kSinPoly3, t, kSinPoly2);
        ps = std::fmaf(ps, t, kSinPoly1);
        ps = std::fmaf(ps, t, kSinPoly0);
        const float sf = x * ps;
        float pc = std::fmaf(kCosPoly4, t, kCosPoly3);
        pc = std::fmaf(pc, t, kCosPoly2);
        pc = std::fmaf(pc, t, kCosPoly1);
        const float cf = std::fmaf(pc, t, kCosPoly0);
        const float tc = lo ? p.tab_h[0][0] : p.tab_h[1][0], ts = lo ? p.tab_h[0][1] : p.tab_h[1][1];
        const float ntc = -tc;
        const float sfts = sf * ts, ntcsf = ntc * sf;
        const float ch = std::fmaf(cf, tc, sfts);
        const float sh = std::fmaf(ts, cf, ntcsf);
        const float shns = sh * -p.sin_h, shs = sh * p.sin_h;
        float c0 = ch, c1 = std::fmaf(ch, p.cos_h, shns);
        float n0 = -ch, n1 = std::fmaf(ch, -p.cos_h, shs);
        const float nhA = -0.5f;
        for (int j = 0; j < (nine ? 9 : 8); ++j) {
            const float tap = std::fmaf(std::fmaf(std::fmaf(1.0f, c0, 1.0f), c0, nhA), c0, nhA);
            const double tt = (double)(jlo + j) - (double)fr;
            const double ex = std::fabs(tt) < hw ? 0.5 * (1.0 + std::cos(wh * tt)) * std::cos(wc * tt) : 0.0;
            err += (double)tap - ex;
            const float c2 = std::fmaf(p.two_cos_h, c1, n0);
            const float n2 = std::fmaf(-p.two_cos_h, c1, c0);
            c0 = c1;
            c1 = c2;
            n0 = n1;
            n1 = n2;
        }
    }
    return (float)(err / N);
}

fq_status make_rf_params(const fq_probe *probe, const fq_tx *tx, int64_t S, RfParams &p)
{
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
    p.ntap_max = (int)std::floor(2.0 * hw) + 1;
    FQ_REQUIRE(p.ntap_max <= kMaxTaps, FQ_ERR_SHAPE,
               "fq_simulate_rf: n_cycles * fs / f0 must be below %d samples", kMaxTaps - 1);
    const double wc = 2.0 * M_PI * probe->f0 / probe->fs;
    const double wh = wc / probe->n_cycles;
    p.w_c = (float)wc;
    p.w_h = (float)wh;
    p.jmin = (int)std::ceil(0.0 - hw);  // frac in [0, 1): jlo in {jmin, jmin + 1}
    p.jmin_f = (float)p.jmin;
    p.theta = (float)(p.jmin + hw);
    p.theta2 = (float)(std::floor(hw) + 1.0 - hw);
    p.att_l2 = (float)(-(double)p.att / std::log(2.0));
    for (int q = 0; q < 2; ++q) {
        double j = p.jmin + q;
        p.tab_h[q][0] = (float)std::cos(wh * j);
        p.tab_h[q][1] = (float)std::sin(wh * j);
        p.tab_c[q][0] = (float)std::cos(wc * j);
        p.tab_c[q][1] = (float)std::sin(wc * j);
    }
    p.cos_h = (float)std::cos(wh);
    p.sin_h = (float)std::sin(wh);
    p.cos_c = (float)std::cos(wc);
    p.sin_c = (float)std::sin(wc);
    p.two_cos_h = (float)(2.0 * std::cos(wh));
    p.two_cos_c = (float)(2.0 * std::cos(wc));
    p.two_cycle = probe->n_cycles == 2;
    fqi::make_angles_ff(probe, tx, p.ang);
    // quad kernel: angle groups as large as the shared memory allows, balanced
    // (FQ_RF_AG_KB, at least 16, lowers the budget in KB for tuning)
    const size_t per_angle = 4 * sizeof(int) * (size_t)probe->n_samples;
    size_t budget = kQuadSmemMax;
    if (const char *env = std::getenv("FQ_RF_AG_KB")) {
        const long kb = std::atol(env);
        if (kb >= 16 && (size_t)kb * 1024 <= kQuadSmemMax) budget = (size_t)kb * 1024;
    }
    int ag = (int)std::max<size_t>(1, budget / per_angle);
    ag = std::min(ag, p.A);
    p.n_ag = (p.A + ag - 1) / ag;
    p.ag = (p.A + p.n_ag - 1) / p.n_ag;
    // taps t of an echo at delay u have |t - u| <= half_w; the pass-1 sample
    // kp (u in binary32, rounded to nearest) is within 0.51 of u
    const double pitch_k = probe->pitch_x * probe->fs / probe->c;  // adjacent elements' delay difference bound
    p.win = (int)std::floor(hw + 0.5 * pitch_k + 0.52);
    {
        const double t = (double)p.kbx * p.kbx;
        p.dbx_far = (float)((1.0 - t / 6.0 + t * t / 120.0) * (1.0 + 1e-6));
    }
    p.bound_margin = (float)(std::exp((double)p.att * (hw + 1.0) / (probe->fs / probe->c)) * (1.0 + 1.0 / 128.0));
    p.n_sg = 1;
    p.dc_corr = p.two_cycle ? -pulse_dc_bias(p, probe->f0, probe->fs, probe->n_cycles) : 0.0f;
    return FQ_OK;
}

// Scatterer groups of the quad kernel for an output type.  A record's
// relative rounding error grows about linearly with the scatterers that
// share its quanta (the quantum follows the sum of |taps| in a window, the
// echo its square root), and with the number of them whose echoes overlap a
// sample: a matrix probe over a volume puts far more scatterers into each
// delay shell than a linear probe over a plane (measured: 1.9e-6 for 20k
// and 4e-5 for 500k scatterers in the 3D workload's 15 mm cube, 8.7e-7 for
// 100k in the 2D one).  FP32 records therefore take groups of at most 65536
// scatterers for matrix probes and 262144 for linear ones (each group adds
// a pass of bounds and a read-modify-write of the records, measured ~0.4%
// per group on the 3D workload); 16-bit outputs keep one group (their
// storage rounding is far coarser).
void set_scatter_groups(RfParams &p, int out_dtype)
{
    // FQ_RF_SCAT_GROUP (tuning, read once): the group size, 0 = one group
    static const int64_t forced = [] {
        const char *env = std::getenv("FQ_RF_SCAT_GROUP");
        return env ? std::max<int64_t>(0, std::atoll(env)) : (int64_t)-1;
    }();
    int64_t g = p.pr.ny > 1 ? 65536 : 262144;
    if (forced >= 0) g = forced ? forced : INT64_MAX;
    p.n_sg = (out_dtype == FQ_F32 && p.S > g) ? (int)((p.S + g - 1) / g) : 1;
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
    FQ_REQUIRE(out_dtype == FQ_F32 || out_dtype == FQ_BF16 || out_dtype == FQ_F16, FQ_ERR_UNSUPPORTED,
               "fq_simulate_rf: out_dtype must be FQ_F32, FQ_BF16 or FQ_F16");
    FQ_REQUIRE(fqi::aligned(rf, 4), FQ_ERR_ALIGN, "fq_simulate_rf: rf must be 4-byte aligned");

    RfParams p;
    fq_status bs = make_rf_params(probe, tx, S, p);
    if (bs) return bs;
    set_scatter_groups(p, out_dtype);
    cudaStream_t st = (cudaStream_t)stream;
    return fqi::with_storage(out_dtype, "fq_simulate_rf", [&](auto *out) {
        return dispatch_rf(p, n_frames, pos, amp, rf_base, (fqi::storage_t<decltype(out)> *)rf, st);
    });
}

namespace fqi {

size_t rf_params_bytes() { return kRfParamBytes; }

fq_status build_rf_params(const fq_probe *probe, const fq_tx *tx, int64_t S, int out_dtype, void *out)
{
    std::memset(out, 0, kRfParamBytes);
    RfParams &p = *reinterpret_cast<RfParams *>(out);
    fq_status s = make_rf_params(probe, tx, S, p);
    if (s) return s;
    set_scatter_groups(p, out_dtype);
    return FQ_OK;
}

// The quad kernel serves probes whose rows hold whole quads (unless
// FQ_RF_QUAD=0); the single-ensemble and batched paths choose alike.
bool use_rf_quad(int nx)
{
    static int off = -1;
    if (off < 0) {
        const char *env = std::getenv("FQ_RF_QUAD");
        off = env && env[0] == '0';
    }
    return !off && nx % 4 == 0;
}

int rf_ntap_ok(const void *rf_params)
{
    return rf_fast_ok(*reinterpret_cast<const RfParams *>(rf_params));
}

void rf_quad_layout(const void *rf_params, int *n_groups, int *group, size_t *smem)
{
    const RfParams &p = *reinterpret_cast<const RfParams *>(rf_params);
    *n_groups = p.n_ag;
    *group = p.ag;
    *smem = quad_smem(p);
}

bool rf_quad_ok(const void *rf_params) { return quad_ok(*reinterpret_cast<const RfParams *>(rf_params)); }

template <int NT, int MINB, bool QUAD, typename OutT>
fq_status launch_rf_batched(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, size_t smem, cudaStream_t st)
{
    void (*kern)(const fqb::EnsDev *, const fqb::StageQueue);
    if constexpr (QUAD)
        kern = rf_quad_batched_kernel<NT, MINB, OutT>;
    else
        kern = rf_pair_batched_kernel<NT, MINB, OutT>;
    fq_status s = cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "batched RF: smem attribute");
    if (s) return s;
    const int grid = fqb::persistent_grid(kern, NT, smem, items);
    kern<<<grid, NT, smem, st>>>(ens, q);
    return launch_check("batched RF");
}

// quad: `tune` = resident warps per SM (32 or 16), split over the CTAs that
// fit by shared memory; pair: `tune` = resident CTAs of 256 threads (2 or 3)
template <typename OutT>
fq_status batched_rf_t(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, size_t smem, int tune, bool quad,
                       cudaStream_t st)
{
    if (quad) {
        const int ctas = quad_ctas_per_sm(smem);
        if (tune == 16) {
            if (ctas == 4) return launch_rf_batched<128, 4, true, OutT>(ens, q, items, smem, st);
            if (ctas == 2) return launch_rf_batched<256, 2, true, OutT>(ens, q, items, smem, st);
            return launch_rf_batched<512, 1, true, OutT>(ens, q, items, smem, st);
        }
        if (ctas == 4) return launch_rf_batched<256, 4, true, OutT>(ens, q, items, smem, st);
        if (ctas == 2) return launch_rf_batched<512, 2, true, OutT>(ens, q, items, smem, st);
        return launch_rf_batched<1024, 1, true, OutT>(ens, q, items, smem, st);
    }
    return tune == 2 ? launch_rf_batched<256, 2, false, OutT>(ens, q, items, smem, st)
                     : launch_rf_batched<256, 3, false, OutT>(ens, q, items, smem, st);
}

fq_status batched_rf(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int rf_dtype, size_t smem, int minb,
                     bool quad, cudaStream_t st)
{
    if (rf_dtype == FQ_F32) return batched_rf_t<float>(ens, q, items, smem, minb, quad, st);
    return batched_rf_t<__nv_bfloat16>(ens, q, items, smem, minb, quad, st);
}

}  // namespace fqi
