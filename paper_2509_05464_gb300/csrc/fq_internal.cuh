// fq_internal.cuh -- helpers shared by the CUDA translation units of libfq.
//
// Float-float ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two binary32 numbers, giving ~48 significant bits at FP32-pipe
// speed.  GB300 executes FP64 at a small fraction of its FP32 rate, so the
// time-of-flight delays that need more than 24 bits (the carrier phase
// 2 pi f0 tau at depth spans hundreds of cycles) are evaluated this way.
// The building blocks are the error-free transforms of Knuth (TwoSum) and
// Dekker (Fast2Sum, and TwoProduct through a fused multiply-add); the
// square root takes one Newton correction of the binary32 root.  Explicit
// _rn intrinsics keep the compiler from contracting or reassociating them.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/fq.h"

namespace fqi {

// ---------------------------------------------------------------- errors --
fq_status set_error(fq_status s, const char *fmt, ...);
fq_status cuda_check(cudaError_t e, const char *where);
fq_status launch_check(const char *where);

#define FQ_REQUIRE(cond, status, ...)                          \
    do {                                                       \
        if (!(cond)) return ::fqi::set_error((status), __VA_ARGS__); \
    } while (0)

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// host-side split of a double into a float pair
struct df2 { float hi, lo; };
__host__ __device__ inline df2 split_double(double d)
{
    float hi = (float)d;
    float lo = (float)(d - (double)hi);
    return {hi, lo};
}

// --------------------------------------------------------- float-float --
struct ff { float hi, lo; };

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)  // |a| >= |b|
{
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ ff ff_two_prod(float a, float b)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.hi, b.hi);
    ff t = ff_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = ff_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_add_f(ff a, float b)
{
    ff s = ff_two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = ff_two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return ff_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    ff p = ff_two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return ff_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_sqr(ff a)
{
    ff p = ff_two_prod(a.hi, a.hi);
    p.lo = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, p.lo);
    return ff_fast_two_sum(p.hi, p.lo);
}
// sqrt of a positive float-float: s = sqrt(hi), then one Newton correction
// (a - s^2) / (2 s) evaluated with s^2 exact through a fused multiply-add.
__device__ __forceinline__ ff ff_sqrt(ff a)
{
    float s = __fsqrt_rn(a.hi);
    float r = __fmaf_rn(-s, s, a.hi);          // a.hi - s^2, exact
    r = __fadd_rn(r, a.lo);
    float corr = __fdiv_rn(r, __fmul_rn(2.0f, s));
    return ff_fast_two_sum(s, corr);
}
// x = n + f with integer n = floor(x) and f in [0, 1) as a float
__device__ __forceinline__ void ff_floor_frac(ff x, int &n, float &f)
{
    float fl = floorf(x.hi);
    float rem = __fadd_rn(__fsub_rn(x.hi, fl), x.lo);  // x.hi - fl is exact
    if (rem < 0.0f) { rem = __fadd_rn(rem, 1.0f); fl -= 1.0f; }
    else if (rem >= 1.0f) { rem = __fsub_rn(rem, 1.0f); fl += 1.0f; }
    n = (int)fl;
    f = rem;
}
// fractional part of x in [0, 1) (x up to ~1e6 in magnitude)
__device__ __forceinline__ float ff_frac(ff x)
{
    int n;
    float f;
    ff_floor_frac(x, n, f);
    return f;
}

__device__ __forceinline__ ff ff_load(const df2 &d) { return {d.hi, d.lo}; }

// -------------------------------------------------------------- storage --
__device__ __forceinline__ float load_f(const float *p, int64_t i) { return p[i]; }
__device__ __forceinline__ float load_f(const __nv_bfloat16 *p, int64_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void store_f(float *p, int64_t i, float v) { p[i] = v; }
__device__ __forceinline__ void store_f(__nv_bfloat16 *p, int64_t i, float v) { p[i] = __float2bfloat16_rn(v); }

// complex element c of an interleaved array
__device__ __forceinline__ float2 load_c(const float *p, int64_t c)
{
    return reinterpret_cast<const float2 *>(p)[c];
}
__device__ __forceinline__ float2 load_c(const __nv_bfloat16 *p, int64_t c)
{
    __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162 *>(p)[c];
    return __bfloat1622float2(v);
}
__device__ __forceinline__ void store_c(float *p, int64_t c, float2 v)
{
    reinterpret_cast<float2 *>(p)[c] = v;
}
__device__ __forceinline__ void store_c(__nv_bfloat16 *p, int64_t c, float2 v)
{
    reinterpret_cast<__nv_bfloat162 *>(p)[c] = __float22bfloat162_rn(v);
}

// ---------------------------------------------------------- parameters --
// Per-angle plane-wave constants: direction and time origin, as float-float.
struct AngleFF {
    df2 ux, uy, uz, origin;  // origin = min_m u . e_m (m)
};

struct ProbeFF {
    int nx, ny, M, ns;
    df2 pitch_x, pitch_y;    // element centres: (i - (n-1)/2) * pitch
    df2 fs_over_c;           // samples per metre of path
    df2 f0_over_fs;          // carrier cycles per sample
};

bool make_probe_ff(const fq_probe *p, ProbeFF &o);
void make_angles_ff(const fq_probe *p, const fq_tx *tx, AngleFF *out);

// element centre as float-float
__device__ __forceinline__ ff elem_coord(int i, int n, df2 pitch)
{
    float k = (float)i - 0.5f * (float)(n - 1);  // exact half-integer
    return ff_mul_f(ff_load(pitch), k);
}

}  // namespace fqi
