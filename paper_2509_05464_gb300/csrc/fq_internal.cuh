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
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

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

// u . r - o for a float-float direction u, binary32 coordinates r and a
// float-float offset o: the three products and two sums of the leading
// words are error-free (TwoProduct, TwoSum); every error term and the
// low-word products are summed in binary32 and renormalised once.
__device__ __forceinline__ ff ff_dot3_minus(df2 ux, df2 uy, df2 uz, df2 o, float x, float y, float z)
{
    ff px = ff_two_prod(ux.hi, x);
    ff pz = ff_two_prod(uz.hi, z);
    ff s = ff_two_sum(px.hi, pz.hi);
    float lo = __fadd_rn(__fadd_rn(px.lo, pz.lo), s.lo);
    if (y != 0.0f) {
        ff py = ff_two_prod(uy.hi, y);
        ff t = ff_two_sum(s.hi, py.hi);
        s.hi = t.hi;
        lo = __fadd_rn(lo, __fadd_rn(py.lo, t.lo));
        lo = __fmaf_rn(uy.lo, y, lo);
    }
    ff t2 = ff_two_sum(s.hi, -o.hi);
    lo = __fadd_rn(lo, t2.lo);
    lo = __fmaf_rn(ux.lo, x, lo);
    lo = __fmaf_rn(uz.lo, z, lo);
    lo = __fsub_rn(lo, o.lo);
    return ff_fast_two_sum(t2.hi, lo);
}

// ------------------------------------------------------ packed FP32 x 2 --
// Blackwell executes add / sub / mul / fma on a pair of binary32 values held
// in one 64-bit register (f32x2) as a single instruction.  On GB300 it does
// not raise the FP32 rate (a throughput probe, fq_alu_probe, measured 79.3
// TFLOP/s packed against 76.9 scalar: a packed instruction holds the FMA
// pipe for two cycles) but it halves the issue slots of paired arithmetic,
// which is what the issue-bound kernels here are short of.  Both lanes round
// to nearest exactly like the scalar _rn forms, so the float-float
// error-free transforms carry over unchanged.
struct f2 { unsigned long long v; };

__device__ __forceinline__ f2 f2_make(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f2 f2_dup(float a) { return f2_make(a, a); }
__device__ __forceinline__ void f2_split(f2 x, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ float f2_lo(f2 x) { float a, b; f2_split(x, a, b); return a; }
__device__ __forceinline__ float f2_hi(f2 x) { float a, b; f2_split(x, a, b); return b; }
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}
__device__ __forceinline__ f2 f2_neg(f2 a) { return f2{a.v ^ 0x8000000080000000ull}; }

// -------------------------------------------------------------- storage --
__device__ __forceinline__ float load_f(const float *p, int64_t i) { return p[i]; }
// two consecutive values starting at an even index
__device__ __forceinline__ float2 load_f2(const float *p, int64_t i) { return *reinterpret_cast<const float2 *>(p + i); }
__device__ __forceinline__ float2 load_f2(const __nv_bfloat16 *p, int64_t i)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p + i));
}
__device__ __forceinline__ float load_f(const __nv_bfloat16 *p, int64_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ void store_f(float *p, int64_t i, float v) { p[i] = v; }
__device__ __forceinline__ void store_f(__nv_bfloat16 *p, int64_t i, float v) { p[i] = __float2bfloat16_rn(v); }
// binary16 storage: values beyond its largest finite magnitude (65504) are
// stored as +-65504 instead of overflowing to infinity
__device__ __forceinline__ float clamp_f16(float v) { return fminf(fmaxf(v, -65504.0f), 65504.0f); }
__device__ __forceinline__ float load_f(const __half *p, int64_t i) { return __half2float(p[i]); }
__device__ __forceinline__ float2 load_f2(const __half *p, int64_t i)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(p + i));
}
__device__ __forceinline__ void store_f(__half *p, int64_t i, float v) { p[i] = __float2half_rn(clamp_f16(v)); }

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
__device__ __forceinline__ float2 load_c(const __half *p, int64_t c)
{
    return __half22float2(reinterpret_cast<const __half2 *>(p)[c]);
}
__device__ __forceinline__ void store_c(__half *p, int64_t c, float2 v)
{
    reinterpret_cast<__half2 *>(p)[c] = __floats2half2_rn(clamp_f16(v.x), clamp_f16(v.y));
}

// Calls fn(T *) with a null pointer of the storage type of `dtype` (float,
// __nv_bfloat16 or __half) and returns its status; any other dtype is
// FQ_ERR_UNSUPPORTED with a message naming `who`.
template <typename Fn>
inline fq_status with_storage(int dtype, const char *who, Fn &&fn)
{
    switch (dtype) {
    case FQ_F32: return fn(static_cast<float *>(nullptr));
    case FQ_BF16: return fn(static_cast<__nv_bfloat16 *>(nullptr));
    case FQ_F16: return fn(static_cast<__half *>(nullptr));
    default: return set_error(FQ_ERR_UNSUPPORTED, "%s: dtype %d is not FQ_F32, FQ_BF16 or FQ_F16", who, dtype);
    }
}
template <typename P>
using storage_t = std::remove_pointer_t<P>;

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

// the driver's cuTensorMapEncodeTiled through the runtime's entry-point query
// (nullptr if unavailable); declared with the driver types by its users
void *tensor_map_encoder_ptr();

// tensor-core Casorati Gram (gram_tc.cu); esz = operand bytes (2 BF16, 4 TF32)
size_t gram_tc_workspace_bytes(int64_t P, int F, int esz);
fq_status gram_tc(const void *S, int dtype, int64_t P, int F, int esz, float2 *G, char *ws, int *status,
                  cudaStream_t st);

// element centre as float-float
__device__ __forceinline__ ff elem_coord(int i, int n, df2 pitch)
{
    float k = (float)i - 0.5f * (float)(n - 1);  // exact half-integer
    return ff_mul_f(ff_load(pitch), k);
}

}  // namespace fqi
