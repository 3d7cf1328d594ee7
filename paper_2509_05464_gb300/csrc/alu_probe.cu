// alu_probe.cu -- a throughput probe of the FP32 pipes, the denominator of
// the ALU rooflines that the RF and DAS kernels are reported against.  Each
// thread runs `iters` rounds of 8 independent FMA chains, as scalar FFMA or
// as packed f32x2 FMAs (two lanes per instruction), so that issue, not
// latency, bounds it; 2 FLOP per lane and FMA.
#include "fq_internal.cuh"

namespace {

template <bool PACKED>
__global__ void __launch_bounds__(256) alu_probe_kernel(int iters, float seed, float *__restrict__ sink)
{
    const float s = seed + 1e-7f * (float)threadIdx.x;
    if constexpr (PACKED) {
        fqi::f2 a[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fqi::f2_make(s + i, s - i);
        const fqi::f2 m = fqi::f2_dup(0.999999f), c = fqi::f2_dup(1e-6f);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fqi::f2_fma(a[i], m, c);
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float x, y;
            fqi::f2_split(a[i], x, y);
            acc += x + y;
        }
        if (acc == 12345.678f) sink[threadIdx.x] = acc;  // keeps the chains live
    } else {
        float a[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = s + i;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], 0.999999f, 1e-6f);
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) acc += a[i];
        if (acc == 12345.678f) sink[threadIdx.x] = acc;
    }
}

}  // namespace

extern "C" fq_status fq_alu_probe(int32_t packed, int32_t blocks, int32_t iters, float *sink, void *stream)
{
    FQ_REQUIRE(sink && blocks >= 1 && iters >= 1, FQ_ERR_INVALID_ARG, "fq_alu_probe: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (packed)
        alu_probe_kernel<true><<<blocks, 256, 0, st>>>(iters, 1.0f, sink);
    else
        alu_probe_kernel<false><<<blocks, 256, 0, st>>>(iters, 1.0f, sink);
    return fqi::launch_check("fq_alu_probe");
}
