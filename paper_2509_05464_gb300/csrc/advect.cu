// advect.cu -- a1 scatterer advection, a2 vessel membership and depth
// binning.
//
// These steps are O(S) per frame (not per scatterer-element pair), so they
// run in IEEE double: the wrap of a scatterer along its vessel and the
// membership / bin decisions are integer-valued, and evaluating them with
// the same double operations in the same order as a plain CPU statement
// makes them bit-identical.  This file is compiled with --fmad=false so that
// no multiply-add is contracted.
#include <cmath>
#include <cstring>

#include "batch.cuh"
#include "fq_internal.cuh"

namespace {

constexpr int kSegDoubles = 20;  // kind, p0[3], a1[3], a2[3], a3[3], length, radius, vmax, arc_radius, phi1, arc_end[2]

struct SegTable {
    int n;
    double t[FQ_MAX_SEGMENTS][kSegDoubles];
};

struct MotionParams {
    int n_terms;
    double amp[4], freq[4], phase[4], dir[4][3];
    double g[3], ce[3], vel[3], omega[3], cr[3];
};

void pack_segments(const fq_flow *flow, SegTable &st)
{
    std::memset(&st, 0, sizeof st);
    st.n = flow ? flow->n_seg : 0;
    for (int i = 0; i < st.n; ++i) {
        const fq_segment &s = flow->seg[i];
        double *t = st.t[i];
        t[0] = (double)s.kind;
        for (int d = 0; d < 3; ++d) {
            t[1 + d] = s.p0[d];
            t[4 + d] = s.a1[d];
            t[7 + d] = s.a2[d];
            t[10 + d] = s.a3[d];
        }
        t[13] = s.length;
        t[14] = s.radius;
        t[15] = s.vmax;
        t[16] = s.arc_radius;
        t[17] = s.phi1;
        t[18] = s.arc_end[0];
        t[19] = s.arc_end[1];
    }
}

__device__ __forceinline__ double wrap_into(double a, double span)
{
    return a - span * floor(a / span);
}

// Frame-constant part of the motion map, evaluated once per block.
struct FrameConst {
    double t, ct, st, kx, ky, kz, wn;
    double dsum[3];
    bool rigid;  // no elastic gain and no drift: out = P + dsum (1 + 0 and + 0 are exact)
};

__device__ void frame_constants(const MotionParams &mp, double t, FrameConst &fc)
{
    fc.t = t;
    const double *om = mp.omega;
    double wn = sqrt(om[0] * om[0] + om[1] * om[1] + om[2] * om[2]);
    fc.wn = wn;
    fc.kx = fc.ky = fc.kz = 0.0;
    fc.ct = 1.0;
    fc.st = 0.0;
    if (wn > 0.0) {
        fc.kx = om[0] / wn;
        fc.ky = om[1] / wn;
        fc.kz = om[2] / wn;
        fc.ct = cos(wn * t);
        fc.st = sin(wn * t);
    }
    fc.rigid = mp.g[0] == 0.0 && mp.g[1] == 0.0 && mp.g[2] == 0.0 && mp.vel[0] == 0.0 && mp.vel[1] == 0.0 &&
               mp.vel[2] == 0.0;
    fc.dsum[0] = fc.dsum[1] = fc.dsum[2] = 0.0;
    for (int j = 0; j < mp.n_terms; ++j) {
        double sj = mp.amp[j] * sin(2.0 * 3.14159265358979323846 * mp.freq[j] * t + mp.phase[j]);
        for (int d = 0; d < 3; ++d) fc.dsum[d] += sj * mp.dir[j][d];
    }
}

// Position of scatterer s at the frame time of fc (written to o[d * S + s]).
__device__ __forceinline__ void advect_point(const float *__restrict__ p0, const int32_t *__restrict__ seg,
                                             const float *__restrict__ flow, int64_t S, int64_t s,
                                             const SegTable &st, const MotionParams &mp, const FrameConst &fc,
                                             float *__restrict__ o)
{
    const double t = fc.t;
    double P[3];
    int si = seg[s];
    if (si < 0 || si >= st.n) {
        P[0] = p0[s];
        P[1] = p0[S + s];
        P[2] = p0[2 * S + s];
    } else {
        const double *sg = st.t[si];
        double q = flow[s], x1 = flow[S + s], x2 = flow[2 * S + s];
        double R = sg[14];
        double v = sg[15] * (1.0 - (x1 * x1 + x2 * x2) / (R * R));
        if ((int)sg[0] == FQ_SEG_LINE) {
            double a = wrap_into(q + v * t, sg[13]);
            for (int d = 0; d < 3; ++d)
                P[d] = sg[1 + d] + a * sg[4 + d] + x1 * sg[7 + d] + x2 * sg[10 + d];
        } else {
            double phi = wrap_into(q + v * t / sg[16], sg[17]);
            double cp, sp;
            sincos(phi, &sp, &cp);
            const double rr = sg[16] + x1;
            for (int d = 0; d < 3; ++d)
                P[d] = sg[1 + d] + rr * (cp * sg[4 + d] + sp * sg[7 + d]) + x2 * sg[10 + d];
        }
    }
    double Q0 = P[0], Q1 = P[1], Q2 = P[2];
    if (fc.wn > 0.0) {
        const double *cr = mp.cr;
        double w0 = P[0] - cr[0], w1 = P[1] - cr[1], w2 = P[2] - cr[2];
        double kw = fc.kx * w0 + fc.ky * w1 + fc.kz * w2;
        double c0 = fc.ky * w2 - fc.kz * w1, c1 = fc.kz * w0 - fc.kx * w2, c2 = fc.kx * w1 - fc.ky * w0;
        double omc = 1.0 - fc.ct;
        P[0] = cr[0] + w0 * fc.ct + c0 * fc.st + fc.kx * kw * omc;
        P[1] = cr[1] + w1 * fc.ct + c1 * fc.st + fc.ky * kw * omc;
        P[2] = cr[2] + w2 * fc.ct + c2 * fc.st + fc.kz * kw * omc;
    }
    if (fc.rigid) {
        // the general form below with gain 1 + 0 = 1 and drift 0 t = 0, whose
        // operations are exact: the same doubles
        for (int d = 0; d < 3; ++d) o[d * S + s] = (float)(P[d] + fc.dsum[d]);
        return;
    }
    double gain = 1.0 + (mp.g[0] * (Q0 - mp.ce[0]) + mp.g[1] * (Q1 - mp.ce[1]) + mp.g[2] * (Q2 - mp.ce[2]));
    for (int d = 0; d < 3; ++d) o[d * S + s] = (float)(P[d] + mp.vel[d] * t + gain * fc.dsum[d]);
}

__global__ void advect_kernel(const float *__restrict__ p0, const int32_t *__restrict__ seg,
                              const float *__restrict__ flow, int64_t S, const SegTable st,
                              const MotionParams mp, double t0, double dt,
                              float *__restrict__ out)
{
    __shared__ FrameConst fc;
    const int f = blockIdx.y;
    if (threadIdx.x == 0) frame_constants(mp, t0 + (double)f * dt, fc);
    __syncthreads();
    float *o = out + (int64_t)f * 3 * S;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x)
        advect_point(p0, seg, flow, S, s, st, mp, fc, o);
}

// ------------------------------------------------------------ membership --
__device__ __forceinline__ bool inside_seg(const double *sg, double px, double py, double pz)
{
    double w0 = px - sg[1], w1 = py - sg[2], w2 = pz - sg[3];
    double R2 = sg[14] * sg[14];
    if ((int)sg[0] == FQ_SEG_LINE) {
        double s = (w0 * sg[4] + w1 * sg[5]) + w2 * sg[6];
        if (s < 0.0 || s > sg[13]) return false;
        double q1 = (w0 * sg[7] + w1 * sg[8]) + w2 * sg[9];
        double q2 = (w0 * sg[10] + w1 * sg[11]) + w2 * sg[12];
        return (q1 * q1 + q2 * q2) < R2;
    }
    double x1 = (w0 * sg[4] + w1 * sg[5]) + w2 * sg[6];
    double x2 = (w0 * sg[7] + w1 * sg[8]) + w2 * sg[9];
    double x3 = (w0 * sg[10] + w1 * sg[11]) + w2 * sg[12];
    if (x2 < 0.0) return false;                        // before the arc start (angle 0)
    if (x1 * sg[19] - x2 * sg[18] < 0.0) return false;  // past the arc end (angle phi1 <= pi)
    double rin = sqrt(x1 * x1 + x2 * x2) - sg[16];
    return (rin * rin + x3 * x3) < R2;
}

__device__ __forceinline__ void classify_point(const float *__restrict__ pos, const int32_t *__restrict__ seg,
                                               int64_t S, int64_t s, const SegTable &st,
                                               const float *__restrict__ amp_in, int32_t *__restrict__ vessel,
                                               float *__restrict__ amp_out)
{
    int v = seg[s];
    if (v < 0) {
        double px = pos[s], py = pos[S + s], pz = pos[2 * S + s];
        for (int i = 0; i < st.n; ++i)
            if (inside_seg(st.t[i], px, py, pz)) { v = i; break; }
    }
    vessel[s] = v;
    if (amp_out) amp_out[s] = (seg[s] < 0 && v >= 0) ? 0.0f : amp_in[s];
}

__global__ void classify_kernel(const float *__restrict__ pos, const int32_t *__restrict__ seg,
                                int64_t S, const SegTable st, const float *__restrict__ amp_in,
                                int32_t *__restrict__ vessel, float *__restrict__ amp_out)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
         s += (int64_t)gridDim.x * blockDim.x)
        classify_point(pos, seg, S, s, st, amp_in, vessel, amp_out);
}

// ----------------------------------------------------------- batched --
// Items of fqb::kItemScat scatterers (classify: one item per chunk; advect:
// one per (chunk, frame)).
using fqb::kItemScat;
constexpr int kBatchThreads = 256;

__global__ void __launch_bounds__(kBatchThreads) classify_batched_kernel(const fqb::EnsDev *__restrict__ ens,
                                                                         const fqb::StageQueue q)
{
    __shared__ int s_buf[2];
    fqb::Item it;
    while (fqb::next_item(q, ens, fqb::ST_CLASSIFY, s_buf, it)) {
        const fqb::EnsDev &e = ens[it.e];
        const SegTable &st = *reinterpret_cast<const SegTable *>(e.seg_table);
        const int64_t beg = (int64_t)it.x * kItemScat;
        const int64_t end = beg + kItemScat < e.S ? beg + kItemScat : e.S;
        for (int64_t s = beg + threadIdx.x; s < end; s += blockDim.x)
            classify_point(e.p0, e.seg, e.S, s, st, e.amp, e.vessel, e.amp_eff);
    }
}

__global__ void __launch_bounds__(kBatchThreads) advect_batched_kernel(const fqb::EnsDev *__restrict__ ens,
                                                                       const fqb::StageQueue q)
{
    __shared__ int s_buf[2];
    __shared__ FrameConst fc;
    fqb::Item it;
    while (fqb::next_item(q, ens, fqb::ST_ADVECT, s_buf, it)) {
        const fqb::EnsDev &e = ens[it.e];
        const SegTable &st = *reinterpret_cast<const SegTable *>(e.seg_table);
        const MotionParams &mp = *reinterpret_cast<const MotionParams *>(e.motion);
        const int f = it.y;
        if (threadIdx.x == 0) frame_constants(mp, e.t0 + (double)f * e.dt, fc);
        __syncthreads();
        float *o = e.pos + (int64_t)f * 3 * e.S;
        const int64_t beg = (int64_t)it.x * kItemScat;
        const int64_t end = beg + kItemScat < e.S ? beg + kItemScat : e.S;
        for (int64_t s = beg + threadIdx.x; s < end; s += blockDim.x)
            advect_point(e.p0, e.seg, e.flow, e.S, s, st, mp, fc, o);
    }
}

void pack_motion(const fq_motion *motion, MotionParams &mp)
{
    std::memset(&mp, 0, sizeof mp);
    if (!motion) return;
    mp.n_terms = motion->n_terms;
    for (int j = 0; j < 4; ++j) {
        mp.amp[j] = motion->amp[j];
        mp.freq[j] = motion->freq[j];
        mp.phase[j] = motion->phase[j];
        for (int d = 0; d < 3; ++d) mp.dir[j][d] = motion->dir[j][d];
    }
    for (int d = 0; d < 3; ++d) {
        mp.g[d] = motion->elastic_grad[d];
        mp.ce[d] = motion->elastic_center[d];
        mp.vel[d] = motion->vel[d];
        mp.omega[d] = motion->omega[d];
        mp.cr[d] = motion->rot_center[d];
    }
}

// ---------------------------------------------------------------- binning --
// Stable counting sort in three passes over fixed chunks of kChunk
// scatterers: (1) per-(bin, chunk) counts, (2) one exclusive scan over the
// bin-major count table, which directly gives the first output slot of every
// (bin, chunk), (3) a single warp per chunk walks its scatterers in index
// order and places them, ranking equal keys with warp match masks.
constexpr int kChunk = 4096;
constexpr int kMaxBins = 8192;

__global__ void bin_count_kernel(const float *__restrict__ z, int64_t S, double z0, double dz, int B,
                                 int32_t *__restrict__ key, int32_t *__restrict__ counts, int n_chunks)
{
    extern __shared__ int32_t hist[];
    const int chunk = blockIdx.x;
    for (int b = threadIdx.x; b < B; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    int64_t beg = (int64_t)chunk * kChunk;
    int64_t end = beg + kChunk < S ? beg + kChunk : S;
    for (int64_t s = beg + threadIdx.x; s < end; s += blockDim.x) {
        double q = floor(((double)z[s] - z0) / dz);
        int b = q < 0.0 ? 0 : (q > (double)(B - 1) ? B - 1 : (int)q);
        key[s] = b;
        atomicAdd(&hist[b], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += blockDim.x) counts[(int64_t)b * n_chunks + chunk] = hist[b];
}

// exclusive scan of n ints in place by one CTA of 1024 threads
__global__ void scan_kernel(int32_t *__restrict__ a, int64_t n)
{
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < n; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int32_t v = i < n ? a[i] : 0;
        int32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int32_t t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;  // inclusive prefix of warp totals
        }
        __syncthreads();
        int32_t before = carry + (wid > 0 ? warp_tot[wid - 1] : 0);
        if (i < n) a[i] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
}

__global__ void bin_place_kernel(const int32_t *__restrict__ key, int64_t S, int B,
                                 const int32_t *__restrict__ offsets, int n_chunks,
                                 int32_t *__restrict__ perm, int32_t *__restrict__ bin_off)
{
    extern __shared__ int32_t next[];
    const int chunk = blockIdx.x;
    const int lane = threadIdx.x;  // one warp
    for (int b = lane; b < B; b += 32) next[b] = offsets[(int64_t)b * n_chunks + chunk];
    if (chunk == 0) {
        for (int b = lane; b < B; b += 32) bin_off[b] = offsets[(int64_t)b * n_chunks];
        if (lane == 0) bin_off[B] = (int32_t)S;
    }
    __syncwarp();
    int64_t beg = (int64_t)chunk * kChunk;
    int64_t end = beg + kChunk < S ? beg + kChunk : S;
    const unsigned lt = (1u << lane) - 1u;
    for (int64_t base = beg; base < end; base += 32) {
        int64_t s = base + lane;
        bool valid = s < end;
        unsigned act = __ballot_sync(0xffffffffu, valid);
        int k = valid ? key[s] : -1 - lane;  // invalid lanes get unique dummy keys
        unsigned peers = __match_any_sync(0xffffffffu, k);
        if (valid) {
            int rank = __popc(peers & lt);
            perm[next[k] + rank] = (int32_t)s;
        }
        __syncwarp();
        // the highest lane of each group advances the bin's cursor
        if (valid && (peers >> lane) == 1u) next[k] += __popc(peers);
        __syncwarp();
        (void)act;
    }
}

}  // namespace

extern "C" {

fq_status fq_advect_scatterers(const float *p0, const int32_t *seg_id, const float *flow_coord,
                               int64_t S, const fq_flow *flow, const fq_motion *motion,
                               double t0, double dt, int32_t n_frames, float *pos_out,
                               void *stream)
{
    FQ_REQUIRE(S >= 0 && n_frames >= 1, FQ_ERR_INVALID_ARG, "fq_advect_scatterers: S=%lld n_frames=%d",
               (long long)S, n_frames);
    if (S == 0) return FQ_OK;
    FQ_REQUIRE(p0 && seg_id && flow_coord && pos_out, FQ_ERR_INVALID_ARG,
               "fq_advect_scatterers: null device pointer");
    FQ_REQUIRE(!flow || (flow->n_seg >= 0 && flow->n_seg <= FQ_MAX_SEGMENTS && (flow->n_seg == 0 || flow->seg)),
               FQ_ERR_SHAPE, "fq_advect_scatterers: n_seg must be in [0, %d]", FQ_MAX_SEGMENTS);
    FQ_REQUIRE(!motion || (motion->n_terms >= 0 && motion->n_terms <= FQ_MAX_MOTION_TERMS), FQ_ERR_SHAPE,
               "fq_advect_scatterers: n_terms must be in [0, 4]");
    SegTable local;
    pack_segments(flow, local);
    MotionParams mp;
    pack_motion(motion, mp);
    const int threads = 256;
    int64_t blocks = (S + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    dim3 grid((unsigned)blocks, (unsigned)n_frames);
    advect_kernel<<<grid, threads, 0, (cudaStream_t)stream>>>(p0, seg_id, flow_coord, S, local, mp, t0, dt,
                                                              pos_out);
    return fqi::launch_check("fq_advect_scatterers");
}

fq_status fq_classify_scatterers(const float *pos, const int32_t *seg_id, int64_t S,
                                 const fq_flow *flow, const float *amp_in, int32_t *vessel_out,
                                 float *amp_out, void *stream)
{
    FQ_REQUIRE(S >= 0, FQ_ERR_INVALID_ARG, "fq_classify_scatterers: S < 0");
    if (S == 0) return FQ_OK;
    FQ_REQUIRE(pos && seg_id && vessel_out && (amp_in || !amp_out), FQ_ERR_INVALID_ARG,
               "fq_classify_scatterers: null device pointer");
    FQ_REQUIRE(!flow || (flow->n_seg >= 0 && flow->n_seg <= FQ_MAX_SEGMENTS && (flow->n_seg == 0 || flow->seg)),
               FQ_ERR_SHAPE, "fq_classify_scatterers: n_seg must be in [0, %d]", FQ_MAX_SEGMENTS);
    SegTable local;
    pack_segments(flow, local);
    const int threads = 256;
    int64_t blocks = (S + threads - 1) / threads;
    if (blocks > 8192) blocks = 8192;
    classify_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(pos, seg_id, S, local, amp_in,
                                                                            vessel_out, amp_out);
    return fqi::launch_check("fq_classify_scatterers");
}

fq_status fq_bin_workspace_size(int64_t S, int32_t B, size_t *bytes)
{
    FQ_REQUIRE(bytes && S >= 0 && B >= 1, FQ_ERR_INVALID_ARG, "fq_bin_workspace_size: bad arguments");
    int64_t n_chunks = (S + kChunk - 1) / kChunk;
    if (n_chunks < 1) n_chunks = 1;
    size_t k = ((size_t)S * 4 + 255) & ~(size_t)255;
    size_t c = ((size_t)n_chunks * B * 4 + 255) & ~(size_t)255;
    *bytes = k + c;
    return FQ_OK;
}

fq_status fq_bin_scatterers(const float *z, int64_t S, double z0, double dz, int32_t B,
                            int32_t *bin_off, int32_t *perm, void *workspace,
                            size_t workspace_bytes, void *stream)
{
    FQ_REQUIRE(S >= 0 && S < ((int64_t)1 << 31), FQ_ERR_SHAPE, "fq_bin_scatterers: S out of range");
    FQ_REQUIRE(B >= 1 && B <= kMaxBins, FQ_ERR_SHAPE, "fq_bin_scatterers: B must be in [1, %d]", kMaxBins);
    FQ_REQUIRE(dz > 0.0, FQ_ERR_INVALID_ARG, "fq_bin_scatterers: dz must be > 0");
    FQ_REQUIRE(bin_off && (S == 0 || (z && perm)), FQ_ERR_INVALID_ARG, "fq_bin_scatterers: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    if (S == 0) {
        return fqi::cuda_check(cudaMemsetAsync(bin_off, 0, sizeof(int32_t) * (B + 1), st), "fq_bin_scatterers");
    }
    size_t need = 0;
    fq_bin_workspace_size(S, B, &need);
    FQ_REQUIRE(workspace && workspace_bytes >= need, FQ_ERR_WORKSPACE,
               "fq_bin_scatterers: workspace needs %zu bytes", need);
    FQ_REQUIRE(fqi::aligned(workspace, 256), FQ_ERR_ALIGN, "fq_bin_scatterers: workspace not 256-byte aligned");
    int n_chunks = (int)((S + kChunk - 1) / kChunk);
    int32_t *key = (int32_t *)workspace;
    int32_t *counts = (int32_t *)((char *)workspace + (((size_t)S * 4 + 255) & ~(size_t)255));
    size_t smem = sizeof(int32_t) * B;
    if (smem > 48 * 1024) {
        fq_status s = fqi::cuda_check(cudaFuncSetAttribute(bin_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)smem), "fq_bin_scatterers");
        if (s) return s;
        s = fqi::cuda_check(cudaFuncSetAttribute(bin_place_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem), "fq_bin_scatterers");
        if (s) return s;
    }
    bin_count_kernel<<<n_chunks, 256, smem, st>>>(z, S, z0, dz, B, key, counts, n_chunks);
    scan_kernel<<<1, 1024, 0, st>>>(counts, (int64_t)n_chunks * B);
    bin_place_kernel<<<n_chunks, 32, smem, st>>>(key, S, B, counts, n_chunks, perm, bin_off);
    return fqi::launch_check("fq_bin_scatterers");
}

}  // extern "C"

namespace fqi {

size_t seg_table_bytes() { return (sizeof(SegTable) + 15) & ~(size_t)15; }
size_t motion_bytes() { return (sizeof(MotionParams) + 15) & ~(size_t)15; }
void build_seg_table(const fq_flow *flow, void *out) { pack_segments(flow, *reinterpret_cast<SegTable *>(out)); }
void build_motion(const fq_motion *m, void *out) { pack_motion(m, *reinterpret_cast<MotionParams *>(out)); }

fq_status batched_classify(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, cudaStream_t st)
{
    const int grid = fqb::persistent_grid(classify_batched_kernel, kBatchThreads, 0, items);
    classify_batched_kernel<<<grid, kBatchThreads, 0, st>>>(ens, q);
    return launch_check("batched classify");
}

fq_status batched_advect(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, cudaStream_t st)
{
    const int grid = fqb::persistent_grid(advect_batched_kernel, kBatchThreads, 0, items);
    advect_batched_kernel<<<grid, kBatchThreads, 0, st>>>(ens, q);
    return launch_check("batched advect");
}

}  // namespace fqi
