// das_matrix.cu -- the explicit DAS-matrix route of Sec. 2.4.1 / Alg. 3
// (steps 2.2-2.4): one sparse matrix per transmit (rows = pixels, columns =
// (element, sample) of the channel IQ) built once and applied to every
// frame, kept here as the paper's design to measure on GB300 beside the
// fused DAS kernel, which recomputes its delays instead of storing them.
//
// Build: a count pass and a fill pass, one thread per (transmit, pixel) row,
// with the same binary32 aperture decision and float-float delays as the
// fused kernel; an exclusive scan of the counts gives the int64 row
// offsets.  Storage: int32 column m Ns + i and a complex binary32 weight
// ((1 - phi) or phi) e^{i 2 pi f0 tau} per entry, two entries per active
// element.  Apply: one warp per pixel walks the rows of every transmit,
// each lane accumulating up to 13 frames (lane, lane + 32, ...); an entry's
// weight is read once per pixel and its channel row of frames is one
// coalesced load per lane and frame group.
#include <cmath>
#include <cstring>

#include "fq_internal.cuh"

namespace {

using fqi::ff;

constexpr int kThreads = 128;
constexpr int kScanBlock = 1024;
constexpr int kMaxFrameGroups = 13;  // F <= 416

struct MatParams {
    fqi::ProbeFF pr;
    int A, gx, gy, gz;
    int64_t P;
    double x0, y0, z0, dx, dy, dz, pitch_x, pitch_y;
    float half_per_z;
    fqi::AngleFF ang[FQ_MAX_ANGLES];
};

// element centres (exact in double, then binary32 and float-float) in
// shared memory: 6 M floats
__device__ __forceinline__ void element_table(const MatParams &p, float *t)
{
    const int M = p.pr.M;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const int ix = m % p.pr.nx, iy = m / p.pr.nx;
        const double ex = __dmul_rn(__dsub_rn((double)ix, __dmul_rn(0.5, (double)(p.pr.nx - 1))), p.pitch_x);
        const double ey = __dmul_rn(__dsub_rn((double)iy, __dmul_rn(0.5, (double)(p.pr.ny - 1))), p.pitch_y);
        const fqi::df2 sx = fqi::split_double(ex), sy = fqi::split_double(ey);
        t[m] = (float)ex;
        t[M + m] = sx.hi;
        t[2 * M + m] = sx.lo;
        t[3 * M + m] = (float)ey;
        t[4 * M + m] = sy.hi;
        t[5 * M + m] = sy.lo;
    }
    __syncthreads();
}

// Walks one row (transmit a, pixel p): calls emit(m, i, phi, u, f0 / fs) for
// every element in the aperture with a valid sample pair; returns the count.
template <typename Emit>
__device__ __forceinline__ int walk_row(const MatParams &p, const float *t, int a, int64_t pix, Emit emit)
{
    const int M = p.pr.M, ns = p.pr.ns;
    const int ix = (int)(pix % p.gx);
    const int iz = (int)((pix / p.gx) % p.gz);
    const int iy = (int)(pix / ((int64_t)p.gx * p.gz));
    const double xd = __dadd_rn(p.x0, __dmul_rn((double)ix, p.dx));
    const double yd = __dadd_rn(p.y0, __dmul_rn((double)iy, p.dy));
    const double zd = __dadd_rn(p.z0, __dmul_rn((double)iz, p.dz));
    const float xf = (float)xd, yf = (float)yd, zf = (float)zd;
    const fqi::df2 xs = fqi::split_double(xd), ys = fqi::split_double(yd), zs = fqi::split_double(zd);
    const ff X = {xs.hi, xs.lo}, Y = {ys.hi, ys.lo}, Z = {zs.hi, zs.lo};
    const ff zz = fqi::ff_sqr(Z);
    const float half = __fmul_rn(zf, p.half_per_z);
    const bool matrix = p.pr.ny > 1;
    const ff fs_c = fqi::ff_load(p.pr.fs_over_c), f0_fs = fqi::ff_load(p.pr.f0_over_fs);
    const fqi::AngleFF an = p.ang[a];
    ff ptx = fqi::ff_add(fqi::ff_mul(fqi::ff_load(an.ux), X), fqi::ff_mul(fqi::ff_load(an.uy), Y));
    ptx = fqi::ff_add(ptx, fqi::ff_mul(fqi::ff_load(an.uz), Z));
    ptx = fqi::ff_add(ptx, fqi::ff_neg(fqi::ff_load(an.origin)));
    int n = 0;
    for (int m = 0; m < M; ++m) {
        if (fabsf(__fsub_rn(xf, t[m])) > half) continue;
        if (matrix && fabsf(__fsub_rn(yf, t[3 * M + m])) > half) continue;
        const ff dxx = fqi::ff_add(X, ff{-t[M + m], -t[2 * M + m]});
        ff r2 = fqi::ff_add(fqi::ff_sqr(dxx), zz);
        if (matrix || yf != 0.0f) {
            const ff dyy = fqi::ff_add(Y, ff{-t[4 * M + m], -t[5 * M + m]});
            r2 = fqi::ff_add(r2, fqi::ff_sqr(dyy));
        }
        const ff path = fqi::ff_add(ptx, fqi::ff_sqrt(r2));
        const ff u = fqi::ff_mul(path, fs_c);
        int i;
        float phi;
        fqi::ff_floor_frac(u, i, phi);
        if (i < 0 || i + 1 >= ns) continue;
        emit(m, i, phi, u, f0_fs);
        n += 2;
    }
    return n;
}

__global__ void __launch_bounds__(kThreads) count_kernel(const MatParams p, int32_t *cnt)
{
    extern __shared__ float etab[];
    element_table(p, etab);
    const int64_t R = (int64_t)p.A * p.P;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < R;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(row / p.P);
        cnt[row] = walk_row(p, etab, a, row - (int64_t)a * p.P, [](int, int, float, ff, ff) {});
    }
}

__global__ void __launch_bounds__(kThreads) fill_kernel(const MatParams p, const int64_t *__restrict__ row_ptr,
                                                        int32_t *__restrict__ col, float2 *__restrict__ val)
{
    extern __shared__ float etab[];
    element_table(p, etab);
    const int64_t R = (int64_t)p.A * p.P;
    const int ns = p.pr.ns;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < R;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(row / p.P);
        int64_t k = row_ptr[row];
        walk_row(p, etab, a, row - (int64_t)a * p.P, [&](int m, int i, float phi, ff u, ff f0_fs) {
            const float cyc = fqi::ff_frac(fqi::ff_mul(u, f0_fs));
            float sn, cs;
            sincospif(2.0f * cyc, &sn, &cs);
            col[k] = m * ns + i;
            val[k] = make_float2((1.0f - phi) * cs, (1.0f - phi) * sn);
            col[k + 1] = m * ns + i + 1;
            val[k + 1] = make_float2(phi * cs, phi * sn);
            k += 2;
        });
    }
}

// exclusive scan of int32 counts into int64 offsets: block sums, a scan of
// the block sums by one block, then each block's local scan plus its offset
__global__ void __launch_bounds__(kScanBlock) block_sum_kernel(const int32_t *cnt, int64_t n, int64_t *bsum)
{
    __shared__ int64_t red[kScanBlock / 32];
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int64_t v = i < n ? cnt[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int w = 0; w < kScanBlock / 32; ++w) s += red[w];
        bsum[blockIdx.x] = s;
    }
}

__global__ void scan_bsum_kernel(int64_t *bsum, int64_t nb, int64_t *total)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t s = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t v = bsum[b];
        bsum[b] = s;
        s += v;
    }
    *total = s;
}

__global__ void __launch_bounds__(kScanBlock) local_scan_kernel(const int32_t *cnt, int64_t n, const int64_t *boff,
                                                                int64_t *row_ptr)
{
    __shared__ int64_t s[kScanBlock];
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    s[threadIdx.x] = i < n ? cnt[i] : 0;
    __syncthreads();
    for (int off = 1; off < kScanBlock; off <<= 1) {  // Hillis-Steele inclusive scan
        const int64_t v = threadIdx.x >= off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    if (i < n) row_ptr[i + 1] = boff[blockIdx.x] + s[threadIdx.x];
    if (i == 0) row_ptr[0] = 0;
}

// one complex channel value (re, im) as float2
__device__ __forceinline__ float2 load_c2(const float *r, int f) { return __ldg(reinterpret_cast<const float2 *>(r) + f); }
__device__ __forceinline__ float2 load_c2(const __nv_bfloat16 *r, int f)
{
    return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(r) + f));
}

template <typename ChT, typename OutT>
__global__ void __launch_bounds__(kThreads) apply_kernel(const int64_t *__restrict__ row_ptr,
                                                         const int32_t *__restrict__ col,
                                                         const float2 *__restrict__ val, int A, int64_t P,
                                                         const ChT *__restrict__ ch, int64_t ch_angle_rows, int Fp,
                                                         int F, float inv_A, OutT *__restrict__ iq)
{
    const int64_t pix = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (pix >= P) return;
    const int groups = (F + 31) >> 5;
    float2 acc[kMaxFrameGroups];
#pragma unroll
    for (int g = 0; g < kMaxFrameGroups; ++g) acc[g] = make_float2(0.0f, 0.0f);
    for (int a = 0; a < A; ++a) {
        const int64_t row = (int64_t)a * P + pix;
        const int64_t k0 = row_ptr[row], k1 = row_ptr[row + 1];
        const ChT *cha = ch + (int64_t)a * ch_angle_rows * Fp * 2;
        // entries come in (i, i + 1) pairs of one element: adjacent channel rows
        for (int64_t k = k0; k < k1; k += 2) {
            const int c = __ldg(col + k);
            const float2 w0 = __ldg(val + k), w1 = __ldg(val + k + 1);
            const ChT *r0 = cha + (int64_t)c * Fp * 2;
            const ChT *r1 = r0 + (int64_t)Fp * 2;
#pragma unroll
            for (int g = 0; g < kMaxFrameGroups; ++g) {
                const int f = g * 32 + lane;
                if (g < groups && f < F) {
                    const float2 v0 = load_c2(r0, f), v1 = load_c2(r1, f);
                    acc[g].x = fmaf(w0.x, v0.x, fmaf(-w0.y, v0.y, fmaf(w1.x, v1.x, fmaf(-w1.y, v1.y, acc[g].x))));
                    acc[g].y = fmaf(w0.x, v0.y, fmaf(w0.y, v0.x, fmaf(w1.x, v1.y, fmaf(w1.y, v1.x, acc[g].y))));
                }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < kMaxFrameGroups; ++g) {
        const int f = g * 32 + lane;
        if (g < groups && f < F) fqi::store_c(iq, pix * F + f, make_float2(acc[g].x * inv_A, acc[g].y * inv_A));
    }
}

fq_status make_params(const fq_probe *probe, const fq_tx *tx, const fq_grid *g, MatParams &p, const char *who)
{
    FQ_REQUIRE(probe && tx && g, FQ_ERR_INVALID_ARG, "%s: null probe/tx/grid", who);
    FQ_REQUIRE(tx->n_angles >= 1 && tx->n_angles <= FQ_MAX_ANGLES && tx->tilt_x && tx->tilt_y, FQ_ERR_SHAPE,
               "%s: n_angles must be in [1, %d]", who, FQ_MAX_ANGLES);
    FQ_REQUIRE(probe->nx >= 1 && probe->ny >= 1 && (int64_t)probe->nx * probe->ny <= 4096, FQ_ERR_SHAPE,
               "%s: element count must be in [1, 4096]", who);
    FQ_REQUIRE(probe->n_samples >= 2 && (int64_t)probe->nx * probe->ny * probe->n_samples < ((int64_t)1 << 31),
               FQ_ERR_SHAPE, "%s: elements x samples must fit int32 columns", who);
    FQ_REQUIRE(g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && g->fnumber > 0.0, FQ_ERR_SHAPE, "%s: bad grid", who);
    std::memset(&p, 0, sizeof p);
    fqi::make_probe_ff(probe, p.pr);
    p.A = tx->n_angles;
    p.gx = g->nx;
    p.gy = g->ny;
    p.gz = g->nz;
    p.P = (int64_t)g->nx * g->ny * g->nz;
    p.x0 = g->x0;
    p.y0 = g->y0;
    p.z0 = g->z0;
    p.dx = g->dx;
    p.dy = g->dy;
    p.dz = g->dz;
    p.pitch_x = probe->pitch_x;
    p.pitch_y = probe->pitch_y;
    p.half_per_z = (float)(0.5 / g->fnumber);
    fqi::make_angles_ff(probe, tx, p.ang);
    return FQ_OK;
}

int64_t n_rows(const fq_tx *tx, const fq_grid *g) { return (int64_t)tx->n_angles * g->nx * g->ny * g->nz; }

}  // namespace

extern "C" fq_status fq_das_matrix_workspace_size(const fq_tx *tx, const fq_grid *grid, size_t *bytes)
{
    FQ_REQUIRE(tx && grid && bytes, FQ_ERR_INVALID_ARG, "fq_das_matrix_workspace_size: null argument");
    const int64_t R = n_rows(tx, grid);
    const int64_t nb = (R + kScanBlock - 1) / kScanBlock;
    *bytes = (((size_t)R * 4 + 255) & ~(size_t)255) + (((size_t)nb * 8 + 255) & ~(size_t)255) + 256;
    return FQ_OK;
}

extern "C" fq_status fq_das_matrix_count(const fq_probe *probe, const fq_tx *tx, const fq_grid *grid,
                                         int64_t *row_ptr, void *workspace, size_t workspace_bytes, void *stream)
{
    MatParams p;
    fq_status s = make_params(probe, tx, grid, p, "fq_das_matrix_count");
    if (s) return s;
    size_t need = 0;
    fq_das_matrix_workspace_size(tx, grid, &need);
    FQ_REQUIRE(row_ptr && workspace && workspace_bytes >= need, FQ_ERR_WORKSPACE,
               "fq_das_matrix_count: workspace needs %zu bytes", need);
    FQ_REQUIRE(fqi::aligned(workspace, 256), FQ_ERR_ALIGN, "fq_das_matrix_count: workspace not 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t R = (int64_t)p.A * p.P;
    const int64_t nb = (R + kScanBlock - 1) / kScanBlock;
    // workspace: counts [R], block sums [nb], the total
    char *w = static_cast<char *>(workspace);
    int32_t *cnt = reinterpret_cast<int32_t *>(w);
    const size_t o1 = ((size_t)R * 4 + 255) & ~(size_t)255;
    int64_t *bsum = reinterpret_cast<int64_t *>(w + o1);
    int64_t *total = reinterpret_cast<int64_t *>(w + o1 + (((size_t)nb * 8 + 255) & ~(size_t)255));
    const size_t smem = 6 * sizeof(float) * (size_t)p.pr.M;
    int64_t blocks = (R + kThreads - 1) / kThreads;
    if (blocks > 65535) blocks = 65535;
    count_kernel<<<(unsigned)blocks, kThreads, smem, st>>>(p, cnt);
    block_sum_kernel<<<(unsigned)nb, kScanBlock, 0, st>>>(cnt, R, bsum);
    scan_bsum_kernel<<<1, 32, 0, st>>>(bsum, nb, total);
    local_scan_kernel<<<(unsigned)nb, kScanBlock, 0, st>>>(cnt, R, bsum, row_ptr);
    return fqi::launch_check("fq_das_matrix_count");
}

extern "C" fq_status fq_das_matrix_fill(const fq_probe *probe, const fq_tx *tx, const fq_grid *grid,
                                        const int64_t *row_ptr, int32_t *col, float *val, void *stream)
{
    MatParams p;
    fq_status s = make_params(probe, tx, grid, p, "fq_das_matrix_fill");
    if (s) return s;
    FQ_REQUIRE(row_ptr && col && val, FQ_ERR_INVALID_ARG, "fq_das_matrix_fill: null pointer");
    FQ_REQUIRE(fqi::aligned(val, 8), FQ_ERR_ALIGN, "fq_das_matrix_fill: val must be 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t R = (int64_t)p.A * p.P;
    const size_t smem = 6 * sizeof(float) * (size_t)p.pr.M;
    int64_t blocks = (R + kThreads - 1) / kThreads;
    if (blocks > 65535) blocks = 65535;
    fill_kernel<<<(unsigned)blocks, kThreads, smem, st>>>(p, row_ptr, col, reinterpret_cast<float2 *>(val));
    return fqi::launch_check("fq_das_matrix_fill");
}

extern "C" fq_status fq_das_matrix_apply(const int64_t *row_ptr, const int32_t *col, const float *val, int32_t A,
                                         int64_t P, int32_t M, int32_t ns, const void *iq_ch, int32_t ch_dtype,
                                         int32_t n_frames, int32_t iq_dtype, void *iq, void *stream)
{
    FQ_REQUIRE(row_ptr && col && val && iq_ch && iq, FQ_ERR_INVALID_ARG, "fq_das_matrix_apply: null pointer");
    FQ_REQUIRE(A >= 1 && P >= 1 && M >= 1 && ns >= 2 && n_frames >= 1, FQ_ERR_INVALID_ARG,
               "fq_das_matrix_apply: bad sizes");
    FQ_REQUIRE(n_frames <= 32 * kMaxFrameGroups, FQ_ERR_UNSUPPORTED, "fq_das_matrix_apply: at most %d frames",
               32 * kMaxFrameGroups);
    FQ_REQUIRE((ch_dtype == FQ_F32 || ch_dtype == FQ_BF16) && (iq_dtype == FQ_F32 || iq_dtype == FQ_BF16),
               FQ_ERR_UNSUPPORTED, "fq_das_matrix_apply: dtypes must be FQ_F32 or FQ_BF16");
    cudaStream_t st = (cudaStream_t)stream;
    const int Fp = fq_frame_pad(n_frames);
    const int64_t threads = P * 32;
    const unsigned blocks = (unsigned)((threads + kThreads - 1) / kThreads);
    const float2 *v = reinterpret_cast<const float2 *>(val);
    const float inv_A = 1.0f / (float)A;
    const int64_t rows = (int64_t)M * ns;
    if (ch_dtype == FQ_F32 && iq_dtype == FQ_F32)
        apply_kernel<float, float><<<blocks, kThreads, 0, st>>>(row_ptr, col, v, A, P, (const float *)iq_ch, rows,
                                                                Fp, n_frames, inv_A, (float *)iq);
    else if (ch_dtype == FQ_F32)
        apply_kernel<float, __nv_bfloat16><<<blocks, kThreads, 0, st>>>(
            row_ptr, col, v, A, P, (const float *)iq_ch, rows, Fp, n_frames, inv_A, (__nv_bfloat16 *)iq);
    else if (iq_dtype == FQ_F32)
        apply_kernel<__nv_bfloat16, float><<<blocks, kThreads, 0, st>>>(
            row_ptr, col, v, A, P, (const __nv_bfloat16 *)iq_ch, rows, Fp, n_frames, inv_A, (float *)iq);
    else
        apply_kernel<__nv_bfloat16, __nv_bfloat16><<<blocks, kThreads, 0, st>>>(
            row_ptr, col, v, A, P, (const __nv_bfloat16 *)iq_ch, rows, Fp, n_frames, inv_A, (__nv_bfloat16 *)iq);
    return fqi::launch_check("fq_das_matrix_apply");
}
