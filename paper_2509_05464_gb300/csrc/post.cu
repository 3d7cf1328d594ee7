// post.cu -- display compression, B-mode, maximum-intensity projections
// and image-quality metrics (Sec. 5.2 logarithmic compression and
// dynamic-range display of B-mode and uPDI; Sec. 6.1 MIPs of 3D uPDI;
// Sec. 5.3 MSE, PSNR, SSIM against ground truth).
//
// These are O(pixels) passes: each kernel reads its image once, coalesced,
// and writes its output once; maxima go through a block reduction and one
// atomicMax on the float's bit pattern (non-negative values order like
// their bits); sums go to per-block FP64 partials that one thread adds in
// block order, so the metrics are deterministic.
#include <cmath>

#include "fq_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kSumBlocks = 304;  // 2 per SM
constexpr int kWin = 11;         // SSIM window
constexpr int kTile = 16;        // SSIM output tile
constexpr int kIn = kTile + kWin - 1;

__device__ __forceinline__ float load_v(const float *p, int64_t i) { return p[i]; }

__device__ __forceinline__ float envelope(const void *iq, int dtype, int64_t i)
{
    float re, im;
    if (dtype == FQ_BF16) {
        const __nv_bfloat162 v = reinterpret_cast<const __nv_bfloat162 *>(iq)[i];
        re = __bfloat162float(v.x);
        im = __bfloat162float(v.y);
    } else {
        const float2 v = reinterpret_cast<const float2 *>(iq)[i];
        re = v.x;
        im = v.y;
    }
    return sqrtf(fmaf(re, re, im * im));
}

__device__ __forceinline__ float block_max(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = 0.0f;
    if (threadIdx.x < 32) {
        v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    v = 0.0;
    if (threadIdx.x < 32) {
        v = threadIdx.x < blockDim.x / 32 ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    return v;
}

// mode 0: plain values (negative -> 0); mode 1: envelope of frame `frame`
// of a Casorati matrix [P][F][2]
__global__ void __launch_bounds__(kThreads) max_kernel(const void *src, int mode, int dtype, int64_t n, int F,
                                                       int frame, unsigned *mx)
{
    __shared__ float red[kThreads / 32];
    float m = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float a = mode == 0 ? load_v(reinterpret_cast<const float *>(src), i)
                                  : envelope(src, dtype, i * F + frame);
        m = fmaxf(m, a);  // NaN-free inputs; negatives count as 0
    }
    m = block_max(m, red);
    if (threadIdx.x == 0 && m > 0.0f) atomicMax(mx, __float_as_uint(m));
}

__global__ void __launch_bounds__(kThreads) compress_kernel(const void *src, int mode, int dtype, int64_t n, int F,
                                                            int frame, float g, float dr, const unsigned *mx,
                                                            float *out)
{
    const float m = __uint_as_float(*mx);
    const float inv_m = m > 0.0f ? 1.0f / m : 0.0f;
    const float inv_dr = 1.0f / dr;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float a = mode == 0 ? load_v(reinterpret_cast<const float *>(src), i)
                                  : envelope(src, dtype, i * F + frame);
        float o = 0.0f;
        if (a > 0.0f && m > 0.0f) o = fminf(fmaxf(fmaf(g, log10f(a * inv_m), dr) * inv_dr, 0.0f), 1.0f);
        out[i] = o;
    }
}

// MIP along x: one warp per (z, y) row
__global__ void __launch_bounds__(kThreads) mip_x_kernel(const float *vol, int nx, int64_t rows, float *out)
{
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= rows) return;
    const float *r = vol + warp * nx;
    float m = -INFINITY;
    for (int x = lane; x < nx; x += 32) m = fmaxf(m, r[x]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) out[warp] = m;
}

// MIP along a strided axis: out[o][i] = max_k vol[o][k][i] (i contiguous)
__global__ void __launch_bounds__(kThreads) mip_strided_kernel(const float *vol, int64_t inner, int nk, int64_t outer,
                                                               float *out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= inner * outer) return;
    const int64_t o = t / inner, i = t - o * inner;
    const float *p = vol + o * nk * inner + i;
    float m = -INFINITY;
    for (int k = 0; k < nk; ++k) m = fmaxf(m, p[k * inner]);
    out[t] = m;
}

__global__ void __launch_bounds__(kThreads) mse_kernel(const float *x, const float *y, int64_t n, double *part)
{
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)x[i] - (double)y[i];
        s += d * d;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

struct Win {
    float w[kWin];
};

// SSIM over one 16 x 16 tile of valid positions: the 11-tap Gaussian is
// separable, so the five weighted sums are taken along rows first (26 rows
// of the tile's input), then along columns
__global__ void __launch_bounds__(kTile * kTile) ssim_kernel(const float *x, const float *y, int H, int W, Win win,
                                                             float C1, float C2, double *part)
{
    __shared__ float sx[kIn][kIn], sy[kIn][kIn];
    __shared__ float hs[5][kIn][kTile];
    __shared__ double red[kTile * kTile / 32];
    const int Ho = H - kWin + 1, Wo = W - kWin + 1;
    const int i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
    const int tid = threadIdx.x;
    // moments about a per-tile shift (the tile's centre values): variances
    // and the covariance do not depend on it, and it keeps the binary32
    // second moments from cancelling in flat regions
    const int ci = min(i0 + kIn / 2, H - 1), cj = min(j0 + kIn / 2, W - 1);
    const float cx = x[(int64_t)ci * W + cj], cy = y[(int64_t)ci * W + cj];
    for (int k = tid; k < kIn * kIn; k += blockDim.x) {
        const int r = k / kIn, c = k - r * kIn;
        const int gi = min(i0 + r, H - 1), gj = min(j0 + c, W - 1);
        sx[r][c] = x[(int64_t)gi * W + gj] - cx;
        sy[r][c] = y[(int64_t)gi * W + gj] - cy;
    }
    __syncthreads();
    for (int k = tid; k < kIn * kTile; k += blockDim.x) {
        const int r = k / kTile, c = k - r * kTile;
        float a = 0.0f, b = 0.0f, aa = 0.0f, bb = 0.0f, ab = 0.0f;
#pragma unroll
        for (int t = 0; t < kWin; ++t) {
            const float wt = win.w[t], u = sx[r][c + t], v = sy[r][c + t];
            a = fmaf(wt, u, a);
            b = fmaf(wt, v, b);
            aa = fmaf(wt, u * u, aa);
            bb = fmaf(wt, v * v, bb);
            ab = fmaf(wt, u * v, ab);
        }
        hs[0][r][c] = a;
        hs[1][r][c] = b;
        hs[2][r][c] = aa;
        hs[3][r][c] = bb;
        hs[4][r][c] = ab;
    }
    __syncthreads();
    const int r = tid / kTile, c = tid - (tid / kTile) * kTile;
    double val = 0.0;
    if (i0 + r < Ho && j0 + c < Wo) {
        float mx = 0.0f, my = 0.0f, xx = 0.0f, yy = 0.0f, xy = 0.0f;
#pragma unroll
        for (int t = 0; t < kWin; ++t) {
            const float wt = win.w[t];
            mx = fmaf(wt, hs[0][r + t][c], mx);
            my = fmaf(wt, hs[1][r + t][c], my);
            xx = fmaf(wt, hs[2][r + t][c], xx);
            yy = fmaf(wt, hs[3][r + t][c], yy);
            xy = fmaf(wt, hs[4][r + t][c], xy);
        }
        const float vx = fmaf(-mx, mx, xx), vy = fmaf(-my, my, yy), cxy = fmaf(-mx, my, xy);
        const float ux = mx + cx, uy = my + cy;  // the window means
        const float num = fmaf(2.0f * ux, uy, C1) * fmaf(2.0f, cxy, C2);
        const float den = (fmaf(ux, ux, fmaf(uy, uy, C1))) * (vx + vy + C2);
        val = (double)num / (double)den;
    }
    val = block_sum(val, red);
    if (tid == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = val;
}

__global__ void finish_quality_kernel(const double *mse_part, int n_mse, const double *ssim_part, int n_ssim,
                                      int64_t n_pix, int64_t n_valid, double L, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n_mse; ++i) s += mse_part[i];
    double q = 0.0;
    for (int i = 0; i < n_ssim; ++i) q += ssim_part[i];
    const double mse = s / (double)n_pix;
    out[0] = mse;
    out[1] = 10.0 * log10(L * L / mse);
    out[2] = q / (double)n_valid;
}

int grid_for(int64_t n)
{
    int64_t b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

fq_status compress_any(const void *src, int mode, int dtype, int64_t n, int F, int frame, float g, double dr_db,
                       float *out, void *ws, cudaStream_t st, const char *who)
{
    unsigned *mx = reinterpret_cast<unsigned *>(ws);
    fq_status s = fqi::cuda_check(cudaMemsetAsync(mx, 0, sizeof(unsigned), st), who);
    if (s) return s;
    const int grid = grid_for(n);
    max_kernel<<<grid, kThreads, 0, st>>>(src, mode, dtype, n, F, frame, mx);
    compress_kernel<<<grid, kThreads, 0, st>>>(src, mode, dtype, n, F, frame, g, (float)dr_db, mx, out);
    return fqi::launch_check(who);
}

int ssim_blocks(int H, int W, dim3 &grid)
{
    grid = dim3((unsigned)((W - kWin + 1 + kTile - 1) / kTile), (unsigned)((H - kWin + 1 + kTile - 1) / kTile));
    return (int)(grid.x * grid.y);
}

}  // namespace

extern "C" fq_status fq_post_workspace_size(int32_t H, int32_t W, size_t *bytes)
{
    FQ_REQUIRE(bytes, FQ_ERR_INVALID_ARG, "fq_post_workspace_size: null bytes");
    size_t n = 256;  // the max accumulator
    if (H >= kWin && W >= kWin) {
        dim3 g;
        n += (size_t)(kSumBlocks + ssim_blocks(H, W, g)) * sizeof(double);
    }
    *bytes = (n + 255) & ~(size_t)255;
    return FQ_OK;
}

extern "C" fq_status fq_log_compress(const float *in, int64_t n, int32_t power, double dr_db, float *out,
                                     void *workspace, void *stream)
{
    FQ_REQUIRE(n >= 0 && dr_db > 0.0, FQ_ERR_INVALID_ARG, "fq_log_compress: n < 0 or dynamic range <= 0");
    if (n == 0) return FQ_OK;
    FQ_REQUIRE(in && out && workspace, FQ_ERR_INVALID_ARG, "fq_log_compress: null pointer");
    FQ_REQUIRE(fqi::aligned(workspace, 256), FQ_ERR_ALIGN, "fq_log_compress: workspace not 256-byte aligned");
    return compress_any(in, 0, FQ_F32, n, 1, 0, power ? 10.0f : 20.0f, dr_db, out, workspace,
                        (cudaStream_t)stream, "fq_log_compress");
}

extern "C" fq_status fq_bmode(const void *iq, int32_t dtype, int64_t P, int32_t F, int32_t frame, double dr_db,
                              float *out, void *workspace, void *stream)
{
    FQ_REQUIRE(P >= 0 && F >= 1 && frame >= 0 && frame < F && dr_db > 0.0, FQ_ERR_INVALID_ARG,
               "fq_bmode: P=%lld F=%d frame=%d dr=%g", (long long)P, F, frame, dr_db);
    FQ_REQUIRE(dtype == FQ_F32 || dtype == FQ_BF16, FQ_ERR_UNSUPPORTED, "fq_bmode: dtype must be FQ_F32 or FQ_BF16");
    if (P == 0) return FQ_OK;
    FQ_REQUIRE(iq && out && workspace, FQ_ERR_INVALID_ARG, "fq_bmode: null pointer");
    FQ_REQUIRE(fqi::aligned(workspace, 256), FQ_ERR_ALIGN, "fq_bmode: workspace not 256-byte aligned");
    return compress_any(iq, 1, dtype, P, F, frame, 20.0f, dr_db, out, workspace, (cudaStream_t)stream, "fq_bmode");
}

extern "C" fq_status fq_mip(const float *vol, int32_t nx, int32_t ny, int32_t nz, int32_t axis, float *out,
                            void *stream)
{
    FQ_REQUIRE(nx >= 1 && ny >= 1 && nz >= 1 && axis >= 0 && axis <= 2, FQ_ERR_INVALID_ARG,
               "fq_mip: sizes must be >= 1 and axis in {0, 1, 2}");
    FQ_REQUIRE(vol && out, FQ_ERR_INVALID_ARG, "fq_mip: null pointer");
    cudaStream_t st = (cudaStream_t)stream;
    if (axis == 0) {
        const int64_t rows = (int64_t)ny * nz;
        const int64_t threads = rows * 32;
        mip_x_kernel<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, st>>>(vol, nx, rows, out);
    } else {
        const int64_t inner = axis == 1 ? nx : (int64_t)nx * ny;
        const int nk = axis == 1 ? ny : nz;
        const int64_t outer = axis == 1 ? nz : 1;
        const int64_t t = inner * outer;
        mip_strided_kernel<<<(unsigned)((t + kThreads - 1) / kThreads), kThreads, 0, st>>>(vol, inner, nk, outer, out);
    }
    return fqi::launch_check("fq_mip");
}

extern "C" fq_status fq_image_quality(const float *x, const float *y, int32_t H, int32_t W, double L, double *out,
                                      void *workspace, size_t workspace_bytes, void *stream)
{
    FQ_REQUIRE(H >= kWin && W >= kWin, FQ_ERR_SHAPE, "fq_image_quality: images need at least 11 x 11 pixels");
    FQ_REQUIRE(L > 0.0, FQ_ERR_INVALID_ARG, "fq_image_quality: data range L must be > 0");
    FQ_REQUIRE(x && y && out && workspace, FQ_ERR_INVALID_ARG, "fq_image_quality: null pointer");
    size_t need = 0;
    fq_post_workspace_size(H, W, &need);
    FQ_REQUIRE(workspace_bytes >= need, FQ_ERR_WORKSPACE, "fq_image_quality: workspace needs %zu bytes", need);
    FQ_REQUIRE(fqi::aligned(workspace, 256), FQ_ERR_ALIGN, "fq_image_quality: workspace not 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    double *mse_part = reinterpret_cast<double *>(static_cast<char *>(workspace) + 256);
    double *ssim_part = mse_part + kSumBlocks;
    const int64_t n = (int64_t)H * W;
    mse_kernel<<<kSumBlocks, kThreads, 0, st>>>(x, y, n, mse_part);
    // normalised 1D Gaussian (sigma 1.5); the 2D window is its outer product
    Win win;
    double g[kWin], sum = 0.0;
    for (int t = 0; t < kWin; ++t) {
        const double r = t - (kWin - 1) / 2.0;
        g[t] = std::exp(-r * r / (2.0 * 1.5 * 1.5));
        sum += g[t];
    }
    for (int t = 0; t < kWin; ++t) win.w[t] = (float)(g[t] / sum);
    dim3 grid;
    const int nb = ssim_blocks(H, W, grid);
    ssim_kernel<<<grid, kTile * kTile, 0, st>>>(x, y, H, W, win, (float)(0.01 * L * 0.01 * L),
                                               (float)(0.03 * L * 0.03 * L), ssim_part);
    finish_quality_kernel<<<1, 32, 0, st>>>(mse_part, kSumBlocks, ssim_part, nb, n,
                                            (int64_t)(H - kWin + 1) * (W - kWin + 1), L, out);
    return fqi::launch_check("fq_image_quality");
}
