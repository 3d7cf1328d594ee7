// clutter.cu -- a6 Casorati Gram, a7 Hermitian eigen-decomposition and
// energy cutoff, a8 clutter projection and power Doppler (Sec. 2.4.2).
//
// The SVD of the Casorati matrix S (pixels x frames) is obtained from the
// eigen-decomposition of its frames x frames Gram matrix G = S^H S
// (eigenvalues sigma^2, eigenvectors = right singular vectors).  Removing
// the k largest components is S_f = S - (S V_k) V_k^H and the power Doppler
// is the mean of |S_f|^2 over frames.  With k << F this is O(P F k) and
// bound by the single read of S.
#include <cfloat>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda.h>  // driver types only: the two driver calls are fetched at run time

#include "batch.cuh"
#include "fq_internal.cuh"

namespace {

// ------------------------------------------------------------ workspace --
struct ClutterLayout {
    size_t status, G, part, V, Vt, lam, k, hv, tau, big, ii, tc, total;
    int n_chunks;
    int64_t chunk_len;
};

constexpr int kGramTile = 32;
constexpr int kFastMaxK = 48;  // top-k eigenvectors by inverse iteration up to this k

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int gram_chunks(int64_t P, int F)
{
    int nt = (F + kGramTile - 1) / kGramTile;
    int pairs = nt * (nt + 1) / 2;
    int want = (4 * 152 + pairs - 1) / pairs;
    int64_t max_chunks = (P + kGramTile - 1) / kGramTile;
    if (want > max_chunks) want = (int)max_chunks;
    if (want > 64) want = 64;
    if (want < 1) want = 1;
    return want;
}

bool eig_in_smem(int F) { return (size_t)F * (F + 1) / 2 * sizeof(float2) <= 190 * 1024; }

// Operand bytes of the tensor-core Gram modes (0 = CUDA-core FP32 Gram).
int tc_esz(int gram_mode) { return gram_mode == FQ_GRAM_BF16 ? 2 : (gram_mode == FQ_GRAM_TF32 ? 4 : 0); }

ClutterLayout layout(int64_t P, int F, int gram_mode = FQ_GRAM_F32, bool force_big = false)
{
    ClutterLayout L;
    size_t o = 0;
    const int esz = tc_esz(gram_mode);
    L.status = o; o += 256;
    L.G = o; o += al256(sizeof(float2) * F * F);
    L.n_chunks = gram_chunks(P, F);
    int64_t per = (P + L.n_chunks - 1) / L.n_chunks;
    L.chunk_len = (per + kGramTile - 1) / kGramTile * kGramTile;
    L.part = o; o += esz ? 0 : al256(sizeof(float2) * (size_t)L.n_chunks * F * F);
    L.tc = o; o += esz ? fqi::gram_tc_workspace_bytes(P, F, esz) : 0;
    L.V = o; o += al256(sizeof(float2) * F * F);
    L.Vt = o; o += al256(sizeof(float2) * F * F);
    L.lam = o; o += al256(sizeof(double) * F);
    L.k = o; o += 256;
    L.hv = o; o += al256(sizeof(float2) * F * F);
    L.tau = o; o += al256(sizeof(float) * F);
    L.big = o; o += (eig_in_smem(F) && !force_big) ? 0 : al256(sizeof(float2) * (size_t)F * (F + 1) / 2);
    L.ii = o; o += al256(sizeof(float) * 6 * (size_t)kFastMaxK * F);
    L.total = o;
    return L;
}

size_t eig_only_bytes(int F)
{
    // status, hv, tau, Vt, k, big
    size_t o = 256 + al256(sizeof(float2) * F * F) + al256(sizeof(float) * F) + al256(sizeof(float2) * F * F) + 256;
    if (!eig_in_smem(F)) o += al256(sizeof(float2) * (size_t)F * (F + 1) / 2);
    return o;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// ----------------------------------------------------------------- Gram --
// Upper-triangular tiles (ti <= tj) of G over pixel chunks; each CTA: one
// 32x32 complex tile over one chunk; 256 threads, 2x2 outputs each.
template <typename T>
__device__ __forceinline__ void gram_tile(const T *__restrict__ S, int64_t P, int F, int nt, int64_t chunk_len,
                                          float2 *__restrict__ part, int pair, int c,
                                          float2 (*As)[kGramTile + 1], float2 (*Bs)[kGramTile + 1])
{
    // decode upper-triangular tile pair
    int t = pair, ti = 0;
    while (t >= nt - ti) { t -= nt - ti; ++ti; }
    const int tj = ti + t;
    const int64_t pbeg = (int64_t)c * chunk_len;
    const int64_t pend = min(P, pbeg + chunk_len);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float2 acc[2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
    for (int64_t p0 = pbeg; p0 < pend; p0 += kGramTile) {
        for (int i = threadIdx.x; i < kGramTile * kGramTile; i += 256) {
            int pr = i / kGramTile, col = i % kGramTile;
            int64_t p = p0 + pr;
            int ci = ti * kGramTile + col, cj = tj * kGramTile + col;
            float2 a = make_float2(0, 0), b = make_float2(0, 0);
            if (p < pend) {
                if (ci < F) a = fqi::load_c(S, p * F + ci);
                if (cj < F) b = fqi::load_c(S, p * F + cj);
            }
            As[pr][col] = a;
            Bs[pr][col] = b;
        }
        __syncthreads();
#pragma unroll 8
        for (int pr = 0; pr < kGramTile; ++pr) {
            float2 a0 = As[pr][2 * ty], a1 = As[pr][2 * ty + 1];
            float2 b0 = Bs[pr][2 * tx], b1 = Bs[pr][2 * tx + 1];
            // conj(a) b
            acc[0][0].x += a0.x * b0.x + a0.y * b0.y; acc[0][0].y += a0.x * b0.y - a0.y * b0.x;
            acc[0][1].x += a0.x * b1.x + a0.y * b1.y; acc[0][1].y += a0.x * b1.y - a0.y * b1.x;
            acc[1][0].x += a1.x * b0.x + a1.y * b0.y; acc[1][0].y += a1.x * b0.y - a1.y * b0.x;
            acc[1][1].x += a1.x * b1.x + a1.y * b1.y; acc[1][1].y += a1.x * b1.y - a1.y * b1.x;
        }
        __syncthreads();
    }
    float2 *out = part + (size_t)c * F * F;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            int i = ti * kGramTile + 2 * ty + a, j = tj * kGramTile + 2 * tx + b;
            if (i < F && j < F) out[(size_t)i * F + j] = acc[a][b];
        }
}

template <typename T>
__global__ void __launch_bounds__(256) gram_partial_kernel(const T *__restrict__ S, int64_t P, int F, int nt,
                                                           int64_t chunk_len, float2 *__restrict__ part)
{
    __shared__ float2 As[kGramTile][kGramTile + 1];
    __shared__ float2 Bs[kGramTile][kGramTile + 1];
    gram_tile<T>(S, P, F, nt, chunk_len, part, blockIdx.x, blockIdx.y, As, Bs);
}

__device__ __forceinline__ void gram_reduce_at(const float2 *__restrict__ part, int n_chunks, int F,
                                               float2 *__restrict__ G, int idx)
{
    if (idx >= F * F) return;
    int i = idx / F, j = idx % F;
    bool upper = (i / kGramTile) <= (j / kGramTile);
    int src = upper ? idx : j * F + i;
    float2 s = make_float2(0, 0);
    for (int c = 0; c < n_chunks; ++c) {
        float2 v = part[(size_t)c * F * F + src];
        s.x += v.x;
        s.y += v.y;
    }
    G[idx] = upper ? s : cconj(s);
}

__global__ void gram_reduce_kernel(const float2 *__restrict__ part, int n_chunks, int F, float2 *__restrict__ G)
{
    gram_reduce_at(part, n_chunks, F, G, blockIdx.x * blockDim.x + threadIdx.x);
}

// ------------------------------------------------------------ eigen (1 CTA) --
constexpr int kEigThreads = 1024;

__device__ __forceinline__ int pidx(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

// block-wide sum of one float per thread
__device__ float block_sum(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        float x = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[32] = x;
    }
    __syncthreads();
    return red[32];
}

// V[:, j] = H_0 ... H_{F-3} D Z[:, perm[j]] for j < ncol (warp per column).
__device__ void back_transform(int F, int ncol, const float *Z, int zs, const int *perm, const float2 *delta,
                               const float2 *__restrict__ hv, const float *__restrict__ tau_g, float2 *__restrict__ V,
                               float2 *__restrict__ Vt, int lane, int wid, int nw)
{
    for (int j = wid; j < ncol; j += nw) {
        const int src = perm[j];
        float2 y[16];  // F <= 512: 16 values per lane
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            int i = lane + 32 * q;
            y[q] = i < F ? make_float2(delta[i].x * Z[i * zs + src], delta[i].y * Z[i * zs + src]) : make_float2(0, 0);
        }
        for (int k = F - 3; k >= 0; --k) {
            const float t = tau_g[k];
            if (t == 0.0f) continue;
            const float2 *v = hv + (size_t)k * F;
            float2 s = make_float2(0, 0);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                int i = lane + 32 * q;
                if (i > k && i < F) {
                    float2 vi = v[i];
                    s.x += vi.x * y[q].x + vi.y * y[q].y;  // conj(v) y
                    s.y += vi.x * y[q].y - vi.y * y[q].x;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
            }
            s.x *= t;
            s.y *= t;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                int i = lane + 32 * q;
                if (i > k && i < F) {
                    float2 u = cmul(v[i], s);
                    y[q].x -= u.x;
                    y[q].y -= u.y;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            int i = lane + 32 * q;
            if (i < F) {
                if (V) V[(size_t)i * F + j] = y[q];
                Vt[(size_t)j * F + i] = y[q];
            }
        }
    }
}

// Number of eigenvalues of the real symmetric tridiagonal (d, e) below x
// (Sturm count by the LDL^T pivot recurrence; tiny pivots are replaced by
// -pivmin so that the count stays monotone).
__device__ int sturm_below(const float *d, const float *e2, int n, float x, float pivmin)
{
    int cnt = 0;
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.0f;
    for (int i = 1; i < n; ++i) {
        q = (d[i] - x) - e2[i - 1] / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt += q < 0.0f;
    }
    return cnt;
}

// The m-th smallest eigenvalue (0-based) by bisection on [lo, hi].
__device__ float bisect_eig(const float *d, const float *e2, int n, int m, float lo, float hi, float pivmin)
{
    for (int it = 0; it < 80; ++it) {
        const float mid = 0.5f * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_below(d, e2, n, mid, pivmin) >= m + 1) hi = mid;
        else lo = mid;
    }
    return 0.5f * (lo + hi);
}

// One eigenvector of the real tridiagonal for eigenvalue sigma by inverse
// iteration: Gaussian elimination with partial pivoting of T - sigma I
// (kept in per-thread local arrays), three solves from a fixed pseudo-random
// start, each normalised.  Writes column `col` of Z (row stride zs).
__device__ void inverse_iteration(const float *d, const float *e, int n, float sigma, float tiny, int seed,
                                  float *Z, int zs, int col, float *__restrict__ scr)
{
    // scratch (global workspace, 6 n floats): u0, u1, u2, multipliers, swaps, x
    float *u0 = scr, *u1 = scr + n, *u2 = scr + 2 * n, *ml = scr + 3 * n, *sw = scr + 4 * n, *x = scr + 5 * n;
    float p0 = d[0] - sigma, p1 = n > 1 ? e[0] : 0.0f, p2 = 0.0f;
    for (int i = 0; i + 1 < n; ++i) {
        const float c = e[i];                       // sub-diagonal of row i + 1
        const float a1 = d[i + 1] - sigma;
        const float b1 = (i + 2 < n) ? e[i + 1] : 0.0f;
        if (fabsf(c) > fabsf(p0)) {
            // pivot on row i + 1
            const float mlt = p0 / c;
            u0[i] = c; u1[i] = a1; u2[i] = b1; ml[i] = mlt; sw[i] = 1.0f;
            p0 = p1 - mlt * a1;
            p1 = p2 - mlt * b1;
            p2 = 0.0f;
        } else {
            const float piv = fabsf(p0) < tiny ? (p0 < 0.0f ? -tiny : tiny) : p0;
            const float mlt = c / piv;
            u0[i] = piv; u1[i] = p1; u2[i] = p2; ml[i] = mlt; sw[i] = 0.0f;
            p0 = a1 - mlt * p1;
            p1 = b1 - mlt * p2;
            p2 = 0.0f;
        }
    }
    u0[n - 1] = fabsf(p0) < tiny ? (p0 < 0.0f ? -tiny : tiny) : p0;
    u1[n - 1] = 0.0f;
    u2[n - 1] = 0.0f;
    unsigned h = 0x9E3779B9u * (unsigned)(seed + 1);
    for (int i = 0; i < n; ++i) {
        h = h * 1664525u + 1013904223u;
        x[i] = 1.0f + 0.25f * ((float)(h >> 8) * (1.0f / 16777216.0f) - 0.5f);
    }
    for (int it = 0; it < 3; ++it) {
        // forward: apply the row swaps and multipliers to the right-hand side
        for (int i = 0; i + 1 < n; ++i) {
            if (sw[i] != 0.0f) {
                const float t = x[i];
                x[i] = x[i + 1];
                x[i + 1] = t - ml[i] * x[i];
            } else {
                x[i + 1] -= ml[i] * x[i];
            }
        }
        // back substitution
        x[n - 1] = x[n - 1] / u0[n - 1];
        if (n > 1) x[n - 2] = (x[n - 2] - u1[n - 2] * x[n - 1]) / u0[n - 2];
        for (int i = n - 3; i >= 0; --i) x[i] = (x[i] - u1[i] * x[i + 1] - u2[i] * x[i + 2]) / u0[i];
        float mx = 0.0f;
        for (int i = 0; i < n; ++i) mx = fmaxf(mx, fabsf(x[i]));
        const float inv = mx > 0.0f ? 1.0f / mx : 1.0f;
        for (int i = 0; i < n; ++i) x[i] *= inv;
    }
    float s2 = 0.0f;
    for (int i = 0; i < n; ++i) s2 += x[i] * x[i];
    const float inv = rsqrtf(s2);
    for (int i = 0; i < n; ++i) Z[i * zs + col] = x[i] * inv;
}

// Householder tridiagonalisation of the Hermitian G (lower triangle used),
// implicit QL with Wilkinson shifts on the real tridiagonal (after a
// diagonal unitary scaling), eigenvalue sort and back-transformation.
// Optional: the energy / fixed cutoff k.
__device__ __forceinline__ void eig_body(const float2 *__restrict__ G, int F, float2 *__restrict__ big,
                                         float2 *__restrict__ hv, float *__restrict__ tau_g,
                                         double *__restrict__ lam_out, float2 *__restrict__ V,
                                         float2 *__restrict__ Vt, int k_cut, double thresh,
                                         int *__restrict__ k_out, int *__restrict__ status,
                                         int topk_only, float *__restrict__ ii_scr)
{
    extern __shared__ float2 dyn[];
    float2 *Ap = big ? big : dyn;                 // packed lower triangle, later Z (real, stride F+1)
    float *Z = reinterpret_cast<float *>(Ap);
    __shared__ float red[33];
    __shared__ float d[512], e[512], rc[512], rs[512];
    __shared__ float2 ec[512], vv[512], pv[512], delta[512];
    __shared__ int perm[512];
    __shared__ float s_tau, s_scale;
    __shared__ int s_m, s_nrot, s_done, s_fail;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;

    // scale to max |G_ij| <= 1 (eigenvectors unchanged, eigenvalues rescaled at the end)
    float amax = 0.0f;
    for (int i = wid; i < F; i += nw)
        for (int j = lane; j <= i; j += 32) {
            float2 g = G[(size_t)i * F + j];
            amax = fmaxf(amax, fmaxf(fabsf(g.x), fabsf(g.y)));
        }
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) red[wid] = amax;
    __syncthreads();
    if (tid == 0) {
        float mx = 0.0f;
        for (int w = 0; w < nw; ++w) mx = fmaxf(mx, red[w]);
        // a power of two, so that the scaling itself is exact
        s_scale = mx > 0.0f ? exp2f(ceilf(log2f(mx))) : 1.0f;
    }
    __syncthreads();
    const float gscale = s_scale, ginv = 1.0f / s_scale;
    for (int i = wid; i < F; i += nw)
        for (int j = lane; j <= i; j += 32) {
            float2 g = G[(size_t)i * F + j];
            Ap[pidx(i, j)] = make_float2(g.x * ginv, g.y * ginv);
        }
    __syncthreads();

    // ---- tridiagonalisation
    for (int k = 0; k + 2 < F; ++k) {
        const int m = F - k - 1;  // length of the column below the diagonal
        float part = 0.0f;
        for (int i = tid; i < m; i += blockDim.x) {
            float2 x = Ap[pidx(k + 1 + i, k)];
            part += x.x * x.x + x.y * x.y;
        }
        float a2 = block_sum(part, red);
        if (tid == 0) {
            d[k] = Ap[pidx(k, k)].x;
            float2 x0 = Ap[pidx(k + 1, k)];
            float ax0 = sqrtf(x0.x * x0.x + x0.y * x0.y);
            float alpha = sqrtf(a2);
            if (alpha <= 1e-30f) {
                s_tau = 0.0f;
                ec[k] = make_float2(0, 0);
                vv[0] = make_float2(0, 0);
            } else {
                float2 th = ax0 > 0.0f ? make_float2(x0.x / ax0, x0.y / ax0) : make_float2(1.0f, 0.0f);
                ec[k] = make_float2(-th.x * alpha, -th.y * alpha);   // beta = -theta alpha
                vv[0] = make_float2(th.x * (ax0 + alpha), th.y * (ax0 + alpha));
                s_tau = 1.0f / (alpha * (alpha + ax0));
            }
        }
        __syncthreads();
        const float tau = s_tau;
        for (int i = 1 + tid; i < m; i += blockDim.x) vv[i] = tau != 0.0f ? Ap[pidx(k + 1 + i, k)] : make_float2(0, 0);
        __syncthreads();
        for (int i = tid; i < m; i += blockDim.x) hv[(size_t)k * F + k + 1 + i] = vv[i];
        if (tid == 0) tau_g[k] = tau;
        if (tau == 0.0f) {
            __syncthreads();
            continue;
        }
        // p = tau A22 v (warp per row)
        for (int i = wid; i < m; i += nw) {
            float2 s = make_float2(0, 0);
            const int gi = k + 1 + i;
            for (int j = lane; j < m; j += 32) {
                const int gj = k + 1 + j;
                float2 a = gj <= gi ? Ap[pidx(gi, gj)] : cconj(Ap[pidx(gj, gi)]);
                float2 t = cmul(a, vv[j]);
                s.x += t.x;
                s.y += t.y;
            }
            for (int o = 16; o > 0; o >>= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
            }
            if (lane == 0) pv[i] = make_float2(tau * s.x, tau * s.y);
        }
        __syncthreads();
        // K = tau / 2 * Re(v^H p)
        float q = 0.0f;
        for (int i = tid; i < m; i += blockDim.x) q += vv[i].x * pv[i].x + vv[i].y * pv[i].y;
        float vhp = block_sum(q, red);
        const float K = 0.5f * tau * vhp;
        // w = p - K v (in place in pv)
        for (int i = tid; i < m; i += blockDim.x) pv[i] = make_float2(pv[i].x - K * vv[i].x, pv[i].y - K * vv[i].y);
        __syncthreads();
        // A22 -= v w^H + w v^H (lower triangle)
        for (int i = wid; i < m; i += nw) {
            const float2 vi = vv[i], wi = pv[i];
            for (int j = lane; j <= i; j += 32) {
                float2 a = Ap[pidx(k + 1 + i, k + 1 + j)];
                float2 t1 = cmul(vi, cconj(pv[j]));
                float2 t2 = cmul(wi, cconj(vv[j]));
                a.x -= t1.x + t2.x;
                a.y -= t1.y + t2.y;
                Ap[pidx(k + 1 + i, k + 1 + j)] = a;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (F >= 2) {
            d[F - 2] = Ap[pidx(F - 2, F - 2)].x;
            ec[F - 2] = Ap[pidx(F - 1, F - 2)];
        }
        d[F - 1] = Ap[pidx(F - 1, F - 1)].x;
        // diagonal unitary scaling making the off-diagonal real and >= 0
        delta[0] = make_float2(1.0f, 0.0f);
        for (int k = 0; k + 1 < F; ++k) {
            float2 x = ec[k];
            float ax = sqrtf(x.x * x.x + x.y * x.y);
            e[k] = ax;
            delta[k + 1] = ax > 0.0f ? cmul(delta[k], make_float2(x.x / ax, x.y / ax)) : delta[k];
        }
        e[F - 1] = 0.0f;
        s_fail = 0;
    }
    __syncthreads();
    const int zs = F + 1;
    if (topk_only) {
        // ---- all eigenvalues by bisection (one thread each), top-k vectors by
        // inverse iteration; the QL path below is the fallback for large k
        __shared__ float e2[512], lamd[512];
        __shared__ float s_lo, s_hi, s_piv, s_tnorm;
        __shared__ int s_k;
        for (int i = tid; i < F; i += blockDim.x) e2[i] = e[i] * e[i];
        if (tid == 0) {
            float lo = 1e30f, hi = -1e30f, tn = 0.0f;
            for (int i = 0; i < F; ++i) {
                const float r = (i > 0 ? e[i - 1] : 0.0f) + e[i];
                lo = fminf(lo, d[i] - r);
                hi = fmaxf(hi, d[i] + r);
                tn = fmaxf(tn, fabsf(d[i]) + r);
            }
            const float pad = 4.0f * FLT_EPSILON * fmaxf(tn, 1e-30f);
            s_lo = lo - pad;
            s_hi = hi + pad;
            s_tnorm = tn;
            s_piv = fmaxf(1e-30f, FLT_MIN * 4.0f);
        }
        __syncthreads();
        for (int j = tid; j < F; j += blockDim.x)
            lamd[j] = bisect_eig(d, e2, F, F - 1 - j, s_lo, s_hi, s_piv);  // descending order
        __syncthreads();
        for (int j = tid; j < F; j += blockDim.x) lam_out[j] = (double)lamd[j] * (double)gscale;
        if (tid == 0) {
            int k = k_cut;
            if (k < 0) {
                double tot = 0.0, acc = 0.0;
                for (int j = 0; j < F; ++j) tot += fmax((double)lamd[j], 0.0);
                k = F;
                for (int j = 0; j < F; ++j) {
                    acc += fmax((double)lamd[j], 0.0);
                    if (acc >= thresh * tot) { k = j + 1; break; }
                }
            }
            if (k_out) *k_out = k;
            s_k = k;
        }
        __syncthreads();
        const int k = s_k;
        if (k <= kFastMaxK && ii_scr) {
            const float tiny = FLT_EPSILON * fmaxf(s_tnorm, 1e-30f);
            for (int j = tid; j < k; j += blockDim.x)
                inverse_iteration(d, e, F, lamd[j], tiny, j, Z, zs, j, ii_scr + (size_t)j * 6 * F);
            __syncthreads();
            // re-orthogonalise vectors of close eigenvalues (modified Gram-Schmidt, warp 0)
            if (wid == 0) {
                const float gap = 1e-3f * s_tnorm;
                for (int j = 1; j < k; ++j) {
                    bool any = false;
                    for (int i = 0; i < j; ++i) {
                        if (fabsf(lamd[i] - lamd[j]) > gap) continue;
                        any = true;
                        float dot = 0.0f;
                        for (int r = lane; r < F; r += 32) dot += Z[r * zs + i] * Z[r * zs + j];
                        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
                        for (int r = lane; r < F; r += 32) Z[r * zs + j] -= dot * Z[r * zs + i];
                        __syncwarp();
                    }
                    if (any) {
                        float n2 = 0.0f;
                        for (int r = lane; r < F; r += 32) n2 += Z[r * zs + j] * Z[r * zs + j];
                        for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
                        const float inv = rsqrtf(n2);
                        for (int r = lane; r < F; r += 32) Z[r * zs + j] *= inv;
                        __syncwarp();
                    }
                }
            }
            for (int j = tid; j < F; j += blockDim.x) perm[j] = j;
            __syncthreads();
            back_transform(F, k, Z, zs, perm, delta, hv, tau_g, V, Vt, lane, wid, nw);
            return;
        }
    }
    // Z = identity (stride F+1), reusing the packed-matrix storage
    for (int i = tid; i < F * zs; i += blockDim.x) Z[i] = ((i / zs) == (i % zs)) ? 1.0f : 0.0f;
    __syncthreads();

    // ---- implicit QL; thread 0 runs the scalar recurrence, everybody applies the rotations
    float tnorm = 0.0f;
    if (tid == 0) {
        for (int i = 0; i < F; ++i) tnorm = fmaxf(tnorm, fabsf(d[i]) + fabsf(e[i]));
    }
    for (int l = 0; l < F; ++l) {
        int iter = 0;
        bool stop_all = false;
        while (true) {
            if (tid == 0) {
                int m = l;
                for (; m < F - 1; ++m) {
                    float dd = fabsf(d[m]) + fabsf(d[m + 1]);
                    if (fabsf(e[m]) <= FLT_EPSILON * dd || fabsf(e[m]) <= 1e-3f * FLT_EPSILON * tnorm) break;
                }
                s_done = (m == l);
                s_nrot = 0;
                if (m != l) {
                    if (++iter > 60) {
                        s_fail = 1;
                        s_done = 1;
                    } else {
                        float g = (d[l + 1] - d[l]) / (2.0f * e[l]);
                        float r = sqrtf(fmaf(g, g, 1.0f));
                        g = d[m] - d[l] + e[l] / (g + copysignf(r, g));
                        float s = 1.0f, c = 1.0f, p = 0.0f;
                        bool early = false;
                        int nrot = 0;
                        for (int i = m - 1; i >= l; --i) {
                            float f = s * e[i], b = c * e[i];
                            // r = |(f, g)| and 1/r from one reciprocal square root plus a
                            // Newton step (the matrix is scaled to max |entry| = 1, so no
                            // overflow is possible)
                            const float q = fmaf(f, f, g * g);
                            if (q == 0.0f) {
                                e[i + 1] = 0.0f;
                                d[i + 1] -= p;
                                e[m] = 0.0f;
                                early = true;
                                break;
                            }
                            float rr = rsqrtf(q);
                            rr = rr * fmaf(-0.5f * q * rr, rr, 1.5f);
                            r = q * rr;
                            e[i + 1] = r;
                            s = f * rr;
                            c = g * rr;
                            g = d[i + 1] - p;
                            r = (d[i] - g) * s + 2.0f * c * b;
                            p = s * r;
                            d[i + 1] = g + p;
                            g = c * r - b;
                            rc[nrot] = c;
                            rs[nrot] = s;
                            ++nrot;
                        }
                        if (!early) {
                            d[l] -= p;
                            e[l] = g;
                            e[m] = 0.0f;
                        }
                        s_nrot = nrot;
                        s_m = m;
                    }
                }
            }
            __syncthreads();
            // every thread reads the sweep description between the two barriers
            const int done = s_done, nrot = s_nrot, mm = s_m, fail = s_fail;
            if (!done) {
                // rotation r acts on columns (i, i+1) with i = m - 1 - r
                for (int row = tid; row < F; row += blockDim.x) {
                    float *zr = Z + row * zs;
                    for (int r = 0; r < nrot; ++r) {
                        int i = mm - 1 - r;
                        float c = rc[r], s = rs[r];
                        float t = zr[i + 1];
                        zr[i + 1] = s * zr[i] + c * t;
                        zr[i] = c * zr[i] - s * t;
                    }
                }
            }
            __syncthreads();
            if (done) {
                stop_all = fail != 0;
                break;
            }
        }
        if (stop_all) break;
    }
    __syncthreads();
    // ---- sort descending (rank by value, ties by index)
    for (int i = tid; i < F; i += blockDim.x) {
        float di = d[i];
        int rank = 0;
        for (int j = 0; j < F; ++j) {
            float dj = d[j];
            rank += (dj > di) || (dj == di && j < i);
        }
        perm[rank] = i;
    }
    __syncthreads();
    for (int j = tid; j < F; j += blockDim.x) lam_out[j] = (double)d[perm[j]] * (double)gscale;
    if (tid == 0) {
        int k = k_cut;
        if (k < 0) {
            double tot = 0.0, acc = 0.0;
            for (int j = 0; j < F; ++j) tot += fmax((double)d[perm[j]], 0.0);
            k = F;
            for (int j = 0; j < F; ++j) {
                acc += fmax((double)d[perm[j]], 0.0);
                if (acc >= thresh * tot) { k = j + 1; break; }
            }
        }
        if (k_out) *k_out = k;
        if (status && s_fail) *status = FQ_ERR_NUMERICAL;
    }
    back_transform(F, F, Z, zs, perm, delta, hv, tau_g, V, Vt, lane, wid, nw);
}

__global__ void __launch_bounds__(kEigThreads) eig_kernel(const float2 *__restrict__ G, int F, float2 *__restrict__ big,
                                                          float2 *__restrict__ hv, float *__restrict__ tau_g,
                                                          double *__restrict__ lam_out, float2 *__restrict__ V,
                                                          float2 *__restrict__ Vt, int k_cut, double thresh,
                                                          int *__restrict__ k_out, int *__restrict__ status,
                                                          int topk_only, float *__restrict__ ii_scr)
{
    eig_body(G, F, big, hv, tau_g, lam_out, V, Vt, k_cut, thresh, k_out, status, topk_only, ii_scr);
}

// One CTA per ensemble of a wave; the packed matrix always in the workspace.
__global__ void __launch_bounds__(kEigThreads) eig_batched_kernel(const fqb::EnsDev *__restrict__ ens,
                                                                  const int *__restrict__ members)
{
    const fqb::EnsDev &e = ens[members[blockIdx.x]];
    char *ws = e.cws;
    double *lam = e.eigvals ? e.eigvals : (double *)(ws + e.cl_lam);
    int *kk = e.k_used ? e.k_used : (int *)(ws + e.cl_k);
    eig_body((const float2 *)(ws + e.cl_G), e.F, (float2 *)(ws + e.cl_big), (float2 *)(ws + e.cl_hv),
             (float *)(ws + e.cl_tau), lam, (float2 *)(ws + e.cl_V), (float2 *)(ws + e.cl_Vt), e.k_cut,
             e.energy_thresh, kk, e.status, 1, (float *)(ws + e.cl_ii));
}

// ------------------------------------------------ projection + power Doppler --
// One warp per pixel: y_j = sum_f S[f] V[f][j] for j < k, then
// S_f = S - sum_j y_j conj(V[:, j]) and pd = mean |S_f|^2.  Lane l holds
// frames l, l + 32, ..: NQ (a power of two, 32 NQ >= F) of them, so that the
// unrolled loops issue no work for frames beyond F (with NQ fixed at 16, the
// loops of a 100-frame ensemble issued four times the instructions they
// needed and the kernel was issue-bound at ~20% of HBM bandwidth).

// the pixel's frames into registers (frames beyond F read as 0)
template <typename T, int NQ>
__device__ __forceinline__ void project_load(const T *__restrict__ S, int64_t p, int F, int lane, float2 (&s)[NQ])
{
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        int f = lane + 32 * q;
        s[q] = f < F ? fqi::load_c(S, p * F + f) : make_float2(0, 0);
    }
}

template <typename T, int NQ>
__device__ __forceinline__ void project_compute(const float2 (&s)[NQ], int64_t p, int F,
                                                const float2 *__restrict__ Vt, int k, T *__restrict__ S_f,
                                                float *__restrict__ pd, float invF, int lane)
{
    float2 sf[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) sf[q] = s[q];
    if (k >= F) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) sf[q] = make_float2(0, 0);
    } else {
        for (int j = 0; j < k; ++j) {
            const float2 *vj = Vt + (size_t)j * F;
            float2 y = make_float2(0, 0);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                int f = lane + 32 * q;
                if (f < F) {
                    float2 t = cmul(s[q], vj[f]);
                    y.x += t.x;
                    y.y += t.y;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                y.x += __shfl_xor_sync(0xffffffffu, y.x, o);
                y.y += __shfl_xor_sync(0xffffffffu, y.y, o);
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                int f = lane + 32 * q;
                if (f < F) {
                    float2 t = cmul(y, cconj(vj[f]));
                    sf[q].x -= t.x;
                    sf[q].y -= t.y;
                }
            }
        }
    }
    float e = 0.0f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        int f = lane + 32 * q;
        if (f < F) {
            e += sf[q].x * sf[q].x + sf[q].y * sf[q].y;
            if (S_f) fqi::store_c(S_f, p * F + f, sf[q]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (pd && lane == 0) pd[p] = e * invF;
}

template <typename T, int NQ = 16>
__device__ __forceinline__ void project_pixel(const T *__restrict__ S, int64_t p, int F, const float2 *__restrict__ Vt,
                                              int k, T *__restrict__ S_f, float *__restrict__ pd, float invF, int lane)
{
    float2 s[NQ];
    project_load<T, NQ>(S, p, F, lane, s);
    project_compute<T, NQ>(s, p, F, Vt, k, S_f, pd, invF, lane);
}

template <typename T, int NQ>
__global__ void __launch_bounds__(256) project_pd_kernel(const T *__restrict__ S, int64_t P, int F,
                                                         const float2 *__restrict__ Vt, const int *__restrict__ k_ptr,
                                                         T *__restrict__ S_f, float *__restrict__ pd)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int k = min(*k_ptr, F);
    const float invF = 1.0f / (float)F;
    // 1.68 GB of FP32 S (2^21 pixels x 100 frames) in 0.58 ms: 43% of HBM
    // bandwidth; loading the next pixel's frames while one is filtered
    // measured the same, so the loop keeps one pixel per warp
    for (int64_t p = warp0; p < P; p += nwarps) project_pixel<T, NQ>(S, p, F, Vt, k, S_f, pd, invF, lane);
}

int pd_blocks(int64_t P);

// the projection for F <= 512 frames with the smallest frames-per-lane count
template <typename T>
fq_status launch_project(const void *S, int64_t P, int F, const float2 *Vt, const int *k, void *S_f, float *pd,
                         cudaStream_t st)
{
    const T *s = (const T *)S;
    T *sf = (T *)S_f;
    const int g = pd_blocks(P);
    if (F <= 32) project_pd_kernel<T, 1><<<g, 256, 0, st>>>(s, P, F, Vt, k, sf, pd);
    else if (F <= 64) project_pd_kernel<T, 2><<<g, 256, 0, st>>>(s, P, F, Vt, k, sf, pd);
    else if (F <= 128) project_pd_kernel<T, 4><<<g, 256, 0, st>>>(s, P, F, Vt, k, sf, pd);
    else if (F <= 256) project_pd_kernel<T, 8><<<g, 256, 0, st>>>(s, P, F, Vt, k, sf, pd);
    else project_pd_kernel<T, 16><<<g, 256, 0, st>>>(s, P, F, Vt, k, sf, pd);
    return fqi::launch_check("projection + power Doppler");
}

// ------------------------------------------------------------- batched --
template <typename T>
__global__ void __launch_bounds__(256) gram_batched_kernel(const fqb::EnsDev *__restrict__ ens, const fqb::StageQueue q)
{
    __shared__ float2 As[kGramTile][kGramTile + 1];
    __shared__ float2 Bs[kGramTile][kGramTile + 1];
    __shared__ int s_buf[2];
    fqb::Item it;
    while (fqb::next_item(q, ens, fqb::ST_GRAM, s_buf, it)) {
        const fqb::EnsDev &e = ens[it.e];
        const int nt = (e.F + kGramTile - 1) / kGramTile;
        gram_tile<T>((const T *)e.iq, e.P, e.F, nt, e.chunk_len, (float2 *)(e.cws + e.cl_part), it.x, it.y, As, Bs);
    }
}

__global__ void __launch_bounds__(256) gram_reduce_batched_kernel(const fqb::EnsDev *__restrict__ ens,
                                                                  const fqb::StageQueue q)
{
    __shared__ int s_buf[2];
    fqb::Item it;
    while (fqb::next_item(q, ens, fqb::ST_GRAM_REDUCE, s_buf, it)) {
        const fqb::EnsDev &e = ens[it.e];
        gram_reduce_at((const float2 *)(e.cws + e.cl_part), e.n_chunks, e.F, (float2 *)(e.cws + e.cl_G),
                       it.x * 256 + threadIdx.x);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) project_batched_kernel(const fqb::EnsDev *__restrict__ ens,
                                                              const fqb::StageQueue q)
{
    __shared__ int s_buf[2];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    fqb::Item it;
    while (fqb::next_item(q, ens, fqb::ST_PROJECT, s_buf, it)) {
        const fqb::EnsDev &e = ens[it.e];
        const int *kk = e.k_used ? e.k_used : (const int *)(e.cws + e.cl_k);
        const int k = min(*kk, e.F);
        const float invF = 1.0f / (float)e.F;
        const int64_t beg = (int64_t)it.x * fqb::kItemPix;
        const int64_t end = beg + fqb::kItemPix < e.P ? beg + fqb::kItemPix : e.P;
        // the frames-per-lane count of the single-ensemble projection, so
        // that both give bit-identical results
        const T *S = (const T *)e.iq;
        const float2 *Vt = (const float2 *)(e.cws + e.cl_Vt);
        for (int64_t p = beg + wid; p < end; p += 8) {
            if (e.F <= 32) project_pixel<T, 1>(S, p, e.F, Vt, k, (T *)nullptr, e.pd, invF, lane);
            else if (e.F <= 64) project_pixel<T, 2>(S, p, e.F, Vt, k, (T *)nullptr, e.pd, invF, lane);
            else if (e.F <= 128) project_pixel<T, 4>(S, p, e.F, Vt, k, (T *)nullptr, e.pd, invF, lane);
            else if (e.F <= 256) project_pixel<T, 8>(S, p, e.F, Vt, k, (T *)nullptr, e.pd, invF, lane);
            else project_pixel<T, 16>(S, p, e.F, Vt, k, (T *)nullptr, e.pd, invF, lane);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) power_doppler_kernel(const T *__restrict__ S, int64_t P, int F,
                                                            float *__restrict__ pd)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp0; p < P; p += nwarps) {
        float e = 0.0f;
        for (int f = lane; f < F; f += 32) {
            float2 v = fqi::load_c(S, p * F + f);
            e += v.x * v.x + v.y * v.y;
        }
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (lane == 0) pd[p] = e / (float)F;
    }
}

// ------------------------------------------------------------- launchers --
template <typename T>
fq_status launch_gram(const void *S, int64_t P, int F, const ClutterLayout &L, char *ws, float2 *G, cudaStream_t st)
{
    int nt = (F + kGramTile - 1) / kGramTile;
    int pairs = nt * (nt + 1) / 2;
    float2 *part = (float2 *)(ws + L.part);
    dim3 grid(pairs, L.n_chunks);
    gram_partial_kernel<T><<<grid, 256, 0, st>>>((const T *)S, P, F, nt, L.chunk_len, part);
    gram_reduce_kernel<<<(F * F + 255) / 256, 256, 0, st>>>(part, L.n_chunks, F, G);
    return fqi::launch_check("fq_casorati_gram");
}

// Gram of gram_mode into G; the tensor-core modes use the L.tc region and
// report a timed-out wait through the status word at ws.
fq_status gram_any(const void *S, int dtype, int64_t P, int F, int gram_mode, const ClutterLayout &L, char *ws,
                   float2 *G, cudaStream_t st)
{
    const int esz = tc_esz(gram_mode);
    if (esz) return fqi::gram_tc(S, dtype, P, F, esz, G, ws + L.tc, (int *)(ws + L.status), st);
    return dtype == FQ_F32 ? launch_gram<float>(S, P, F, L, ws, G, st) : launch_gram<__nv_bfloat16>(S, P, F, L, ws, G, st);
}

fq_status launch_eig(const float2 *G, int F, float2 *big, float2 *hv, float *tau, double *lam, float2 *V, float2 *Vt,
                     int k_cut, double thresh, int *k_out, int *status, cudaStream_t st, int topk_only = 0,
                     float *ii_scr = nullptr)
{
    size_t smem = big ? 0 : sizeof(float2) * (size_t)F * (F + 1) / 2;
    if (smem > 0) {
        // the kernel's static arrays count against the same 48 KB default,
        // so the opt-in is needed for much smaller packed matrices too
        fq_status s = fqi::cuda_check(cudaFuncSetAttribute(eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                           (int)smem), "eig: smem attribute");
        if (s) return s;
    }
    eig_kernel<<<1, kEigThreads, smem, st>>>(G, F, big, hv, tau, lam, V, Vt, k_cut, thresh, k_out, status,
                                             topk_only, ii_scr);
    return fqi::launch_check("fq_hermitian_eig");
}

// ---------------------------------------------------- no-allocation variant --
// Scratch for fq_clutter_svd_noalloc: one fixed array per device that loads
// the library.  Its host-side name is only a stand-in; kernels get the
// device address that cudaGetSymbolAddress returns for the current device.
constexpr size_t kNoallocBytes = (size_t)12 << 20;
constexpr int kNoallocMaxF = 256;
constexpr int kNoallocMaxChunks = 16;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// The workspace layout of the clutter filter with at most max_chunks Gram
// partial sums (fewer pixel chunks, each longer), so that its size depends
// on F only.
ClutterLayout layout_capped(int64_t P, int F, int max_chunks)
{
    ClutterLayout L = layout(P, F);
    if (L.n_chunks <= max_chunks) return L;
    size_t o = 0;
    L.status = o; o += 256;
    L.G = o; o += al256(sizeof(float2) * F * F);
    L.n_chunks = max_chunks;
    int64_t per = (P + L.n_chunks - 1) / L.n_chunks;
    L.chunk_len = (per + kGramTile - 1) / kGramTile * kGramTile;
    L.part = o; o += al256(sizeof(float2) * (size_t)L.n_chunks * F * F);
    L.V = o; o += al256(sizeof(float2) * F * F);
    L.Vt = o; o += al256(sizeof(float2) * F * F);
    L.lam = o; o += al256(sizeof(double) * F);
    L.k = o; o += 256;
    L.hv = o; o += al256(sizeof(float2) * F * F);
    L.tau = o; o += al256(sizeof(float) * F);
    L.big = o; o += eig_in_smem(F) ? 0 : al256(sizeof(float2) * (size_t)F * (F + 1) / 2);
    L.ii = o; o += al256(sizeof(float) * 6 * (size_t)kFastMaxK * F);
    L.tc = o;
    L.total = o;
    return L;
}

// Unique ID of the calling thread's current CUDA context (0 if none), from
// the driver's cuCtxGetCurrent / cuCtxGetId, fetched once through the
// runtime so that the library needs no link to the driver library.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetId)f;
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device.  It is looked
// up (with that device current) the first time and again whenever the
// device's current context has changed since (a device reset destroys the
// context that the cached address belongs to), and cached otherwise.
fq_status noalloc_scratch(char **out)
{
    constexpr int kMaxDevices = 64;
    static void *addr[kMaxDevices] = {};
    static unsigned long long ctx_id[kMaxDevices] = {};
    static std::mutex mu;
    int dev = 0;
    fq_status s = fqi::cuda_check(cudaGetDevice(&dev), "fq_clutter_svd_noalloc: cudaGetDevice");
    if (s) return s;
    FQ_REQUIRE(dev >= 0 && dev < kMaxDevices, FQ_ERR_UNSUPPORTED, "fq_clutter_svd_noalloc: device ordinal %d", dev);
    std::lock_guard<std::mutex> lock(mu);
    const unsigned long long id = current_context_id();
    if (!addr[dev] || id == 0 || id != ctx_id[dev]) {
        void *p = nullptr;
        s = fqi::cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch),
                            "fq_clutter_svd_noalloc: cudaGetSymbolAddress");
        if (s) return s;
        addr[dev] = p;
        ctx_id[dev] = current_context_id();  // the lookup makes the device's context current if it was not
    }
    *out = (char *)addr[dev];
    return FQ_OK;
}

int pd_blocks(int64_t P)
{
    int64_t b = (P + 7) / 8;
    return (int)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

extern "C" {

fq_status fq_gram_workspace_size(int64_t P, int32_t F, int32_t gram_mode, size_t *bytes)
{
    FQ_REQUIRE(bytes && P >= 1 && F >= 2 && F <= 512, FQ_ERR_INVALID_ARG, "fq_gram_workspace_size: bad arguments");
    FQ_REQUIRE(gram_mode >= FQ_GRAM_F32 && gram_mode <= FQ_GRAM_BF16, FQ_ERR_INVALID_ARG,
               "fq_gram_workspace_size: gram_mode %d", gram_mode);
    const int esz = tc_esz(gram_mode);
    if (esz) {
        *bytes = 256 + fqi::gram_tc_workspace_bytes(P, F, esz);  // status word + operands + partials
        return FQ_OK;
    }
    ClutterLayout L = layout(P, F);
    *bytes = al256(sizeof(float2) * (size_t)L.n_chunks * F * F);
    return FQ_OK;
}

fq_status fq_casorati_gram(const void *S, int32_t dtype, int64_t P, int32_t F, int32_t gram_mode, float *G,
                           void *workspace, size_t workspace_bytes, void *stream)
{
    FQ_REQUIRE(S && G && P >= 1 && F >= 2 && F <= 512, FQ_ERR_INVALID_ARG, "fq_casorati_gram: bad arguments");
    FQ_REQUIRE(gram_mode >= FQ_GRAM_F32 && gram_mode <= FQ_GRAM_BF16, FQ_ERR_INVALID_ARG,
               "fq_casorati_gram: gram_mode %d", gram_mode);
    FQ_REQUIRE(dtype == FQ_F32 || dtype == FQ_BF16, FQ_ERR_UNSUPPORTED, "fq_casorati_gram: dtype");
    size_t need = 0;
    fq_gram_workspace_size(P, F, gram_mode, &need);
    FQ_REQUIRE(workspace && workspace_bytes >= need, FQ_ERR_WORKSPACE, "fq_casorati_gram: workspace needs %zu bytes",
               need);
    FQ_REQUIRE(fqi::aligned(workspace, 256) && fqi::aligned(S, 8) && fqi::aligned(G, 8), FQ_ERR_ALIGN,
               "fq_casorati_gram: alignment");
    cudaStream_t st = (cudaStream_t)stream;
    const int esz = tc_esz(gram_mode);
    if (esz) {
        fq_status s = fqi::cuda_check(cudaMemsetAsync(workspace, 0, 256, st), "fq_casorati_gram: status reset");
        if (s) return s;
        return fqi::gram_tc(S, dtype, P, F, esz, (float2 *)G, (char *)workspace + 256, (int *)workspace, st);
    }
    ClutterLayout L = layout(P, F);
    L.part = 0;  // the partials are the only workspace content here
    if (dtype == FQ_F32) return launch_gram<float>(S, P, F, L, (char *)workspace, (float2 *)G, st);
    return launch_gram<__nv_bfloat16>(S, P, F, L, (char *)workspace, (float2 *)G, st);
}

fq_status fq_eig_workspace_size(int32_t F, size_t *bytes)
{
    FQ_REQUIRE(bytes && F >= 1 && F <= 512, FQ_ERR_INVALID_ARG, "fq_eig_workspace_size: F must be in [1, 512]");
    *bytes = eig_only_bytes(F);
    return FQ_OK;
}

fq_status fq_hermitian_eig(const float *G, int32_t F, double *eigvals, float *V, void *workspace,
                           size_t workspace_bytes, void *stream)
{
    FQ_REQUIRE(G && eigvals && V && F >= 1 && F <= 512, FQ_ERR_INVALID_ARG, "fq_hermitian_eig: bad arguments");
    size_t need = eig_only_bytes(F);
    FQ_REQUIRE(workspace && workspace_bytes >= need, FQ_ERR_WORKSPACE, "fq_hermitian_eig: workspace needs %zu bytes",
               need);
    FQ_REQUIRE(fqi::aligned(workspace, 256) && fqi::aligned(G, 8) && fqi::aligned(V, 8), FQ_ERR_ALIGN,
               "fq_hermitian_eig: alignment");
    char *ws = (char *)workspace;
    size_t o = 256;
    float2 *hv = (float2 *)(ws + o); o += al256(sizeof(float2) * F * F);
    float *tau = (float *)(ws + o); o += al256(sizeof(float) * F);
    float2 *Vt = (float2 *)(ws + o); o += al256(sizeof(float2) * F * F);
    int *kk = (int *)(ws + o); o += 256;
    float2 *big = eig_in_smem(F) ? nullptr : (float2 *)(ws + o);
    cudaStream_t st = (cudaStream_t)stream;
    fq_status s = fqi::cuda_check(cudaMemsetAsync(ws, 0, 256, st), "fq_hermitian_eig: status reset");
    if (s) return s;
    return launch_eig((const float2 *)G, F, big, hv, tau, eigvals, (float2 *)V, Vt, 0, 0.0, kk, (int *)ws, st);
}

fq_status fq_clutter_svd_workspace_size(int64_t P, int32_t F, int32_t gram_mode, size_t *bytes)
{
    FQ_REQUIRE(bytes && P >= 1 && F >= 2 && F <= 512, FQ_ERR_INVALID_ARG,
               "fq_clutter_svd_workspace_size: bad arguments");
    FQ_REQUIRE(gram_mode >= FQ_GRAM_F32 && gram_mode <= FQ_GRAM_BF16, FQ_ERR_INVALID_ARG,
               "fq_clutter_svd_workspace_size: gram_mode %d", gram_mode);
    *bytes = layout(P, F, gram_mode).total;
    return FQ_OK;
}

fq_status fq_clutter_svd(const void *iq, int32_t dtype, int64_t P, int32_t F, int32_t k_cut, double energy_thresh,
                         int32_t gram_mode, void *iq_f, float *pd, double *eigvals, int32_t *k_used, void *workspace,
                         size_t workspace_bytes, void *stream)
{
    FQ_REQUIRE(iq && P >= 1 && F >= 2 && F <= 512, FQ_ERR_INVALID_ARG, "fq_clutter_svd: bad arguments");
    FQ_REQUIRE(k_cut <= F, FQ_ERR_INVALID_ARG, "fq_clutter_svd: k_cut %d > F %d", k_cut, F);
    FQ_REQUIRE(k_cut >= 0 || (energy_thresh > 0.0 && energy_thresh <= 1.0), FQ_ERR_INVALID_ARG,
               "fq_clutter_svd: energy_thresh must be in (0, 1] when k_cut < 0");
    FQ_REQUIRE(dtype == FQ_F32 || dtype == FQ_BF16, FQ_ERR_UNSUPPORTED, "fq_clutter_svd: dtype");
    FQ_REQUIRE(gram_mode >= FQ_GRAM_F32 && gram_mode <= FQ_GRAM_BF16, FQ_ERR_INVALID_ARG,
               "fq_clutter_svd: gram_mode %d", gram_mode);
    ClutterLayout L = layout(P, F, gram_mode);
    FQ_REQUIRE(workspace && workspace_bytes >= L.total, FQ_ERR_WORKSPACE,
               "fq_clutter_svd: workspace needs %zu bytes", L.total);
    FQ_REQUIRE(fqi::aligned(workspace, 256) && fqi::aligned(iq, 8) && fqi::aligned(iq_f, 8), FQ_ERR_ALIGN,
               "fq_clutter_svd: alignment");
    char *ws = (char *)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    fq_status s = fqi::cuda_check(cudaMemsetAsync(ws, 0, 256, st), "fq_clutter_svd: status reset");
    if (s) return s;
    float2 *G = (float2 *)(ws + L.G);
    s = gram_any(iq, dtype, P, F, gram_mode, L, ws, G, st);
    if (s) return s;
    double *lam = eigvals ? eigvals : (double *)(ws + L.lam);
    int *kk = k_used ? (int *)k_used : (int *)(ws + L.k);
    float2 *big = eig_in_smem(F) ? nullptr : (float2 *)(ws + L.big);
    s = launch_eig(G, F, big, (float2 *)(ws + L.hv), (float *)(ws + L.tau), lam, (float2 *)(ws + L.V),
                   (float2 *)(ws + L.Vt), k_cut, energy_thresh, kk, (int *)ws, st, 1, (float *)(ws + L.ii));
    if (s) return s;
    if (!iq_f && !pd) return FQ_OK;
    if (dtype == FQ_F32) return launch_project<float>(iq, P, F, (const float2 *)(ws + L.Vt), kk, iq_f, pd, st);
    return launch_project<__nv_bfloat16>(iq, P, F, (const float2 *)(ws + L.Vt), kk, iq_f, pd, st);
}

fq_status fq_power_doppler(const void *iq_f, int32_t dtype, int64_t P, int32_t F, float *pd, void *stream)
{
    FQ_REQUIRE(iq_f && pd && P >= 1 && F >= 1, FQ_ERR_INVALID_ARG, "fq_power_doppler: bad arguments");
    FQ_REQUIRE(fqi::aligned(iq_f, 8), FQ_ERR_ALIGN, "fq_power_doppler: iq_f must be 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == FQ_F32)
        power_doppler_kernel<float><<<pd_blocks(P), 256, 0, st>>>((const float *)iq_f, P, F, pd);
    else if (dtype == FQ_BF16)
        power_doppler_kernel<__nv_bfloat16><<<pd_blocks(P), 256, 0, st>>>((const __nv_bfloat16 *)iq_f, P, F, pd);
    else
        return fqi::set_error(FQ_ERR_UNSUPPORTED, "fq_power_doppler: dtype");
    return fqi::launch_check("fq_power_doppler");
}

fq_status fq_clutter_status(void *workspace, void *stream)
{
    if (!workspace) {  // the built-in array of fq_clutter_svd_noalloc on the current device
        char *ws = nullptr;
        fq_status s = noalloc_scratch(&ws);
        if (s) return s;
        workspace = ws;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int flag = 0;
    fq_status s = fqi::cuda_check(cudaMemcpyAsync(&flag, workspace, sizeof(int), cudaMemcpyDeviceToHost, st),
                                  "fq_clutter_status: read");
    if (s) return s;
    s = fqi::cuda_check(cudaStreamSynchronize(st), "fq_clutter_status: sync");
    if (s) return s;
    s = fqi::cuda_check(cudaMemsetAsync(workspace, 0, sizeof(int), st), "fq_clutter_status: clear");
    if (s) return s;
    if (flag) return fqi::set_error((fq_status)flag, "device solver reported %s", fq_status_string((fq_status)flag));
    return FQ_OK;
}


fq_status fq_clutter_svd_noalloc(const void *iq, int32_t dtype, int64_t P, int32_t F, int32_t k_cut,
                                 double energy_thresh, void *iq_f, float *pd, double *eigvals, int32_t *k_used,
                                 void *stream)
{
    FQ_REQUIRE(iq && P >= 1 && F >= 2, FQ_ERR_INVALID_ARG, "fq_clutter_svd_noalloc: bad arguments");
    FQ_REQUIRE(F <= kNoallocMaxF, FQ_ERR_SHAPE,
               "fq_clutter_svd_noalloc: F = %d frames exceeds the built-in scratch limit of %d frames; "
               "use fq_clutter_svd with a workspace", F, kNoallocMaxF);
    FQ_REQUIRE(k_cut <= F, FQ_ERR_INVALID_ARG, "fq_clutter_svd_noalloc: k_cut %d > F %d", k_cut, F);
    FQ_REQUIRE(k_cut >= 0 || (energy_thresh > 0.0 && energy_thresh <= 1.0), FQ_ERR_INVALID_ARG,
               "fq_clutter_svd_noalloc: energy_thresh must be in (0, 1] when k_cut < 0");
    FQ_REQUIRE(dtype == FQ_F32 || dtype == FQ_BF16, FQ_ERR_UNSUPPORTED, "fq_clutter_svd_noalloc: dtype");
    FQ_REQUIRE(fqi::aligned(iq, 8) && fqi::aligned(iq_f, 8), FQ_ERR_ALIGN, "fq_clutter_svd_noalloc: alignment");
    ClutterLayout L = layout_capped(P, F, kNoallocMaxChunks);
    FQ_REQUIRE(L.total <= kNoallocBytes, FQ_ERR_SHAPE,
               "fq_clutter_svd_noalloc: needs %zu scratch bytes, the built-in array has %zu", L.total, kNoallocBytes);
    char *ws = nullptr;
    fq_status s = noalloc_scratch(&ws);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // the status word must start at zero; everything else is fully rewritten
    s = fqi::cuda_check(cudaMemsetAsync(ws, 0, 256, st), "fq_clutter_svd_noalloc: status reset");
    if (s) return s;
    float2 *G = (float2 *)(ws + L.G);
    s = dtype == FQ_F32 ? launch_gram<float>(iq, P, F, L, ws, G, st) : launch_gram<__nv_bfloat16>(iq, P, F, L, ws, G, st);
    if (s) return s;
    double *lam = eigvals ? eigvals : (double *)(ws + L.lam);
    int *kk = k_used ? (int *)k_used : (int *)(ws + L.k);
    float2 *big = eig_in_smem(F) ? nullptr : (float2 *)(ws + L.big);
    s = launch_eig(G, F, big, (float2 *)(ws + L.hv), (float *)(ws + L.tau), lam, (float2 *)(ws + L.V),
                   (float2 *)(ws + L.Vt), k_cut, energy_thresh, kk, (int *)ws, st, 1, (float *)(ws + L.ii));
    if (s) return s;
    if (!iq_f && !pd) return FQ_OK;
    if (dtype == FQ_F32) return launch_project<float>(iq, P, F, (const float2 *)(ws + L.Vt), kk, iq_f, pd, st);
    return launch_project<__nv_bfloat16>(iq, P, F, (const float2 *)(ws + L.Vt), kk, iq_f, pd, st);
}

}  // extern "C"

namespace fqi {

void clutter_layout_batched(int64_t P, int F, size_t off[10], int *n_chunks, int64_t *chunk_len, size_t *total)
{
    const ClutterLayout L = layout(P, F, FQ_GRAM_F32, true);
    const size_t o[10] = {L.G, L.part, L.V, L.Vt, L.lam, L.k, L.hv, L.tau, L.big, L.ii};
    for (int i = 0; i < 10; ++i) off[i] = o[i];
    *n_chunks = L.n_chunks;
    *chunk_len = L.chunk_len;
    *total = L.total;
}

fq_status batched_gram(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int iq_dtype, cudaStream_t st)
{
    if (iq_dtype == FQ_F32)
        gram_batched_kernel<float><<<fqb::persistent_grid(gram_batched_kernel<float>, 256, 0, items), 256, 0, st>>>(
            ens, q);
    else
        gram_batched_kernel<__nv_bfloat16>
            <<<fqb::persistent_grid(gram_batched_kernel<__nv_bfloat16>, 256, 0, items), 256, 0, st>>>(ens, q);
    return launch_check("batched Gram");
}

fq_status batched_gram_reduce(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, cudaStream_t st)
{
    gram_reduce_batched_kernel<<<fqb::persistent_grid(gram_reduce_batched_kernel, 256, 0, items), 256, 0, st>>>(ens,
                                                                                                               q);
    return launch_check("batched Gram reduce");
}

fq_status batched_eig(const fqb::EnsDev *ens, const int *members, int n, cudaStream_t st)
{
    eig_batched_kernel<<<n, kEigThreads, 0, st>>>(ens, members);
    return launch_check("batched eig");
}

fq_status batched_project(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int iq_dtype, cudaStream_t st)
{
    if (iq_dtype == FQ_F32)
        project_batched_kernel<float>
            <<<fqb::persistent_grid(project_batched_kernel<float>, 256, 0, items), 256, 0, st>>>(ens, q);
    else
        project_batched_kernel<__nv_bfloat16>
            <<<fqb::persistent_grid(project_batched_kernel<__nv_bfloat16>, 256, 0, items), 256, 0, st>>>(ens, q);
    return launch_check("batched projection");
}

}  // namespace fqi
