/*
 * fq_oracle.c -- plain, slow FP64 CPU statement of the uPDI hot path of
 * 3D-FQFlow (arXiv 2509.05464).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this code:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code, header, table or constant with the CUDA
 * library; both read the same seeded inputs and nothing else.
 *
 * Every quantity is evaluated in double precision from its definition, in
 * the order the definition states, with no blocking, fusion or reordering.
 * Build with -ffp-contract=off so that the integer-valued decisions
 * (classification, binning) follow plain IEEE double arithmetic.
 *
 * Parity status of each function is listed in its comment ("pinned by"):
 * the pins live in tests/test_oracle_*.py.
 *
 * Parity unpinned: the absolute RF scale against the paper's
 * frequency-domain PFIELD model (Eq. 1).  The paper prints no echo values,
 * and the narrowband time-domain restatement used here differs from Eq. 1
 * by design (ideal plane-wave transmit, single point per element, no
 * elevation focusing); its internal physics (time of flight, pulse energy,
 * attenuation, directivity, superposition, symmetry) is pinned, and so is
 * its agreement with this file's frequency-domain form in the narrowband
 * limit.  The transmit sum over elements and sub-elements of Eq. 1-2
 * (or_simulate_rf_pfield) is pinned on its own (single-element spectrum,
 * superposition over weights, far-field limit, steered arrival time); the
 * ratio between an ideal unit plane wave and that sum is the free constant.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Probe geometry (Sec. 2.3 / App. D): element centres on the z = 0 plane,
 * x fastest.  Linear arrays have ny = 1.
 * ---------------------------------------------------------------------- */
static void element_pos(int m, int nx, int ny, double px, double py, double *ex, double *ey)
{
    int ix = m % nx, iy = m / nx;
    *ex = ((double)ix - 0.5 * (double)(nx - 1)) * px;
    *ey = ((double)iy - 0.5 * (double)(ny - 1)) * py;
}

/* plane-wave direction for tilts (tx, ty) */
static void pw_dir(double tx, double ty, double u[3])
{
    u[0] = sin(tx);
    u[1] = sin(ty);
    u[2] = sqrt(1.0 - u[0] * u[0] - u[1] * u[1]);
}

/* min over elements of u . e_m: the transmit time origin (first firing) */
static double pw_origin(const double u[3], int nx, int ny, double px, double py)
{
    double best = 1e300;
    for (int m = 0; m < nx * ny; ++m) {
        double ex, ey;
        element_pos(m, nx, ny, px, py, &ex, &ey);
        double d = u[0] * ex + u[1] * ey;
        if (d < best) best = d;
    }
    return best;
}

static double sinc_unnorm(double x) { return x == 0.0 ? 1.0 : sin(x) / x; }

/* ------------------------------------------------------------------------
 * Two-way pulse p(t) = 1/2 (1 + cos(2 pi t / T)) cos(2 pi f0 t), |t| < T/2,
 * T = n_cycles / f0: an n-cycle Hann-windowed tone (the transmit waveform of
 * Eq. 1 restated in time; reading recorded in the design notes).
 * ---------------------------------------------------------------------- */
static double pulse(double t, double f0, double T)
{
    if (fabs(t) >= 0.5 * T) return 0.0;
    return 0.5 * (1.0 + cos(2.0 * OR_PI * t / T)) * cos(2.0 * OR_PI * f0 * t);
}

/* ------------------------------------------------------------------------
 * RF synthesis (Eq. 1 restated as a narrowband time-domain sum; Sec. 2.3,
 * App. D; weak scattering => linear superposition over scatterers):
 *
 *   RF_{a,m}[k] = sum_s A_{s,m,a} p(k/fs - tau_{s,m,a})
 *   tau = (u_a . r_s - min_m' u_a . e_m') / c + |r_s - e_m| / c
 *   A   = R_s * D * exp(-alpha f0 c tau) / |r_s - e_m|
 *   D   = sinc(k0 bx (x_s - x_m)/r) [* sinc(k0 by (y_s - y_m)/r) if ny > 1]
 *
 * pos: float [3][S] (x, y, z rows), amp: float [S]; rf: double [A][M][Ns].
 * If accumulate != 0 the sum is added to rf, otherwise rf is overwritten.
 * Pinned by: single-scatterer closed form (T1), superposition (T3),
 * attenuation ratio, mirror symmetry (T11).
 * ---------------------------------------------------------------------- */
/* one RF line (transmit a, element m) of the sum above, added to line[Ns] */
static void rf_line(int nx, int ny, double px, double py, double wx, double wy, double f0, double fs, double c,
                    double alpha_db_cm_mhz, int n_cycles, int ns, double tilt_x, double tilt_y, int m, int64_t S,
                    const float *pos, const float *amp, double *line)
{
    const double T = (double)n_cycles / f0;
    const double k0 = 2.0 * OR_PI * f0 / c;
    const double alpha_np = alpha_db_cm_mhz * 100.0 / (20.0 / log(10.0)); /* Np / (m MHz) */
    const double f0_mhz = f0 * 1e-6;
    const float *X = pos, *Y = pos + S, *Z = pos + 2 * S;
    double u[3];
    pw_dir(tilt_x, tilt_y, u);
    double origin = pw_origin(u, nx, ny, px, py);
    double ex, ey;
    element_pos(m, nx, ny, px, py, &ex, &ey);
    for (int64_t s = 0; s < S; ++s) {
        double x = X[s], y = Y[s], z = Z[s];
        double dx = x - ex, dy = y - ey, dz = z;
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r == 0.0) continue;
        double path_tx = u[0] * x + u[1] * y + u[2] * z - origin;
        double path = path_tx + r;
        double tau = path / c;
        double D = sinc_unnorm(k0 * 0.5 * wx * dx / r);
        if (ny > 1) D *= sinc_unnorm(k0 * 0.5 * wy * dy / r);
        double A = (double)amp[s] * D * exp(-alpha_np * f0_mhz * path) / r;
        int64_t kmin = (int64_t)ceil((tau - 0.5 * T) * fs);
        int64_t kmax = (int64_t)floor((tau + 0.5 * T) * fs);
        if (kmin < 0) kmin = 0;
        if (kmax > ns - 1) kmax = ns - 1;
        for (int64_t k = kmin; k <= kmax; ++k)
            line[k] += A * pulse((double)k / fs - tau, f0, T);
    }
}

void or_simulate_rf(int nx, int ny, double px, double py, double wx, double wy,
                    double f0, double fs, double c, double alpha_db_cm_mhz, int n_cycles, int ns,
                    int n_ang, const double *tilt_x, const double *tilt_y,
                    int64_t S, const float *pos, const float *amp, int accumulate, double *rf)
{
    const int M = nx * ny;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int am = 0; am < n_ang * M; ++am) {
        int a = am / M, m = am % M;
        double *line = rf + (int64_t)am * ns;
        if (!accumulate)
            for (int k = 0; k < ns; ++k) line[k] = 0.0;
        rf_line(nx, ny, px, py, wx, wy, f0, fs, c, alpha_db_cm_mhz, n_cycles, ns, tilt_x[a], tilt_y[a], m, S,
                pos, amp, line);
    }
}

/* The same sum for a list of lines only: rf[i] (double [n_lines][Ns]) is
 * line lines[i] = a * M + m of or_simulate_rf (overwritten).  For sampled
 * checks of workloads whose full RF is too large for this oracle. */
void or_simulate_rf_lines(int nx, int ny, double px, double py, double wx, double wy,
                          double f0, double fs, double c, double alpha_db_cm_mhz, int n_cycles, int ns,
                          const double *tilt_x, const double *tilt_y, int n_lines, const int32_t *lines,
                          int64_t S, const float *pos, const float *amp, double *rf)
{
    const int M = nx * ny;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < n_lines; ++i) {
        int a = lines[i] / M, m = lines[i] % M;
        double *line = rf + (int64_t)i * ns;
        for (int k = 0; k < ns; ++k) line[k] = 0.0;
        rf_line(nx, ny, px, py, wx, wy, f0, fs, c, alpha_db_cm_mhz, n_cycles, ns, tilt_x[a], tilt_y[a], m, S,
                pos, amp, line);
    }
}

/* ------------------------------------------------------------------------
 * rf2iq (Alg. 3 step 2.3.2.1): mix down by f0 then low-pass:
 *   IQ[k] = 2 sum_{j=-J..J} h_j RF[k-j] exp(-i 2 pi f0 (k-j) / fs)
 * h: Hann-windowed ideal low-pass with cutoff f0, 2J+1 taps with
 * J = 2 round(fs/f0), window w_j = 1/2 (1 + cos(pi j / (J+1))), normalised
 * to sum 1.  Samples outside [0, Ns) are zero.  (The paper does not specify
 * the filter; this reading is recorded in the design notes.)
 * rf: float [n_lines][Ns]; iq: double complex interleaved [n_lines][Ns][2].
 * Pinned by: np.convolve of the mixed signal, pure tone / DC responses.
 * ---------------------------------------------------------------------- */
int or_rf2iq_taps(double f0, double fs, double *h /* [2J+1] or NULL */)
{
    int J = 2 * (int)lround(fs / f0);
    if (h) {
        double sum = 0.0;
        for (int j = -J; j <= J; ++j) {
            double x = 2.0 * f0 / fs * (double)j;            /* normalised-sinc argument */
            double ideal = 2.0 * f0 / fs * (j == 0 ? 1.0 : sin(OR_PI * x) / (OR_PI * x));
            double w = 0.5 * (1.0 + cos(OR_PI * (double)j / (double)(J + 1)));
            h[j + J] = w * ideal;
            sum += h[j + J];
        }
        for (int j = 0; j < 2 * J + 1; ++j) h[j] /= sum;
    }
    return 2 * J + 1;
}

void or_rf2iq(double f0, double fs, int ns, int64_t n_lines, const float *rf, double *iq)
{
    int ntap = or_rf2iq_taps(f0, fs, NULL);
    int J = (ntap - 1) / 2;
    double *h = (double *)malloc(sizeof(double) * ntap);
    or_rf2iq_taps(f0, fs, h);
    #pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < n_lines; ++l) {
        const float *x = rf + l * ns;
        double *o = iq + l * ns * 2;
        for (int k = 0; k < ns; ++k) {
            double re = 0.0, im = 0.0;
            for (int j = -J; j <= J; ++j) {
                int n = k - j;
                if (n < 0 || n >= ns) continue;
                double ph = 2.0 * OR_PI * f0 * (double)n / fs;
                re += h[j + J] * (double)x[n] * cos(ph);
                im -= h[j + J] * (double)x[n] * sin(ph);
            }
            o[2 * k] = 2.0 * re;
            o[2 * k + 1] = 2.0 * im;
        }
    }
    free(h);
}

/* ------------------------------------------------------------------------
 * Delay-and-sum with coherent compounding (Sec. 2.4.1, Alg. 3):
 *   tau_{p,m,a} = (u_a . r_p - min u_a . e) / c + |r_p - e_m| / c
 *   u = tau fs, i = floor(u), phi = u - i,
 *   v = (1 - phi) IQ[i] + phi IQ[i+1]   (0 if i < 0 or i + 1 >= Ns)
 *   IQ(p, f) = (1/A) sum_a sum_m w_m(p) v exp(+i 2 pi f0 tau)
 *   w_m(p) = 1 iff |x_p - x_m| <= z_p / (2 f#) (and the same in y for
 *   matrix arrays), else 0.  This integer decision is taken in binary32 on
 *   the coordinates rounded to float, exactly as the kernel takes it.
 * iq_ch: double complex [F][A][M][Ns][2]; pixels p = (iy*nz + iz)*nx + ix;
 * out: double complex [P][F][2] (Casorati layout: frames contiguous).
 * Pinned by: PSF peak (T2), the paper's explicit DAS-matrix form (T7),
 * mirror symmetry (T11).
 * ---------------------------------------------------------------------- */
void or_das(int nx, int ny, double px, double py, double f0, double fs, double c, int ns,
            int n_ang, const double *tilt_x, const double *tilt_y, int F, const double *iq_ch,
            int gx, int gy, int gz, double x0, double y0, double z0, double dx, double dy,
            double dz, double fnum, double *out)
{
    const int M = nx * ny;
    const int64_t P = (int64_t)gx * gy * gz;
    double *ux = (double *)malloc(sizeof(double) * 4 * n_ang);
    for (int a = 0; a < n_ang; ++a) {
        double u[3];
        pw_dir(tilt_x[a], tilt_y[a], u);
        ux[4 * a] = u[0]; ux[4 * a + 1] = u[1]; ux[4 * a + 2] = u[2];
        ux[4 * a + 3] = pw_origin(u, nx, ny, px, py);
    }
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < P; ++p) {
        int ix = (int)(p % gx);
        int iz = (int)((p / gx) % gz);
        int iy = (int)(p / ((int64_t)gx * gz));
        double x = x0 + ix * dx, y = y0 + iy * dy, z = z0 + iz * dz;
        double *o = out + p * F * 2;
        for (int f = 0; f < 2 * F; ++f) o[f] = 0.0;
        for (int a = 0; a < n_ang; ++a) {
            const double *u = ux + 4 * a;
            double path_tx = u[0] * x + u[1] * y + u[2] * z - u[3];
            for (int m = 0; m < M; ++m) {
                double ex, ey;
                element_pos(m, nx, ny, px, py, &ex, &ey);
                /* aperture decision in binary32, as the kernel takes it:
                   |x_p - x_m| <= z_p / (2 f#) on the rounded coordinates */
                float half = (float)z * (float)(0.5 / fnum);
                if (fabsf((float)x - (float)ex) > half) continue;
                if (ny > 1 && fabsf((float)y - (float)ey) > half) continue;
                double r = sqrt((x - ex) * (x - ex) + (y - ey) * (y - ey) + z * z);
                double tau = (path_tx + r) / c;
                double uu = tau * fs;
                double fi = floor(uu);
                double phi = uu - fi;
                int64_t i = (int64_t)fi;
                if (i < 0 || i + 1 >= ns) continue;
                double ph = 2.0 * OR_PI * f0 * tau;
                double cr = cos(ph), ci = sin(ph);
                for (int f = 0; f < F; ++f) {
                    const double *line = iq_ch + ((((int64_t)f * n_ang + a) * M + m) * ns) * 2;
                    double vr = (1.0 - phi) * line[2 * i] + phi * line[2 * i + 2];
                    double vi = (1.0 - phi) * line[2 * i + 1] + phi * line[2 * i + 3];
                    o[2 * f] += vr * cr - vi * ci;
                    o[2 * f + 1] += vr * ci + vi * cr;
                }
            }
        }
        for (int f = 0; f < 2 * F; ++f) o[f] /= (double)n_ang;
    }
    free(ux);
}

/* ------------------------------------------------------------------------
 * Complex one-sided (Hestenes) Jacobi SVD of a P x F column set, FP64.
 * On return the columns of A hold A V = U Sigma (column norms = singular
 * values) and V (F x F, row-major, complex) is the accumulated rotation,
 * both sorted by decreasing singular value.  A: [P][F][2] row-major.
 * Rotations are applied in the round-robin (tournament) order so that the
 * disjoint pairs of one round can be processed in parallel; the result does
 * not depend on the thread count.
 * ---------------------------------------------------------------------- */
static void rr_pair(int n, int round, int k, int *i, int *j)
{
    /* round-robin schedule over n (even) players: player n-1 fixed */
    int a, b;
    if (k == 0) { a = n - 1; b = round % (n - 1); }
    else {
        a = (round + k) % (n - 1);
        b = (round - k + (n - 1)) % (n - 1);
    }
    *i = a < b ? a : b;
    *j = a < b ? b : a;
}

int or_jacobi_svd(int64_t P, int F, double *A, double *V, double *sigma)
{
    int n = F + (F & 1);
    for (int i = 0; i < F; ++i)
        for (int j = 0; j < F; ++j) {
            V[2 * ((int64_t)i * F + j)] = (i == j) ? 1.0 : 0.0;
            V[2 * ((int64_t)i * F + j) + 1] = 0.0;
        }
    int sweep, converged = 0;
    for (sweep = 0; sweep < 80 && !converged; ++sweep) {
        converged = 1;
        for (int round = 0; round < n - 1; ++round) {
            int changed = 0;
            #pragma omp parallel for schedule(dynamic, 1) reduction(|:changed)
            for (int k = 0; k < n / 2; ++k) {
                int i, j;
                rr_pair(n, round, k, &i, &j);
                if (j >= F) continue;
                double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
                for (int64_t p = 0; p < P; ++p) {
                    double xr = A[2 * (p * F + i)], xi = A[2 * (p * F + i) + 1];
                    double yr = A[2 * (p * F + j)], yi = A[2 * (p * F + j) + 1];
                    al += xr * xr + xi * xi;
                    be += yr * yr + yi * yi;
                    gr += xr * yr + xi * yi; /* conj(x) y */
                    gi += xr * yi - xi * yr;
                }
                double g = sqrt(gr * gr + gi * gi);
                if (g <= 1e-15 * sqrt(al * be) || g == 0.0) continue;
                changed = 1;
                /* phase e^{-i phi} aligns column j with column i */
                double er = gr / g, ei = -gi / g;
                double zeta = (be - al) / (2.0 * g);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int64_t p = 0; p < P; ++p) {
                    double *x = A + 2 * (p * F + i), *y = A + 2 * (p * F + j);
                    double yr = y[0] * er - y[1] * ei, yi = y[0] * ei + y[1] * er;
                    double xr = x[0], xi = x[1];
                    x[0] = cs * xr - sn * yr; x[1] = cs * xi - sn * yi;
                    y[0] = sn * xr + cs * yr; y[1] = sn * xi + cs * yi;
                }
                for (int r = 0; r < F; ++r) {
                    double *x = V + 2 * ((int64_t)r * F + i), *y = V + 2 * ((int64_t)r * F + j);
                    double yr = y[0] * er - y[1] * ei, yi = y[0] * ei + y[1] * er;
                    double xr = x[0], xi = x[1];
                    x[0] = cs * xr - sn * yr; x[1] = cs * xi - sn * yi;
                    y[0] = sn * xr + cs * yr; y[1] = sn * xi + cs * yi;
                }
            }
            if (changed) converged = 0;
        }
    }
    /* singular values = column norms; sort decreasing (selection sort) */
    for (int i = 0; i < F; ++i) {
        double s = 0.0;
        for (int64_t p = 0; p < P; ++p)
            s += A[2 * (p * F + i)] * A[2 * (p * F + i)] + A[2 * (p * F + i) + 1] * A[2 * (p * F + i) + 1];
        sigma[i] = sqrt(s);
    }
    for (int i = 0; i < F; ++i) {
        int best = i;
        for (int j = i + 1; j < F; ++j)
            if (sigma[j] > sigma[best]) best = j;
        if (best != i) {
            double ts = sigma[i]; sigma[i] = sigma[best]; sigma[best] = ts;
            for (int64_t p = 0; p < P; ++p)
                for (int q = 0; q < 2; ++q) {
                    double tv = A[2 * (p * F + i) + q];
                    A[2 * (p * F + i) + q] = A[2 * (p * F + best) + q];
                    A[2 * (p * F + best) + q] = tv;
                }
            for (int r = 0; r < F; ++r)
                for (int q = 0; q < 2; ++q) {
                    double tv = V[2 * ((int64_t)r * F + i) + q];
                    V[2 * ((int64_t)r * F + i) + q] = V[2 * ((int64_t)r * F + best) + q];
                    V[2 * ((int64_t)r * F + best) + q] = tv;
                }
        }
    }
    return converged ? sweep : -sweep;
}

/* ------------------------------------------------------------------------
 * SVD clutter filter and power Doppler (Sec. 2.4.2; Figs. 11-13):
 *   S = U Sigma V^H (Casorati matrix, pixels x frames)
 *   S_f = S - sum_{i<=k} sigma_i u_i v_i^H     (remove the k largest)
 *   k = k_cut if k_cut >= 0, else the smallest k with
 *       sum_{i<=k} sigma_i^2 >= energy_thresh * sum_i sigma_i^2
 *   PD(p) = (1/F) sum_f |S_f(p, f)|^2
 * S: double complex [P][F][2].  Outputs (each nullable): sigma [F],
 * s_f double complex [P][F][2], pd double [P].  Returns k, or -1 on bad k.
 * Pinned by: exact removal of a rank-k clutter with a spectral gap (T5),
 * numpy's SVD, and PD = (1/F) sum_{j>k} sigma_j^2 |u_pj|^2.
 * ---------------------------------------------------------------------- */
int or_svd_filter(int64_t P, int F, const double *S, int k_cut, double energy_thresh,
                  double *sigma_out, double *s_f, double *pd)
{
    if (k_cut > F) return -1;
    double *A = (double *)malloc(sizeof(double) * 2 * P * F);
    double *V = (double *)malloc(sizeof(double) * 2 * (int64_t)F * F);
    double *sg = (double *)malloc(sizeof(double) * F);
    memcpy(A, S, sizeof(double) * 2 * P * F);
    or_jacobi_svd(P, F, A, V, sg);
    int k = k_cut;
    if (k < 0) {
        double tot = 0.0, acc = 0.0;
        for (int i = 0; i < F; ++i) tot += sg[i] * sg[i];
        k = F;
        for (int i = 0; i < F; ++i) {
            acc += sg[i] * sg[i];
            if (acc >= energy_thresh * tot) { k = i + 1; break; }
        }
    }
    if (sigma_out) memcpy(sigma_out, sg, sizeof(double) * F);
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        double e = 0.0;
        for (int f = 0; f < F; ++f) {
            double re = S[2 * (p * F + f)], im = S[2 * (p * F + f) + 1];
            for (int i = 0; i < k; ++i) {
                /* (A V)_{p,i} conj(V_{f,i}) */
                double ar = A[2 * (p * F + i)], ai = A[2 * (p * F + i) + 1];
                double vr = V[2 * ((int64_t)f * F + i)], vi = -V[2 * ((int64_t)f * F + i) + 1];
                re -= ar * vr - ai * vi;
                im -= ar * vi + ai * vr;
            }
            if (s_f) { s_f[2 * (p * F + f)] = re; s_f[2 * (p * F + f) + 1] = im; }
            e += re * re + im * im;
        }
        if (pd) pd[p] = e / (double)F;
    }
    free(A); free(V); free(sg);
    return k;
}

/* Plain SVD access for tests: A [P][F][2] in, U Sigma (in A), V, sigma out. */
int or_svd(int64_t P, int F, double *A, double *V, double *sigma)
{
    return or_jacobi_svd(P, F, A, V, sigma);
}

/* Casorati Gram G = S^H S (F x F complex, row-major [F][F][2]) by its
 * definition G_ij = sum_p conj(S_pi) S_pj.  Pinned by brute force (T6). */
void or_gram(int64_t P, int F, const double *S, double *G)
{
    #pragma omp parallel for schedule(static)
    for (int ij = 0; ij < F * F; ++ij) {
        int i = ij / F, j = ij % F;
        double re = 0.0, im = 0.0;
        for (int64_t p = 0; p < P; ++p) {
            double xr = S[2 * (p * F + i)], xi = S[2 * (p * F + i) + 1];
            double yr = S[2 * (p * F + j)], yi = S[2 * (p * F + j) + 1];
            re += xr * yr + xi * yi;
            im += xr * yi - xi * yr;
        }
        G[2 * ij] = re;
        G[2 * ij + 1] = im;
    }
}

/* Power Doppler of an already filtered ensemble: PD(p) = (1/F) sum_f |S_f|^2 */
void or_power_doppler(int64_t P, int F, const double *s_f, double *pd)
{
    for (int64_t p = 0; p < P; ++p) {
        double e = 0.0;
        for (int f = 0; f < F; ++f)
            e += s_f[2 * (p * F + f)] * s_f[2 * (p * F + f)] + s_f[2 * (p * F + f) + 1] * s_f[2 * (p * F + f) + 1];
        pd[p] = e / (double)F;
    }
}

/* ------------------------------------------------------------------------
 * Scatterer advection (Sec. 2.2.2 steady-velocity-field trajectories in
 * closed form; Poiseuille flow along the vessel centreline):
 *
 *  blood in segment i with flow coordinates (q, xi1, xi2):
 *    v = vmax (1 - (xi1^2 + xi2^2) / R^2)
 *    line: a = q + v t wrapped into [0, L): P = p0 + a a1 + xi1 a2 + xi2 a3
 *    arc:  phi = q + v t / Rc wrapped into [0, phi1):
 *          P = p0 + (Rc + xi1)(cos phi a1 + sin phi a2) + xi2 a3
 *  tissue: P = P0.
 *  then the tissue motion map (applied to both, evaluated with the
 *  unperturbed position Q = P):
 *    rotation about c_r by |omega| t around omega/|omega| (Rodrigues),
 *    plus translation vel t,
 *    plus (1 + g . (Q - c_e)) sum_j A_j sin(2 pi f_j t + phase_j) dir_j.
 *
 * seg table: [n_seg][24] (see workload.segment_table); motion: [40].
 * Output float [3][S].  Pinned by: Poiseuille mean = vmax/2 over a disc and
 * 2 vmax/3 over a stripe (T4), lumen confinement, translation and rotation
 * closed forms (T10).
 * ---------------------------------------------------------------------- */
static double wrap_into(double a, double span)
{
    return a - span * floor(a / span);
}

void or_advect(int64_t S, const float *p0, const int32_t *seg, const float *flow,
               const double *segt, const double *mot, double t, float *out)
{
    int nterm = (int)mot[0];
    const double *om = mot + 34, *cr = mot + 37, *g = mot + 25, *ce = mot + 28, *vel = mot + 31;
    double wn = sqrt(om[0] * om[0] + om[1] * om[1] + om[2] * om[2]);
    double kx = 0, ky = 0, kz = 0, ct = 1.0, st = 0.0;
    if (wn > 0.0) {
        kx = om[0] / wn; ky = om[1] / wn; kz = om[2] / wn;
        ct = cos(wn * t); st = sin(wn * t);
    }
    double dsum[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < nterm; ++j) {
        double sj = mot[1 + j] * sin(2.0 * OR_PI * mot[5 + j] * t + mot[9 + j]);
        for (int d = 0; d < 3; ++d) dsum[d] += sj * mot[13 + 3 * j + d];
    }
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < S; ++s) {
        double P[3];
        int si = seg[s];
        if (si < 0) {
            P[0] = p0[s]; P[1] = p0[S + s]; P[2] = p0[2 * S + s];
        } else {
            const double *sg = segt + 24 * (int64_t)si;
            double q = flow[s], x1 = flow[S + s], x2 = flow[2 * S + s];
            double R = sg[14];
            double v = sg[15] * (1.0 - (x1 * x1 + x2 * x2) / (R * R));
            if ((int)sg[0] == 0) {
                double a = wrap_into(q + v * t, sg[13]);
                for (int d = 0; d < 3; ++d)
                    P[d] = sg[1 + d] + a * sg[4 + d] + x1 * sg[7 + d] + x2 * sg[10 + d];
            } else {
                double phi = wrap_into(q + v * t / sg[16], sg[17]);
                double cp = cos(phi), sp = sin(phi), rr = sg[16] + x1;
                for (int d = 0; d < 3; ++d)
                    P[d] = sg[1 + d] + rr * (cp * sg[4 + d] + sp * sg[7 + d]) + x2 * sg[10 + d];
            }
        }
        double Q[3] = {P[0], P[1], P[2]};
        if (wn > 0.0) {
            double w0 = P[0] - cr[0], w1 = P[1] - cr[1], w2 = P[2] - cr[2];
            double kw = kx * w0 + ky * w1 + kz * w2;
            double c0 = ky * w2 - kz * w1, c1 = kz * w0 - kx * w2, c2 = kx * w1 - ky * w0;
            P[0] = cr[0] + w0 * ct + c0 * st + kx * kw * (1.0 - ct);
            P[1] = cr[1] + w1 * ct + c1 * st + ky * kw * (1.0 - ct);
            P[2] = cr[2] + w2 * ct + c2 * st + kz * kw * (1.0 - ct);
        }
        double gain = 1.0 + (g[0] * (Q[0] - ce[0]) + g[1] * (Q[1] - ce[1]) + g[2] * (Q[2] - ce[2]));
        for (int d = 0; d < 3; ++d) out[d * S + s] = (float)(P[d] + vel[d] * t + gain * dsum[d]);
    }
}

/* ------------------------------------------------------------------------
 * Vessel membership (replaces the band-limited delta projection of App. D,
 * Eqs. 3-5, by an exact distance-to-centreline test):
 *   blood scatterers keep their segment; a tissue scatterer gets the first
 *   segment whose lumen strictly contains it, or -1.
 *   line: w = P - p0, s = w.a1 in [0, L], (w.a2)^2 + (w.a3)^2 < R^2
 *   arc:  w = P - C, x_k = w.a_k; angle in [0, phi1]:
 *         x2 >= 0 if phi1 <= pi (sector test by signs of cross products with
 *         the start (1,0) and end (cos phi1, sin phi1) directions);
 *         (sqrt(x1^2 + x2^2) - Rc)^2 + x3^2 < R^2
 * All arithmetic is IEEE double in the written order (integer result).
 * Also returns the effective amplitude (tissue inside a lumen -> 0).
 * Pinned by: brute-force geometric construction of inside/outside points.
 * ---------------------------------------------------------------------- */
static int inside_seg(const double *sg, double px, double py, double pz)
{
    double w0 = px - sg[1], w1 = py - sg[2], w2 = pz - sg[3];
    double R2 = sg[14] * sg[14];
    if ((int)sg[0] == 0) {
        double s = (w0 * sg[4] + w1 * sg[5]) + w2 * sg[6];
        if (s < 0.0 || s > sg[13]) return 0;
        double q1 = (w0 * sg[7] + w1 * sg[8]) + w2 * sg[9];
        double q2 = (w0 * sg[10] + w1 * sg[11]) + w2 * sg[12];
        return (q1 * q1 + q2 * q2) < R2;
    } else {
        double x1 = (w0 * sg[4] + w1 * sg[5]) + w2 * sg[6];
        double x2 = (w0 * sg[7] + w1 * sg[8]) + w2 * sg[9];
        double x3 = (w0 * sg[10] + w1 * sg[11]) + w2 * sg[12];
        /* start direction (1, 0): cross((1,0),(x1,x2)) = x2 >= 0
           end direction (c1, s1): cross((x1,x2),(c1,s1)) = x1 s1 - x2 c1 >= 0
           (arcs span at most pi) */
        if (x2 < 0.0) return 0;
        if (x1 * sg[19] - x2 * sg[18] < 0.0) return 0;
        double rin = sqrt(x1 * x1 + x2 * x2) - sg[16];
        return (rin * rin + x3 * x3) < R2;
    }
}

void or_classify(int64_t S, const float *pos, const int32_t *seg, int n_seg, const double *segt,
                 const float *amp_in, int32_t *vessel, float *amp_out)
{
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < S; ++s) {
        int v = seg[s];
        if (v < 0) {
            double px = pos[s], py = pos[S + s], pz = pos[2 * S + s];
            for (int i = 0; i < n_seg; ++i)
                if (inside_seg(segt + 24 * (int64_t)i, px, py, pz)) { v = i; break; }
        }
        vessel[s] = v;
        if (amp_out) amp_out[s] = (seg[s] < 0 && v >= 0) ? 0.0f : amp_in[s];
    }
}

/* ------------------------------------------------------------------------
 * Depth binning: b(s) = clamp(floor(((double) z_s - z0) / dz), 0, B - 1);
 * stable counting sort: bin_off[b] = #{s : bin(s) < b}, perm lists the
 * scatterer indices ordered by (bin, index).  Pinned by: numpy's stable
 * argsort and bincount on the same keys.
 * ---------------------------------------------------------------------- */
void or_bin(int64_t S, const float *z, double z0, double dz, int B, int32_t *bin_off, int32_t *perm)
{
    int32_t *key = (int32_t *)malloc(sizeof(int32_t) * (S > 0 ? S : 1));
    for (int b = 0; b <= B; ++b) bin_off[b] = 0;
    for (int64_t s = 0; s < S; ++s) {
        double q = floor(((double)z[s] - z0) / dz);
        int b = q < 0.0 ? 0 : (q > (double)(B - 1) ? B - 1 : (int)q);
        key[s] = b;
        bin_off[b + 1] += 1;
    }
    for (int b = 0; b < B; ++b) bin_off[b + 1] += bin_off[b];
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (B > 0 ? B : 1));
    for (int b = 0; b < B; ++b) fill[b] = bin_off[b];
    for (int64_t s = 0; s < S; ++s) perm[fill[key[s]]++] = (int32_t)s;
    free(fill);
    free(key);
}

/* ------------------------------------------------------------------------
 * Trajectories of a steady gridded velocity field (Sec. 2.2.2:
 * P(t) = P0 + integral_0^t v(P(s)) ds; App. C: scatterers follow the local
 * flow), by the classical fourth-order Runge-Kutta method with the fixed
 * step h = dt / n_sub, with blood scatterers confined to their vessel lumen
 * (Sec. 2.2.2: the vessel geometry constrains the integration).
 *
 *  v(P): trilinear interpolation of the samples v[iz][iy][ix][0..2] (four
 *        floats per sample, the fourth unused) at the grid coordinates
 *        g = (P - origin) / spacing, each clamped to [0, n - 1] (the field
 *        continues constant beyond the grid); the cell is
 *        i = min(floor(g), n - 2) (i = 0 when n = 1), weight f = g - i.
 *  step: k1 = v(P), k2 = v(P + h/2 k1), k3 = v(P + h/2 k2), k4 = v(P + h k3),
 *        P <- P + h/6 (k1 + 2 k2 + 2 k3 + k4).
 *  confinement of a scatterer with 0 <= seg < n_seg, after every step
 *  (segment table as for or_advect):
 *    line: w = P - p0, a = w.a1, x = (w.a2, w.a3); if |x| > R, x <- x R/|x|;
 *          a wrapped into [0, L); P = p0 + a a1 + x1 a2 + x2 a3.
 *    arc:  w = P - C, u_k = w.a_k, phi = atan2(u2, u1),
 *          e = (sqrt(u1^2 + u2^2) - Rc, u3); if |e| > R, e <- e R/|e|;
 *          phi wrapped into [0, phi1);
 *          P = C + (Rc + e1)(cos phi a1 + sin phi a2) + e2 a3.
 *  (the wrap re-injects a scatterer that leaves one end at the other, as
 *  the closed-form advection does.)
 * Output: out[f - f0] = (float) P(f dt) for f = f0 .. f0 + F - 1, P(0) = p0.
 * Pinned by: uniform and linear fields (exact solutions: translation,
 * matrix exponential, rigid rotation), the fourth-order convergence of the
 * step, lumen confinement and axial wrap, constant continuation outside
 * the grid.
 * ---------------------------------------------------------------------- */
static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

static void field_cell(double g, int n, int *i0, int *i1, double *f)
{
    if (n <= 1) { *i0 = 0; *i1 = 0; *f = 0.0; return; }
    g = clampd(g, 0.0, (double)(n - 1));
    int i = (int)floor(g);
    if (i > n - 2) i = n - 2;
    *i0 = i; *i1 = i + 1; *f = g - (double)i;
}

static void field_eval(const float *v, int nx, int ny, int nz, const double *org, const double *sp,
                       const double P[3], double out[3])
{
    int x0, x1, y0, y1, z0, z1;
    double fx, fy, fz;
    field_cell((P[0] - org[0]) / sp[0], nx, &x0, &x1, &fx);
    field_cell((P[1] - org[1]) / sp[1], ny, &y0, &y1, &fy);
    field_cell((P[2] - org[2]) / sp[2], nz, &z0, &z1, &fz);
    for (int c = 0; c < 3; ++c) {
        double vz[2];
        for (int kz = 0; kz < 2; ++kz) {
            int iz = kz ? z1 : z0;
            double vy[2];
            for (int ky = 0; ky < 2; ++ky) {
                int iy = ky ? y1 : y0;
                const float *row = v + (((int64_t)iz * ny + iy) * nx) * 4;
                double a = row[4 * x0 + c], b = row[4 * x1 + c];
                vy[ky] = a + fx * (b - a);
            }
            vz[kz] = vy[0] + fy * (vy[1] - vy[0]);
        }
        out[c] = vz[0] + fz * (vz[1] - vz[0]);
    }
}

static void confine(const double *sg, double P[3])
{
    double w[3] = {P[0] - sg[1], P[1] - sg[2], P[2] - sg[3]};
    double u1 = w[0] * sg[4] + w[1] * sg[5] + w[2] * sg[6];
    double u2 = w[0] * sg[7] + w[1] * sg[8] + w[2] * sg[9];
    double u3 = w[0] * sg[10] + w[1] * sg[11] + w[2] * sg[12];
    double R = sg[14];
    if ((int)sg[0] == 0) {
        double r = sqrt(u2 * u2 + u3 * u3);
        if (r > R) { u2 *= R / r; u3 *= R / r; }
        double a = wrap_into(u1, sg[13]);
        for (int d = 0; d < 3; ++d) P[d] = sg[1 + d] + a * sg[4 + d] + u2 * sg[7 + d] + u3 * sg[10 + d];
    } else {
        double Rc = sg[16];
        double phi = atan2(u2, u1);
        double e1 = sqrt(u1 * u1 + u2 * u2) - Rc, e2 = u3;
        double r = sqrt(e1 * e1 + e2 * e2);
        if (r > R) { e1 *= R / r; e2 *= R / r; }
        phi = wrap_into(phi, sg[17]);
        double cp = cos(phi), s = sin(phi);
        for (int d = 0; d < 3; ++d)
            P[d] = sg[1 + d] + (Rc + e1) * (cp * sg[4 + d] + s * sg[7 + d]) + e2 * sg[10 + d];
    }
}

void or_advect_field(int64_t S, const float *p0, const int32_t *seg, int n_seg, const double *segt,
                     const float *v, int nx, int ny, int nz, const double *origin, const double *spacing,
                     double dt, int n_sub, int f0, int F, float *out)
{
    const double h = dt / (double)n_sub;
    #pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < S; ++s) {
        double P[3] = {p0[s], p0[S + s], p0[2 * S + s]};
        const double *sg = (seg && seg[s] >= 0 && seg[s] < n_seg) ? segt + 24 * (int64_t)seg[s] : NULL;
        for (int f = 0; f < f0 + F; ++f) {
            if (f > 0) {
                for (int j = 0; j < n_sub; ++j) {
                    double k1[3], k2[3], k3[3], k4[3], Q[3];
                    field_eval(v, nx, ny, nz, origin, spacing, P, k1);
                    for (int d = 0; d < 3; ++d) Q[d] = P[d] + 0.5 * h * k1[d];
                    field_eval(v, nx, ny, nz, origin, spacing, Q, k2);
                    for (int d = 0; d < 3; ++d) Q[d] = P[d] + 0.5 * h * k2[d];
                    field_eval(v, nx, ny, nz, origin, spacing, Q, k3);
                    for (int d = 0; d < 3; ++d) Q[d] = P[d] + h * k3[d];
                    field_eval(v, nx, ny, nz, origin, spacing, Q, k4);
                    for (int d = 0; d < 3; ++d) P[d] += h / 6.0 * (k1[d] + 2.0 * k2[d] + 2.0 * k3[d] + k4[d]);
                    if (sg) confine(sg, P);
                }
            }
            if (f >= f0)
                for (int d = 0; d < 3; ++d) out[((int64_t)(f - f0) * 3 + d) * S + s] = (float)P[d];
        }
    }
}

/* ------------------------------------------------------------------------
 * The explicit DAS matrices of Sec. 2.4.1 / Alg. 3 (steps 2.2-2.3): one
 * sparse matrix per transmit, rows = pixels, columns = (element, sample)
 * of the channel IQ, built once and applied to every frame.  Row (a, p)
 * holds, for every element m in the receive aperture with a valid sample
 * pair, the two linear-interpolation weights times the phase rotation of
 * or_das:  (m Ns + i, (1 - phi) e^{i 2 pi f0 tau}), (m Ns + i + 1, phi e^{...}).
 * Rows are numbered a * P + p.  With col == NULL only row_ptr is written
 * (row_ptr[r + 1] - row_ptr[r] = entries of row r, row_ptr[0] = 0); then
 * col [nnz], val [nnz][2] are filled in the same order.
 * Pinned by: applying the matrices (scipy.sparse) equals or_das.
 * ---------------------------------------------------------------------- */
void or_das_matrix(int nx, int ny, double px, double py, double f0, double fs, double c, int ns,
                   int n_ang, const double *tilt_x, const double *tilt_y,
                   int gx, int gy, int gz, double x0, double y0, double z0, double dx, double dy,
                   double dz, double fnum, int64_t *row_ptr, int32_t *col, double *val)
{
    const int M = nx * ny;
    const int64_t P = (int64_t)gx * gy * gz;
    const int64_t R = (int64_t)n_ang * P;
    double *ux = (double *)malloc(sizeof(double) * 4 * n_ang);
    for (int a = 0; a < n_ang; ++a) {
        double u[3];
        pw_dir(tilt_x[a], tilt_y[a], u);
        ux[4 * a] = u[0]; ux[4 * a + 1] = u[1]; ux[4 * a + 2] = u[2];
        ux[4 * a + 3] = pw_origin(u, nx, ny, px, py);
    }
    int64_t *cnt = col ? NULL : (int64_t *)malloc(sizeof(int64_t) * (R > 0 ? R : 1));
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t row = 0; row < R; ++row) {
        int a = (int)(row / P);
        int64_t p = row % P;
        int ix = (int)(p % gx);
        int iz = (int)((p / gx) % gz);
        int iy = (int)(p / ((int64_t)gx * gz));
        double x = x0 + ix * dx, y = y0 + iy * dy, z = z0 + iz * dz;
        const double *u = ux + 4 * a;
        double path_tx = u[0] * x + u[1] * y + u[2] * z - u[3];
        int64_t k = col ? row_ptr[row] : 0;
        for (int m = 0; m < M; ++m) {
            double ex, ey;
            element_pos(m, nx, ny, px, py, &ex, &ey);
            float half = (float)z * (float)(0.5 / fnum);
            if (fabsf((float)x - (float)ex) > half) continue;
            if (ny > 1 && fabsf((float)y - (float)ey) > half) continue;
            double r = sqrt((x - ex) * (x - ex) + (y - ey) * (y - ey) + z * z);
            double tau = (path_tx + r) / c;
            double uu = tau * fs;
            double fi = floor(uu);
            double phi = uu - fi;
            int64_t i = (int64_t)fi;
            if (i < 0 || i + 1 >= ns) continue;
            if (col) {
                double ph = 2.0 * OR_PI * f0 * tau;
                double cr = cos(ph), ci = sin(ph);
                col[k] = (int32_t)(m * ns + i);
                val[2 * k] = (1.0 - phi) * cr;
                val[2 * k + 1] = (1.0 - phi) * ci;
                col[k + 1] = (int32_t)(m * ns + i + 1);
                val[2 * k + 2] = phi * cr;
                val[2 * k + 3] = phi * ci;
            }
            k += 2;
        }
        if (!col) cnt[row] = k;
    }
    if (!col) {
        row_ptr[0] = 0;
        for (int64_t r = 0; r < R; ++r) row_ptr[r + 1] = row_ptr[r] + cnt[r];
        free(cnt);
    }
    free(ux);
}

/* ------------------------------------------------------------------------
 * RF synthesis in the frequency domain (Eq. 1 evaluated per frequency, as
 * Alg. 2 step 2.6 does: wavenumber, attenuation and directivity at each
 * frequency, spectral weights, then the inverse transform), with the same
 * geometry as or_simulate_rf (ideal plane-wave transmit, receive at the
 * element centre):
 *
 *   RF_{a,m}[n] = df sum_s sum_{j=0}^{N/2-1} w_j Re{ S(f_j) A_j e^{i 2 pi f_j (n/fs - tau)} }
 *   A_j = R_s D_j exp(-alpha f_j c tau) / |r_s - e_m|,  D_j = sinc(k_j b sin theta),
 *   f_j = j df, df = fs / N, k_j = 2 pi f_j / c, w_0 = 1, w_j = 2 (j >= 1),
 *   S(f) = Fourier transform of the pulse p(t) of or_simulate_rf:
 *     p = rect_T(t) [1/2 cos(2 pi f0 t) + 1/4 cos(2 pi (f0 + 1/T) t) + 1/4 cos(2 pi (f0 - 1/T) t)]
 *     S(f) = T/2 sum_g c_g [sinc(pi (f - g) T) + sinc(pi (f + g) T)],
 *     (g, c_g) = (f0, 1/2), (f0 + 1/T, 1/4), (f0 - 1/T, 1/4).
 * The sum over frequencies represents the echo periodised with period
 * N / fs (N = n_fft >= Ns; 2 Ns keeps every echo of the record inside one
 * period) and band-limited to fs / 2.  The spectrum of each line is summed
 * over scatterers first, then transformed by a direct inverse sum.
 * rf: double [A][M][Ns].  Pinned by: the discrete spectrum of a single
 * echo (numpy FFT of the output over one full period) equals
 * N df S(f_j) A_j e^{-i 2 pi f_j tau} with S from numerical integration of
 * p(t); superposition.
 * ---------------------------------------------------------------------- */
static double pulse_spectrum(double f, double f0, double T)
{
    const double g[3] = {f0, f0 + 1.0 / T, f0 - 1.0 / T}, c[3] = {0.5, 0.25, 0.25};
    double s = 0.0;
    for (int k = 0; k < 3; ++k)
        s += c[k] * (sinc_unnorm(OR_PI * (f - g[k]) * T) + sinc_unnorm(OR_PI * (f + g[k]) * T));
    return 0.5 * T * s;
}

void or_simulate_rf_freq(int nx, int ny, double px, double py, double wx, double wy,
                         double f0, double fs, double c, double alpha_db_cm_mhz, int n_cycles, int ns,
                         int n_fft, int n_ang, const double *tilt_x, const double *tilt_y,
                         int64_t S, const float *pos, const float *amp, double *rf)
{
    const int M = nx * ny;
    const double T = (double)n_cycles / f0;
    const double alpha_np = alpha_db_cm_mhz * 100.0 / (20.0 / log(10.0)); /* Np / (m MHz) */
    const double df = fs / (double)n_fft;
    const int J = n_fft / 2;
    const float *X = pos, *Y = pos + S, *Z = pos + 2 * S;
    double *Sw = (double *)malloc(sizeof(double) * J);
    for (int j = 0; j < J; ++j) Sw[j] = pulse_spectrum(j * df, f0, T);

    #pragma omp parallel for schedule(dynamic, 1)
    for (int am = 0; am < n_ang * M; ++am) {
        int a = am / M, m = am % M;
        double u[3];
        pw_dir(tilt_x[a], tilt_y[a], u);
        double origin = pw_origin(u, nx, ny, px, py);
        double ex, ey;
        element_pos(m, nx, ny, px, py, &ex, &ey);
        double *Pre = (double *)calloc(J, sizeof(double)), *Pim = (double *)calloc(J, sizeof(double));
        for (int64_t s = 0; s < S; ++s) {
            double x = X[s], y = Y[s], z = Z[s];
            double dx = x - ex, dy = y - ey;
            double r = sqrt(dx * dx + dy * dy + z * z);
            if (r == 0.0) continue;
            double tau = (u[0] * x + u[1] * y + u[2] * z - origin + r) / c;
            for (int j = 0; j < J; ++j) {
                double f = j * df, k = 2.0 * OR_PI * f / c;
                double D = sinc_unnorm(k * 0.5 * wx * dx / r);
                if (ny > 1) D *= sinc_unnorm(k * 0.5 * wy * dy / r);
                double A = (double)amp[s] * D * exp(-alpha_np * f * 1e-6 * c * tau) / r;
                double ph = -2.0 * OR_PI * f * tau;
                Pre[j] += A * cos(ph);
                Pim[j] += A * sin(ph);
            }
        }
        double *line = rf + (int64_t)am * ns;
        for (int n = 0; n < ns; ++n) {
            double t = n / fs, acc = 0.0;
            for (int j = 0; j < J; ++j) {
                double w = j == 0 ? 1.0 : 2.0;
                double ph = 2.0 * OR_PI * j * df * t;
                /* Re{S_j P_j e^{i ph}} with S_j real */
                acc += w * Sw[j] * (Pre[j] * cos(ph) - Pim[j] * sin(ph));
            }
            line[n] = df * acc;
        }
        free(Pre);
        free(Pim);
    }
    free(Sw);
}

/* ------------------------------------------------------------------------
 * RF synthesis with the transmit sum of Eq. 1 and the sub-elements of
 * Eq. 2 (App. D), per frequency like or_simulate_rf_freq (Alg. 2 step 2.6):
 * every element e of the probe transmits with weight W_e (the transmit
 * aperture weighting) and the plane-wave steering delay
 *   dtau_{a,e} = (u_a . e - min_e' u_a . e') / c,
 * each element is split into v sub-elements along x (Eq. 2: the element's
 * pressure is the coherent sum over its sub-elements), and a sub-element q
 * radiates to or receives from a scatterer at distance d the Green's function
 *   g_q(f) = D_q(f) exp(-alpha f d) e^{-i 2 pi f d / c} / d,
 *   D_q(f) = sinc(k (w_x / 2v) (x_s - x_q) / d) [* sinc(k (w_y / 2) (y_s - y_q) / d)],
 *   sub-element centres x_q = x_e + (mu - (v - 1)/2) w_x / v, y_q = y_e.
 *   T_{a,s}(f) = sum_e W_e e^{-i 2 pi f dtau_{a,e}} (1/v) sum_mu g_{e mu}(f)
 *   G_{m,s}(f) = (1/v) sum_mu g_{m mu}(f)
 *   RF_{a,m}[n] = df sum_{j < N/2} w_j Re{ S(f_j) sum_s R_s T_{a,s}(f_j) G_{m,s}(f_j) e^{i 2 pi f_j n / fs} }
 * with f_j, df, w_j, S(f) as in or_simulate_rf_freq; elevation focusing
 * delta(Y, r, k) = 1 (unfocused elements).  apod: double [M] transmit
 * weights; rf: double [A][M][Ns].  Pinned by: the discrete spectrum of a
 * single-element transmit and receive (closed form), superposition over
 * transmit weights, the far-field limit of the sub-element sum, and the
 * arrival time of a steered full-aperture transmit on the array axis.
 * ---------------------------------------------------------------------- */
static void or_green(double x, double y, double z, double qx, double qy, double bx, double by, int matrix,
                     double f, double c, double alpha_np, double *re, double *im)
{
    double dx = x - qx, dy = y - qy;
    double d = sqrt(dx * dx + dy * dy + z * z);
    double k = 2.0 * OR_PI * f / c;
    double D = sinc_unnorm(k * bx * dx / d);
    if (matrix) D *= sinc_unnorm(k * by * dy / d);
    double a = D * exp(-alpha_np * f * 1e-6 * d) / d;
    *re = a * cos(-k * d);
    *im = a * sin(-k * d);
}

void or_simulate_rf_pfield(int nx, int ny, double px, double py, double wx, double wy,
                           double f0, double fs, double c, double alpha_db_cm_mhz, int n_cycles, int ns,
                           int n_fft, int n_ang, const double *tilt_x, const double *tilt_y, const double *apod,
                           int n_sub, int64_t S, const float *pos, const float *amp, double *rf)
{
    const int M = nx * ny;
    const int v = n_sub;
    const int matrix = ny > 1;
    const double T = (double)n_cycles / f0;
    const double alpha_np = alpha_db_cm_mhz * 100.0 / (20.0 / log(10.0)); /* Np / (m MHz) */
    const double df = fs / (double)n_fft;
    const int J = n_fft / 2;
    const double bx = 0.5 * wx / v, by = 0.5 * wy;
    const float *X = pos, *Y = pos + S, *Z = pos + 2 * S;
    double *Sw = (double *)malloc(sizeof(double) * J);
    for (int j = 0; j < J; ++j) Sw[j] = pulse_spectrum(j * df, f0, T);
    double *Tre = (double *)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1) * J);
    double *Tim = (double *)malloc(sizeof(double) * (size_t)(S > 0 ? S : 1) * J);

    for (int a = 0; a < n_ang; ++a) {
        double u[3];
        pw_dir(tilt_x[a], tilt_y[a], u);
        double origin = pw_origin(u, nx, ny, px, py);
        /* transmit field at every scatterer and frequency */
        #pragma omp parallel for schedule(dynamic, 16)
        for (int64_t s = 0; s < S; ++s) {
            double x = X[s], y = Y[s], z = Z[s];
            for (int j = 0; j < J; ++j) {
                double f = j * df, tr = 0.0, ti = 0.0;
                for (int e = 0; e < M; ++e) {
                    if (apod[e] == 0.0) continue;
                    double ex, ey;
                    element_pos(e, nx, ny, px, py, &ex, &ey);
                    double dtau = (u[0] * ex + u[1] * ey - origin) / c;
                    double sr = 0.0, si = 0.0;
                    for (int mu = 0; mu < v; ++mu) {
                        double qx = ex + ((double)mu - 0.5 * (v - 1)) * wx / v;
                        double gr, gi;
                        or_green(x, y, z, qx, ey, bx, by, matrix, f, c, alpha_np, &gr, &gi);
                        sr += gr;
                        si += gi;
                    }
                    double w = apod[e] / v;
                    double ph = -2.0 * OR_PI * f * dtau;
                    double cr = cos(ph), ci = sin(ph);
                    tr += w * (sr * cr - si * ci);
                    ti += w * (sr * ci + si * cr);
                }
                Tre[s * J + j] = tr;
                Tim[s * J + j] = ti;
            }
        }
        /* receive per element, then the inverse transform */
        #pragma omp parallel for schedule(dynamic, 1)
        for (int m = 0; m < M; ++m) {
            double ex, ey;
            element_pos(m, nx, ny, px, py, &ex, &ey);
            double *Pre = (double *)calloc(J, sizeof(double)), *Pim = (double *)calloc(J, sizeof(double));
            for (int64_t s = 0; s < S; ++s) {
                double x = X[s], y = Y[s], z = Z[s];
                double R = (double)amp[s];
                for (int j = 0; j < J; ++j) {
                    double f = j * df, gr = 0.0, gi = 0.0;
                    for (int mu = 0; mu < v; ++mu) {
                        double qx = ex + ((double)mu - 0.5 * (v - 1)) * wx / v;
                        double hr, hi;
                        or_green(x, y, z, qx, ey, bx, by, matrix, f, c, alpha_np, &hr, &hi);
                        gr += hr;
                        gi += hi;
                    }
                    gr /= v;
                    gi /= v;
                    double tr = Tre[s * J + j], ti = Tim[s * J + j];
                    Pre[j] += R * (tr * gr - ti * gi);
                    Pim[j] += R * (tr * gi + ti * gr);
                }
            }
            double *line = rf + ((int64_t)a * M + m) * ns;
            for (int n = 0; n < ns; ++n) {
                double t = n / fs, acc = 0.0;
                for (int j = 0; j < J; ++j) {
                    double w = j == 0 ? 1.0 : 2.0;
                    double ph = 2.0 * OR_PI * j * df * t;
                    acc += w * Sw[j] * (Pre[j] * cos(ph) - Pim[j] * sin(ph));
                }
                line[n] = df * acc;
            }
            free(Pre);
            free(Pim);
        }
    }
    free(Tre);
    free(Tim);
    free(Sw);
}
