/*
 * fq.h -- C ABI of the GB300 (sm_103a) uPDI hot path of 3D-FQFlow
 * (arXiv 2509.05464): scatterer advection, vessel membership, depth binning,
 * pulse-echo RF synthesis, rf2iq, plane-wave delay-and-sum compounding, the
 * SVD clutter filter and power Doppler.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Plain C types only.  "device" pointers are CUDA device (or managed)
 *    memory owned by the caller; "host" pointers are ordinary host memory
 *    read during the call only.  The library never allocates device memory:
 *    scratch comes from a caller-provided workspace whose size the matching
 *    *_workspace_size call returns (workspace pointers must be 256-byte
 *    aligned).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call
 *    only enqueues work on that stream and returns; outputs are valid once
 *    the stream has reached that point.  Calls may be captured into CUDA
 *    graphs unless stated otherwise.
 *  - Inputs are never modified.  Outputs are fully overwritten unless a flag
 *    says otherwise.
 *  - Every call returns an fq_status.  On failure nothing has been enqueued
 *    (argument errors) or the CUDA error is reported (FQ_ERR_CUDA);
 *    fq_last_error() gives a message for the calling host thread.  No call
 *    aborts, exits, throws or traps.
 *  - Units are SI (m, s, Hz), angles in radians.
 *  - Complex arrays are interleaved (re, im) pairs of the element type.
 *  - Element m of a probe sits at x = (ix - (nx-1)/2) pitch_x,
 *    y = (iy - (ny-1)/2) pitch_y, z = 0, with m = iy * nx + ix.
 *    Linear arrays have ny = 1 (no elevation directivity).
 *  - Pixel p of a grid sits at (x0 + ix dx, y0 + iy dy, z0 + iz dz) with
 *    p = (iy * nz + iz) * nx + ix.
 */
#ifndef FQ_H
#define FQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fq_status {
    FQ_OK = 0,
    FQ_ERR_INVALID_ARG = 1, /* null pointer, bad enum, negative size ... */
    FQ_ERR_SHAPE = 2,       /* sizes out of the supported range */
    FQ_ERR_ALIGN = 3,       /* pointer not aligned as documented */
    FQ_ERR_WORKSPACE = 4,   /* workspace missing or too small */
    FQ_ERR_CUDA = 5,        /* a CUDA runtime error (message has details) */
    FQ_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out */
    FQ_ERR_NUMERICAL = 7,   /* an iterative solver did not converge */
    FQ_ERR_UNSUPPORTED = 8  /* valid request the library does not implement */
} fq_status;

typedef enum fq_dtype {
    FQ_F32 = 0,  /* IEEE binary32 */
    FQ_BF16 = 1, /* bfloat16 storage, FP32 arithmetic (8 significant bits) */
    FQ_F16 = 2   /* binary16 storage, FP32 arithmetic (11 significant bits);
                    magnitudes above 65504 are stored as +-65504.  Accepted
                    for RF (fq_simulate_rf, fq_rf2iq input) and channel IQ
                    (fq_rf2iq output, fq_das / fq_beamform_das ch_dtype). */
} fq_dtype;

typedef enum fq_gram_mode {
    FQ_GRAM_F32 = 0,  /* FP32 FMA Gram (CUDA cores) */
    FQ_GRAM_TF32 = 1, /* TF32 operands on tcgen05 tensor cores, FP32 accumulate */
    FQ_GRAM_BF16 = 2  /* BF16 operands on tcgen05 tensor cores, FP32 accumulate */
} fq_gram_mode;

enum { FQ_SEG_LINE = 0, FQ_SEG_ARC = 1 };
enum { FQ_MAX_SEGMENTS = 128, FQ_MAX_ANGLES = 64, FQ_MAX_MOTION_TERMS = 4 };

/* Transducer and medium (Sec. 2.3, App. D; Eq. 1 parameters).
 * The two-way pulse is p(t) = 1/2 (1 + cos(2 pi t / T)) cos(2 pi f0 t) for
 * |t| < T/2, T = n_cycles / f0. */
typedef struct fq_probe {
    int32_t nx, ny;             /* elements along x and y (ny = 1: linear) */
    double pitch_x, pitch_y;    /* element pitch (m) */
    double width_x, width_y;    /* element width (m); directivity half-width b = width/2 */
    double f0;                  /* centre frequency (Hz) */
    double fs;                  /* sampling frequency (Hz) */
    double c;                   /* speed of sound (m/s) */
    double alpha_db_cm_mhz;     /* amplitude attenuation (dB / cm / MHz) */
    int32_t n_cycles;           /* pulse length in cycles */
    int32_t n_samples;          /* samples per channel, Ns */
} fq_probe;

/* Plane-wave transmits: direction u = (sin tx, sin ty, sqrt(1 - sin^2 tx - sin^2 ty));
 * time zero is when the first element fires. Arrays are host memory. */
typedef struct fq_tx {
    int32_t n_angles;           /* 1 .. FQ_MAX_ANGLES */
    const double *tilt_x;       /* host [n_angles] */
    const double *tilt_y;       /* host [n_angles] */
} fq_tx;

/* Reconstruction grid and receive aperture (f-number). */
typedef struct fq_grid {
    int32_t nx, ny, nz;
    double x0, y0, z0;
    double dx, dy, dz;
    double fnumber;             /* element m is used for pixel p iff |x_p - x_m| <= z_p / (2 f#) */
} fq_grid;

/* One vessel piece with Poiseuille flow v(rho) = vmax (1 - rho^2 / radius^2).
 * (a1, a2, a3) is a right-handed orthonormal frame.  line: p0 = start,
 * a1 = axis, centreline p0 + s a1, s in [0, length).  arc: p0 = centre,
 * centreline p0 + arc_radius (cos phi a1 + sin phi a2), phi in [0, phi1),
 * phi1 <= pi, arc_end = (cos phi1, sin phi1). */
typedef struct fq_segment {
    int32_t kind;               /* FQ_SEG_LINE or FQ_SEG_ARC */
    double p0[3];
    double a1[3], a2[3], a3[3];
    double length;              /* line only */
    double radius;              /* lumen radius */
    double vmax;                /* centreline speed (m/s) */
    double arc_radius;          /* arc only */
    double phi1;                /* arc only: angular span */
    double arc_end[2];          /* arc only: (cos phi1, sin phi1) */
} fq_segment;

typedef struct fq_flow {
    int32_t n_seg;              /* 0 .. FQ_MAX_SEGMENTS */
    const fq_segment *seg;      /* host [n_seg] */
} fq_flow;

/* Tissue motion (Sec. 2.2.2, Sec. 3.2): rigid rotation by |omega| t about
 * rot_center, translation vel t, and a periodic displacement
 * (1 + g.(Q - elastic_center)) sum_j amp_j sin(2 pi freq_j t + phase_j) dir_j
 * evaluated at the unperturbed position Q. */
typedef struct fq_motion {
    int32_t n_terms;            /* 0 .. FQ_MAX_MOTION_TERMS */
    double amp[4], freq[4], phase[4];
    double dir[4][3];
    double elastic_grad[3];
    double elastic_center[3];
    double vel[3];
    double omega[3];
    double rot_center[3];
} fq_motion;

/* ------------------------------------------------------------------ */
/* library information                                                 */
/* ------------------------------------------------------------------ */

/* Message of the last failing call on this host thread ("" if none). */
const char *fq_last_error(void);
/* Static name of a status code. */
const char *fq_status_string(fq_status s);
/* ABI version (major * 10000 + minor * 100 + patch). */
int32_t fq_version(void);

/* ------------------------------------------------------------------ */
/* a1: scatterer advection                                              */
/* ------------------------------------------------------------------ */

/* Positions of S scatterers at the frame times t_f = t0 + f dt, f < n_frames
 * (Sec. 2.2.2: trajectories of a steady velocity field, here in closed form;
 * App. C: scatterers follow the local flow velocity).
 *   blood (seg_id >= 0), flow coordinates (q, xi1, xi2):
 *     v = vmax (1 - (xi1^2 + xi2^2) / R^2)
 *     line: a = q + v t wrapped into [0, length), P = p0 + a a1 + xi1 a2 + xi2 a3
 *     arc:  phi = q + v t / arc_radius wrapped into [0, phi1),
 *           P = p0 + (arc_radius + xi1)(cos phi a1 + sin phi a2) + xi2 a3
 *   tissue (seg_id = -1): P = p0.
 * Then the tissue motion map is applied to every scatterer.
 *   p0        device float [3][S]  initial positions (x row, y row, z row)
 *   seg_id    device int32 [S]     segment index or -1
 *   flow_coord device float [3][S] (q, xi1, xi2) rows, read for blood only
 *   pos_out   device float [n_frames][3][S]
 * Arithmetic is FP64 (wrap decisions bit-identical to IEEE double).
 * Errors: FQ_ERR_INVALID_ARG (null pointer, S < 0, n_frames < 1, seg_id
 * outside [-1, n_seg) is not checked on the device: such scatterers are
 * treated as tissue), FQ_ERR_SHAPE (n_seg or n_terms above the maximum). */
fq_status fq_advect_scatterers(const float *p0, const int32_t *seg_id, const float *flow_coord,
                               int64_t S, const fq_flow *flow, const fq_motion *motion,
                               double t0, double dt, int32_t n_frames, float *pos_out,
                               void *stream);

/* Trajectories of a steady gridded velocity field (Sec. 2.2.2: the
 * position is P(t) = P0 + integral_0^t v(P(s)) ds for a user-defined steady
 * field v(x, y, z), and the vessel geometry confines the intravascular
 * scatterers; App. C: scatterers follow the local flow).  The paper
 * integrates with an adaptive ODE23 (PROTEUS); this call uses the classical
 * fourth-order Runge-Kutta method with the fixed step h = dt / n_sub:
 *   k1 = v(P), k2 = v(P + h/2 k1), k3 = v(P + h/2 k2), k4 = v(P + h k3),
 *   P <- P + h/6 (k1 + 2 k2 + 2 k3 + k4).
 * v(P) is the trilinear interpolation of the samples at the grid
 * coordinates g = (P - origin) / spacing, each clamped to [0, n - 1] (the
 * field continues constant beyond the grid; an axis with n = 1 is
 * constant along it).  After every step a scatterer with
 * 0 <= seg_id < n_seg is confined to that segment's lumen and re-injected
 * at the other end when it leaves one (fq_segment frame (a1, a2, a3)):
 *   line: a = (P - p0).a1, x = ((P - p0).a2, (P - p0).a3); |x| > radius ->
 *         x radius / |x|; a wrapped into [0, length).
 *   arc:  u_k = (P - p0).a_k, phi = atan2(u2, u1), e = (|(u1, u2)| - arc_radius, u3);
 *         |e| > radius -> e radius / |e|; phi wrapped into [0, phi1).
 * Other scatterers (seg_id NULL, < 0 or >= n_seg) move freely.
 *   p0       device float [3][S]   positions at t = 0
 *   seg_id   device int32 [S] or NULL
 *   grid     host fq_vfield (sample counts, origin, spacing)
 *   v        device float [nz][ny][nx][4] (vx, vy, vz, unused) in m/s, 16-byte aligned
 *   pos_out  device float [n_frames][3][S]: P(f dt) for f = first_frame ..
 *            first_frame + n_frames - 1 (P(0) = p0)
 * Arithmetic is binary32 (the displacement from p0 is accumulated, not the
 * position).  Errors: FQ_ERR_INVALID_ARG (null pointer, S < 0,
 * n_frames < 1, first_frame < 0, n_sub < 1, dt <= 0, a segment with no
 * extent), FQ_ERR_SHAPE (a grid axis with n < 1 or spacing <= 0, more than
 * 2^31 samples, n_seg above the maximum), FQ_ERR_ALIGN (v). */
typedef struct fq_vfield {
    int32_t nx, ny, nz;         /* samples per axis (>= 1) */
    double x0, y0, z0;          /* position of sample (0, 0, 0) (m) */
    double dx, dy, dz;          /* spacing (m) */
} fq_vfield;

fq_status fq_advect_field(const float *p0, const int32_t *seg_id, int64_t S, const fq_flow *flow,
                          const fq_vfield *grid, const float *v, double dt, int32_t n_sub,
                          int32_t first_frame, int32_t n_frames, float *pos_out, void *stream);

/* ------------------------------------------------------------------ */
/* RF synthesis in the frequency domain (Eq. 1 per frequency, Alg. 2)   */
/* ------------------------------------------------------------------ */

/* Eq. 1 evaluated at each frequency of the transform grid (Alg. 2 step
 * 2.6: wavenumber, attenuation and directivity per frequency, spectral
 * weights, then the inverse transform), with the geometry of
 * fq_simulate_rf (ideal plane-wave transmit, receive at the element
 * centre):
 *   RF[f][a][m][n] = df sum_s sum_{j < N/2} w_j Re{ S(f_j) A_j e^{i 2 pi f_j (n/fs - tau)} },
 *   A_j = R_s D_j exp(-alpha f_j c tau) / |r_s - e_m|, D_j = sinc(k_j b sin theta)
 *   (matrix arrays: the product of the x and y factors), f_j = j df,
 *   df = fs / N, w_0 = 1, w_j = 2, S = Fourier transform of the pulse of
 *   fq_probe, N = n_fft (a power of two, n_samples <= N <= 8192; 2
 *   n_samples keeps every echo of the record inside one period of the
 *   transform).  Compared with fq_simulate_rf it drops the narrowband
 *   approximation (attenuation and directivity at f0) and adds the band
 *   limit fs / 2.
 *   pos device float [n_frames][3][S], amp device float [S],
 *   rf device [n_frames][A][M][n_samples] in out_dtype (FQ_F32 or FQ_BF16),
 *   workspace device, 256-byte aligned, fq_simulate_rf_freq_workspace_size
 *   bytes (the spectra [n_frames][A][M][N/2] complex and the weights).
 * Errors: FQ_ERR_INVALID_ARG, FQ_ERR_SHAPE (n_fft, sizes), FQ_ERR_UNSUPPORTED
 * (out_dtype), FQ_ERR_WORKSPACE, FQ_ERR_ALIGN. */
fq_status fq_simulate_rf_freq_workspace_size(const fq_probe *probe, const fq_tx *tx, int32_t n_frames,
                                             int32_t n_fft, size_t *bytes);
fq_status fq_simulate_rf_freq(const fq_probe *probe, const fq_tx *tx, const float *pos, const float *amp,
                              int64_t S, int32_t n_frames, int32_t n_fft, int32_t out_dtype, void *rf,
                              void *workspace, size_t workspace_bytes, void *stream);

/* Eq. 1 with its transmit sum over elements and Eq. 2's sub-elements (App.
 * D; Alg. 2 steps 2.2 and 2.6), per frequency like fq_simulate_rf_freq:
 *   RF[f][a][m][n] = df sum_j w_j Re{ S(f_j) sum_s R_s T_{a,s}(f_j) G_{m,s}(f_j) e^{i 2 pi f_j n / fs} }
 *   T_{a,s}(f) = sum_e W_e e^{-i 2 pi f dtau_{a,e}} (1/v) sum_{mu < v} g_{e mu,s}(f)   (transmit)
 *   G_{m,s}(f) = (1/v) sum_{mu < v} g_{m mu,s}(f)                                       (receive)
 *   g_{q,s}(f) = D_q(f) exp(-alpha f d) e^{-i 2 pi f d / c} / d,  d = |r_s - q|,
 *   D_q(f) = sinc(k (width_x / 2v) (x_s - x_q) / d) [* sinc(k (width_y / 2) (y_s - y_q) / d)],
 *   dtau_{a,e} = (u_a . e - min_e' u_a . e') / c  (plane-wave steering delays),
 *   sub-element centres x_q = x_e + (mu - (v - 1)/2) width_x / v, y_q = y_e.
 * S(f), w_j, df, f_j as for fq_simulate_rf_freq; elevation focusing is
 * not modelled (unfocused elements).
 *   apod    host double [M] transmit weights W_e, or NULL (all 1)
 *   n_sub   sub-elements per element v, 1 .. 8 (M v <= 4096)
 *   pos     device float [n_frames][3][S], amp device float [S]
 *   rf      device [n_frames][A][M][n_samples] of out_dtype (FQ_F32 or FQ_BF16)
 *   workspace device, 256-byte aligned, fq_simulate_rf_pfield_workspace_size
 *           bytes (the spectra, one transmit field [S][N/2] complex, tables).
 * The call synchronises `stream` once after uploading its host tables.
 * Errors: FQ_ERR_INVALID_ARG, FQ_ERR_SHAPE (n_fft, M v), FQ_ERR_UNSUPPORTED
 * (out_dtype), FQ_ERR_WORKSPACE, FQ_ERR_ALIGN. */
fq_status fq_simulate_rf_pfield_workspace_size(const fq_probe *probe, const fq_tx *tx, int64_t S, int32_t n_frames,
                                               int32_t n_fft, int32_t n_sub, size_t *bytes);
fq_status fq_simulate_rf_pfield(const fq_probe *probe, const fq_tx *tx, const double *apod, int32_t n_sub,
                                const float *pos, const float *amp, int64_t S, int32_t n_frames, int32_t n_fft,
                                int32_t out_dtype, void *rf, void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* the paper's explicit DAS-matrix route (Sec. 2.4.1, Alg. 3)           */
/* ------------------------------------------------------------------ */

/* One sparse matrix per transmit, rows = pixels, columns = (element,
 * sample) of the channel IQ, computed once and applied to every frame (Alg.
 * 3 steps 2.2-2.4).  Row a * P + p holds, for every element m in the
 * receive aperture with a valid sample pair (i, i + 1) at u = tau fs
 * (i = floor u, phi = u - i), the entries
 *   (m Ns + i, (1 - phi) e^{i 2 pi f0 tau}) and (m Ns + i + 1, phi e^{i 2 pi f0 tau}),
 * with the same aperture decision and delays as fq_das, so that
 *   iq[p][f] = (1/A) sum_a sum_k val[k] iq_ch[a][col[k]][f]   equals fq_das.
 * Build in two calls: fq_das_matrix_count writes the exclusive row offsets
 * row_ptr (device int64 [A P + 1]; nnz = row_ptr[A P], read it back to
 * size col and val), fq_das_matrix_fill writes col (device int32 [nnz]) and
 * val (device float [nnz][2], 8-byte aligned).  The library keeps fq_das as
 * its hot path (it recomputes delays instead of storing the matrices:
 * 627 MB for the 2D compounded workload, ~470 GB for the 3D one).
 * Errors: FQ_ERR_INVALID_ARG, FQ_ERR_SHAPE (sizes, elements x samples
 * beyond int32), FQ_ERR_WORKSPACE, FQ_ERR_ALIGN. */
fq_status fq_das_matrix_workspace_size(const fq_tx *tx, const fq_grid *grid, size_t *bytes);
fq_status fq_das_matrix_count(const fq_probe *probe, const fq_tx *tx, const fq_grid *grid,
                              int64_t *row_ptr, void *workspace, size_t workspace_bytes, void *stream);
fq_status fq_das_matrix_fill(const fq_probe *probe, const fq_tx *tx, const fq_grid *grid,
                             const int64_t *row_ptr, int32_t *col, float *val, void *stream);
/* Applies the matrices to the channel IQ of fq_rf2iq ([A M][Ns][F_pad][2],
 * F_pad = fq_frame_pad(n_frames)): iq device [P][n_frames][2].  At most 416
 * frames (FQ_ERR_UNSUPPORTED beyond). */
fq_status fq_das_matrix_apply(const int64_t *row_ptr, const int32_t *col, const float *val, int32_t A,
                              int64_t P, int32_t M, int32_t ns, const void *iq_ch, int32_t ch_dtype,
                              int32_t n_frames, int32_t iq_dtype, void *iq, void *stream);

/* ------------------------------------------------------------------ */
/* display and image quality (Sec. 5.2, 5.3, 6.1)                       */
/* ------------------------------------------------------------------ */

/* Workspace for fq_log_compress / fq_bmode (any H, W) and
 * fq_image_quality (images of H x W pixels). */
fq_status fq_post_workspace_size(int32_t H, int32_t W, size_t *bytes);

/* Logarithmic compression and dynamic-range display (Sec. 5.2):
 *   out[i] = clamp((g log10(in[i] / max_j in[j]) + dr_db) / dr_db, 0, 1),
 * g = 10 for powers (power Doppler, power != 0), 20 for amplitudes;
 * in[i] <= 0 gives 0, an all-zero image all 0.  The paper shows B-mode over
 * 75 dB and uPDI over 60 dB (Sec. 6.1).
 *   in, out   device float [n]
 *   workspace device, 256-byte aligned, fq_post_workspace_size bytes
 * Errors: FQ_ERR_INVALID_ARG (null pointer, n < 0, dr_db <= 0),
 * FQ_ERR_ALIGN. */
fq_status fq_log_compress(const float *in, int64_t n, int32_t power, double dr_db, float *out,
                          void *workspace, void *stream);

/* B-mode of one frame of a Casorati matrix (Sec. 5.2): the envelope
 * |S[p, frame]| compressed as above with g = 20.
 *   iq   device [P][F][2] (re, im) in dtype FQ_F32 or FQ_BF16
 *   out  device float [P]
 * Errors: FQ_ERR_INVALID_ARG (frame outside [0, F), ...), FQ_ERR_UNSUPPORTED
 * (dtype), FQ_ERR_ALIGN. */
fq_status fq_bmode(const void *iq, int32_t dtype, int64_t P, int32_t F, int32_t frame, double dr_db,
                   float *out, void *workspace, void *stream);

/* Maximum-intensity projection of a volume (Sec. 6.1, Fig. 9d):
 *   vol device float [nz][ny][nx]; axis 0 (x) -> out [nz][ny],
 *   axis 1 (y) -> out [nz][nx], axis 2 (z) -> out [ny][nx].
 * Errors: FQ_ERR_INVALID_ARG (size < 1, axis outside {0, 1, 2}, null). */
fq_status fq_mip(const float *vol, int32_t nx, int32_t ny, int32_t nz, int32_t axis, float *out,
                 void *stream);

/* Image quality of x against the reference y (Sec. 5.3: MSE, PSNR, SSIM),
 * both device float [H][W] with data range L:
 *   out[0] = MSE = mean (x - y)^2, out[1] = PSNR = 10 log10(L^2 / MSE),
 *   out[2] = SSIM = mean over the (H - 10)(W - 10) valid positions of
 *   ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
 *   weighted statistics of an 11 x 11 Gaussian window (sigma 1.5, weights
 *   sum 1), C1 = (0.01 L)^2, C2 = (0.03 L)^2 (Wang et al. 2004).
 *   out device double [3]; sums are per-block FP64 partials added in block
 *   order (deterministic).
 * Errors: FQ_ERR_SHAPE (H or W < 11), FQ_ERR_INVALID_ARG (L <= 0, null),
 * FQ_ERR_WORKSPACE, FQ_ERR_ALIGN. */
fq_status fq_image_quality(const float *x, const float *y, int32_t H, int32_t W, double L, double *out,
                           void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* a2: vessel membership and depth binning                              */
/* ------------------------------------------------------------------ */

/* Vessel membership (App. D decides whether a scatterer lies inside a
 * vessel; here by an exact distance-to-centreline test in IEEE double).
 * vessel_out[s] = seg_id[s] for blood; for tissue the first segment whose
 * lumen strictly contains pos[:, s], else -1.  amp_out (nullable) = amp_in
 * with tissue scatterers inside a lumen set to 0.
 *   pos device float [3][S]; seg_id, vessel_out device int32 [S];
 *   amp_in, amp_out device float [S].
 * The integer result is bit-identical to IEEE double evaluation. */
fq_status fq_classify_scatterers(const float *pos, const int32_t *seg_id, int64_t S,
                                 const fq_flow *flow, const float *amp_in, int32_t *vessel_out,
                                 float *amp_out, void *stream);

/* Depth bins b(s) = clamp(floor(((double) z_s - z0) / dz), 0, B - 1) and a
 * stable counting sort: bin_off[b] = #{s : b(s) < b} (device int32 [B+1]),
 * perm (device int32 [S]) = scatterer indices ordered by (bin, index).
 * Bit-identical to IEEE double evaluation.  Needs a workspace of
 * fq_bin_workspace_size bytes.  S < 2^31, 1 <= B <= 8192. */
fq_status fq_bin_workspace_size(int64_t S, int32_t B, size_t *bytes);
fq_status fq_bin_scatterers(const float *z, int64_t S, double z0, double dz, int32_t B,
                            int32_t *bin_off, int32_t *perm, void *workspace,
                            size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* a3: pulse-echo RF synthesis                                          */
/* ------------------------------------------------------------------ */

/* RF channel data of n_frames frames (Eq. 1 restated as a narrowband
 * time-domain sum under the weak-scattering assumption, App. D; Sec. 2.3):
 *   RF[f][a][m][k] = base[a][m][k]
 *       + sum_s A_{s,m,a} p(k / fs - tau_{s,m,a})
 *   tau = ((u_a . r_s - min_m' u_a . e_m') + |r_s - e_m|) / c
 *   A   = amp_s D exp(-alpha f0[MHz] c tau) / |r_s - e_m|,
 *   alpha = alpha_db_cm_mhz * 100 / (20 / ln 10)  (Np / m / MHz)
 *   D   = sinc(k0 b_x (x_s - x_m) / r) [* sinc(k0 b_y (y_s - y_m) / r) if ny > 1]
 *   sinc(u) = sin(u) / u, k0 = 2 pi f0 / c.
 * Samples outside [0, Ns) are dropped.  Alg. 1's static-tissue reuse is the
 * `rf_base` term: pass the tissue RF of one frame (computed by an earlier
 * call) and only the moving scatterers here.
 *   pos     device float [n_frames][3][S]
 *   amp     device float [S]
 *   rf_base device float [A][M][Ns] or NULL
 *   rf      device [n_frames][A][M][Ns] of out_dtype (FQ_F32, FQ_BF16 or
 *           FQ_F16), 4-byte aligned
 * Delays use float-float (~48-bit) arithmetic.  Taps are accumulated in
 * fixed point, so results are bit-reproducible.  For probes whose rows hold
 * whole groups of 4 elements (two-cycle pulse of 8-9 taps, elements up to
 * 5/pi wavelengths wide, S < 2^30) every (transmit, element) record is one
 * int32 per sample with its own quantum, about 2^-31 of an upper bound of
 * the sum of |taps| at any of its samples (plus the largest |rf_base|), so
 * the record cannot overflow and its precision is relative to its largest
 * possible sum; otherwise records are 47-bit (resolution 2^-20 of the
 * largest |amp|, range 2^27 of it).  1/r is capped at 2^17 per metre:
 * scatterers closer than ~8 um to an element centre (far inside the
 * element's near field, outside the model) saturate.
 * Errors: FQ_ERR_INVALID_ARG, FQ_ERR_SHAPE (Ns > 8192, n_angles outside
 * [1, FQ_MAX_ANGLES], M > 65536), FQ_ERR_UNSUPPORTED (another out_dtype). */
fq_status fq_simulate_rf(const fq_probe *probe, const fq_tx *tx, const float *pos,
                         const float *amp, int64_t S, int32_t n_frames, const float *rf_base,
                         int32_t out_dtype, void *rf, void *stream);

/* ------------------------------------------------------------------ */
/* a4 + a5: rf2iq and delay-and-sum compounding                          */
/* ------------------------------------------------------------------ */

/* rf2iq (Alg. 3 step 2.3.2.1): IQ[k] = 2 sum_{j=-J..J} h_j RF[k-j]
 * exp(-i 2 pi f0 (k-j) / fs), h = Hann-windowed ideal low-pass with cutoff
 * f0, J = 2 round(fs/f0), w_j = (1 + cos(pi j / (J+1))) / 2, normalised to
 * sum 1; RF outside [0, Ns) is 0.
 *   rf      device [n_frames][n_lines][Ns] of rf_dtype (FQ_F32 / FQ_BF16 / FQ_F16)
 *   iq_ch   device complex [n_lines][Ns][F_pad] of iq_dtype (the same
 *           three), frames
 *           innermost, F_pad = fq_frame_pad(n_frames); padded frames are 0.
 * n_lines = A * M.  J <= 32. */
int32_t fq_frame_pad(int32_t n_frames);
fq_status fq_rf2iq(const fq_probe *probe, int32_t n_lines, int32_t n_frames, const void *rf,
                   int32_t rf_dtype, int32_t iq_dtype, void *iq_ch, void *stream);

/* DAS with coherent compounding (Sec. 2.4.1, Alg. 3):
 *   tau = ((u_a . r_p - min u_a . e) + |r_p - e_m|) / c,  u = tau fs,
 *   i = floor(u), phi = u - i,
 *   v = (1 - phi) IQ[i] + phi IQ[i+1]   (0 if i < 0 or i + 1 >= Ns)
 *   iq[p][f] = (1/A) sum_a sum_m w_m(p) v exp(+i 2 pi f0 tau)
 * w_m(p) = 1 iff |x_p - x_m| <= z_p / (2 f#) (and in y for matrix arrays),
 * decided in binary32 on the coordinates rounded to float.
 * Delays are computed once per (pixel, angle, element) and shared by all
 * frames (the paper's precomputed-DAS-matrix idea, without the matrix).
 *   iq_ch  device complex [A*M][Ns][F_pad] of ch_dtype (fq_rf2iq layout;
 *          FQ_F32, FQ_BF16 or FQ_F16)
 *   iq     device complex [P][n_frames] of iq_dtype (Casorati, frames
 *          contiguous; FQ_F32 or FQ_BF16), 8-byte aligned.
 * FP32 accumulation, float-float delays. */
fq_status fq_das(const fq_probe *probe, const fq_tx *tx, const void *iq_ch, int32_t ch_dtype,
                 int32_t n_frames, const fq_grid *grid, int32_t iq_dtype, void *iq, void *stream);

/* rf2iq followed by DAS; the channel IQ lives in the workspace. */
fq_status fq_beamform_das_workspace_size(const fq_probe *probe, const fq_tx *tx,
                                         int32_t n_frames, int32_t ch_dtype, size_t *bytes);
fq_status fq_beamform_das(const fq_probe *probe, const fq_tx *tx, const void *rf,
                          int32_t rf_dtype, int32_t n_frames, const fq_grid *grid,
                          int32_t ch_dtype, int32_t iq_dtype, void *iq, void *workspace,
                          size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* a6 - a8: SVD clutter filter and power Doppler                        */
/* ------------------------------------------------------------------ */

/* Casorati Gram G = S^H S (Sec. 2.4.2: the SVD of S is obtained from the
 * eigen-decomposition of its frames x frames Gram matrix).
 *   S  device complex [P][F] of dtype
 *   G  device float complex [F][F] (row-major, Hermitian, full matrix)
 * dtype FQ_F32 or FQ_BF16, any gram_mode, 2 <= F <= 512, P >= 1.
 *   FQ_GRAM_F32   FP32 products and sums on the CUDA cores.
 *   FQ_GRAM_BF16  tcgen05 tensor cores: S is rounded to BF16 (nearest even),
 *                 products are exact, sums FP32 (G is the Gram of the
 *                 rounded S up to FP32 accumulation).
 *   FQ_GRAM_TF32  as BF16 with TF32 operands (10 mantissa bits, nearest,
 *                 ties away from zero).
 * The tensor-core modes keep their scratch (a 2F x P operand copy plus
 * FP32 partial tiles) in the workspace and a status word in its first 256
 * bytes: a device-side wait that runs out (bounded at ~2 s) sets it to
 * FQ_ERR_TIMEOUT, readable with fq_clutter_status(workspace). */
fq_status fq_gram_workspace_size(int64_t P, int32_t F, int32_t gram_mode, size_t *bytes);
fq_status fq_casorati_gram(const void *S, int32_t dtype, int64_t P, int32_t F, int32_t gram_mode,
                           float *G, void *workspace, size_t workspace_bytes, void *stream);

/* Eigen-decomposition of a Hermitian F x F matrix, G = V diag(lambda) V^H,
 * lambda descending (= sigma^2 of S when G = S^H S).
 *   G       device float complex [F][F]
 *   eigvals device double [F]
 *   V       device float complex [F][F], column j = eigenvector j
 * Householder tridiagonalisation + implicit QL with Wilkinson shifts on one
 * CTA (FP32).  FQ_ERR_NUMERICAL (reported through fq_clutter_status after
 * the stream reaches the call) if QL needs more than 60 iterations for one
 * eigenvalue; the outputs are then unspecified. */
fq_status fq_eig_workspace_size(int32_t F, size_t *bytes);
fq_status fq_hermitian_eig(const float *G, int32_t F, double *eigvals, float *V, void *workspace,
                           size_t workspace_bytes, void *stream);

/* SVD clutter filter + power Doppler (Sec. 2.4.2):
 *   S_f = S - (S V_k) V_k^H   (the k largest singular components removed)
 *   k   = k_cut if k_cut >= 0, else the smallest k with
 *         sum_{i<k} lambda_i >= energy_thresh * sum_i lambda_i
 *   pd[p] = (1/F) sum_f |S_f[p][f]|^2
 *   iq       device complex [P][F] of dtype (FQ_F32 / FQ_BF16)
 *   iq_f     device complex [P][F] of dtype, nullable (may equal iq)
 *   pd       device float [P], nullable
 *   eigvals  device double [F], nullable
 *   k_used   device int32 [1], nullable
 * k_cut > F -> FQ_ERR_INVALID_ARG; k == F -> S_f = 0.
 * gram_mode selects the Gram arithmetic as for fq_casorati_gram; the
 * projection always reads iq in its own dtype.
 * Everything stays on the device (k is decided on the device). */
fq_status fq_clutter_svd_workspace_size(int64_t P, int32_t F, int32_t gram_mode, size_t *bytes);
fq_status fq_clutter_svd(const void *iq, int32_t dtype, int64_t P, int32_t F, int32_t k_cut,
                         double energy_thresh, int32_t gram_mode, void *iq_f, float *pd,
                         double *eigvals, int32_t *k_used, void *workspace,
                         size_t workspace_bytes, void *stream);

/* No-allocation variant of fq_clutter_svd.  The paper has no counterpart:
 * it serves callers that cannot hand the library a workspace.  Some hosts
 * cannot call cudaMalloc, or create device buffers, at the point where they
 * filter an ensemble: their device memory belongs to an allocator they
 * cannot reach (for instance a framework's caching allocator seen through a
 * plugin interface), or their acquisition loop forbids device allocation
 * after start-up.  This call takes all its scratch from one array built
 * into the library instead, and allocates nothing itself (no cudaMalloc,
 * no cudaFree, no library routine that allocates).
 *   - The array holds 12 MiB of device memory on every GPU that loads the
 *     library, until the process exits.
 *   - Limit: F <= 256 frames (any P).  Larger F returns FQ_ERR_SHAPE with
 *     a message; use fq_clutter_svd with a workspace instead.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture.
 *   - Every call uses the same array and leaves its contents behind: calls
 *     whose work overlaps on the GPU (unordered streams, or several host
 *     threads) race with each other and give wrong results.
 *   - The device-side status word (eigen-solver convergence) is kept in
 *     the array: fq_clutter_status(NULL, stream) reads and clears it, as
 *     for the workspace of fq_clutter_svd.
 *   - The cached address is looked up again when the device's current
 *     context has changed (for instance after cudaDeviceReset).
 * Arguments and results are those of fq_clutter_svd with gram_mode
 * FQ_GRAM_F32 (iq_f, pd, eigvals, k_used nullable; everything stays on the
 * device). */
fq_status fq_clutter_svd_noalloc(const void *iq, int32_t dtype, int64_t P, int32_t F, int32_t k_cut,
                                 double energy_thresh, void *iq_f, float *pd, double *eigvals, int32_t *k_used,
                                 void *stream);

/* Power Doppler of a filtered ensemble: pd[p] = (1/F) sum_f |iq_f[p][f]|^2
 * (Sec. 2.4.2).  iq_f device complex [P][F] of dtype; pd device float [P]. */
fq_status fq_power_doppler(const void *iq_f, int32_t dtype, int64_t P, int32_t F, float *pd,
                           void *stream);

/* Device-side status word of the calls that decide on the device
 * (eigen-solver convergence, a timed-out tensor-core wait).  Reads and
 * clears the flag the last fq_hermitian_eig / fq_clutter_svd (or
 * tensor-core fq_casorati_gram) on this workspace wrote; workspace NULL
 * reads the built-in array of fq_clutter_svd_noalloc on the current device.
 * Synchronises `stream`. */
fq_status fq_clutter_status(void *workspace, void *stream);

/* Test hook (the paper has no counterpart).  FQ_DEBUG_SKIP_TC_LOADS = 1
 * makes the tensor-core Gram kernels issue no operand loads, so that every
 * bounded wait inside them runs out (~2 s per launch) and the call reports
 * FQ_ERR_TIMEOUT through its status word; 0 (the default) restores normal
 * operation.  For testing the timeout path only. */
enum { FQ_DEBUG_SKIP_TC_LOADS = 1 };
fq_status fq_debug_set(int32_t what, int32_t value);

/* Throughput probe of the FP32 pipes (the paper has no counterpart): the
 * denominator of the ALU rooflines the RF and DAS kernels are reported
 * against.  `blocks` CTAs of 256 threads each run `iters` rounds of 8
 * independent fused multiply-adds, scalar (packed = 0) or as packed f32x2
 * instructions that issue two lanes' FMAs at once (packed = 1): 2 FLOP per
 * lane and FMA, i.e. blocks x 256 x iters x 8 x 2 (x 2 when packed) FLOP.
 * The caller times the launch on `stream` (CUDA events).  sink: device float
 * [256], written only to keep the chains from being optimised away. */
fq_status fq_alu_probe(int32_t packed, int32_t blocks, int32_t iters, float *sink, void *stream);

/* sizeof of the ABI's structs as this library was compiled, for bindings
 * that check their own layouts: 0 fq_probe, 1 fq_tx, 2 fq_grid,
 * 3 fq_segment, 4 fq_flow, 5 fq_motion, 6 fq_ensemble_desc,
 * 7 fq_tile_choice, 8 fq_vfield; 0 for any other index.  The paper has no counterpart. */
size_t fq_sizeof(int32_t which);

/* ------------------------------------------------------------------ */
/* a11: many uneven ensembles in one persistent kernel per stage        */
/* ------------------------------------------------------------------ */
/* The paper simulates its ensembles one after another and processes each
 * in chunks (Alg. 2-3); a batch instead puts the work items of all its
 * ensembles into one queue per stage.  One persistent kernel per stage
 * takes items from that queue (an atomic counter), most expensive
 * ensembles first, and runs the same tile code as the single-ensemble
 * calls above, so every ensemble's result equals what fq_classify_scatterers
 * -> fq_advect_scatterers -> fq_simulate_rf -> fq_beamform_das ->
 * fq_clutter_svd (gram_mode FQ_GRAM_F32) give for it.  A stage's queue
 * covers one wave of ensembles: the plan groups ensembles into waves whose
 * scratch (positions, RF, channel IQ, Casorati matrix, clutter workspace)
 * fits the arena budget and runs the waves in turn. */

/* One ensemble: host descriptions read by fq_batch_plan, device pointers
 * read by the kernels.  Requirements: two-cycle pulse with
 * n_cycles fs / f0 <= 9 samples, n_samples <= 8192, 2 <= n_frames <= 512,
 * element count <= 4096, S >= 1. */
typedef struct fq_ensemble_desc {
    fq_probe probe;
    fq_tx tx;                   /* host arrays */
    fq_grid grid;
    fq_flow flow;               /* host segment array */
    fq_motion motion;
    int64_t S;                  /* scatterers */
    int32_t n_frames;           /* F */
    double t0, dt;              /* frame f is at time t0 + f dt */
    int32_t k_cut;              /* as fq_clutter_svd */
    double energy_thresh;
    const float *p0;            /* device [3][S] */
    const int32_t *seg_id;      /* device [S] */
    const float *flow_coord;    /* device [3][S] */
    const float *amp;           /* device [S] */
    float *pd;                  /* device [P] output: power Doppler */
    double *eigvals;            /* device [F] output, nullable */
    int32_t *k_used;            /* device [1] output, nullable */
} fq_ensemble_desc;

typedef struct fq_batch fq_batch;  /* opaque plan (host memory) */
typedef struct fq_graph fq_graph;  /* opaque captured batch */

enum { FQ_OP_RF = 0, FQ_OP_DAS = 1 };

/* A tile shape the autotuner chose for one stage.
 *   FQ_OP_RF : choice = the RF kernel's register budget, for the
 *              4-element kernel that probes whose rows are multiples of 4
 *              use as resident warps per SM (32: 64 registers per thread,
 *              16: 128), for the 2-element kernel as resident CTAs of 256
 *              threads per SM (2 or 3)
 *   FQ_OP_DAS: choice = threads per DAS CTA (64, 128 or 256) */
typedef struct fq_tile_choice {
    int32_t op;
    int32_t choice;
    int32_t n_tried;
    int32_t tried[4];           /* the candidates, in the order timed */
    float tried_ms[4];          /* their device times (ms) */
    float ms;                   /* time of the chosen one */
} fq_tile_choice;

/* Plan a batch of n >= 1 ensembles (host only, no CUDA call).
 *   rf_dtype, ch_dtype, iq_dtype  FQ_F32 / FQ_BF16 storage of the RF, the
 *       channel IQ and the Casorati matrix
 *   max_arena_bytes  budget for the arena; 0 = no budget (one wave).  An
 *       ensemble that alone exceeds the budget gets a wave of its own.
 *   *arena_bytes  receives the size of the arena fq_batch_launch needs
 *       (256-byte aligned device memory the caller owns).
 * Errors: FQ_ERR_INVALID_ARG / FQ_ERR_SHAPE / FQ_ERR_UNSUPPORTED naming
 * the first bad ensemble. */
fq_status fq_batch_plan(const fq_ensemble_desc *ens, int32_t n, int32_t rf_dtype, int32_t ch_dtype,
                        int32_t iq_dtype, size_t max_arena_bytes, fq_batch **plan, size_t *arena_bytes);

/* Plan facts: waves, and work items per stage (9 stages: classify, advect,
 * RF, rf2iq, DAS, Gram, Gram reduce, eigen-solver, projection). */
fq_status fq_batch_info(const fq_batch *plan, int32_t *n_waves, int64_t items[9]);

/* Use a tile choice (from fq_autotune) for every wave of the plan. */
fq_status fq_batch_set_tile(fq_batch *plan, const fq_tile_choice *choice);

/* Enqueue the whole batch on `stream`: the plan's tables are copied into
 * the arena (synchronously, the first time this arena is used with this
 * plan), then per wave one persistent kernel per stage.  Outputs are valid
 * once the stream reaches the end of the call.  The arena holds a status
 * word per ensemble; fq_batch_status reads them. */
fq_status fq_batch_launch(fq_batch *plan, void *arena, size_t arena_bytes, void *stream);

/* fq_batch_launch that also records events[0] before the first stage and
 * events[1 + w * 9 + s] after stage s of wave w (events: host array of
 * n_events >= 1 + 9 n_waves cudaEvent_t, created by the caller), for
 * per-stage device times. */
fq_status fq_batch_launch_profiled(fq_batch *plan, void *arena, size_t arena_bytes, void *stream, void **events,
                                   int32_t n_events);

/* Reads (and clears) every ensemble's device status word; synchronises the
 * stream.  Returns the first non-OK status with the ensemble index in the
 * message. */
fq_status fq_batch_status(fq_batch *plan, void *arena, void *stream);

void fq_batch_free(fq_batch *plan);

/* Plan + launch + free in one call (arena sized by a previous plan). */
fq_status fq_run_batched(const fq_ensemble_desc *ens, int32_t n, int32_t dtype, void *arena, size_t arena_bytes,
                         void *stream);

/* Capture a planned batch on this arena into a CUDA graph (the tables are
 * uploaded first, outside the capture), and replay it.  The graph keeps
 * the arena pointer and the descriptors' device pointers: they must stay
 * valid while the graph is used.  Replays on one arena must not overlap. */
fq_status fq_graph_capture(fq_batch *plan, void *arena, size_t arena_bytes, fq_graph **graph);
fq_status fq_graph_launch(fq_graph *graph, void *stream);
void fq_graph_free(fq_graph *graph);

/* Autotuner: time every candidate tile shape of `op` on one ensemble (its
 * batch of one, on this arena), keep the fastest.  Results are cached per
 * (op, probe, frames, scatterers, grid) in the process; a cached answer is
 * returned without timing (out->n_tried = 0).  Synchronises `stream`. */
fq_status fq_autotune(int32_t op, const fq_ensemble_desc *ens, int32_t rf_dtype, void *arena, size_t arena_bytes,
                      fq_tile_choice *out, void *stream);

/* ------------------------------------------------------------------ */
/* a10: learned clutter filter (3D convolutional network)              */
/* ------------------------------------------------------------------ */
/* Filters learned from simulated ensembles are the paper's future work
 * (Sec. 1, Sec. 4).  Network: four 3D convolutions over the IQ ensemble,
 * 2 -> 32 -> 32 -> 32 -> 2 channels, kernels of 5 frames x 3 x 3 pixels,
 * zero "same" padding, bias, ReLU after the first three; input = (Re, Im)
 * of the IQ times a normalisation `scale`, output = estimated blood IQ,
 * power Doppler = mean over frames of |output|^2 / scale^2.  Convention:
 *   y[v, o] = b[o] + sum_t sum_i x[v + d_t, i] W[t][i][o],
 *   d_t = (dt, dz, dx), dt in -2..2, dz, dx in -1..1, t = (dt+2) 9 + (dz+1) 3 + (dx+1).
 * Volumes are channels-last [n_vol][F][Z][X][32] (X a multiple of 128, or
 * of 32 with Z a multiple of 4), BF16 activations (channels beyond the real
 * ones are 0), FP32 network output.  Convolutions run on the tcgen05 tensor cores (BF16
 * in, FP32 accumulate); weight gradients on the CUDA cores in FP32.
 *
 * Parameters: one device block of fq_cnn_param_bytes() (256-byte aligned),
 * owned by the caller.  FP32 master weights W[layer] [45][32][32] (tap, in,
 * out; entries beyond the layer's channels must be 0) and biases b[layer]
 * [32], then the Adam moments m and v over the same span, then the BF16
 * tap tiles the kernels read.  fq_cnn_param_offset(what, layer) gives byte
 * offsets: what = 0 W[layer], 1 b[layer], 2 m, 3 v, 4 size of the trainable
 * span (W and b of all layers, the layout of `grads`).  After writing the
 * master weights call fq_cnn_pack; fq_cnn_adam repacks by itself.
 * `status`: device int, set to FQ_ERR_TIMEOUT if a bounded wait inside a
 * convolution ran out. */
size_t fq_cnn_param_bytes(void);
size_t fq_cnn_param_offset(int32_t what, int32_t layer);
/* Activation workspace for n_vol volumes; fq_cnn_act_offset(which, ...)
 * gives the byte offset of hidden layer `which` (0..2) or, for 3, of the
 * FP32 output [n_vol][F][Z][X][32] (channels 0, 1 used). */
size_t fq_cnn_act_bytes(int32_t n_vol, int32_t F, int32_t Z, int32_t X);
size_t fq_cnn_act_offset(int32_t which, int32_t n_vol, int32_t F, int32_t Z, int32_t X);
fq_status fq_cnn_pack(void *params, void *stream);
/* Casorati [P][F][2] FP32 (pixel p = x + X z) -> input volume (BF16,
 * nullable) and / or training target [F][Z][X][2] FP32 (nullable):
 * (s - m_p) * scale * gain, m_p = the pixel's temporal mean when
 * remove_mean != 0 (the static part of the echo), else 0.  scale = *scale_in
 * (device float) if given, else 1 / RMS of the deviations of this ensemble,
 * written to *scale_out (device float).  Workspace: fq_cnn_prep_bytes(Z, X)
 * bytes, 256-byte aligned. */
size_t fq_cnn_prep_bytes(int32_t Z, int32_t X);
fq_status fq_cnn_from_casorati(const float *iq, int32_t F, int32_t Z, int32_t X, int32_t remove_mean,
                               const float *scale_in, float *scale_out, float gain, void *vol, float *target,
                               void *workspace, size_t workspace_bytes, void *stream);
/* One convolution layer: mode 0 = bias + ReLU -> BF16, 1 = bias -> FP32,
 * 2 = (no bias) x (mask > 0) -> BF16; backward != 0 uses the flipped,
 * channel-swapped kernel of the data gradient. */
fq_status fq_cnn_conv(int32_t mode, const void *in, const void *params, int32_t layer, int32_t backward,
                      void *out, const void *mask, int32_t n_vol, int32_t F, int32_t Z, int32_t X,
                      int32_t *status, void *stream);
fq_status fq_cnn_forward(const void *params, const void *vol, int32_t n_vol, int32_t F, int32_t Z, int32_t X,
                         void *acts, size_t act_bytes, int32_t *status, void *stream);
/* After fq_cnn_forward on the same acts: MSE against target [n_vol][F][Z][X][2]
 * into *loss (device float), gradients of W and b into grads (device FP32,
 * the trainable-span layout). */
fq_status fq_cnn_backward(const void *params, const void *vol, const float *target, int32_t n_vol, int32_t F,
                          int32_t Z, int32_t X, void *acts, size_t act_bytes, float *grads, float *loss,
                          int32_t *status, void *stream);
/* Adam (beta 0.9, 0.999, eps 1e-8), step >= 1, then repack. */
fq_status fq_cnn_adam(void *params, const float *grads, float lr, int32_t step, void *stream);
fq_status fq_cnn_power_doppler(const float *out, int32_t F, int32_t Z, int32_t X, float scale, float *pd,
                               void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FQ_H */
