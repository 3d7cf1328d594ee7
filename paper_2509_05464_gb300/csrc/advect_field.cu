// advect_field.cu -- scatterer trajectories of a steady gridded velocity
// field (Sec. 2.2.2: P(t) = P0 + integral_0^t v(P(s)) ds, with the vessel
// geometry confining intravascular scatterers; App. C: scatterers follow
// the local flow), by the classical fourth-order Runge-Kutta method.
//
// Design (GB300): one thread per scatterer walks every step of every frame
// and writes the frames it is asked for; the field is an L2-resident array
// of float4 samples (vx, vy, vz, unused), so one trilinear evaluation is
// eight 16-byte loads.  Arithmetic is binary32 (FP64 only for the lumen
// projection of blood scatterers), arranged so that rounding
// at centimetre coordinates (~1e-9 m) does not enter the trajectory: a
// Poiseuille profile shears at a few hundred 1/s, which turns a lateral
// error of 1e-9 m into ~1e-7 m of axial error over 200 frames.  So each
// thread carries (i) its displacement D = P - P0 as an unevaluated float
// pair, updated by an exact two-sum each step, and (ii) its grid
// coordinate as an integer cell plus a binary32 fraction in [0, 1), started
// in FP64 and advanced by each step's increment, so that every sampling
// point is cell + (fraction + small offset / spacing).  Lumen confinement
// adds its corrections to both only when a scatterer crosses its vessel's
// wall or end, where the definition moves it.
#include <cmath>
#include <cstring>

#include "fq_internal.cuh"

namespace {

// binary32 view of a segment for the per-step wall projection (copied into
// registers once per scatterer)
struct FSegF {
    int kind;
    float a1[3], a2[3], a3[3];
    float len, R, c1, s1;
};

struct FSeg {
    int kind;
    double p[3], a1[3], a2[3], a3[3];
    double len, R, Rc, phi1, c1, s1;  // c1, s1 = cos, sin phi1
    FSegF f;
};

// binary32 coordinates along a vessel (millimetres) are good to ~1e-9 m; a
// scatterer farther than this from a vessel end takes no wrap decision
constexpr float kInsideMargin = 1e-8f;

struct FSegTable {
    int n;
    FSeg s[FQ_MAX_SEGMENTS];
};

struct FieldParams {
    const float4 *v;
    int nx, ny, nz;
    double ox, oy, oz;  // origin (m)
    double ixd, iyd, izd;  // 1 / spacing (1/m)
    float ix, iy, iz;
    float h, h2, h6;   // step, h / 2, h / 6 (s)
    int n_sub, f0, F;
    int64_t S;
};

// Starting grid coordinate g0 = (p - o) / spacing as an integer cell and a
// binary32 fraction in [0, 1) (FP64 once per scatterer; far-away starts are
// clamped to +-2^20 cells, beyond any grid).
__device__ __forceinline__ void start_cell(double p, double o, double inv, int &c, float &fr)
{
    double g = (p - o) * inv;
    g = fmin(fmax(g, -1048576.0), 1048576.0);
    const double fl = floor(g);
    c = (int)fl;
    fr = (float)(g - fl);
}

// Cell and weight along one axis at g = c0 + fr0 + e * inv, clamped to
// [0, n - 1]: i = min(floor(g), n - 2), f = g - i (i = 0, f = 0 if n = 1);
// e is a stage offset (a fraction of one step's displacement).
__device__ __forceinline__ void cell(int c0, float fr0, float e, float inv, int n, int &i0, int &i1, float &f)
{
    if (n <= 1) {
        i0 = i1 = 0;
        f = 0.0f;
        return;
    }
    const float t = fmaf(e, inv, fr0);
    const float k = floorf(t);
    int i = c0 + (int)k;
    float w = t - k;
    if (i < 0) {
        i = 0;
        w = 0.0f;
    } else if (i > n - 2) {
        i = n - 2;
        w = 1.0f;
    }
    i0 = i;
    i1 = i + 1;
    f = w;
}

struct Start {
    int cx, cy, cz;
    float fx, fy, fz;
};

// advance one axis of the grid coordinate by the displacement d
__device__ __forceinline__ void advance(int &c, float &fr, float d, float inv)
{
    const float t = fmaf(d, inv, fr);
    const float k = floorf(t);
    c += (int)k;
    fr = t - k;
}

// (hi, lo) += d exactly up to the final rounding of lo (two-sum)
__device__ __forceinline__ void ff_acc(float &hi, float &lo, float d)
{
    const float s = hi + d;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (d - bb);
    const float l = lo + e;
    hi = s + l;
    lo = l - (hi - s);
}

// p + (hi + lo) rounded once to binary32 (to within the final rounding)
__device__ __forceinline__ float ff_out(float p, float hi, float lo)
{
    const float s = p + hi;
    const float bb = s - p;
    const float e = (p - (s - bb)) + (hi - bb);
    return s + (e + lo);
}

__device__ __forceinline__ float3 lerp3(float3 a, float3 b, float t)
{
    return make_float3(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y), fmaf(t, b.z - a.z, a.z));
}

__device__ __forceinline__ float3 ld3(const float4 *v, int64_t i)
{
    const float4 q = __ldg(v + i);
    return make_float3(q.x, q.y, q.z);
}

// trilinear interpolation at P0 + E, coordinates clamped to the grid
// (constant continuation beyond it)
__device__ __forceinline__ float3 field_eval(const FieldParams &fp, const Start &g, float ex, float ey, float ez)
{
    int x0, x1, y0, y1, z0, z1;
    float fx, fy, fz;
    cell(g.cx, g.fx, ex, fp.ix, fp.nx, x0, x1, fx);
    cell(g.cy, g.fy, ey, fp.iy, fp.ny, y0, y1, fy);
    cell(g.cz, g.fz, ez, fp.iz, fp.nz, z0, z1, fz);
    const int64_t r00 = ((int64_t)z0 * fp.ny + y0) * fp.nx, r01 = ((int64_t)z0 * fp.ny + y1) * fp.nx;
    const int64_t r10 = ((int64_t)z1 * fp.ny + y0) * fp.nx, r11 = ((int64_t)z1 * fp.ny + y1) * fp.nx;
    const float3 c00 = lerp3(ld3(fp.v, r00 + x0), ld3(fp.v, r00 + x1), fx);
    const float3 c01 = lerp3(ld3(fp.v, r01 + x0), ld3(fp.v, r01 + x1), fx);
    const float3 c10 = lerp3(ld3(fp.v, r10 + x0), ld3(fp.v, r10 + x1), fx);
    const float3 c11 = lerp3(ld3(fp.v, r11 + x0), ld3(fp.v, r11 + x1), fx);
    return lerp3(lerp3(c00, c01, fy), lerp3(c10, c11, fy), fz);
}

__device__ __forceinline__ float dot3(const float a[3], float x, float y, float z)
{
    return fmaf(a[0], x, fmaf(a[1], y, a[2] * z));
}

__device__ __forceinline__ double dotd(const double a[3], double x, double y, double z)
{
    return fma(a[0], x, fma(a[1], y, a[2] * z));
}

__device__ __forceinline__ float dotf(const float a[3], float x, float y, float z)
{
    return fmaf(a[0], x, fmaf(a[1], y, a[2] * z));
}

// Local vessel coordinates of a blood scatterer, taken in FP64 at an
// anchor displacement DA and followed in binary32 through the motion since
// then, Delta = D - DA: line (u1 axial, u2, u3 across), arc (u1, u2 in the
// arc plane, u3 across; e1 = in-plane radius - Rc).  The cross-lumen
// offsets are small (below the lumen radius) and the arc's radial offset
// comes from the exact identity r^2 - r0^2 = 2 u0.Delta + |Delta|^2, so a
// wall projection is accurate to ~1e-11 m without FP64.
struct Anchor {
    float3 DA, DAl;      // displacement at the anchor (float pair)
    float u1, u2, u3;    // local coordinates at the anchor
    float r0, e1;        // arc: in-plane radius and its offset from Rc
};

__device__ __forceinline__ void set_anchor(const FSeg &sg, float3 P0, float3 D, float3 Dl, Anchor &an)
{
    const double wx = ((double)P0.x - sg.p[0]) + ((double)D.x + (double)Dl.x);
    const double wy = ((double)P0.y - sg.p[1]) + ((double)D.y + (double)Dl.y);
    const double wz = ((double)P0.z - sg.p[2]) + ((double)D.z + (double)Dl.z);
    const double u1 = dotd(sg.a1, wx, wy, wz), u2 = dotd(sg.a2, wx, wy, wz), u3 = dotd(sg.a3, wx, wy, wz);
    an.DA = D;
    an.DAl = Dl;
    an.u1 = (float)u1;
    an.u2 = (float)u2;
    an.u3 = (float)u3;
    const double r0 = sqrt(u1 * u1 + u2 * u2);
    an.r0 = (float)r0;
    an.e1 = (float)(r0 - sg.Rc);
}

// Wall projection in binary32 from the anchor; returns false when the
// scatterer is within kInsideMargin of a vessel end or arc end, where the
// FP64 projection (and wrap) decides.  c = correction to add to D.
__device__ __forceinline__ bool wall_fp32(const FSegF &sg, const Anchor &an, float3 D, float3 Dl, float3 &c)
{
    const float dx = (D.x - an.DA.x) + (Dl.x - an.DAl.x);
    const float dy = (D.y - an.DA.y) + (Dl.y - an.DAl.y);
    const float dz = (D.z - an.DA.z) + (Dl.z - an.DAl.z);
    const float d1 = dotf(sg.a1, dx, dy, dz), d2 = dotf(sg.a2, dx, dy, dz), d3 = dotf(sg.a3, dx, dy, dz);
    const float u1 = an.u1 + d1, u2 = an.u2 + d2, u3 = an.u3 + d3;
    c = make_float3(0.0f, 0.0f, 0.0f);
    const float R = sg.R;
    if (sg.kind == FQ_SEG_LINE) {
        if (!(u1 > kInsideMargin && u1 < sg.len - kInsideMargin)) return false;
        const float q2 = fmaf(u2, u2, u3 * u3);
        if (q2 > R * R) {
            const float k = R * rsqrtf(q2) - 1.0f;  // move (u2, u3) onto the wall
            const float m2 = k * u2, m3 = k * u3;
            c = make_float3(fmaf(m2, sg.a2[0], m3 * sg.a3[0]), fmaf(m2, sg.a2[1], m3 * sg.a3[1]),
                            fmaf(m2, sg.a2[2], m3 * sg.a3[2]));
        }
        return true;
    }
    if (!(u2 > kInsideMargin && fmaf(u1, sg.s1, -u2 * sg.c1) > kInsideMargin)) return false;
    // approximate division and square root: they shape corrections of
    // nanometres, where a few ulps are below 1e-15 m
    const float dr2 = fmaf(2.0f * an.u1 + d1, d1, (2.0f * an.u2 + d2) * d2);  // r^2 - r0^2
    const float r2 = fmaf(an.r0, an.r0, dr2);
    const float rr = rsqrtf(r2);
    const float r = r2 * rr;
    const float e1 = an.e1 + __fdividef(dr2, r + an.r0);
    const float q2 = fmaf(e1, e1, u3 * u3);
    if (q2 > R * R) {
        const float k = R * rsqrtf(q2) - 1.0f;  // move (e1, u3) onto the wall
        const float de = k * e1 * rr, m3 = k * u3;  // radial step along (u1, u2) / r
        const float m1 = de * u1, m2 = de * u2;
        c = make_float3(fmaf(m1, sg.a1[0], fmaf(m2, sg.a2[0], m3 * sg.a3[0])),
                        fmaf(m1, sg.a1[1], fmaf(m2, sg.a2[1], m3 * sg.a3[1])),
                        fmaf(m1, sg.a1[2], fmaf(m2, sg.a2[2], m3 * sg.a3[2])));
    }
    return true;
}

// Moves the scatterer (P = P0 + D) back into its segment's lumen and wraps
// it along the vessel; returns the correction (zero when it stays).  FP64:
// it runs once per step for blood only, and binary32 coordinates relative
// to a vessel centre (millimetres) would round the wall by ~5e-10 m.
__device__ __forceinline__ double3 confine(const FSeg &sg, float3 P0, float3 D, float3 Dl)
{
    const double wx = ((double)P0.x - sg.p[0]) + ((double)D.x + (double)Dl.x);
    const double wy = ((double)P0.y - sg.p[1]) + ((double)D.y + (double)Dl.y);
    const double wz = ((double)P0.z - sg.p[2]) + ((double)D.z + (double)Dl.z);
    const double u1 = dotd(sg.a1, wx, wy, wz), u2 = dotd(sg.a2, wx, wy, wz), u3 = dotd(sg.a3, wx, wy, wz);
    double d1 = 0.0, d2 = 0.0, d3 = 0.0;  // change of (u1, u2, u3)
    if (sg.kind == FQ_SEG_LINE) {
        const double r2 = u2 * u2 + u3 * u3;
        if (r2 > sg.R * sg.R) {
            const double k = sg.R / sqrt(r2) - 1.0;
            d2 = k * u2;
            d3 = k * u3;
        }
        if (u1 < 0.0 || u1 >= sg.len) d1 = -sg.len * floor(u1 / sg.len);
    } else {
        const double r = sqrt(u1 * u1 + u2 * u2);
        const double e1 = r - sg.Rc;
        const double q2 = e1 * e1 + u3 * u3;
        double n1 = u1, n2 = u2;
        if (q2 > sg.R * sg.R) {
            const double k = sg.R / sqrt(q2);
            const double sc = (sg.Rc + k * e1) / r;  // new in-plane radius over the old
            n1 = u1 * sc;
            n2 = u2 * sc;
            d3 = (k - 1.0) * u3;
        }
        // inside the angular span [0, phi1) unless before the start or at /
        // past the end (arcs span at most pi)
        if (n2 < 0.0 || n1 * sg.s1 - n2 * sg.c1 <= 0.0) {
            const double phi = atan2(n2, n1);
            const double turns = floor(phi / sg.phi1);
            if (turns != 0.0) {
                double sn, cs;
                sincos(turns * sg.phi1, &sn, &cs);  // rotate back by turns * phi1
                const double m1 = n1 * cs + n2 * sn, m2 = n2 * cs - n1 * sn;
                n1 = m1;
                n2 = m2;
            }
        }
        d1 = n1 - u1;
        d2 = n2 - u2;
    }
    if (d1 == 0.0 && d2 == 0.0 && d3 == 0.0) return make_double3(0.0, 0.0, 0.0);
    return make_double3(d1 * sg.a1[0] + d2 * sg.a2[0] + d3 * sg.a3[0], d1 * sg.a1[1] + d2 * sg.a2[1] + d3 * sg.a3[1],
                        d1 * sg.a1[2] + d2 * sg.a2[2] + d3 * sg.a3[2]);
}

// a confinement correction added to the float-pair displacement in two
// parts; the grid coordinate advances by it (a wall projection, below a
// micrometre) or is taken afresh from the corrected position in FP64 (a
// wrap, up to a vessel length)
__device__ __forceinline__ void jump(const FieldParams &fp, float3 P0, double3 c, float3 &D, float3 &Dl, Start &g)
{
    const float hx = (float)c.x, hy = (float)c.y, hz = (float)c.z;
    ff_acc(D.x, Dl.x, hx);
    ff_acc(D.y, Dl.y, hy);
    ff_acc(D.z, Dl.z, hz);
    ff_acc(D.x, Dl.x, (float)(c.x - (double)hx));
    ff_acc(D.y, Dl.y, (float)(c.y - (double)hy));
    ff_acc(D.z, Dl.z, (float)(c.z - (double)hz));
    if (fabs(c.x) + fabs(c.y) + fabs(c.z) < 1e-6) {  // a wall projection: advance like a step
        advance(g.cx, g.fx, hx, fp.ix);
        advance(g.cy, g.fy, hy, fp.iy);
        advance(g.cz, g.fz, hz, fp.iz);
        return;
    }
    start_cell((double)P0.x + ((double)D.x + (double)Dl.x), fp.ox, fp.ixd, g.cx, g.fx);
    start_cell((double)P0.y + ((double)D.y + (double)Dl.y), fp.oy, fp.iyd, g.cy, g.fy);
    start_cell((double)P0.z + ((double)D.z + (double)Dl.z), fp.oz, fp.izd, g.cz, g.fz);
}

// D += d in both carried forms (float-pair displacement, grid coordinate)
__device__ __forceinline__ void move(const FieldParams &fp, float3 d, float3 &D, float3 &Dl, Start &g)
{
    ff_acc(D.x, Dl.x, d.x);
    ff_acc(D.y, Dl.y, d.y);
    ff_acc(D.z, Dl.z, d.z);
    advance(g.cx, g.fx, d.x, fp.ix);
    advance(g.cy, g.fy, d.y, fp.iy);
    advance(g.cz, g.fz, d.z, fp.iz);
}

// the rare path: within kInsideMargin of a vessel end
__device__ __forceinline__ void end_of_vessel(const FieldParams &fp, const FSeg &sg, float3 P0, float3 &D, float3 &Dl,
                                           Start &g, Anchor &an)
{
    const double3 c = confine(sg, P0, D, Dl);
    if (c.x != 0.0 || c.y != 0.0 || c.z != 0.0) jump(fp, P0, c, D, Dl, g);
    set_anchor(sg, P0, D, Dl, an);
}

__global__ void __launch_bounds__(256) advect_field_kernel(const FieldParams fp, const FSegTable st,
                                                           const float *__restrict__ p0,
                                                           const int32_t *__restrict__ seg_id,
                                                           float *__restrict__ out)
{
    const int64_t S = fp.S;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const float3 P0 = make_float3(p0[s], p0[S + s], p0[2 * S + s]);
        const int si = seg_id ? seg_id[s] : -1;
        const bool confined = si >= 0 && si < st.n;
        Start g;
        start_cell((double)P0.x, fp.ox, fp.ixd, g.cx, g.fx);
        start_cell((double)P0.y, fp.oy, fp.iyd, g.cy, g.fy);
        start_cell((double)P0.z, fp.oz, fp.izd, g.cz, g.fz);
        float3 D = make_float3(0.0f, 0.0f, 0.0f), Dl = make_float3(0.0f, 0.0f, 0.0f);
        Anchor an;
        FSegF sf;
        if (confined) {
            sf = st.s[si].f;
            set_anchor(st.s[si], P0, D, Dl, an);
        }
        for (int f = 0; f < fp.f0 + fp.F; ++f) {
            if (f > 0) {
                for (int j = 0; j < fp.n_sub; ++j) {
                    const float3 k1 = field_eval(fp, g, 0.0f, 0.0f, 0.0f);
                    const float3 k2 = field_eval(fp, g, fp.h2 * k1.x, fp.h2 * k1.y, fp.h2 * k1.z);
                    const float3 k3 = field_eval(fp, g, fp.h2 * k2.x, fp.h2 * k2.y, fp.h2 * k2.z);
                    const float3 k4 = field_eval(fp, g, fp.h * k3.x, fp.h * k3.y, fp.h * k3.z);
                    const float3 inc = make_float3(fp.h6 * (k1.x + 2.0f * (k2.x + k3.x) + k4.x),
                                                   fp.h6 * (k1.y + 2.0f * (k2.y + k3.y) + k4.y),
                                                   fp.h6 * (k1.z + 2.0f * (k2.z + k3.z) + k4.z));
                    move(fp, inc, D, Dl, g);
                    if (confined) {
                        float3 cf;
                        if (wall_fp32(sf, an, D, Dl, cf)) {
                            if (cf.x != 0.0f || cf.y != 0.0f || cf.z != 0.0f) move(fp, cf, D, Dl, g);
                        } else {  // near a vessel end: FP64 projection and wrap, new anchor
                            end_of_vessel(fp, st.s[si], P0, D, Dl, g, an);
                        }
                    }
                }
            }
            if (f >= fp.f0) {
                float *o = out + (int64_t)(f - fp.f0) * 3 * S;
                o[s] = ff_out(P0.x, D.x, Dl.x);
                o[S + s] = ff_out(P0.y, D.y, Dl.y);
                o[2 * S + s] = ff_out(P0.z, D.z, Dl.z);
            }
        }
    }
}

void pack_fsegments(const fq_flow *flow, FSegTable &st)
{
    std::memset(&st, 0, sizeof st);
    st.n = flow ? flow->n_seg : 0;
    for (int i = 0; i < st.n; ++i) {
        const fq_segment &s = flow->seg[i];
        FSeg &t = st.s[i];
        t.kind = s.kind;
        for (int d = 0; d < 3; ++d) {
            t.p[d] = s.p0[d];
            t.a1[d] = s.a1[d];
            t.a2[d] = s.a2[d];
            t.a3[d] = s.a3[d];
        }
        t.len = s.length;
        t.R = s.radius;
        t.Rc = s.arc_radius;
        t.phi1 = s.phi1;
        t.c1 = std::cos(s.phi1);
        t.s1 = std::sin(s.phi1);
        t.f.kind = t.kind;
        for (int d = 0; d < 3; ++d) {
            t.f.a1[d] = (float)t.a1[d];
            t.f.a2[d] = (float)t.a2[d];
            t.f.a3[d] = (float)t.a3[d];
        }
        t.f.len = (float)t.len;
        t.f.R = (float)t.R;
        t.f.c1 = (float)t.c1;
        t.f.s1 = (float)t.s1;
    }
}

}  // namespace

extern "C" fq_status fq_advect_field(const float *p0, const int32_t *seg_id, int64_t S, const fq_flow *flow,
                                     const fq_vfield *grid, const float *v, double dt, int32_t n_sub,
                                     int32_t first_frame, int32_t n_frames, float *pos_out, void *stream)
{
    FQ_REQUIRE(S >= 0 && n_frames >= 1 && first_frame >= 0 && n_sub >= 1, FQ_ERR_INVALID_ARG,
               "fq_advect_field: S=%lld n_frames=%d first_frame=%d n_sub=%d", (long long)S, n_frames,
               first_frame, n_sub);
    FQ_REQUIRE(grid && grid->nx >= 1 && grid->ny >= 1 && grid->nz >= 1 && grid->dx > 0.0 && grid->dy > 0.0 &&
                   grid->dz > 0.0 && (int64_t)grid->nx * grid->ny * grid->nz < ((int64_t)1 << 31),
               FQ_ERR_SHAPE, "fq_advect_field: grid needs n >= 1 samples and spacing > 0 on every axis");
    FQ_REQUIRE(dt > 0.0, FQ_ERR_INVALID_ARG, "fq_advect_field: dt must be > 0");
    FQ_REQUIRE(!flow || (flow->n_seg >= 0 && flow->n_seg <= FQ_MAX_SEGMENTS && (flow->n_seg == 0 || flow->seg)),
               FQ_ERR_SHAPE, "fq_advect_field: n_seg must be in [0, %d]", FQ_MAX_SEGMENTS);
    if (S == 0) return FQ_OK;
    FQ_REQUIRE(p0 && v && pos_out, FQ_ERR_INVALID_ARG, "fq_advect_field: null device pointer");
    FQ_REQUIRE(fqi::aligned(v, 16), FQ_ERR_ALIGN, "fq_advect_field: v must be 16-byte aligned");
    if (flow)
        for (int i = 0; i < flow->n_seg; ++i) {
            const fq_segment &s = flow->seg[i];
            FQ_REQUIRE((s.kind == FQ_SEG_LINE && s.length > 0.0) || (s.kind == FQ_SEG_ARC && s.phi1 > 0.0 &&
                                                                     s.phi1 <= M_PI && s.arc_radius > 0.0),
                       FQ_ERR_INVALID_ARG, "fq_advect_field: segment %d has no extent", i);
        }
    FieldParams fp;
    fp.v = reinterpret_cast<const float4 *>(v);
    fp.nx = grid->nx;
    fp.ny = grid->ny;
    fp.nz = grid->nz;
    fp.ox = grid->x0;
    fp.oy = grid->y0;
    fp.oz = grid->z0;
    fp.ixd = 1.0 / grid->dx;
    fp.iyd = 1.0 / grid->dy;
    fp.izd = 1.0 / grid->dz;
    fp.ix = (float)fp.ixd;
    fp.iy = (float)fp.iyd;
    fp.iz = (float)fp.izd;
    const double h = dt / n_sub;
    fp.h = (float)h;
    fp.h2 = (float)(0.5 * h);
    fp.h6 = (float)(h / 6.0);
    fp.n_sub = n_sub;
    fp.f0 = first_frame;
    fp.F = n_frames;
    fp.S = S;
    FSegTable st;
    pack_fsegments(flow, st);
    const int threads = 256;
    int64_t blocks = (S + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    advect_field_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(fp, st, p0, seg_id, pos_out);
    return fqi::launch_check("fq_advect_field");
}
