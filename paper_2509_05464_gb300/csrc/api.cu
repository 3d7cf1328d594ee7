// api.cu -- error reporting, library information and host-side parameter
// preparation shared by the entry points of libfq.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "fq_internal.cuh"

namespace fqi {

static thread_local char g_err[1024] = "";

fq_status set_error(fq_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return s;
}

fq_status cuda_check(cudaError_t e, const char *where)
{
    if (e == cudaSuccess) return FQ_OK;
    return set_error(FQ_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

fq_status launch_check(const char *where)
{
    return cuda_check(cudaGetLastError(), where);
}

bool make_probe_ff(const fq_probe *p, ProbeFF &o)
{
    o.nx = p->nx;
    o.ny = p->ny;
    o.M = p->nx * p->ny;
    o.ns = p->n_samples;
    o.pitch_x = split_double(p->pitch_x);
    o.pitch_y = split_double(p->pitch_y);
    o.fs_over_c = split_double(p->fs / p->c);
    o.f0_over_fs = split_double(p->f0 / p->fs);
    return true;
}

void make_angles_ff(const fq_probe *p, const fq_tx *tx, AngleFF *out)
{
    for (int a = 0; a < tx->n_angles; ++a) {
        double ux = std::sin(tx->tilt_x[a]);
        double uy = std::sin(tx->tilt_y[a]);
        double uz = std::sqrt(1.0 - ux * ux - uy * uy);
        double best = 1e300;
        for (int m = 0; m < p->nx * p->ny; ++m) {
            int ix = m % p->nx, iy = m / p->nx;
            double ex = ((double)ix - 0.5 * (double)(p->nx - 1)) * p->pitch_x;
            double ey = ((double)iy - 0.5 * (double)(p->ny - 1)) * p->pitch_y;
            double d = ux * ex + uy * ey;
            if (d < best) best = d;
        }
        out[a].ux = split_double(ux);
        out[a].uy = split_double(uy);
        out[a].uz = split_double(uz);
        out[a].origin = split_double(best);
    }
}

}  // namespace fqi

extern "C" {

const char *fq_last_error(void) { return fqi::g_err; }

const char *fq_status_string(fq_status s)
{
    switch (s) {
    case FQ_OK: return "FQ_OK";
    case FQ_ERR_INVALID_ARG: return "FQ_ERR_INVALID_ARG";
    case FQ_ERR_SHAPE: return "FQ_ERR_SHAPE";
    case FQ_ERR_ALIGN: return "FQ_ERR_ALIGN";
    case FQ_ERR_WORKSPACE: return "FQ_ERR_WORKSPACE";
    case FQ_ERR_CUDA: return "FQ_ERR_CUDA";
    case FQ_ERR_TIMEOUT: return "FQ_ERR_TIMEOUT";
    case FQ_ERR_NUMERICAL: return "FQ_ERR_NUMERICAL";
    case FQ_ERR_UNSUPPORTED: return "FQ_ERR_UNSUPPORTED";
    }
    return "FQ_ERR_UNKNOWN";
}

int32_t fq_version(void) { return 100; }

}  // extern "C"
