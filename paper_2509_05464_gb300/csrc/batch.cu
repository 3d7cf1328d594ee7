// batch.cu -- a11 batched persistent execution of many uneven ensembles:
// the host plan (validation, waves under an arena budget, per-stage work
// queues ordered most expensive first, arena layout), the upload of the
// device tables, one persistent launch per stage and wave, CUDA graph
// capture of the whole batch, and the tile-shape autotuner.
//
// The per-item tile code is the single-ensemble code of each stage (see
// the *_batched_kernel functions next to each stage), so a batch gives the
// results of the single-ensemble calls, ensemble by ensemble.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "batch.cuh"
#include "fq_internal.cuh"

using fqb::EnsDev;
using fqb::StageQueue;

namespace {

constexpr int NS = fqb::N_STAGES;
inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
inline size_t elem(int dt) { return dt == FQ_F32 ? 4 : 2; }
inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

struct EnsHost {
    fq_ensemble_desc d;
    int64_t P = 0;
    int A = 0, M = 0, ns = 0, F = 0, Fp = 0, L = 0, J = 0;
    size_t off_pos = 0, off_vessel = 0, off_amp = 0, off_rf = 0, off_ch = 0, off_iq = 0, off_cws = 0, scratch = 0;
    size_t cl[10] = {};
    int n_chunks = 1;
    int64_t chunk_len = 0;
    int gx[NS] = {}, gy[NS] = {};
    int items[NS] = {};
    double cost[NS] = {};
    int wave = 0;
    size_t wave_off = 0;
    size_t par_seg = 0, par_mot = 0, par_rf = 0, par_iq = 0, par_das = 0;  // offsets in the parameter image
};

struct Wave {
    std::vector<int> members;
    size_t scratch = 0;
    std::vector<int> order[NS];  // ensemble indices in execution order
    std::vector<int> off[NS];    // prefix of item counts in that order
    int total[NS] = {};
    size_t q_off[NS] = {}, q_ens[NS] = {};
    size_t members_off = 0;      // eigen-solver members, largest F first
};

}  // namespace

struct fq_batch {
    int n = 0;
    int rf_dtype = FQ_F32, ch_dtype = FQ_F32, iq_dtype = FQ_F32;
    size_t budget = 0;
    std::vector<EnsHost> e;
    std::vector<Wave> waves;
    int rf_tune = 3, das_threads = 128;  // RF register budget (see fq_tile_choice), DAS CTA size
    bool rf_quad = true;  // every member's rows hold whole element quads
    int ns_max = 0, J_max = 0, M_max = 0, A_max = 0;
    size_t rf_smem = 0;  // dynamic shared memory of the RF stage kernel
    size_t off_counters = 0, off_status = 0, off_ens = 0, off_params = 0, off_queues = 0, off_scratch = 0, total = 0;
    std::vector<unsigned char> params;  // host image of the parameter blocks
    const void *uploaded = nullptr;     // arena holding the current tables
};

struct fq_graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
};

namespace {

// ------------------------------------------------------------ validation --
fq_status check_desc(const fq_ensemble_desc &d, int i, int rf_dtype)
{
    const fq_probe &p = d.probe;
    FQ_REQUIRE(d.S >= 1 && d.S < ((int64_t)1 << 31), FQ_ERR_SHAPE, "batch: ensemble %d: S = %lld", i, (long long)d.S);
    FQ_REQUIRE(d.n_frames >= 2 && d.n_frames <= 512, FQ_ERR_SHAPE, "batch: ensemble %d: n_frames must be in [2, 512]",
               i);
    FQ_REQUIRE(p.nx >= 1 && p.ny >= 1 && (int64_t)p.nx * p.ny <= 4096, FQ_ERR_SHAPE,
               "batch: ensemble %d: element count must be in [1, 4096]", i);
    FQ_REQUIRE(p.n_samples >= 2 && p.n_samples <= 8192, FQ_ERR_SHAPE, "batch: ensemble %d: n_samples in [2, 8192]", i);
    FQ_REQUIRE(p.f0 > 0 && p.fs > 0 && p.c > 0, FQ_ERR_INVALID_ARG, "batch: ensemble %d: f0, fs, c must be > 0", i);
    FQ_REQUIRE(p.n_cycles == 2, FQ_ERR_UNSUPPORTED, "batch: ensemble %d: the batched RF kernel needs a two-cycle pulse",
               i);
    FQ_REQUIRE(d.tx.n_angles >= 1 && d.tx.n_angles <= FQ_MAX_ANGLES && d.tx.tilt_x && d.tx.tilt_y, FQ_ERR_SHAPE,
               "batch: ensemble %d: n_angles must be in [1, %d]", i, FQ_MAX_ANGLES);
    FQ_REQUIRE(d.grid.nx >= 1 && d.grid.ny >= 1 && d.grid.nz >= 1 && d.grid.fnumber > 0.0, FQ_ERR_SHAPE,
               "batch: ensemble %d: bad grid", i);
    FQ_REQUIRE(d.flow.n_seg >= 0 && d.flow.n_seg <= FQ_MAX_SEGMENTS && (d.flow.n_seg == 0 || d.flow.seg),
               FQ_ERR_SHAPE, "batch: ensemble %d: n_seg must be in [0, %d]", i, FQ_MAX_SEGMENTS);
    FQ_REQUIRE(d.motion.n_terms >= 0 && d.motion.n_terms <= FQ_MAX_MOTION_TERMS, FQ_ERR_SHAPE,
               "batch: ensemble %d: motion n_terms must be in [0, 4]", i);
    FQ_REQUIRE(d.k_cut <= d.n_frames, FQ_ERR_INVALID_ARG, "batch: ensemble %d: k_cut > F", i);
    FQ_REQUIRE(d.k_cut >= 0 || (d.energy_thresh > 0.0 && d.energy_thresh <= 1.0), FQ_ERR_INVALID_ARG,
               "batch: ensemble %d: energy_thresh must be in (0, 1] when k_cut < 0", i);
    FQ_REQUIRE(d.p0 && d.seg_id && d.flow_coord && d.amp && d.pd, FQ_ERR_INVALID_ARG,
               "batch: ensemble %d: null device pointer", i);
    FQ_REQUIRE(rf_dtype == FQ_F32 || rf_dtype == FQ_BF16, FQ_ERR_UNSUPPORTED, "batch: dtype");
    return FQ_OK;
}

// ------------------------------------------------------------------ plan --
void item_grids(fq_batch *b, EnsHost &h)
{
    using namespace fqb;
    const int sc = cdiv(h.d.S, kItemScat);
    h.gx[ST_CLASSIFY] = sc; h.gy[ST_CLASSIFY] = 1; h.items[ST_CLASSIFY] = sc;
    h.gx[ST_ADVECT] = sc; h.gy[ST_ADVECT] = h.F; h.items[ST_ADVECT] = sc * h.F;
    int rf_groups = h.A, rf_group = 1;
    if (b->rf_quad) {
        size_t smem = 0;
        fqi::rf_quad_layout(b->params.data() + h.par_rf, &rf_groups, &rf_group, &smem);
    }
    h.gx[ST_RF] = cdiv(h.M, b->rf_quad ? 4 : kRfItemElems); h.gy[ST_RF] = rf_groups;
    h.items[ST_RF] = h.gx[ST_RF] * rf_groups * h.F;
    h.gx[ST_RF2IQ] = cdiv(h.ns, kIqTile); h.gy[ST_RF2IQ] = h.L;
    h.items[ST_RF2IQ] = h.gx[ST_RF2IQ] * h.L * (h.Fp / kFrameChunkB);
    // DAS tiles: voxels along x of one (y, z) row, das_threads / 4 of them and
    // 16 frames for FP32 channel data, das_threads / 32 (one warp each) and
    // 128 frames for 16-bit channel data
    const bool das_w = b->ch_dtype != FQ_F32;
    h.gx[ST_DAS] = cdiv(h.d.grid.nx, b->das_threads / (das_w ? 32 : kDasThreadsPerPixel)) * h.d.grid.ny * h.d.grid.nz;
    h.gy[ST_DAS] = das_w ? cdiv(h.Fp, kDasWarpFramesB) : h.Fp / kFrameChunkB;
    h.items[ST_DAS] = h.gx[ST_DAS] * h.gy[ST_DAS];
    const int nt = cdiv(h.F, 32);
    h.gx[ST_GRAM] = nt * (nt + 1) / 2; h.gy[ST_GRAM] = h.n_chunks; h.items[ST_GRAM] = h.gx[ST_GRAM] * h.n_chunks;
    h.gx[ST_GRAM_REDUCE] = cdiv((int64_t)h.F * h.F, 256); h.gy[ST_GRAM_REDUCE] = 1;
    h.items[ST_GRAM_REDUCE] = h.gx[ST_GRAM_REDUCE];
    h.gx[ST_EIG] = 1; h.gy[ST_EIG] = 1; h.items[ST_EIG] = 1;
    h.gx[ST_PROJECT] = cdiv(h.P, kItemPix); h.gy[ST_PROJECT] = 1; h.items[ST_PROJECT] = h.gx[ST_PROJECT];
    // relative cost of one item: what its inner loop runs over
    for (int s = 0; s < NS; ++s) h.cost[s] = 1.0;
    h.cost[ST_CLASSIFY] = 1.0 + h.d.flow.n_seg;
    h.cost[ST_RF] = (double)h.d.S * rf_group;
    h.cost[ST_RF2IQ] = 2.0 * h.J + 1.0;
    h.cost[ST_DAS] = (double)h.A * h.M;
    h.cost[ST_GRAM] = (double)h.chunk_len;
    h.cost[ST_GRAM_REDUCE] = h.n_chunks;
    h.cost[ST_EIG] = (double)h.F * h.F * h.F;
    h.cost[ST_PROJECT] = h.F;
}

// Queues, arena layout (everything but the waves and the scratch offsets).
void layout(fq_batch *b)
{
    for (auto &h : b->e) item_grids(b, h);
    size_t o = 0;
    b->off_counters = o; o += al256(sizeof(int) * b->waves.size() * NS);
    b->off_status = o; o += al256(sizeof(int) * b->n);
    b->off_ens = o; o += al256(sizeof(EnsDev) * b->n);
    b->off_params = o; o += al256(b->params.size());
    b->off_queues = o;
    for (auto &w : b->waves) {
        const int m = (int)w.members.size();
        for (int s = 0; s < NS; ++s) {
            w.order[s] = w.members;
            std::stable_sort(w.order[s].begin(), w.order[s].end(),
                             [&](int x, int y) { return b->e[x].cost[s] > b->e[y].cost[s]; });
            w.off[s].assign(m + 1, 0);
            for (int i = 0; i < m; ++i) w.off[s][i + 1] = w.off[s][i] + b->e[w.order[s][i]].items[s];
            w.total[s] = w.off[s][m];
            w.q_off[s] = o; o += al16(sizeof(int) * (m + 1));
            w.q_ens[s] = o; o += al16(sizeof(int) * m);
        }
        w.members_off = o; o += al16(sizeof(int) * m);
    }
    o = al256(o);
    b->off_scratch = o;
    size_t scratch = 0;
    for (auto &w : b->waves) scratch = std::max(scratch, w.scratch);
    b->total = o + scratch;
    b->uploaded = nullptr;
}

void scratch_sizes(fq_batch *b, EnsHost &h)
{
    size_t o = 0;
    h.off_pos = o; o += al256(sizeof(float) * 3 * (size_t)h.F * h.d.S);
    h.off_vessel = o; o += al256(sizeof(int32_t) * (size_t)h.d.S);
    h.off_amp = o; o += al256(sizeof(float) * (size_t)h.d.S);
    h.off_rf = o; o += al256(elem(b->rf_dtype) * (size_t)h.F * h.L * h.ns);
    h.off_ch = o; o += al256(elem(b->ch_dtype) * 2 * (size_t)h.L * h.ns * h.Fp);
    h.off_iq = o; o += al256(elem(b->iq_dtype) * 2 * (size_t)h.P * h.F);
    size_t cl_total = 0;
    fqi::clutter_layout_batched(h.P, h.F, h.cl, &h.n_chunks, &h.chunk_len, &cl_total);
    h.off_cws = o; o += al256(cl_total);
    h.scratch = o;
}

// ---------------------------------------------------------------- upload --
fq_status upload(fq_batch *b, char *arena, cudaStream_t st)
{
    if (b->uploaded == arena) return FQ_OK;
    const size_t lo = b->off_ens, hi = b->off_scratch;
    std::vector<unsigned char> img(hi - lo, 0);
    EnsDev *ed = reinterpret_cast<EnsDev *>(img.data());
    for (int i = 0; i < b->n; ++i) {
        const EnsHost &h = b->e[i];
        EnsDev &x = ed[i];
        std::memset(&x, 0, sizeof x);
        char *base = arena + b->off_scratch + h.wave_off;
        char *par = arena + b->off_params;
        x.p0 = h.d.p0;
        x.seg = h.d.seg_id;
        x.flow = h.d.flow_coord;
        x.amp = h.d.amp;
        x.pos = (float *)(base + h.off_pos);
        x.vessel = (int32_t *)(base + h.off_vessel);
        x.amp_eff = (float *)(base + h.off_amp);
        x.rf = base + h.off_rf;
        x.ch = base + h.off_ch;
        x.iq = base + h.off_iq;
        x.cws = base + h.off_cws;
        x.pd = h.d.pd;
        x.eigvals = h.d.eigvals;
        x.k_used = h.d.k_used;
        x.status = (int *)(arena + b->off_status) + i;
        x.seg_table = par + h.par_seg;
        x.motion = par + h.par_mot;
        x.rf_params = par + h.par_rf;
        x.iq_params = par + h.par_iq;
        x.das_params = par + h.par_das;
        x.S = h.d.S;
        x.P = h.P;
        x.F = h.F;
        x.Fp = h.Fp;
        x.A = h.A;
        x.M = h.M;
        x.ns = h.ns;
        x.L = h.L;
        x.t0 = h.d.t0;
        x.dt = h.d.dt;
        x.k_cut = h.d.k_cut;
        x.energy_thresh = h.d.energy_thresh;
        x.n_chunks = h.n_chunks;
        x.chunk_len = h.chunk_len;
        x.cl_G = h.cl[0]; x.cl_part = h.cl[1]; x.cl_V = h.cl[2]; x.cl_Vt = h.cl[3]; x.cl_lam = h.cl[4];
        x.cl_k = h.cl[5]; x.cl_hv = h.cl[6]; x.cl_tau = h.cl[7]; x.cl_big = h.cl[8]; x.cl_ii = h.cl[9];
        for (int s = 0; s < NS; ++s) {
            x.gx[s] = h.gx[s];
            x.gy[s] = h.gy[s];
        }
    }
    std::memcpy(img.data() + (b->off_params - lo), b->params.data(), b->params.size());
    for (auto &w : b->waves) {
        for (int s = 0; s < NS; ++s) {
            std::memcpy(img.data() + (w.q_off[s] - lo), w.off[s].data(), sizeof(int) * w.off[s].size());
            std::memcpy(img.data() + (w.q_ens[s] - lo), w.order[s].data(), sizeof(int) * w.order[s].size());
        }
        std::vector<int> eig = w.order[fqb::ST_EIG];
        std::memcpy(img.data() + (w.members_off - lo), eig.data(), sizeof(int) * eig.size());
    }
    fq_status s = fqi::cuda_check(cudaMemcpyAsync(arena + lo, img.data(), img.size(), cudaMemcpyHostToDevice, st),
                                  "batch: table upload");
    if (s) return s;
    s = fqi::cuda_check(cudaStreamSynchronize(st), "batch: table upload");
    if (s) return s;
    b->uploaded = arena;
    return FQ_OK;
}

// ---------------------------------------------------------------- launch --
fq_status launch_stage(fq_batch *b, char *arena, int w, int s, cudaStream_t st)
{
    const Wave &wv = b->waves[w];
    if (wv.total[s] == 0) return FQ_OK;
    const EnsDev *ens = reinterpret_cast<const EnsDev *>(arena + b->off_ens);
    StageQueue q;
    q.n = (int)wv.members.size();
    q.total = wv.total[s];
    q.off = reinterpret_cast<const int *>(arena + wv.q_off[s]);
    q.ens = reinterpret_cast<const int *>(arena + wv.q_ens[s]);
    q.counter = reinterpret_cast<int *>(arena + b->off_counters) + w * NS + s;
    switch (s) {
    case fqb::ST_CLASSIFY: return fqi::batched_classify(ens, q, q.total, st);
    case fqb::ST_ADVECT: return fqi::batched_advect(ens, q, q.total, st);
    case fqb::ST_RF: return fqi::batched_rf(ens, q, q.total, b->rf_dtype, b->rf_smem, b->rf_tune, b->rf_quad, st);
    case fqb::ST_RF2IQ: return fqi::batched_rf2iq(ens, q, q.total, b->rf_dtype, b->ch_dtype, b->J_max, st);
    case fqb::ST_DAS:
        return fqi::batched_das(ens, q, q.total, b->ch_dtype, b->iq_dtype, b->M_max, b->A_max, b->ns_max, b->das_threads, st);
    case fqb::ST_GRAM: return fqi::batched_gram(ens, q, q.total, b->iq_dtype, st);
    case fqb::ST_GRAM_REDUCE: return fqi::batched_gram_reduce(ens, q, q.total, st);
    case fqb::ST_EIG:
        return fqi::batched_eig(ens, reinterpret_cast<const int *>(arena + wv.members_off), q.n, st);
    case fqb::ST_PROJECT: return fqi::batched_project(ens, q, q.total, b->iq_dtype, st);
    default: return fqi::set_error(FQ_ERR_INVALID_ARG, "batch: stage %d", s);
    }
}

// Everything after the upload: counter and status reset, then the stages of
// every wave in order (stream-ordered, so each stage sees the previous one).
// With `ev`, ev[0] is recorded after the reset and ev[1 + w NS + s] after
// each stage.
fq_status launch_all(fq_batch *b, char *arena, cudaStream_t st, cudaEvent_t *ev = nullptr)
{
    fq_status s = fqi::cuda_check(cudaMemsetAsync(arena, 0, b->off_ens, st), "batch: counter reset");
    if (s) return s;
    if (ev) {
        s = fqi::cuda_check(cudaEventRecord(ev[0], st), "batch: event");
        if (s) return s;
    }
    for (int w = 0; w < (int)b->waves.size(); ++w)
        for (int stage = 0; stage < NS; ++stage) {
            s = launch_stage(b, arena, w, stage, st);
            if (s) return s;
            if (ev) {
                s = fqi::cuda_check(cudaEventRecord(ev[1 + w * NS + stage], st), "batch: event");
                if (s) return s;
            }
        }
    return FQ_OK;
}

fq_status check_arena(const fq_batch *b, const void *arena, size_t bytes, const char *who)
{
    FQ_REQUIRE(b, FQ_ERR_INVALID_ARG, "%s: null plan", who);
    FQ_REQUIRE(arena && bytes >= b->total, FQ_ERR_WORKSPACE, "%s: arena needs %zu bytes", who, b->total);
    FQ_REQUIRE(fqi::aligned(arena, 256), FQ_ERR_ALIGN, "%s: arena must be 256-byte aligned", who);
    return FQ_OK;
}

// ------------------------------------------------------------- autotune --
std::mutex g_tune_mu;
std::map<std::string, fq_tile_choice> g_tune;

std::string tune_key(int op, const fq_ensemble_desc &d, int dtype)
{
    char buf[256];
    std::snprintf(buf, sizeof buf, "%d|%d,%d,%d|%d|%d|%lld|%d,%d,%d|%d", op, d.probe.nx, d.probe.ny, d.probe.n_samples,
                  d.tx.n_angles, d.n_frames, (long long)d.S, d.grid.nx, d.grid.ny, d.grid.nz, dtype);
    return buf;
}

}  // namespace

extern "C" {

size_t fq_sizeof(int32_t which)
{
    switch (which) {
    case 0: return sizeof(fq_probe);
    case 1: return sizeof(fq_tx);
    case 2: return sizeof(fq_grid);
    case 3: return sizeof(fq_segment);
    case 4: return sizeof(fq_flow);
    case 5: return sizeof(fq_motion);
    case 6: return sizeof(fq_ensemble_desc);
    case 7: return sizeof(fq_tile_choice);
    case 8: return sizeof(fq_vfield);
    default: return 0;
    }
}

fq_status fq_batch_plan(const fq_ensemble_desc *ens, int32_t n, int32_t rf_dtype, int32_t ch_dtype, int32_t iq_dtype,
                        size_t max_arena_bytes, fq_batch **plan, size_t *arena_bytes)
{
    FQ_REQUIRE(ens && n >= 1 && plan, FQ_ERR_INVALID_ARG, "fq_batch_plan: null argument or n < 1");
    FQ_REQUIRE((ch_dtype == FQ_F32 || ch_dtype == FQ_BF16) && (iq_dtype == FQ_F32 || iq_dtype == FQ_BF16),
               FQ_ERR_UNSUPPORTED, "fq_batch_plan: dtypes must be FQ_F32 or FQ_BF16");
    *plan = nullptr;
    fq_batch *b = new fq_batch;
    b->n = n;
    b->rf_dtype = rf_dtype;
    b->ch_dtype = ch_dtype;
    b->iq_dtype = iq_dtype;
    b->budget = max_arena_bytes;
    b->e.resize(n);
    const size_t seg_b = fqi::seg_table_bytes(), mot_b = fqi::motion_bytes(), rf_b = fqi::rf_params_bytes(),
                 iq_b = fqi::iq_params_bytes(), das_b = fqi::das_params_bytes();
    b->params.assign((size_t)n * (seg_b + mot_b + rf_b + iq_b + das_b), 0);
    size_t po = 0;
    for (int i = 0; i < n; ++i) {
        const fq_ensemble_desc &d = ens[i];
        fq_status s = check_desc(d, i, rf_dtype);
        if (s) { delete b; return s; }
        EnsHost &h = b->e[i];
        h.d = d;
        h.d.tx.tilt_x = h.d.tx.tilt_y = nullptr;  // host arrays are read here only
        h.d.flow.seg = nullptr;
        h.A = d.tx.n_angles;
        h.M = d.probe.nx * d.probe.ny;
        h.ns = d.probe.n_samples;
        h.F = d.n_frames;
        h.Fp = fq_frame_pad(d.n_frames);
        h.L = h.A * h.M;
        h.P = (int64_t)d.grid.nx * d.grid.ny * d.grid.nz;
        unsigned char *pb = b->params.data();
        h.par_seg = po; fqi::build_seg_table(&d.flow, pb + po); po += seg_b;
        h.par_mot = po; fqi::build_motion(&d.motion, pb + po); po += mot_b;
        h.par_rf = po;
        s = fqi::build_rf_params(&d.probe, &d.tx, d.S, rf_dtype, pb + po);
        if (!s && !fqi::rf_ntap_ok(pb + po))
            s = fqi::set_error(FQ_ERR_UNSUPPORTED, "batch: ensemble %d: the batched RF kernel needs 8 <= n_cycles fs / f0 < 9", i);
        po += rf_b;
        if (!s) {
            h.par_iq = po;
            s = fqi::build_iq_params(&d.probe, h.L, h.F, pb + po, &h.J);
            po += iq_b;
        }
        if (!s) {
            h.par_das = po;
            s = fqi::build_das_params(&d.probe, &d.tx, h.F, &d.grid, pb + po);
            po += das_b;
        }
        if (s) { delete b; return s; }
        scratch_sizes(b, h);
        b->ns_max = std::max(b->ns_max, h.ns);
        b->J_max = std::max(b->J_max, h.J);
        b->M_max = std::max(b->M_max, h.M);
        b->A_max = std::max(b->A_max, h.A);
    }
    for (int i = 0; i < n; ++i)
        b->rf_quad = b->rf_quad && fqi::use_rf_quad(b->e[i].d.probe.nx) && fqi::rf_quad_ok(b->params.data() + b->e[i].par_rf);
    for (int i = 0; i < n; ++i) {
        size_t smem = 4 * sizeof(int) * (size_t)b->e[i].ns;  // paired kernel: hi and lo of 2 elements
        if (b->rf_quad) {
            int groups = 0, group = 0;
            fqi::rf_quad_layout(b->params.data() + b->e[i].par_rf, &groups, &group, &smem);
        }
        b->rf_smem = std::max(b->rf_smem, smem);
    }
    b->rf_tune = b->rf_quad ? 32 : 3;  // quad: resident warps per SM; pair: resident CTAs
    // waves: greedy in the given order under the budget
    for (int i = 0; i < n; ++i) {
        EnsHost &h = b->e[i];
        if (b->waves.empty() ||
            (max_arena_bytes && b->waves.back().scratch + h.scratch > max_arena_bytes && !b->waves.back().members.empty()))
            b->waves.emplace_back();
        Wave &w = b->waves.back();
        h.wave = (int)b->waves.size() - 1;
        h.wave_off = w.scratch;
        w.scratch += h.scratch;
        w.members.push_back(i);
    }
    layout(b);
    *plan = b;
    if (arena_bytes) *arena_bytes = b->total;
    return FQ_OK;
}

fq_status fq_batch_info(const fq_batch *plan, int32_t *n_waves, int64_t items[9])
{
    FQ_REQUIRE(plan, FQ_ERR_INVALID_ARG, "fq_batch_info: null plan");
    if (n_waves) *n_waves = (int32_t)plan->waves.size();
    if (items)
        for (int s = 0; s < NS; ++s) {
            items[s] = 0;
            for (const auto &w : plan->waves) items[s] += w.total[s];
        }
    return FQ_OK;
}

fq_status fq_batch_set_tile(fq_batch *plan, const fq_tile_choice *c)
{
    FQ_REQUIRE(plan && c, FQ_ERR_INVALID_ARG, "fq_batch_set_tile: null argument");
    if (c->op == FQ_OP_RF) {
        const bool ok = plan->rf_quad ? (c->choice == 16 || c->choice == 32) : (c->choice == 2 || c->choice == 3);
        FQ_REQUIRE(ok, FQ_ERR_INVALID_ARG, "fq_batch_set_tile: RF choice %d", c->choice);
        plan->rf_tune = c->choice;
        return FQ_OK;
    }
    if (c->op == FQ_OP_DAS) {
        FQ_REQUIRE(c->choice == 64 || c->choice == 128 || c->choice == 256, FQ_ERR_INVALID_ARG,
                   "fq_batch_set_tile: DAS choice %d", c->choice);
        if (plan->das_threads != c->choice) {
            plan->das_threads = c->choice;
            layout(plan);  // DAS item grid changes; tables are uploaded again
        }
        return FQ_OK;
    }
    return fqi::set_error(FQ_ERR_INVALID_ARG, "fq_batch_set_tile: op %d", c->op);
}

fq_status fq_batch_launch(fq_batch *plan, void *arena, size_t arena_bytes, void *stream)
{
    fq_status s = check_arena(plan, arena, arena_bytes, "fq_batch_launch");
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    s = upload(plan, (char *)arena, st);
    if (s) return s;
    return launch_all(plan, (char *)arena, st);
}

fq_status fq_batch_launch_profiled(fq_batch *plan, void *arena, size_t arena_bytes, void *stream, void **events,
                                   int32_t n_events)
{
    fq_status s = check_arena(plan, arena, arena_bytes, "fq_batch_launch_profiled");
    if (s) return s;
    FQ_REQUIRE(events && n_events >= 1 + NS * (int)plan->waves.size(), FQ_ERR_INVALID_ARG,
               "fq_batch_launch_profiled: needs %d events", 1 + NS * (int)plan->waves.size());
    cudaStream_t st = (cudaStream_t)stream;
    s = upload(plan, (char *)arena, st);
    if (s) return s;
    return launch_all(plan, (char *)arena, st, reinterpret_cast<cudaEvent_t *>(events));
}

fq_status fq_batch_status(fq_batch *plan, void *arena, void *stream)
{
    FQ_REQUIRE(plan && arena, FQ_ERR_INVALID_ARG, "fq_batch_status: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> flags(plan->n, 0);
    char *a = (char *)arena;
    fq_status s = fqi::cuda_check(cudaMemcpyAsync(flags.data(), a + plan->off_status, sizeof(int) * plan->n,
                                                  cudaMemcpyDeviceToHost, st), "fq_batch_status: read");
    if (s) return s;
    s = fqi::cuda_check(cudaStreamSynchronize(st), "fq_batch_status: sync");
    if (s) return s;
    s = fqi::cuda_check(cudaMemsetAsync(a + plan->off_status, 0, sizeof(int) * plan->n, st), "fq_batch_status: clear");
    if (s) return s;
    for (int i = 0; i < plan->n; ++i)
        if (flags[i])
            return fqi::set_error((fq_status)flags[i], "batch: ensemble %d reported %s", i,
                                  fq_status_string((fq_status)flags[i]));
    return FQ_OK;
}

void fq_batch_free(fq_batch *plan) { delete plan; }

fq_status fq_run_batched(const fq_ensemble_desc *ens, int32_t n, int32_t dtype, void *arena, size_t arena_bytes,
                         void *stream)
{
    fq_batch *b = nullptr;
    size_t need = 0;
    fq_status s = fq_batch_plan(ens, n, dtype, dtype, dtype, arena_bytes, &b, &need);
    if (s) return s;
    s = fq_batch_launch(b, arena, arena_bytes, stream);
    fq_batch_free(b);
    return s;
}

fq_status fq_graph_capture(fq_batch *plan, void *arena, size_t arena_bytes, fq_graph **graph)
{
    FQ_REQUIRE(graph, FQ_ERR_INVALID_ARG, "fq_graph_capture: null graph");
    *graph = nullptr;
    fq_status s = check_arena(plan, arena, arena_bytes, "fq_graph_capture");
    if (s) return s;
    cudaStream_t cs = nullptr;
    s = fqi::cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "fq_graph_capture: stream");
    if (s) return s;
    s = upload(plan, (char *)arena, cs);
    if (!s) s = fqi::cuda_check(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed), "fq_graph_capture: begin");
    cudaGraph_t g = nullptr;
    if (!s) {
        fq_status ls = launch_all(plan, (char *)arena, cs);
        cudaError_t ce = cudaStreamEndCapture(cs, &g);
        s = ls ? ls : fqi::cuda_check(ce, "fq_graph_capture: end");
    }
    fq_graph *out = nullptr;
    if (!s) {
        out = new fq_graph;
        out->g = g;
        s = fqi::cuda_check(cudaGraphInstantiate(&out->x, g, 0), "fq_graph_capture: instantiate");
        if (s) {
            cudaGraphDestroy(g);
            delete out;
            out = nullptr;
        }
    } else if (g) {
        cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    *graph = out;
    return s;
}

fq_status fq_graph_launch(fq_graph *graph, void *stream)
{
    FQ_REQUIRE(graph && graph->x, FQ_ERR_INVALID_ARG, "fq_graph_launch: null graph");
    return fqi::cuda_check(cudaGraphLaunch(graph->x, (cudaStream_t)stream), "fq_graph_launch");
}

void fq_graph_free(fq_graph *graph)
{
    if (!graph) return;
    if (graph->x) cudaGraphExecDestroy(graph->x);
    if (graph->g) cudaGraphDestroy(graph->g);
    delete graph;
}

fq_status fq_autotune(int32_t op, const fq_ensemble_desc *ens, int32_t rf_dtype, void *arena, size_t arena_bytes,
                      fq_tile_choice *out, void *stream)
{
    FQ_REQUIRE(ens && out, FQ_ERR_INVALID_ARG, "fq_autotune: null argument");
    FQ_REQUIRE(op == FQ_OP_RF || op == FQ_OP_DAS, FQ_ERR_INVALID_ARG, "fq_autotune: op %d", op);
    const std::string key = tune_key(op, *ens, rf_dtype);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *out = it->second;
            out->n_tried = 0;
            return FQ_OK;
        }
    }
    fq_batch *b = nullptr;
    size_t need = 0;
    fq_status s = fq_batch_plan(ens, 1, rf_dtype, rf_dtype, rf_dtype, 0, &b, &need);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    fq_tile_choice c;
    std::memset(&c, 0, sizeof c);
    c.op = op;
    const int cands_rf_pair[2] = {3, 2}, cands_rf_quad[2] = {32, 16}, cands_das[3] = {128, 64, 256};
    const int *cands = op == FQ_OP_RF ? (b->rf_quad ? cands_rf_quad : cands_rf_pair) : cands_das;
    const int nc = op == FQ_OP_RF ? 2 : 3;
    const int stage = op == FQ_OP_RF ? fqb::ST_RF : fqb::ST_DAS;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    s = check_arena(b, arena, arena_bytes, "fq_autotune");
    if (!s) s = fqi::cuda_check(cudaEventCreate(&e0), "fq_autotune: event");
    if (!s) s = fqi::cuda_check(cudaEventCreate(&e1), "fq_autotune: event");
    if (!s) s = fq_batch_launch(b, arena, arena_bytes, stream);  // inputs of every stage in place
    float best = 1e30f;
    for (int i = 0; i < nc && !s; ++i) {
        fq_tile_choice t;
        std::memset(&t, 0, sizeof t);
        t.op = op;
        t.choice = cands[i];
        s = fq_batch_set_tile(b, &t);
        if (!s) s = upload(b, (char *)arena, st);
        const int reps = 3;
        float ms = 0.0f;
        for (int r = 0; r <= reps && !s; ++r) {  // first run warms up
            int *ctr = reinterpret_cast<int *>((char *)arena + b->off_counters) + stage;
            s = fqi::cuda_check(cudaMemsetAsync(ctr, 0, sizeof(int), st), "fq_autotune: counter");
            if (!s && r == 1) s = fqi::cuda_check(cudaEventRecord(e0, st), "fq_autotune: event");
            if (!s) s = launch_stage(b, (char *)arena, 0, stage, st);
        }
        if (!s) s = fqi::cuda_check(cudaEventRecord(e1, st), "fq_autotune: event");
        if (!s) s = fqi::cuda_check(cudaEventSynchronize(e1), "fq_autotune: sync");
        if (!s) s = fqi::cuda_check(cudaEventElapsedTime(&ms, e0, e1), "fq_autotune: elapsed");
        if (s) break;
        ms /= reps;
        c.tried[c.n_tried] = cands[i];
        c.tried_ms[c.n_tried] = ms;
        ++c.n_tried;
        if (ms < best) {
            best = ms;
            c.choice = cands[i];
            c.ms = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    fq_batch_free(b);
    if (s) return s;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[key] = c;
    }
    *out = c;
    return FQ_OK;
}

}  // extern "C"
