// batch.cuh -- shared pieces of the batched persistent execution (many
// uneven ensembles, one persistent kernel per stage; Alg. 2-3 process the
// work in chunks, here the chunks of all ensembles form one queue).
//
// Each stage of a wave has a queue of work items: the items of every
// ensemble of the wave, laid out ensemble after ensemble in the order the
// host chose (most expensive items first).  A persistent CTA takes the next
// item with one atomicAdd on the stage's counter, finds its ensemble by a
// binary search over the prefix of item counts, and runs the same tile body
// as the single-ensemble kernel of that stage with the ensemble's own
// parameters.
#pragma once

#include "fq_internal.cuh"

namespace fqb {

constexpr int kItemScat = 2048;   // scatterers per classify / advect item
constexpr int kItemPix = 64;      // pixels per projection item (8 warps x 8)
constexpr int kRfItemElems = 2;   // receive elements per RF item (the paired kernel; 4 for the quad kernel)
constexpr int kIqTile = 128;      // rf2iq output samples per item
constexpr int kFrameChunkB = 16;  // frames per rf2iq / DAS item
constexpr int kDasThreadsPerPixel = 4;  // FP32 channel data (8 measured slower on the 2D benchmark)
constexpr int kDasWarpFramesB = 128;     // frames per DAS item of 16-bit channel data (one warp per voxel)

enum Stage {
    ST_CLASSIFY = 0,
    ST_ADVECT,
    ST_RF,
    ST_RF2IQ,
    ST_DAS,
    ST_GRAM,
    ST_GRAM_REDUCE,
    ST_EIG,
    ST_PROJECT,
    N_STAGES
};

// Per-ensemble device record (arena-resident; pointers are device pointers).
struct EnsDev {
    const float *p0;
    const int32_t *seg;
    const float *flow;
    const float *amp;
    float *pos;        // [F][3][S]
    int32_t *vessel;   // [S]
    float *amp_eff;    // [S]
    void *rf;          // [F][A][M][Ns]
    void *ch;          // [A*M][Ns][Fp][2]
    void *iq;          // [P][F][2]
    char *cws;         // clutter workspace (status word first)
    float *pd;         // [P]
    double *eigvals;   // [F]
    int32_t *k_used;   // [1]
    int *status;       // persistent status word of the ensemble (eigen-solver convergence)
    const void *seg_table;   // advect / classify segment table
    const void *motion;      // advect motion parameters
    const void *rf_params;   // RF synthesis parameters
    const void *iq_params;   // rf2iq parameters
    const void *das_params;  // DAS parameters
    int64_t S, P;
    int F, Fp, A, M, ns, L;
    double t0, dt;
    int k_cut;
    double energy_thresh;
    int n_chunks;            // Gram pixel chunks
    int64_t chunk_len;
    size_t cl_G, cl_part, cl_V, cl_Vt, cl_lam, cl_k, cl_hv, cl_tau, cl_big, cl_ii;  // clutter layout offsets
    int gx[N_STAGES], gy[N_STAGES];  // per-stage item grid (x fastest, then y, then z)
};

// One stage of one wave.
struct StageQueue {
    int n;             // ensembles in the wave
    int total;         // work items
    const int *off;    // [n + 1] prefix of item counts in execution order
    const int *ens;    // [n] ensemble index of each execution slot
    int *counter;      // reset to 0 before the launch
};

struct Item {
    int e;             // ensemble index
    int x, y, z;       // tile coordinates within the ensemble's grid for the stage
};

// Take the next item; every thread of the CTA calls it and gets the same
// answer.  False when the queue is empty.  Starts with a barrier so that the
// previous item's shared-memory use is finished.
__device__ __forceinline__ bool next_item(const StageQueue &q, const EnsDev *ens, int stage, int *s_buf, Item &it)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const int i = atomicAdd(q.counter, 1);
        int slot = -1;
        if (i < q.total) {
            int lo = 0, hi = q.n - 1;  // largest slot with off[slot] <= i
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (q.off[mid] <= i) lo = mid;
                else hi = mid - 1;
            }
            slot = lo;
        }
        s_buf[0] = i;
        s_buf[1] = slot;
    }
    __syncthreads();
    const int i = s_buf[0];
    if (i >= q.total) return false;
    const int slot = s_buf[1];
    it.e = q.ens[slot];
    const int local = i - q.off[slot];
    const int gx = ens[it.e].gx[stage], gy = ens[it.e].gy[stage];
    it.x = local % gx;
    it.y = (local / gx) % gy;
    it.z = local / (gx * gy);
    return true;
}

// Copy a parameter block of `bytes` (multiple of 16) from global to shared
// memory with the whole CTA; the caller synchronises.
__device__ __forceinline__ void copy_block(void *dst, const void *src, int bytes)
{
    const int4 *s = reinterpret_cast<const int4 *>(src);
    int4 *d = reinterpret_cast<int4 *>(dst);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
}

// Persistent grid: as many CTAs as fit on the GPU at once, at most one per
// item.  The kernel's dynamic shared-memory attribute must already be set.
template <typename K>
inline int persistent_grid(K kern, int threads, size_t smem, int items)
{
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return items < 1 ? 1 : items;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (occ < 1) occ = 1;
    if (sms < 1) sms = 1;
    const long g = (long)sms * occ;
    const long n = items < 1 ? 1 : items;
    return (int)(n < g ? n : g);
}

}  // namespace fqb

namespace fqi {

// Host launchers of the persistent stage kernels (one per source file).
// `ens` and the queue arrays are device pointers into the batch arena.
fq_status batched_classify(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, cudaStream_t st);
fq_status batched_advect(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, cudaStream_t st);
fq_status batched_rf(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int rf_dtype, size_t smem,
                     int minb, bool quad, cudaStream_t st);
fq_status batched_rf2iq(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int rf_dtype, int ch_dtype,
                        int J_max, cudaStream_t st);
fq_status batched_das(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int ch_dtype, int iq_dtype,
                      int M_max, int A_max, int ns_max, int threads, cudaStream_t st);
fq_status batched_gram(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int iq_dtype, cudaStream_t st);
fq_status batched_gram_reduce(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, cudaStream_t st);
fq_status batched_eig(const fqb::EnsDev *ens, const int *members, int n, cudaStream_t st);
fq_status batched_project(const fqb::EnsDev *ens, const fqb::StageQueue &q, int items, int iq_dtype,
                          cudaStream_t st);

// Parameter blocks of the stages (sizes rounded up to 16 bytes) and their
// host-side builders; the blocks are copied into the arena by the batch.
size_t seg_table_bytes();
size_t motion_bytes();
void build_seg_table(const fq_flow *flow, void *out);
void build_motion(const fq_motion *m, void *out);
size_t rf_params_bytes();
fq_status build_rf_params(const fq_probe *probe, const fq_tx *tx, int64_t S, int out_dtype, void *out);
int rf_ntap_ok(const void *rf_params);  // the packed-pair pulse kernel applies
bool use_rf_quad(int nx);               // the quad-element RF kernel applies to this probe
bool rf_quad_ok(const void *rf_params);  // ... and to these sizes (records fit in shared memory)
// quad RF kernel: angle groups per (frame, quad), angles per group, shared-memory bytes per CTA
void rf_quad_layout(const void *rf_params, int *n_groups, int *group, size_t *smem);
size_t iq_params_bytes();
fq_status build_iq_params(const fq_probe *probe, int L, int F, void *out, int *J);
size_t das_params_bytes();
fq_status build_das_params(const fq_probe *probe, const fq_tx *tx, int F, const fq_grid *g, void *out);
// clutter layout for the batched path: the eigen-solver's packed matrix
// always in the workspace (one CTA per ensemble, any F)
void clutter_layout_batched(int64_t P, int F, size_t off[10], int *n_chunks, int64_t *chunk_len, size_t *total);

}  // namespace fqi
