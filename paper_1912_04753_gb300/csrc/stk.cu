// C ABI of libstk.so: handles, argument checking and the job pipeline
//   (observed upload) -> CSR generation -> cell keys -> counting sort -> work list
//   -> persistent pair kernel -> finalize (K, L) -> envelope.
// Everything after argument checking runs on the handle's CUDA stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <vector>

#include "stk.h"
#include "stk_internal.h"

using namespace stk;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky launch error where possible
    if (e == cudaErrorMemoryAllocation)
        return fail(STK_ENOMEM, "%s: out of device memory", what);
    return fail(STK_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(expr, what)                                    \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

int ensure(DevBuf& b, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return STK_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(STK_ENOMEM, "cannot allocate %zu bytes of device memory for %s", bytes, what);
    }
    b.bytes = bytes;
    return STK_OK;
}

template <class T>
T* as(DevBuf& b) {
    return reinterpret_cast<T*>(b.p);
}

// byte offset of a polygon's band lists in its device buffer (after the vertices, the edge
// boxes, the FP32 edge table and the bucket lists)
size_t poly_band_offset(int nv) {
    return 96 * (size_t)nv + (size_t)kPolyBucketsMax * kPolyBucketsMax * kPolyBucketBytes;
}

}  // namespace

namespace stk {
// The y-band edge lists of a polygon (Polygon::band): band b of kPolyBands equal bands over the
// vertices' y-range lists the edges whose closed y-range meets the band widened by eps, far
// above the rounding of the band index on the device.
void build_poly_bands(const double* vx, const double* vy, int nv, uint8_t* out, double* ylo,
                      double* yhi) {
    (void)vx;
    double lo = vy[0], hi = vy[0];
    for (int k = 1; k < nv; ++k) {
        lo = std::min(lo, vy[k]);
        hi = std::max(hi, vy[k]);
    }
    const double bh = (hi - lo) / kPolyBands;
    const double eps = 1e-9 * (hi - lo) + 1e-12 * (fabs(lo) + fabs(hi));
    for (int b = 0; b < kPolyBands; ++b) {
        const double blo = lo + b * bh - eps, bhi = lo + (b + 1) * bh + eps;
        uint8_t* L = out + (size_t)b * kPolyBandBytes;
        int c = 0;
        for (int k = 0; k < nv; ++k) {
            const int k1 = (k + 1) % nv;
            if (std::min(vy[k], vy[k1]) <= bhi && std::max(vy[k], vy[k1]) >= blo)
                L[1 + c++] = (uint8_t)k;
        }
        L[0] = (uint8_t)c;
    }
    *ylo = lo;
    *yhi = hi;
}

void stk_note_error(int code, const char* msg) {
    (void)code;
    snprintf(g_err, sizeof g_err, "%s", msg);
}
}  // namespace stk

struct stk_handle {
    int device = 0;
    int num_sms = 0;
    int64_t n = 0;
    double box[6] = {0, 0, 0, 0, 0, 0};
    double* d_x = nullptr;
    double* d_y = nullptr;
    double* d_t = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // workspace (grow-only, resident between calls)
    DevBuf ux, uy, ut, key, rank, counts, start, scan_tmp;
    DevBuf X, Y, T, P, Plo, cell_start, chunks, chunk_off, items, counter;
    DevBuf acc_cnt, acc_lo, acc_hi, stats, pc, thr, self_pairs, mask_in, mask_sorted;
    DevBuf oK, oL, oS, oC, env, xq_e, xq_count, simseed, simid;
    DevBuf oA;  // raw accumulators of the last job's realizations, [R][4][nbins]
    DevBuf F;   // the pair filter's coordinate arrays, [m][3][filter_stride(n)]
    DevBuf stg; // the scatter's staging records, [m][n] x 32 bytes
    DevBuf fused;  // descriptors of a fused pair launch issued on this handle's stream
    // resident index of the observed pattern: its sorted arrays, cell counts and filter arrays
    // from the last job, reused while the grid and the record constants (obs_key) are the same
    DevBuf obs;
    std::vector<unsigned char> obs_key;
    int last_rows = 0, last_nbins = 0;  // shape of oA
    PairConsts* h_pc = nullptr;  // pinned host copy of the pair constants
    // pinned staging of the other per-job host inputs (graph-capturable copies)
    double* h_thr = nullptr;     // [2][STK_MAX_THRESHOLDS]
    uint64_t* h_seed = nullptr;  // [h_sim_cap]
    uint32_t* h_id = nullptr;
    size_t h_sim_cap = 0;
    // the last job, captured as one CUDA graph per wave, and what it was captured for
    std::vector<cudaGraphExec_t> gexecs;
    std::vector<unsigned char> gkey;
    std::vector<unsigned char> last_key;  // the shape of the last batched job (captured or not)
    stk_stats last;
    size_t smem32 = 0, smem64 = 0;
    int reps32 = 1, reps64 = 1;
    int configured_nbins = -1;
    size_t wave_budget = 0;  // device bytes a job may hold (0: a share of the free memory)
    // polygon study area (nv = 0: the box), vertices in device memory, and the area A of Eq. 2
    DevBuf poly;  // [nv] x, [nv] y (FP64), [nv] edge boxes (float4), [4 nv] float4 (pe32),
                  // the bucket lists (kPolyBucketsMax^2 x kPolyBucketBytes), the band lists
    int nv = 0;
    int poly_ccw = 1;
    double poly_span = 0.0;  // larger side of the polygon's bounding box
    double poly_bb[4] = {0.0, 0.0, 0.0, 0.0};  // its bounding box in the box frame
    double band_ylo = 0.0, band_yhi = 0.0;     // the band lists' y-range
    double area = 0.0;
    // inhomogeneous K: the relative intensity (device tables hcell and cum, [2][cells]), h of
    // the observed points in input order, and the per-wave h arrays (unsorted, sorted) and
    // whole-part accumulators
    DevBuf inh, inh_obs, uh, Hs, acc_whole;
    Intensity inten;    // inten.nix = 0: none
    int inh_zero = 0;   // some cell has rho = 0
    uint64_t inh_gen = 0;
};

namespace {

bool finite_in(double v, double lo, double hi) { return v >= lo && v <= hi; }

// The FP32-guarded pair kernel (every estimator has an instantiation of it).
bool fp32_path(const stk_handle* h, const stk_request* q) {
    (void)h;
    return q->prec == STK_PREC_FP32_GUARDED;
}

int check_box(const stk_box* b) {
    if (!b) return fail(STK_EINVAL, "box is NULL");
    const double v[6] = {b->x0, b->x1, b->y0, b->y1, b->t0, b->t1};
    for (double d : v)
        if (!isfinite(d)) return fail(STK_EINVAL, "box bounds must be finite");
    if (!(b->x0 < b->x1 && b->y0 < b->y1 && b->t0 < b->t1))
        return fail(STK_EINVAL, "box must satisfy x0<x1, y0<y1, t0<t1");
    return STK_OK;
}

int init_handle(stk_handle* h, int64_t n, const stk_box* box) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(STK_ENODEV, "no CUDA device: %s", cudaGetErrorString(e));
    }
    h->device = dev;
    CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev), "device query");
    h->n = n;
    h->box[0] = box->x0;
    h->box[1] = box->x1;
    h->box[2] = box->y0;
    h->box[3] = box->y1;
    h->box[4] = box->t0;
    h->box[5] = box->t1;
    h->area = (box->x1 - box->x0) * (box->y1 - box->y0);
    CK(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking), "stream create");
    h->stream = h->own_stream;
    CK(cudaEventCreate(&h->ev0), "event create");
    CK(cudaEventCreate(&h->ev1), "event create");
    CK(cudaMallocHost(reinterpret_cast<void**>(&h->h_pc), sizeof(PairConsts)), "pinned alloc");
    CK(cudaMallocHost(reinterpret_cast<void**>(&h->h_thr), 16 * STK_MAX_THRESHOLDS),
       "pinned alloc");
    const size_t bytes = sizeof(double) * (size_t)n;
    CK(cudaMalloc(reinterpret_cast<void**>(&h->d_x), bytes), "point upload");
    CK(cudaMalloc(reinterpret_cast<void**>(&h->d_y), bytes), "point upload");
    CK(cudaMalloc(reinterpret_cast<void**>(&h->d_t), bytes), "point upload");
    memset(&h->last, 0, sizeof h->last);
    return STK_OK;
}

void free_buf(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

int check_thresholds(const stk_handle* h, const double* s, int cs, const double* tt, int ct) {
    char err[256];
    if (validate_thresholds(h->box, s, cs, tt, ct, err, sizeof err)) return fail(STK_EINVAL, "%s", err);
    return STK_OK;
}

int configure_kernels(stk_handle* h, int nbins) {
    if (h->configured_nbins == nbins) return STK_OK;
    h->smem32 = pair_fp32_smem(nbins, &h->reps32);
    h->smem64 = pair_fp64_smem(nbins, &h->reps64);
    CK(pair_kernels_configure(h->smem32, h->smem64), "pair kernel configuration");
    h->configured_nbins = nbins;
    return STK_OK;
}

// FP64 queue entries for a wave of `points` points: four per point (the workloads measured
// push at most two per point), at most 2^27 (2 GiB).  An overflow is still evaluated exactly,
// but inside the pair kernel, where its FP64 work holds up the warp that meets it: the 2M-point
// job's 1.3e8 entries overflowing a queue of 2^24 cost its pair kernel 18%.
unsigned int exact_queue_cap(int64_t points) {
    int64_t c = 1 << 16;
    while (c < 4 * points && c < (int64_t(1) << 27)) c <<= 1;
    return (unsigned int)c;
}

// Device bytes of a job: `per_real` for every realization resident in a wave, `fixed` for the
// job's output rows and constants.
Footprint footprint(int64_t n, const Grid& g, int nbins, int R, int groups, bool fp32,
                    bool inh = false) {
    const size_t ncells = (size_t)g.ncells, nrows = (size_t)g.ny * g.nt, un = (size_t)n;
    Footprint f;
    // unsorted + keys/ranks + sorted FP64 + FP32 records + low parts; counts, starts, cell
    // starts, scan scratch; work counts/offsets and units; histograms; seeds; FP64 queue
    f.per_real = un * (24 + 8 + 24 + 32 + 8) + ncells * 12 + ncells / 256 + 8 +
                 (nrows + 1) * 8 + (nrows + un / kUnit + 1) * 16 + 4 + (size_t)nbins * 24 +
                 8 + 12 + (fp32 ? 64 * un : 0) + un /* role flags */ +
                 4 * 3 * (size_t)filter_stride(n) /* filter arrays */ +
                 32 * un /* scatter staging */ +
                 (inh ? 16 * un + 8 * (size_t)nbins : 0);
    f.fixed = 32 * 8 + 64 * (size_t)R * nbins +
              32 * (size_t)nbins * (size_t)(groups > 0 ? groups : 1) + sizeof(PairConsts) +
              16 * kMaxThr + 2 * un + ((size_t)1 << 16) * 16 + 4096;
    return f;
}

size_t workspace_bytes(const stk_handle* h) {
    const DevBuf* bufs[] = {&h->xq_e, &h->xq_count, &h->ux, &h->uy, &h->ut, &h->key, &h->rank,
                            &h->counts, &h->start, &h->scan_tmp, &h->X, &h->Y, &h->T, &h->P,
                            &h->Plo, &h->cell_start, &h->chunks, &h->chunk_off, &h->items,
                            &h->counter, &h->acc_cnt, &h->acc_lo, &h->acc_hi, &h->stats, &h->pc,
                            &h->thr, &h->self_pairs, &h->mask_in, &h->mask_sorted, &h->oK,
                            &h->oL, &h->oS, &h->oC, &h->env, &h->simseed, &h->simid, &h->uh,
                            &h->Hs, &h->acc_whole, &h->oA, &h->F, &h->stg, &h->fused, &h->obs};
    size_t b = 0;
    for (const DevBuf* d : bufs) b += d->bytes;
    return b;
}

// Runs the observed pattern (optional) and the simulations of `plan`; leaves per-realization
// K, L, S, C rows in h->oK/oL/oS/oC ([R][nbins], observed first) and one envelope per group of
// the plan in h->env ([groups][4][nbins]).
// Part of a fused pair launch (run_plans_fused): Prepare issues a job's generation and grid
// index, stops before its pair kernel and describes that kernel's work in `job`; Finish (the
// same job, after the fused launch) issues only what follows the pair kernel.
enum class FusePhase { Prepare, Finish };
struct FuseCtx {
    FusePhase phase = FusePhase::Prepare;
    FusedJob job{};
    bool even = false, edge = false;
    int nbins = 0;
    float ms_pair = 0.0f;            // Finish: the fused launch's time
    bool count_pair_launch = false;  // Finish: the fused launch counts in this job's launches
    int shape = 0;  // Prepare's launch shape (shape_code), which Finish repeats
};
constexpr int kNotFusable = -1000;  // run_job with a FuseCtx: the job cannot be fused

int run_job(stk_handle* h, const stk_request* q, bool include_obs, const SimPlan& plan,
            int* R_out, int f_force = 0, FuseCtx* fuse = nullptr);

// Launch-shape tuner: the first batched job of a problem shape (n, box, largest thresholds,
// precision, edge mode, simulation method, sectors) times the pair kernel on a few CSR
// realizations (about 4e6 point-realizations) for the grid refinement, the unit tile and the
// blocks per SM (tuned_refinement), and every later job of the shape takes that choice for the
// life of the process.
struct TuneKey {
    int64_t n;
    double box[6], s_max, t_max;
    int prec, edge, method, nsec;
    bool operator<(const TuneKey& o) const {
        return memcmp(this, &o, sizeof(TuneKey)) < 0;
    }
};
// A launch shape: grid refinement (fs | ft << 8), work units per tile claim and blocks per SM
// of the FP32 pair kernel; 0 = not chosen (planner / defaults).
struct TuneChoice {
    int f = 0, tile = 0, bps = 0;
};
// run_job's forced shape for the tuner's trials: f | tile << 16 | bps << 24
inline int shape_code(const TuneChoice& c) { return c.f | (c.tile << 16) | (c.bps << 24); }
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tuned;
thread_local bool t_tuning = false;  // the tuner's trial jobs are running (not logged)

// The problem shape of a job, for the tuner's table.
TuneKey tune_key(const stk_handle* h, const stk_request* q) {
    TuneKey key;
    memset(&key, 0, sizeof key);
    key.n = h->n;
    memcpy(key.box, h->box, sizeof key.box);
    key.s_max = q->s[q->cs - 1];
    key.t_max = q->tt[q->ct - 1];
    key.prec = q->prec;
    key.edge = q->edge_mode;
    key.nsec = q->n_sectors;
    key.method = q->sim_method;
    return key;
}

// The refinement tuned for this problem shape, if any (0: none yet).
// Launch shape for a job shape, timed once per process on a few CSR realizations and kept:
// first the grid refinement (fs = ft = 1, 2, 3, then the time axis one step either side), then
// with it the tile of work units a block claims (8, 32, 64 against 16), then, for the plain
// rectangle kernels, three blocks per SM (85 registers) against two.  The incumbent of each
// step (the planner's refinement, tile 16, two blocks) is replaced only by a shape 3% faster:
// trial timings of a few realizations differ by about 1% from run to run.
int tuned_refinement(stk_handle* h, const stk_request* q, TuneChoice* out) {
    const TuneKey key = tune_key(h, q);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            *out = it->second;
            return STK_OK;
        }
    }
    // a few realizations (about 4e6 point-realizations, at most 4) so that the timing is stable
    SimPlan trial;
    const int k_trial = (int)std::min<int64_t>(4, std::max<int64_t>(1, 4000000 / h->n));
    for (int k = 0; k < k_trial; ++k) {
        trial.seed.push_back(0x9E3779B97F4A7C15ull);
        trial.id.push_back((uint32_t)k);
    }
    stk_request tq = *q;
    tq.centre_mask = nullptr;
    tq.exec = STK_EXEC_BATCHED;  // the shape serves plain jobs too; trials run batched
    Grid gp;
    char err[256];
    if (build_grid(h->box, key.s_max, key.t_max, h->n, 0, &gp, err, sizeof err))
        return fail(STK_EINVAL, "%s", err);
    TuneChoice best;
    best.f = gp.fs | (gp.ft << 8);
    best.tile = (int)kTileUnitsDefault;
    best.bps = 2;
    float best_ms = -1.0f;
    // times shape c; `incumbent`: the step's default, which others must beat by 3%
    auto trial_run = [&](TuneChoice c, bool incumbent) -> int {
        int R = 0;
        t_tuning = true;
        const int rc = run_job(h, &tq, false, trial, &R, shape_code(c));
        t_tuning = false;
        if (rc == STK_ENOMEM) return STK_OK;  // a shape that does not fit is no candidate
        if (rc) return rc;
        float ms = (float)h->last.ms_pair;
        if (!incumbent) ms *= 1.03f;
        if (best_ms < 0.0f || ms < best_ms) best_ms = ms, best = c;
        return STK_OK;
    };
    const int planned = best.f;
    for (int f = 1; f <= 3; ++f) {
        TuneChoice c = best;
        c.f = f | (f << 8);
        const int rc = trial_run(c, c.f == planned);
        if (rc) return rc;
    }
    const int fs0 = best.f & 0xff;
    for (int ft = fs0 - 1; ft <= fs0 + 1; ft += 2) {
        if (ft < 1 || ft > 3) continue;
        TuneChoice c = best;
        c.f = fs0 | (ft << 8);
        const int rc = trial_run(c, c.f == planned);
        if (rc) return rc;
    }
    // the refinement's own time with the default shape is the incumbent of the next steps;
    // the tile and the block shape are the FP32 kernel's (the FP64 kernel has neither)
    if (fp32_path(h, q)) {
        const TuneChoice base = best;
        best_ms = -1.0f;
        int rc = trial_run(base, true);
        if (rc) return rc;
        for (int tile : {8, 32, 64}) {
            TuneChoice c = base;
            c.tile = tile;
            if ((rc = trial_run(c, false))) return rc;
        }
        if (pair_fp32_shape_tunable(*h->h_pc, h->inten.nix > 0)) {
            TuneChoice c = best;
            c.bps = 3;
            if ((rc = trial_run(c, false))) return rc;
        }
    }
    // a shape tuned meanwhile by another thread keeps its first choice
    std::lock_guard<std::mutex> lock(g_tune_mu);
    *out = g_tuned.emplace(key, best).first->second;
    return STK_OK;
}

// With STK_JOB_LOG set, every job appends one JSON line with its parameters and statistics
// to that file (jobs of several threads are serialised).
std::mutex g_log_mu;

void log_job(const stk_handle* h, const stk_request* q, int nsec) {
    if (t_tuning) return;
    const char* path = getenv("STK_JOB_LOG");
    if (!path || !*path) return;
    const stk_stats& st = h->last;
    std::lock_guard<std::mutex> lock(g_log_mu);
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"n\": %lld, \"realizations\": %d, \"waves\": %d, \"cs\": %d, \"ct\": %d, "
            "\"n_sectors\": %d, \"prec\": %d, \"edge_mode\": %d, \"norm\": %d, "
            "\"sim_method\": %d, \"polygon_vertices\": %d, \"intensity_cells\": %d, "
            "\"qualifying_pairs\": %lld, \"candidate_pairs\": %lld, \"fp64_recomputed\": %lld, "
            "\"ms_total\": %.3f, \"ms_pair\": %.3f, \"pairs_per_s\": %.6g, "
            "\"grid_refinement\": [%d, %d], \"graph_replays\": %d, \"kernel_launches\": %lld, "
            "\"internal_errors\": %lld}\n",
            (long long)h->n, st.realizations, st.waves, q->cs, q->ct, nsec, q->prec, q->edge_mode,
            q->norm, q->sim_method, h->nv, h->inten.nix * h->inten.niy * h->inten.nit,
            (long long)st.qualifying_pairs, (long long)st.candidate_pairs,
            (long long)st.fp64_recomputed, st.ms_total, st.ms_pair,
            st.ms_pair > 0 ? (double)st.qualifying_pairs / (st.ms_pair * 1e-3) : 0.0,
            st.grid_refinement, st.grid_refinement_t, st.graph_replays,
            (long long)st.kernel_launches, (long long)st.internal_errors);
    fclose(f);
}

// Eq. 2 normalisation of a request on h: A * D / (n (n - 1)) (A * D / n^2 with STK_NORM_N2);
// for a cross K the label counts take n's place: n_a n_b for two labels, n_a (n_a - 1) (or
// n_a^2) for a label with itself.
int job_coef(const stk_handle* h, const stk_request* q, double* coef) {
    const double nn = (double)h->n;
    double denom = q->norm == STK_NORM_N2 ? nn * nn : nn * (nn - 1.0);
    if (q->labels) {
        int64_t n_a = 0, n_b = 0;
        for (int64_t i = 0; i < h->n; ++i) {
            n_a += q->labels[i] == q->cross_a ? 1 : 0;
            n_b += q->labels[i] == q->cross_b ? 1 : 0;
        }
        if (n_a < 1 || n_b < 1 || (q->cross_a == q->cross_b && n_a < 2))
            return fail(STK_EINVAL, "cross K needs points of both labels");
        const double fa = (double)n_a, fb = (double)n_b;
        denom = q->cross_a != q->cross_b ? fa * fb
                                         : (q->norm == STK_NORM_N2 ? fa * fa : fa * (fa - 1.0));
    }
    *coef = h->area * (h->box[5] - h->box[4]) / denom;
    return STK_OK;
}

int run_job(stk_handle* h, const stk_request* q, bool include_obs, const SimPlan& plan,
            int* R_out, int f_force, FuseCtx* fuse) {
    const bool finish = fuse && fuse->phase == FusePhase::Finish;
    if (finish) f_force = fuse->shape;  // the grid and tile Prepare built
    using clock = std::chrono::steady_clock;
    const auto t_start = clock::now();
    h->last_rows = 0;  // the raw accumulator rows are the new job's from here on
    int rc = check_thresholds(h, q->s, q->cs, q->tt, q->ct);
    if (rc) return rc;
    if (q->edge_mode != STK_EDGE_NONE && q->edge_mode != STK_EDGE_ISOTROPIC &&
        q->edge_mode != STK_EDGE_TRANSLATION)
        return fail(STK_EINVAL, "unknown edge_mode %d", q->edge_mode);
    if (q->n_sectors < 0 || q->n_sectors > kMaxSectors)
        return fail(STK_EINVAL, "n_sectors must be in 0..%d", kMaxSectors);
    const int nsec = q->n_sectors > 1 ? q->n_sectors : 1;
    const bool dir = nsec > 1 || q->edge_mode == STK_EDGE_TRANSLATION;
    if (nsec > 1 && q->edge_mode == STK_EDGE_ISOTROPIC)
        return fail(STK_EINVAL,
                    "the directional K takes edge_mode NONE or TRANSLATION (the isotropic "
                    "weight is not unbiased direction by direction)");
    if (nsec > 1 && (int64_t)nsec * q->cs * q->ct > (int64_t)kMaxThr * kMaxThr)
        return fail(STK_EINVAL, "n_sectors * cs * ct must be at most %d", kMaxThr * kMaxThr);
    if (q->edge_mode == STK_EDGE_TRANSLATION && q->ct >= 1 && q->tt &&
        q->tt[q->ct - 1] > 0.5 * (h->box[5] - h->box[4]))
        return fail(STK_EINVAL,
                    "the translation correction needs t_ct <= half the study period (its "
                    "temporal factor D / (D - u) then stays <= 2)");
    if (dir && (h->nv > 0 || h->inten.nix > 0 || q->labels))
        return fail(STK_EINVAL,
                    "the translation correction and the directional K need the rectangle, no "
                    "intensity and no labels");
    if (q->prec != STK_PREC_FP64 && q->prec != STK_PREC_FP32_GUARDED)
        return fail(STK_EINVAL, "unknown prec %d", q->prec);
    if (q->shard_count < 0 || q->shard_count > (1 << 16) ||
        (q->shard_count > 1 && (q->shard_index < 0 || q->shard_index >= q->shard_count)))
        return fail(STK_EINVAL, "shard_index must be in 0 .. shard_count - 1 (shard_count <= 65536)");
    if (q->norm != STK_NORM_N_NM1 && q->norm != STK_NORM_N2)
        return fail(STK_EINVAL, "unknown norm %d", q->norm);
    if (q->exec != STK_EXEC_BATCHED && q->exec != STK_EXEC_PLAIN)
        return fail(STK_EINVAL, "unknown exec %d", q->exec);
    if (q->sim_method < STK_SIM_CSR || q->sim_method > STK_SIM_BOOTSTRAP)
        return fail(STK_EINVAL, "unknown sim_method %d", q->sim_method);
    if (q->labels && q->centre_mask)
        return fail(STK_EINVAL, "labels (cross K) and centre_mask cannot be combined");
    if (q->labels && q->sim_method == STK_SIM_BOOTSTRAP)
        return fail(STK_EINVAL, "cross K takes CSR or permutation simulations");
    if (q->labels && (q->cross_a < 0 || q->cross_a > 255 || q->cross_b < 0 || q->cross_b > 255))
        return fail(STK_EINVAL, "cross labels must be in 0..255");
    if (h->inten.nix > 0 && q->labels)
        return fail(STK_EINVAL, "the inhomogeneous K takes no labels (cross K)");
    if (h->nv > 0 && q->labels)
        return fail(STK_EINVAL, "cross K takes the rectangle, not a polygon study area");
    if (h->inten.nix > 0 && h->inh_zero && q->sim_method == STK_SIM_PERMUTATION &&
        plan.seed.size() > 0)
        return fail(STK_EINVAL,
                    "permutation simulations need rho > 0 in every cell (a permuted point "
                    "may fall in a cell with rho = 0)");
    const int n_sims = (int)plan.seed.size();
    if (n_sims > (1 << 24) || plan.id.size() != plan.seed.size())
        return fail(STK_EINVAL, "n_sims out of range");
    const int n_groups = (int)plan.groups.size();
    for (const auto& gr : plan.groups)
        if (gr.second <= 0 || gr.first < 0 || gr.first + gr.second > n_sims)
            return fail(STK_EINVAL, "bad envelope group");
    const int R = (include_obs ? 1 : 0) + n_sims;
    if (R < 1) return fail(STK_EINVAL, "nothing to compute (no observed pattern, n_sims = 0)");
    *R_out = R;
    const int64_t n = h->n;
    // a directional K holds nsec grids of cs x ct per realization
    const int cs = q->cs, ct = q->ct, nbins = cs * ct * nsec;
    const double lfac = (double)nsec;
    char err[256];
    Grid g;
    // launch shape: forced (tuner trials: shape_code), STK_GRID_F (and STK_GRID_FT for the time
    // axis), STK_TILE_UNITS, STK_BLOCKS_PER_SM, the tuner (STK_TUNE=0 disables it), or the
    // density planner with the default tile and two blocks per SM
    int f_req = f_force & 0xffff;
    int tile_req = (f_force >> 16) & 0xff, bps_req = (f_force >> 24) & 0xf;
    if (f_force == 0) {
        if (const char* fe = getenv("STK_GRID_F")) f_req = atoi(fe);
        if (const char* ft = getenv("STK_GRID_FT")) f_req |= atoi(ft) << 8;
        if (const char* te = getenv("STK_TILE_UNITS")) tile_req = atoi(te);
        if (const char* be = getenv("STK_BLOCKS_PER_SM")) bps_req = atoi(be);
    }
    const char* tune_env = getenv("STK_TUNE");
    const bool tune_on = !(tune_env && atoi(tune_env) == 0) && f_req == 0 && tile_req == 0 &&
                         bps_req == 0;
    if (tune_on) {
        // the first job of a problem shape tunes it, whatever its size, and every later job of
        // the shape takes that choice: a job's grids then never depend on which jobs came
        // before it or shared its batch (a served job equals the same job run alone)
        TuneChoice c;
        rc = tuned_refinement(h, q, &c);
        if (rc) return rc;
        f_req = c.f;
        tile_req = c.tile;
        bps_req = c.bps;
    }
    if (tile_req < 1 || tile_req > 255) tile_req = (int)kTileUnitsDefault;
    if (bps_req != 3 || fuse) bps_req = 2;  // the fused kernel has the 2-block shape only
    if (build_grid(h->box, q->s[cs - 1], q->tt[ct - 1], n, f_req, &g, err, sizeof err))
        return fail(STK_EINVAL, "%s", err);
    if (fuse && !finish) fuse->shape = (g.fs | (g.ft << 8)) | (tile_req << 16) | (bps_req << 24);
    cudaStream_t st = h->stream;
    CK(cudaStreamSynchronize(st), "stream sync");  // the pinned constants are reused below
    build_pair_consts(g, n, q->s, cs, q->tt, ct, q->edge_mode, h->h_pc);
    h->h_pc->nsec = nsec;
    h->h_pc->nbins = nbins;
    h->h_pc->tile_units = (uint32_t)tile_req;
    {  // failure-detection test hook, see PairConsts::never_publish
        const char* np = getenv("STK_TEST_NEVER_PUBLISH");
        h->h_pc->never_publish = (np && atoi(np) != 0) ? 1 : 0;
    }
    for (int m = 1; m < nsec; ++m) {  // sector boundaries m pi / nsec
        const double ang = (double)m * 3.14159265358979323846 / (double)nsec;
        h->h_pc->sec_bx[m - 1] = cos(ang);
        h->h_pc->sec_by[m - 1] = sin(ang);
    }
    h->h_pc->tw = h->box[1] - h->box[0];
    h->h_pc->th = h->box[3] - h->box[2];
    h->h_pc->td = h->box[5] - h->box[4];
    // FP32 directional kernel: boundaries and sides rounded to FP32.  Its offset is the exact
    // hi-part difference plus the low parts (x relative to the box with quantum qX, y relative
    // to the cell with quantum q_y; q the larger): within 2^-24 |d| + 3 2^-24 q of the offset the
    // points' FP64 coordinates give, which is itself within half an ulp of the largest
    // coordinate of the FP64 offset.  With the boundaries' rounding (2^-24 per component) and
    // the FP32 cross product's (2^-24 of each product), |cross_FP32 - cross_FP64| stays below
    // 2^-21 s_max + 2^-22 q + 4e-16 max|coordinate|, inside sec_g; the sign of d_y is certain
    // beyond sec_gd.
    for (int m = 1; m < nsec; ++m) {
        h->h_pc->sec_bxf[m - 1] = (float)h->h_pc->sec_bx[m - 1];
        h->h_pc->sec_byf[m - 1] = (float)h->h_pc->sec_by[m - 1];
    }
    h->h_pc->twf = (float)h->h_pc->tw;
    h->h_pc->thf = (float)h->h_pc->th;
    h->h_pc->tdf = (float)h->h_pc->td;
    {
        const double qm = std::max((double)g.qX, (double)g.qy);  // x: the box-frame quantum
        const double big = std::max(std::max(fabs(h->box[0]), fabs(h->box[1])),
                                    std::max(fabs(h->box[2]), fabs(h->box[3])));
        h->h_pc->sec_g = (float)(1.0e-6 * q->s[cs - 1] + 1.0e-6 * qm + 4.0e-16 * big + 1e-30);
        h->h_pc->sec_gd = (float)(1.0e-6 * qm + 4.0e-16 * big + 1e-30);
    }
    Polygon poly;
    double pb_bs = 0.0, pb_reach = 0.0;
    int pb_nx = 0, pb_ny = 0;
    if (h->nv > 0) {
        poly.vx = as<double>(h->poly);
        poly.vy = as<double>(h->poly) + h->nv;
        poly.nv = h->nv;
        poly.band = as<uint8_t>(h->poly) + poly_band_offset(h->nv);
        poly.band_ylo = h->band_ylo;
        poly.band_yhi = h->band_yhi;
        poly.band_inv = kPolyBands / (h->band_yhi - h->band_ylo);
        h->h_pc->pband = poly.band;
        h->h_pc->band_ylo = poly.band_ylo;
        h->h_pc->band_yhi = poly.band_yhi;
        h->h_pc->band_inv = poly.band_inv;
        h->h_pc->nv = h->nv;
        h->h_pc->pccw = h->poly_ccw;
        h->h_pc->pvx = poly.vx;
        h->h_pc->pvy = poly.vy;
        h->h_pc->pebox = reinterpret_cast<const float4*>(as<double>(h->poly) + 2 * h->nv);
        h->h_pc->pe32 = reinterpret_cast<const float4*>(as<double>(h->poly) + 4 * h->nv);
        h->h_pc->poly_f32 = 1;
        // bound on the error of the FP32 pair positions the polygon weight works with (box
        // frame): the records' hi + low parts (acc_x, acc_y, as for the pair offsets; they
        // bound one point's position and the vertices' FP64 box-frame values too), a row
        // origin row (chq + chl) (chl rounded: up to ny q_y 2^-24) and the pair arithmetic on
        // box-frame lengths (2^-44 of the box's extent each step); doubled
        const double acc_x = ldexp((double)g.qX, -24) + ldexp(fabs(g.x0) + fabs(g.x1), -50);
        const double acc_y = ldexp((double)g.qy, -22) + ldexp(fabs(g.y0) + fabs(g.y1), -50);
        const double ext = (g.x1 - g.x0) + (g.y1 - g.y0);
        const double eh = 2.0 * (2.0 * (acc_x + acc_y) + ldexp((double)g.ny * g.qy, -23) +
                                 ldexp(ext, -43));
        h->h_pc->poly_eh = (float)(eh * 1.001);
        h->h_pc->poly_span = (float)(h->poly_span * (1.0 - 1e-6));
        // bucket grid over the polygon's bounding box: side at least half the largest pair
        // radius, at most 64 buckets a side; a bucket lists the edges within the largest radius
        // plus half its diagonal of its centre, with a margin for the FP32 bucket index
        const double r_max = sqrt((double)h->h_pc->s2_cut) * (1.0 + 1e-6);
        const double bw = h->poly_bb[1] - h->poly_bb[0], bh = h->poly_bb[3] - h->poly_bb[2];
        pb_bs = std::max(0.5 * r_max, std::max(bw, bh) / (kPolyBucketsMax - 0.5));
        pb_nx = std::max(1, std::min(kPolyBucketsMax, (int)ceil(bw / pb_bs)));
        pb_ny = std::max(1, std::min(kPolyBucketsMax, (int)ceil(bh / pb_bs)));
        pb_reach = r_max + 0.5 * sqrt(2.0) * pb_bs * 1.001 +
                   1e-5 * (fabs(h->poly_bb[0]) + fabs(h->poly_bb[2]) + bw + bh);
        h->h_pc->pb_ox = (float)h->poly_bb[0];
        h->h_pc->pb_oy = (float)h->poly_bb[2];
        h->h_pc->pb_inv = (float)(1.0 / pb_bs);
        h->h_pc->pb_rmax = (float)(r_max * (1.0 - 1e-6));
        h->h_pc->pb_nx = pb_nx;
        h->h_pc->pb_ny = pb_ny;
        h->h_pc->pb_list = as<uint8_t>(h->poly) + 96 * (size_t)h->nv;
        // the deep-unit shortcut is derived for the rectangle: none in a polygon
        for (int a = 0; a < 2; ++a) {
            h->h_pc->deep_x[a] = 1 - a;
            h->h_pc->deep_y[a] = 1 - a;
        }
    }
    rc = configure_kernels(h, nbins);
    if (rc) return rc;

    // wave size: every realization of the wave is resident at once
    const int64_t ncells = g.ncells;
    const int64_t nrows = (int64_t)g.ny * g.nt;
    const bool inh = h->inten.nix > 0;
    const Footprint fp = footprint(n, g, nbins, R, n_groups, fp32_path(h, q), inh);
    int m_w = 1;
    size_t budget_job = 0;  // device bytes this job may hold (batched jobs)
    if (q->exec == STK_EXEC_BATCHED) {
        size_t budget = h->wave_budget;
        if (budget == 0) {
            size_t free_b = 0, total_b = 0;
            CK(cudaMemGetInfo(&free_b, &total_b), "memory query");
            budget = (size_t)(0.6 * (double)(free_b + workspace_bytes(h)));
            const char* env = getenv("STK_MEM_BUDGET_MB");
            if (env) budget = (size_t)atoll(env) << 20;
        }
        int64_t fit = budget > fp.fixed ? (int64_t)((budget - fp.fixed) / fp.per_real) : 1;
        if (fit < 1) fit = 1;
        const int64_t cap_idx = ((int64_t)1 << 31) / (n > 0 ? n : 1);  // 32-bit sorted offsets
        m_w = (int)std::min<int64_t>(std::min<int64_t>(fit, cap_idx > 0 ? cap_idx : 1), R);
        budget_job = budget;
    }
    const int64_t mn = (int64_t)m_w * n;
    const int64_t mc = (int64_t)m_w * ncells;
    const int64_t mr = (int64_t)m_w * nrows + 1;
    const size_t max_items = (size_t)m_w * ((size_t)nrows + (size_t)n / kUnit + 1);
    const int64_t tmp_words = std::max(scan_tmp_words(mc), scan_tmp_words(mr));
    if ((rc = ensure(h->ux, 8 * mn, "unsorted x")) || (rc = ensure(h->uy, 8 * mn, "unsorted y")) ||
        (rc = ensure(h->ut, 8 * mn, "unsorted t")) || (rc = ensure(h->key, 4 * mn, "keys")) ||
        (rc = ensure(h->rank, 4 * mn, "ranks")) || (rc = ensure(h->counts, 4 * mc, "counts")) ||
        (rc = ensure(h->start, 4 * mc, "starts")) ||
        (rc = ensure(h->scan_tmp, 4 * tmp_words, "scan scratch")) ||
        (rc = ensure(h->X, 8 * mn, "sorted x")) || (rc = ensure(h->Y, 8 * mn, "sorted y")) ||
        (rc = ensure(h->T, 8 * mn, "sorted t")) || (rc = ensure(h->P, 32 * (mn + 8), "FP32 points")) ||
        (rc = ensure(h->Plo, 8 * mn, "FP32 low parts")) ||
        (rc = ensure(h->F, 12 * (size_t)m_w * (size_t)filter_stride(n), "filter arrays")) ||
        (rc = ensure(h->stg, stage_bytes(m_w, n), "scatter staging")) ||
        (rc = ensure(h->cell_start, 4 * (mc + m_w), "cell starts")) ||
        (rc = ensure(h->chunks, 4 * mr, "work counts")) ||
        (rc = ensure(h->chunk_off, 4 * mr, "work offsets")) ||
        (rc = ensure(h->items, sizeof(WorkItem) * max_items, "work units")) ||
        (rc = ensure(h->counter, 4 * (size_t)m_w + 16, "unit counters")) ||
        (rc = ensure(h->acc_cnt, 8 * (size_t)m_w * nbins, "histograms")) ||
        (rc = ensure(h->acc_lo, 8 * (size_t)m_w * nbins, "histograms")) ||
        (rc = ensure(h->acc_hi, 8 * (size_t)m_w * nbins, "histograms")) ||
        (rc = ensure(h->stats, 64, "statistics")) || (rc = ensure(h->pc, sizeof(PairConsts), "constants")) ||
        (rc = ensure(h->thr, 8 * 2 * STK_MAX_THRESHOLDS, "thresholds")) ||
        (rc = ensure(h->self_pairs, 8 * (size_t)m_w * nsec, "self pairs")) ||
        (rc = ensure(h->oK, 8 * (size_t)R * nbins, "K grids")) ||
        (rc = ensure(h->oL, 8 * (size_t)R * nbins, "L grids")) ||
        (rc = ensure(h->oS, 8 * (size_t)R * nbins, "S grids")) ||
        (rc = ensure(h->oC, 8 * (size_t)R * nbins, "C grids")) ||
        (rc = ensure(h->oA, 32 * (size_t)R * nbins, "raw accumulators")) ||
        (rc = ensure(h->env, 8 * 4 * (size_t)nbins * (size_t)(n_groups > 0 ? n_groups : 1),
                     "envelope")) ||
        (rc = ensure(h->simseed, 8 * (size_t)m_w, "simulation seeds")) ||
        (rc = ensure(h->simid, 4 * (size_t)m_w, "simulation ids")))
        return rc;
    // FP64 queue: pairs the FP32 kernel cannot decide (well under 0.1% of pairs in practice);
    // overflow is still exact, evaluated inside the pair kernel
    const unsigned int xq_cap = exact_queue_cap((int64_t)m_w * n);
    if (inh && ((rc = ensure(h->uh, 8 * mn, "intensity ratios")) ||
                (rc = ensure(h->Hs, 8 * mn, "intensity ratios")) ||
                (rc = ensure(h->acc_whole, 8 * (size_t)m_w * nbins, "histograms"))))
        return rc;
    if (fp32_path(h, q) && ((rc = ensure(h->xq_e, sizeof(uint4) * (size_t)xq_cap, "FP64 queue")) ||
                         (rc = ensure(h->xq_count, 16, "FP64 queue"))))
        return rc;
    // per-point role flags (bit 0 centre, bit 1 neighbour): the sampled-centre mask of the
    // observed pattern, or the labels of a cross K for every realization
    const bool cross = q->labels != nullptr;
    const bool centre_mode = include_obs && q->centre_mask != nullptr;
    const bool use_mask = centre_mode || cross;
    int64_t n_a = n, n_b = n;
    if (use_mask) {
        if ((rc = ensure(h->mask_in, (size_t)n, "role flags")) ||
            (rc = ensure(h->mask_sorted, (size_t)n * (cross ? (size_t)m_w : 1), "role flags")))
            return rc;
        std::vector<uint8_t> flags((size_t)n);
        n_a = n_b = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (cross) {
                const bool fa = q->labels[i] == q->cross_a, fb = q->labels[i] == q->cross_b;
                flags[(size_t)i] = (uint8_t)((fa ? 1 : 0) | (fb ? 2 : 0));
                n_a += fa;
                n_b += fb;
            } else {
                flags[(size_t)i] = (uint8_t)((q->centre_mask[i] != 0 ? 1 : 0) | 2);
            }
        }
        if (cross && (n_a < 1 || n_b < 1 || (q->cross_a == q->cross_b && n_a < 2)))
            return fail(STK_EINVAL, "cross K needs points of both labels");
        // pageable source: staged before the call returns
        CK(cudaMemcpyAsync(h->mask_in.p, flags.data(), (size_t)n, cudaMemcpyHostToDevice, st),
           "role flags upload");
    }
    CK(cudaMemcpyAsync(h->pc.p, h->h_pc, sizeof(PairConsts), cudaMemcpyHostToDevice, st),
       "constants upload");
    if (h->nv > 0)
        CK(launch_poly_buckets(poly, h->box[0], h->box[2], h->poly_bb[0], h->poly_bb[2], pb_bs,
                               pb_nx, pb_ny, pb_reach, as<uint8_t>(h->poly) + 96 * (size_t)h->nv,
                               st),
           "polygon buckets");
    for (int a = 0; a < 2 * STK_MAX_THRESHOLDS; ++a) h->h_thr[a] = 0.0;
    for (int a = 0; a < cs; ++a) h->h_thr[a] = q->s[a];
    for (int b = 0; b < ct; ++b) h->h_thr[STK_MAX_THRESHOLDS + b] = q->tt[b];
    CK(cudaMemcpyAsync(h->thr.p, h->h_thr, 16 * STK_MAX_THRESHOLDS, cudaMemcpyHostToDevice, st),
       "threshold upload");
    // simulation keys and indices: pinned staging (the stream was idle at the start)
    if ((size_t)n_sims > h->h_sim_cap) {
        if (h->h_seed) cudaFreeHost(h->h_seed);
        if (h->h_id) cudaFreeHost(h->h_id);
        h->h_seed = nullptr;
        h->h_id = nullptr;
        h->h_sim_cap = 0;
        CK(cudaMallocHost(reinterpret_cast<void**>(&h->h_seed), 8 * (size_t)n_sims), "pinned alloc");
        CK(cudaMallocHost(reinterpret_cast<void**>(&h->h_id), 4 * (size_t)n_sims), "pinned alloc");
        h->h_sim_cap = (size_t)n_sims;
    }
    for (int k = 0; k < n_sims; ++k) {
        h->h_seed[k] = plan.seed[(size_t)k];
        h->h_id[k] = plan.id[(size_t)k];
    }
    if (!finish) CK(cudaMemsetAsync(h->stats.p, 0, 64, st), "memset");

    double coef = 0.0;
    if ((rc = job_coef(h, q, &coef))) return rc;
    const double* d_s = as<double>(h->thr);
    const double* d_tt = as<double>(h->thr) + STK_MAX_THRESHOLDS;
    const bool fp32 = fp32_path(h, q);
    int reps = fp32 ? h->reps32 : h->reps64;
    size_t smem = fp32 ? h->smem32 : h->smem64;
    if (inh) smem = fp32 ? pair_fp32_smem(nbins, &reps, true) : pair_fp64_smem(nbins, &reps, true);
    if (fp32 && !inh && h->nv > 0) smem += pair_fp32_poly_extra(nbins, reps);
    // the launch shape's blocks per SM: 3 only where the kernel has that instantiation
    const int shape_bps = fp32 && bps_req == 3 && pair_fp32_shape_tunable(*h->h_pc, inh) ? 3 : 2;
    const int bps = fp32 ? pair_fp32_blocks_per_sm(smem, shape_bps)
                         : pair_fp64_blocks_per_sm(smem, inh);
    const int grid = bps * h->num_sms;
    if (fuse && (!fp32 || q->exec != STK_EXEC_BATCHED || use_mask || inh || h->nv > 0 || dir ||
                 q->shard_count > 1 || (R + m_w - 1) / m_w != 1))
        return kNotFusable;  // fused jobs: plain FP32 rectangle kernels, one wave
    float ms_pair = 0.0f;
    int waves = 0;
    int64_t launches = h->nv > 0 ? 1 : 0;  // the polygon's bucket lists
    // resident observed index: reused when the grid, the record constants and the study area
    // are those of the cached copy (no role flags, no intensity: their per-point data differ)
    const int64_t nF = filter_stride(n);
    auto a256 = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t oc_cnt = 0, oc_x = a256(4 * (size_t)ncells), oc_y = oc_x + a256(8 * (size_t)n),
                 oc_t = oc_y + a256(8 * (size_t)n), oc_p = oc_t + a256(8 * (size_t)n),
                 oc_lo = oc_p + a256(32 * (size_t)n), oc_f = oc_lo + a256(8 * (size_t)n),
                 oc_end = oc_f + a256(12 * (size_t)nF);
    // (STK_RESIDENT=0 rebuilds the index every job)
    const char* resident_env = getenv("STK_RESIDENT");
    bool obs_cacheable = include_obs && !use_mask && !inh &&
                         !(resident_env && atoi(resident_env) == 0);
    std::vector<unsigned char> okey;
    if (obs_cacheable) {
        auto put = [&okey](const void* p, size_t b) {
            const unsigned char* c = reinterpret_cast<const unsigned char*>(p);
            okey.insert(okey.end(), c, c + b);
        };
        put(&g, sizeof g);
        const float rc3[3] = {h->h_pc->tan_rel, h->h_pc->tan_abs, h->h_pc->fast_abs};
        put(rc3, sizeof rc3);
        const void* pp[2] = {h->poly.p, (const void*)(intptr_t)h->nv};
        put(pp, sizeof pp);
    }
    // the resident index is kept only beside a job's workspace that leaves room for it
    if (obs_cacheable && budget_job > 0 &&
        fp.fixed + fp.per_real * (size_t)m_w + oc_end > budget_job) {
        obs_cacheable = false;
        free_buf(h->obs);
        h->obs_key.clear();
    }
    const bool obs_hit = obs_cacheable && !h->obs_key.empty() && okey == h->obs_key &&
                         h->obs.bytes >= oc_end;
    if (obs_cacheable && !obs_hit) {
        h->obs_key.clear();
        if (ensure(h->obs, oc_end, "observed index") != STK_OK) obs_cacheable = false;
    }
    unsigned char* oc = reinterpret_cast<unsigned char*>(h->obs.p);
    // kernels of one exclusive scan over `count` entries (tile pass + add pass per level)
    auto scan_launches = [](int64_t count) {
        int64_t k = 0;
        while (count > 2048) {
            k += 2;
            count = (count + 2047) / 2048;
        }
        return k + 1;
    };
    // every stream operation of the wave holding realizations r0 .. r0+m-1 (in_graph: being
    // captured; the events around the pair kernel then become event-record nodes of the graph)
    auto issue_wave = [&](int r0, int m, bool in_graph) -> int {
        const bool obs_here = include_obs && r0 == 0;
        const int first_sim_slot = obs_here ? 1 : 0;
        if (!finish) {  // generation, grid index, work list, cleared accumulators
        CK(cudaMemsetAsync(h->counts.p, 0, 4 * (size_t)m * ncells, st), "memset");
        if (obs_here && obs_hit) {  // the resident index: its cell counts feed the scan
            CK(cudaMemcpyAsync(h->counts.p, oc + oc_cnt, 4 * (size_t)ncells,
                               cudaMemcpyDeviceToDevice, st),
               "copy");
        } else if (obs_here) {
            CK(cudaMemcpyAsync(h->ux.p, h->d_x, 8 * n, cudaMemcpyDeviceToDevice, st), "copy");
            CK(cudaMemcpyAsync(h->uy.p, h->d_y, 8 * n, cudaMemcpyDeviceToDevice, st), "copy");
            CK(cudaMemcpyAsync(h->ut.p, h->d_t, 8 * n, cudaMemcpyDeviceToDevice, st), "copy");
            if (inh)
                CK(cudaMemcpyAsync(h->uh.p, h->inh_obs.p, 8 * n, cudaMemcpyDeviceToDevice, st),
                   "copy");
            CK(launch_keys_observed(h->d_x, h->d_y, h->d_t, n, g, as<uint32_t>(h->key),
                                    as<uint32_t>(h->rank), as<uint32_t>(h->counts),
                                    reinterpret_cast<int*>(as<unsigned long long>(h->stats) + 3), st),
               "cell keys");
        }
        if (m > first_sim_slot) {
            const int r_first = r0 + first_sim_slot;
            const int s_first = r_first - (include_obs ? 1 : 0);
            const int ms = m - first_sim_slot;
            CK(cudaMemcpyAsync(h->simseed.p, h->h_seed + s_first, 8 * (size_t)ms,
                               cudaMemcpyHostToDevice, st), "seeds");
            CK(cudaMemcpyAsync(h->simid.p, h->h_id + s_first, 4 * (size_t)ms,
                               cudaMemcpyHostToDevice, st), "seeds");
            const int64_t off = (int64_t)first_sim_slot * n;
            uint32_t* cnt0 = as<uint32_t>(h->counts) + (int64_t)first_sim_slot * ncells;
            if (q->sim_method == STK_SIM_CSR && inh)
                CK(launch_gen_inhom(n, ms, as<uint64_t>(h->simseed), as<uint32_t>(h->simid), g,
                                    h->inten, as<double>(h->ux) + off, as<double>(h->uy) + off,
                                    as<double>(h->ut) + off, as<double>(h->uh) + off,
                                    as<uint32_t>(h->key) + off, as<uint32_t>(h->rank) + off,
                                    cnt0, st),
                   "intensity-weighted generation");
            else if (q->sim_method == STK_SIM_CSR)
                CK(launch_gen_csr(n, ms, as<uint64_t>(h->simseed), as<uint32_t>(h->simid), g,
                                  as<double>(h->ux) + off, as<double>(h->uy) + off,
                                  as<double>(h->ut) + off, as<uint32_t>(h->key) + off,
                                  as<uint32_t>(h->rank) + off, cnt0, st, poly,
                                  as<unsigned long long>(h->stats) + 2),
                   "CSR generation");
            else
                CK(launch_gen_resample(q->sim_method, n, ms, as<uint64_t>(h->simseed),
                                       as<uint32_t>(h->simid), g, h->d_x, h->d_y, h->d_t,
                                       as<double>(h->ux) + off, as<double>(h->uy) + off,
                                       as<double>(h->ut) + off, as<uint32_t>(h->key) + off,
                                       as<uint32_t>(h->rank) + off, cnt0,
                                       as<unsigned long long>(h->stats) + 2, st),
                   "resampling");
            // resampled points take h from the cell they lie in (rho > 0 there: a bootstrap
            // point is an observed one; permutations need rho > 0 everywhere)
            if (inh && q->sim_method != STK_SIM_CSR)
                CK(launch_intensity_lookup(as<double>(h->ux) + off, as<double>(h->uy) + off,
                                           as<double>(h->ut) + off, (int64_t)ms * n, h->box,
                                           h->inten, as<double>(h->uh) + off,
                                           as<unsigned long long>(h->stats) + 2, st),
                   "intensity lookup");
        }
        CK(launch_exclusive_scan(as<uint32_t>(h->counts), as<uint32_t>(h->start),
                                 (int64_t)m * ncells, as<uint32_t>(h->scan_tmp), tmp_words, st),
           "cell scan");
        // with the resident index the observed slot is copied, not scattered
        const int s0 = (obs_here && obs_hit) ? 1 : 0;
        const int64_t so = (int64_t)s0 * n;
        if (m > s0)
            CK(launch_scatter(m - s0, n, g, as<double>(h->ux) + so, as<double>(h->uy) + so,
                              as<double>(h->ut) + so, as<uint32_t>(h->key) + so,
                              as<uint32_t>(h->rank) + so, as<uint32_t>(h->start),
                              (cross || (obs_here && centre_mode)) ? as<uint8_t>(h->mask_in)
                                                                   : nullptr,
                              as<double>(h->X), as<double>(h->Y), as<double>(h->T),
                              as<float4>(h->P), as<float2>(h->Plo), as<uint8_t>(h->mask_sorted),
                              h->h_pc->tan_rel, h->h_pc->tan_abs, h->h_pc->fast_abs,
                              as<float>(h->F), nF, as<double2>(h->stg), st, poly, cross,
                              inh ? as<double>(h->uh) + so : nullptr,
                              inh ? as<double>(h->Hs) : nullptr, s0),
               "scatter");
        if (obs_here && (obs_hit || obs_cacheable)) {
            // slot 0 <- resident index (hit), or resident index <- slot 0 (miss: fill it)
            struct Span {
                void* slot;
                size_t off, bytes;
            } sp[6] = {{h->X.p, oc_x, 8 * (size_t)n},       {h->Y.p, oc_y, 8 * (size_t)n},
                       {h->T.p, oc_t, 8 * (size_t)n},       {h->P.p, oc_p, 32 * (size_t)n},
                       {h->Plo.p, oc_lo, 8 * (size_t)n},    {h->F.p, oc_f, 12 * (size_t)nF}};
            for (const Span& q2 : sp) {
                void* dst = obs_hit ? q2.slot : (void*)(oc + q2.off);
                const void* src = obs_hit ? (const void*)(oc + q2.off) : q2.slot;
                CK(cudaMemcpyAsync(dst, src, q2.bytes, cudaMemcpyDeviceToDevice, st), "copy");
            }
            if (!obs_hit)
                CK(cudaMemcpyAsync(oc + oc_cnt, h->counts.p, 4 * (size_t)ncells,
                                   cudaMemcpyDeviceToDevice, st),
                   "copy");
        }
        CK(launch_cell_starts(m, n, ncells, as<uint32_t>(h->start), as<uint32_t>(h->cell_start),
                              st),
           "cell starts");
        CK(launch_work_counts(m, g, as<uint32_t>(h->cell_start), as<uint32_t>(h->chunks), st),
           "work counts");
        CK(launch_exclusive_scan(as<uint32_t>(h->chunks), as<uint32_t>(h->chunk_off),
                                 (int64_t)m * nrows + 1, as<uint32_t>(h->scan_tmp), tmp_words, st),
           "work scan");
        CK(launch_work_fill(m, g, as<uint32_t>(h->cell_start), as<uint32_t>(h->chunk_off),
                            as<WorkItem>(h->items), st),
           "work fill");
        const size_t accb = 8 * (size_t)m * nbins;
        CK(cudaMemsetAsync(h->acc_cnt.p, 0, accb, st), "memset");
        CK(cudaMemsetAsync(h->acc_lo.p, 0, accb, st), "memset");
        CK(cudaMemsetAsync(h->acc_hi.p, 0, accb, st), "memset");
        if (inh) CK(cudaMemsetAsync(h->acc_whole.p, 0, accb, st), "memset");
        CK(cudaMemsetAsync(h->counter.p, 0, 4 * (size_t)m, st), "memset");
        if (fp32) CK(cudaMemsetAsync(h->xq_count.p, 0, 16, st), "memset");
        // each unordered pair is evaluated once, never a point with itself
        CK(cudaMemsetAsync(h->self_pairs.p, 0, 8 * (size_t)m * nsec, st), "memset");
        }
        RealBatch rb;
        rb.P = as<float4>(h->P);
        rb.Plo = as<float2>(h->Plo);
        rb.X = as<double>(h->X);
        rb.Y = as<double>(h->Y);
        rb.T = as<double>(h->T);
        rb.cell_start = as<uint32_t>(h->cell_start);
        rb.mask = (cross || (obs_here && centre_mode)) ? as<uint8_t>(h->mask_sorted) : nullptr;
        rb.mask_all = cross ? 1 : 0;
        rb.n = n;
        rb.ncells = ncells;
        rb.H = inh ? as<double>(h->Hs) : nullptr;
        rb.F = as<float>(h->F);
        rb.nF = filter_stride(n);
        if (obs_here && q->shard_count > 1) {
            rb.shard_count = q->shard_count;
            rb.shard_index = q->shard_index;
        }
        Accum acc;
        acc.cnt = as<unsigned long long>(h->acc_cnt);
        acc.exc_lo = as<unsigned long long>(h->acc_lo);
        acc.exc_hi = as<unsigned long long>(h->acc_hi);
        acc.stats = as<unsigned long long>(h->stats);
        acc.whole = inh ? as<unsigned long long>(h->acc_whole) : nullptr;
        ExactQueue xq;
        xq.e = as<uint4>(h->xq_e);
        xq.count = as<unsigned int>(h->xq_count);
        xq.cap = xq_cap;
        if (fuse && !finish) {  // the fused launch runs this job's pair kernel
            fuse->job.pc = as<PairConsts>(h->pc);
            fuse->job.rb = rb;
            fuse->job.units = as<WorkItem>(h->items);
            fuse->job.unit_off = as<uint32_t>(h->chunk_off);
            fuse->job.counters = as<uint32_t>(h->counter);
            fuse->job.acc = acc;
            fuse->job.xq = xq;
            fuse->job.m = m;
            fuse->even = h->h_pc->even_s && h->h_pc->even_t;
            fuse->edge = h->h_pc->edge != 0;
            fuse->nbins = nbins;
            return STK_OK;
        }
        if (!finish)
            CK(cudaEventRecordWithFlags(h->ev0, st, in_graph ? cudaEventRecordExternal : 0),
               "event");
        if (finish) {
        } else if (fp32)
            CK(launch_pair_fp32(*h->h_pc, as<PairConsts>(h->pc), h->h_pc->even_s && h->h_pc->even_t,
                                h->h_pc->edge != 0, smem, reps, grid, m, rb,
                                as<WorkItem>(h->items), as<uint32_t>(h->chunk_off),
                                as<uint32_t>(h->counter), acc, xq, st, shape_bps),
               "pair kernel (FP32)");
        else
            CK(launch_pair_fp64(as<PairConsts>(h->pc), smem, reps, grid, m, rb,
                                as<WorkItem>(h->items), as<uint32_t>(h->chunk_off),
                                as<uint32_t>(h->counter), acc, st, h->nv > 0, inh, dir),
               "pair kernel (FP64)");
        if (!finish)
            CK(cudaEventRecordWithFlags(h->ev1, st, in_graph ? cudaEventRecordExternal : 0),
               "event");
        if (fp32) {
            CK(launch_exact(as<PairConsts>(h->pc), 4 * h->num_sms, rb, acc, xq, st, h->nv > 0,
                            dir),
               "FP64 queue");
        }
        // the wave's raw accumulators into the job's rows [R][4][nbins] (count, excess low and
        // high halves, whole part)
        {
            const size_t w8 = 8 * (size_t)nbins, pitch = 4 * w8;
            unsigned char* dst = reinterpret_cast<unsigned char*>(h->oA.p) + (size_t)r0 * pitch;
            const void* src[3] = {h->acc_cnt.p, h->acc_lo.p, h->acc_hi.p};
            for (int c = 0; c < 3; ++c)
                CK(cudaMemcpy2DAsync(dst + c * w8, pitch, src[c], w8, w8, (size_t)m,
                                     cudaMemcpyDeviceToDevice, st),
                   "accumulator copy");
            if (inh)
                CK(cudaMemcpy2DAsync(dst + 3 * w8, pitch, h->acc_whole.p, w8, w8, (size_t)m,
                                     cudaMemcpyDeviceToDevice, st),
                   "accumulator copy");
            else
                CK(cudaMemset2DAsync(dst + 3 * w8, pitch, 0, w8, (size_t)m, st), "memset");
        }
        const int64_t row = (int64_t)r0 * nbins;
        CK(launch_finalize(m * nsec, cs, ct, d_s, d_tt, coef, as<int64_t>(h->self_pairs), acc,
                           as<double>(h->oK) + row, as<double>(h->oL) + row,
                           as<double>(h->oS) + row, as<int64_t>(h->oC) + row, st, lfac),
           "finalize");
        return STK_OK;
    };
    // A batched job without role flags (centre mask, labels) whose shape, constants and buffers
    // repeat those of the job before it is captured as one CUDA graph per wave and replayed for
    // as long as they stay the same, so a one-off job pays no capture (STK_GRAPHS=1 captures a
    // shape at its first occurrence, 0 disables graphs).  The pair kernel is timed by
    // event-record nodes inside the graph.
    const char* graphs_env = getenv("STK_GRAPHS");
    const int graphs = graphs_env ? atoi(graphs_env) : -1;
    const bool graph_ok = q->exec == STK_EXEC_BATCHED && !use_mask && graphs != 0 && !fuse;
    std::vector<unsigned char> key;
    if (graph_ok) {
        auto put = [&key](const void* p, size_t b) {
            const unsigned char* c = reinterpret_cast<const unsigned char*>(p);
            key.insert(key.end(), c, c + b);
        };
        const int64_t sc[] = {n, R, include_obs, fp32, q->edge_mode, q->norm, cs, ct, grid,
                              (int64_t)smem, reps, (int64_t)xq_cap, tmp_words, ncells, nrows,
                              q->sim_method, inh, (int64_t)h->inh_gen, nsec, q->shard_count,
                              q->shard_index, obs_hit, obs_cacheable, shape_bps};
        put(sc, sizeof sc);
        put(&coef, sizeof coef);
        put(h->h_pc, sizeof(PairConsts));
        const void* ptrs[] = {h->ux.p, h->uy.p, h->ut.p, h->key.p, h->rank.p, h->counts.p,
                              h->start.p, h->scan_tmp.p, h->X.p, h->Y.p, h->T.p, h->P.p,
                              h->Plo.p, h->cell_start.p, h->chunks.p, h->chunk_off.p,
                              h->items.p, h->counter.p, h->acc_cnt.p, h->acc_lo.p, h->acc_hi.p,
                              h->stats.p, h->pc.p, h->thr.p, h->self_pairs.p, h->oK.p, h->oL.p,
                              h->oS.p, h->oC.p, h->xq_e.p, h->xq_count.p, h->simseed.p,
                              h->simid.p, h->d_x, h->d_y, h->d_t, h->h_seed, h->h_id,
                              (void*)h->ev0, (void*)h->ev1, (void*)st, h->uh.p, h->Hs.p,
                              h->acc_whole.p, h->inh.p, h->inh_obs.p, h->oA.p, h->F.p,
                              h->obs.p, h->stg.p};
        put(ptrs, sizeof ptrs);
    }
    int replays = 0;
    const int n_waves = (R + m_w - 1) / m_w;
    const bool replay = graph_ok && (int)h->gexecs.size() == n_waves && key == h->gkey;
    const bool use_graph = replay || (graph_ok && (graphs == 1 || key == h->last_key));
    if (graph_ok) h->last_key = key;
    if (use_graph && !replay) {
        for (cudaGraphExec_t ge : h->gexecs) cudaGraphExecDestroy(ge);
        h->gexecs.clear();
        h->gkey.clear();
    }
    for (int r0 = 0, wi = 0; r0 < R; r0 += m_w, ++wi) {
        const int m = std::min(m_w, R - r0);
        const bool obs_here = include_obs && r0 == 0;
        const int first_sim_slot = obs_here ? 1 : 0;
        if (use_graph && !replay) {  // capture this wave (its events become graph nodes)
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "graph capture");
            const int irc = issue_wave(r0, m, true);
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(st, &graph);
            if (irc) {
                if (graph) cudaGraphDestroy(graph);
                return irc;
            }
            CK(ec, "graph capture");
            cudaGraphExec_t ex = nullptr;
            const cudaError_t ei = cudaGraphInstantiate(&ex, graph, 0);
            cudaGraphDestroy(graph);
            CK(ei, "graph instantiate");
            h->gexecs.push_back(ex);
        }
        if (use_graph) {
            CK(cudaGraphLaunch(h->gexecs[(size_t)wi], st), "graph launch");
            if (replay) ++replays;
        } else {
            rc = issue_wave(r0, m, false);
            if (rc) return rc;
        }
        if (fuse && !finish) return STK_OK;  // Prepare ends before the pair kernel (one wave)
        float ms = 0.0f;
        if (finish) {
            ms = fuse->ms_pair;
        } else {
            CK(cudaEventSynchronize(h->ev1), "pair kernel");
            CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1), "event timing");
        }
        ms_pair += ms;
        ++waves;
        if (finish && !fuse->count_pair_launch) --launches;  // counted with another job
        launches += (obs_here && !obs_hit ? 1 : 0) + (m > first_sim_slot ? 1 : 0) +
                    scan_launches((int64_t)m * ncells) + scan_launches((int64_t)m * nrows + 1) +
                    4 /* scatter, starts, counts, fill */ -
                    (obs_here && obs_hit && m == 1 ? 1 : 0) /* no scatter */ +
                    2 /* pair, finalize */ + (fp32 ? 1 : 0) /* FP64 queue */;
    }
    if (use_graph && !replay) h->gkey = key;
    const int first_sim_row = include_obs ? 1 : 0;
    for (int gi = 0; gi < n_groups; ++gi) {
        const int g0 = plan.groups[gi].first, gn = plan.groups[gi].second;
        double* env = as<double>(h->env) + (size_t)gi * 4 * nbins;
        CK(launch_envelope(gn, nbins, cs, ct,
                           as<double>(h->oK) + (int64_t)(first_sim_row + g0) * nbins, d_s, d_tt,
                           env, env + nbins, env + 2 * nbins, env + 3 * nbins, st, lfac),
           "envelope");
    }
    unsigned long long stats[8];
    CK(cudaMemcpyAsync(stats, h->stats.p, sizeof stats, cudaMemcpyDeviceToHost, st), "stats");
    // qualifying pairs: the last cell of every grid (one per sector)
    std::vector<int64_t> lastC((size_t)R * nsec);
    CK(cudaMemcpy2DAsync(lastC.data(), 8, as<int64_t>(h->oC) + cs * ct - 1, 8 * (size_t)cs * ct,
                         8, (size_t)R * nsec, cudaMemcpyDeviceToHost, st),
       "counts");
    CK(cudaStreamSynchronize(st), "job");
    if (stats[3] != 0) return fail(STK_EDOMAIN, "a point lies outside the study box");
    if (stats[4] != 0)
        return fail(STK_ETIMEOUT,
                    "%llu bounded waits for work in the pair kernel ran out; the job's results "
                    "are incomplete",
                    stats[4]);
    h->last.qualifying_pairs = 0;
    for (int64_t c : lastC) h->last.qualifying_pairs += c;
    h->last.candidate_pairs = (int64_t)stats[0];
    h->last.fp64_recomputed = (int64_t)stats[1];
    h->last.work_items = 0;
    h->last.realizations = R;
    h->last.waves = waves;
    h->last.ms_pair = ms_pair;
    h->last.kernel_launches = launches;
    h->last.internal_errors = (int64_t)stats[2];
    h->last.grid_refinement = g.fs;
    h->last.grid_refinement_t = g.ft;
    h->last.tile_units = fp32 ? tile_req : 0;
    h->last.blocks_per_sm = bps;
    h->last.graph_replays = replays;
    h->last_rows = R;
    h->last_nbins = nbins;
    if (obs_cacheable && !obs_hit) h->obs_key = okey;
    h->last.obs_index_reused = obs_hit ? 1 : 0;
    h->last.ms_total =
        std::chrono::duration<double, std::milli>(clock::now() - t_start).count();
    log_job(h, q, nsec);
    return STK_OK;
}

SimPlan default_plan(const stk_request* q) {
    SimPlan p;
    const int ns = q->n_sims > 0 ? q->n_sims : 0;
    p.seed.assign((size_t)ns, q->seed);
    p.id.resize((size_t)ns);
    for (int k = 0; k < ns; ++k) p.id[(size_t)k] = q->first_sim + (uint32_t)k;
    if (ns > 0) p.groups.push_back({0, ns});
    return p;
}

int copy_rows(stk_handle* h, DevBuf& b, int64_t row0, int rows, int nbins, void* dst) {
    if (!dst) return STK_OK;
    CK(cudaMemcpyAsync(dst, reinterpret_cast<char*>(b.p) + 8 * row0 * nbins,
                       8 * (size_t)rows * nbins, cudaMemcpyDeviceToHost, h->stream),
       "result copy");
    return STK_OK;
}

}  // namespace

namespace stk {

int run_plan(stk_handle* h, const stk_request* q, const SimPlan& plan, bool include_obs) {
    int R = 0;
    return run_job(h, q, include_obs, plan, &R);
}

bool fusable_job(const stk_handle* h, const stk_request* q, int64_t R) {
    return q->exec == STK_EXEC_BATCHED && q->prec == STK_PREC_FP32_GUARDED &&
           (q->edge_mode == STK_EDGE_NONE || q->edge_mode == STK_EDGE_ISOTROPIC) &&
           q->n_sectors <= 1 && q->labels == nullptr && q->centre_mask == nullptr &&
           q->shard_count <= 1 && h->nv == 0 && h->inten.nix == 0 &&
           (double)h->n * (double)R < kFuseMaxPointRealizations;
}

int run_plans_fused(const std::vector<FusePart>& parts, int* fused_launches) {
    const size_t np = parts.size();
    if (fused_launches) *fused_launches = 0;
    std::vector<FuseCtx> ctx(np);
    std::vector<char> in_launch(np, 0);
    int rc = STK_OK;
    // 1. each part's generation and grid index on its own stream
    for (size_t i = 0; i < np; ++i) {
        int R = 0;
        if (!fusable_job(parts[i].h, parts[i].q, 1 + (int64_t)parts[i].plan->seed.size()))
            continue;  // runs alone below
        ctx[i].phase = FusePhase::Prepare;
        rc = run_job(parts[i].h, parts[i].q, true, *parts[i].plan, &R, 0, &ctx[i]);
        if (rc == kNotFusable) continue;  // runs alone below
        if (rc) return rc;
        in_launch[i] = 1;
    }
    // 2. one persistent pair launch per kernel class present (usually one), on the first
    // part's stream once every part's index is built; the parts' streams wait for it
    std::vector<cudaEvent_t> evs;
    auto new_event = [&evs](unsigned flags) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, flags) != cudaSuccess) return (cudaEvent_t) nullptr;
        evs.push_back(e);
        return e;
    };
    auto cleanup = [&evs]() {
        for (cudaEvent_t e : evs) cudaEventDestroy(e);
        evs.clear();
    };
    for (int cls = 0; cls < 4 && rc == STK_OK; ++cls) {
        std::vector<size_t> members;
        for (size_t i = 0; i < np; ++i)
            if (in_launch[i] && (ctx[i].even ? 2 : 0) + (ctx[i].edge ? 1 : 0) == cls)
                members.push_back(i);
        if (members.empty()) continue;
        stk_handle* h0 = parts[members[0]].h;
        cudaStream_t st0 = h0->stream;
        int nbins_max = 0;
        std::vector<FusedJob> jobs;
        for (size_t i : members) {
            nbins_max = std::max(nbins_max, ctx[i].nbins);
            jobs.push_back(ctx[i].job);
            cudaEvent_t built = new_event(cudaEventDisableTiming);
            if (!built || cudaEventRecord(built, parts[i].h->stream) != cudaSuccess ||
                cudaStreamWaitEvent(st0, built, 0) != cudaSuccess) {
                cleanup();
                return fail(STK_ECUDA, "fused launch: event");
            }
        }
        int reps = 1, reps64 = 1;
        const size_t smem = pair_fp32_smem(nbins_max, &reps);
        if (pair_kernels_configure(smem, pair_fp64_smem(nbins_max, &reps64)) != cudaSuccess ||
            ensure(h0->fused, sizeof(FusedJob) * jobs.size(), "fused launch") != STK_OK) {
            cleanup();
            return fail(STK_ECUDA, "fused launch: set-up");
        }
        cudaEvent_t t0 = new_event(cudaEventDefault), t1 = new_event(cudaEventDefault);
        cudaEvent_t done = new_event(cudaEventDisableTiming);
        const int grid = pair_fp32_fused_blocks_per_sm(smem) * h0->num_sms;
        cudaError_t e = (t0 && t1 && done) ? cudaSuccess : cudaErrorMemoryAllocation;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h0->fused.p, jobs.data(), sizeof(FusedJob) * jobs.size(),
                                cudaMemcpyHostToDevice, st0);
        if (e == cudaSuccess) e = cudaEventRecord(t0, st0);
        if (e == cudaSuccess)
            e = launch_pair_fp32_fused(ctx[members[0]].even, ctx[members[0]].edge, smem, reps,
                                       nbins_max, grid, as<FusedJob>(h0->fused),
                                       (int)jobs.size(), st0);
        if (e == cudaSuccess) e = cudaEventRecord(t1, st0);
        if (e == cudaSuccess) e = cudaEventRecord(done, st0);
        for (size_t i : members)
            if (e == cudaSuccess) e = cudaStreamWaitEvent(parts[i].h->stream, done, 0);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventSynchronize(t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        if (e != cudaSuccess) {
            cleanup();
            return fail(STK_ECUDA, "fused pair launch: %s", cudaGetErrorString(e));
        }
        for (size_t k = 0; k < members.size(); ++k) {
            ctx[members[k]].ms_pair = ms;
            ctx[members[k]].count_pair_launch = k == 0;
        }
        if (fused_launches) *fused_launches += 1;
    }
    cleanup();
    // 3. what follows each part's pair kernel, on its own stream
    for (size_t i = 0; i < np && rc == STK_OK; ++i) {
        if (!in_launch[i]) continue;
        int R = 0;
        ctx[i].phase = FusePhase::Finish;
        rc = run_job(parts[i].h, parts[i].q, true, *parts[i].plan, &R, 0, &ctx[i]);
    }
    // 4. parts that could not join the launch run alone
    for (size_t i = 0; i < np && rc == STK_OK; ++i) {
        if (in_launch[i]) continue;
        int R = 0;
        rc = run_job(parts[i].h, parts[i].q, true, *parts[i].plan, &R);
    }
    return rc;
}

int fetch_rows(stk_handle* h, int what, int row0, int rows, void* dst) {
    DevBuf* b = what == 0   ? &h->oK
                : what == 1 ? &h->oL
                : what == 2 ? &h->oS
                : what == 3 ? &h->oC
                            : &h->env;
    return copy_rows(h, *b, row0, rows, h->configured_nbins, dst);
}

int handle_sync(stk_handle* h) {
    CK(cudaStreamSynchronize(h->stream), "synchronise");
    return STK_OK;
}

int job_footprint(stk_handle* h, const stk_request* q, int R, int groups, Footprint* out) {
    int rc = check_thresholds(h, q->s, q->cs, q->tt, q->ct);
    if (rc) return rc;
    char err[256];
    Grid g;
    // the finest refinement the tuner may pick bounds the cell-dependent part
    int f_req = 3 | (3 << 8);
    if (const char* fe = getenv("STK_GRID_F")) f_req = atoi(fe);
    if (const char* ft = getenv("STK_GRID_FT")) f_req = (f_req & 0xff) | (atoi(ft) << 8);
    if (build_grid(h->box, q->s[q->cs - 1], q->tt[q->ct - 1], h->n, f_req, &g, err, sizeof err))
        return fail(STK_EINVAL, "%s", err);
    *out = footprint(h->n, g, q->cs * q->ct * (q->n_sectors > 1 ? q->n_sectors : 1), R, groups,
                     fp32_path(h, q), h->inten.nix > 0);
    return STK_OK;
}

size_t handle_workspace_bytes(const stk_handle* h) { return workspace_bytes(h); }

void handle_trim(stk_handle* h) {
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_buf(h->obs);
    h->obs_key.clear();
    DevBuf* bufs[] = {&h->xq_e, &h->xq_count, &h->ux, &h->uy, &h->ut, &h->key, &h->rank,
                      &h->counts, &h->start, &h->scan_tmp, &h->X, &h->Y, &h->T, &h->P,
                      &h->Plo, &h->cell_start, &h->chunks, &h->chunk_off, &h->items,
                      &h->counter, &h->acc_cnt, &h->acc_lo, &h->acc_hi, &h->stats, &h->pc,
                      &h->thr, &h->self_pairs, &h->mask_in, &h->mask_sorted, &h->oK, &h->oL,
                      &h->oS, &h->oC, &h->env, &h->simseed, &h->simid, &h->uh, &h->Hs,
                      &h->acc_whole, &h->oA, &h->F, &h->stg, &h->fused};
    for (DevBuf* b : bufs) free_buf(*b);
}

void handle_set_wave_budget(stk_handle* h, size_t bytes) { h->wave_budget = bytes; }

int64_t handle_points(const stk_handle* h) { return h->n; }

}  // namespace stk

extern "C" {

const char* stk_last_error(void) { return g_err; }

const char* stk_version(void) { return "stk-gb300 0.1 (sm_103a)"; }

int stk_create(const double* x, const double* y, const double* t, int64_t n, const stk_box* box,
               stk_handle** out) {
    if (!out) return fail(STK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!x || !y || !t) return fail(STK_EINVAL, "point arrays must not be NULL");
    if (n < 2) return fail(STK_EINVAL, "need n >= 2 points (got %lld)", (long long)n);
    if (n > ((int64_t)1 << 31) - 1) return fail(STK_EINVAL, "n too large");
    int rc = check_box(box);
    if (rc) return rc;
    for (int64_t i = 0; i < n; ++i) {
        if (!finite_in(x[i], box->x0, box->x1) || !finite_in(y[i], box->y0, box->y1) ||
            !finite_in(t[i], box->t0, box->t1))
            return fail(STK_EDOMAIN, "point %lld lies outside the study box or is not finite",
                        (long long)i);
    }
    stk_handle* h = new stk_handle();
    rc = init_handle(h, n, box);
    if (rc) {
        stk_destroy(h);
        return rc;
    }
    const size_t bytes = sizeof(double) * (size_t)n;
    cudaError_t e = cudaMemcpyAsync(h->d_x, x, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_y, y, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_t, t, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "point upload");
        stk_destroy(h);
        return rc;
    }
    *out = h;
    return STK_OK;
}

int stk_create_device(const double* d_x, const double* d_y, const double* d_t, int64_t n,
                      const stk_box* box, void* stream, stk_handle** out) {
    if (!out) return fail(STK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d_x || !d_y || !d_t) return fail(STK_EINVAL, "point arrays must not be NULL");
    if (n < 2) return fail(STK_EINVAL, "need n >= 2 points (got %lld)", (long long)n);
    if (n > ((int64_t)1 << 31) - 1) return fail(STK_EINVAL, "n too large");
    int rc = check_box(box);
    if (rc) return rc;
    stk_handle* h = new stk_handle();
    rc = init_handle(h, n, box);
    if (rc) {
        stk_destroy(h);
        return rc;
    }
    if (stream) h->stream = reinterpret_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(double) * (size_t)n;
    int bad = 0;
    cudaError_t e = cudaMemcpyAsync(h->d_x, d_x, bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_y, d_y, bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_t, d_t, bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) {
        rc = ensure(h->stats, 64, "statistics");
        if (rc) {
            stk_destroy(h);
            return rc;
        }
        e = cudaMemsetAsync(h->stats.p, 0, 64, h->stream);
    }
    if (e == cudaSuccess) e = launch_validate(h->d_x, h->d_y, h->d_t, n, h->box,
                                              reinterpret_cast<int*>(h->stats.p), h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&bad, h->stats.p, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "point copy");
        stk_destroy(h);
        return rc;
    }
    if (bad) {
        stk_destroy(h);
        return fail(STK_EDOMAIN, "a point lies outside the study box or is not finite");
    }
    *out = h;
    return STK_OK;
}

int stk_set_stream(stk_handle* h, void* stream) {
    if (!h) return fail(STK_EINVAL, "handle is NULL");
    h->stream = stream ? reinterpret_cast<cudaStream_t>(stream) : h->own_stream;
    return STK_OK;
}

// Copies the last job's observed grids, envelope and per-simulation grids into res (the
// pointers that are not NULL) and waits for the copies.
int download_result(stk_handle* h, const stk_request* req, stk_result* res) {
    int rc = STK_OK;
    const int nbins = req->cs * req->ct * (req->n_sectors > 1 ? req->n_sectors : 1);
    if ((rc = copy_rows(h, h->oK, 0, 1, nbins, res->K)) ||
        (rc = copy_rows(h, h->oL, 0, 1, nbins, res->L)) ||
        (rc = copy_rows(h, h->oS, 0, 1, nbins, res->raw_sum)) ||
        (rc = copy_rows(h, h->oC, 0, 1, nbins, res->pair_count)))
        return rc;
    if (req->n_sims > 0) {
        if ((rc = copy_rows(h, h->env, 0, 1, nbins, res->K_lo)) ||
            (rc = copy_rows(h, h->env, 1, 1, nbins, res->K_hi)) ||
            (rc = copy_rows(h, h->env, 2, 1, nbins, res->L_lo)) ||
            (rc = copy_rows(h, h->env, 3, 1, nbins, res->L_hi)) ||
            (rc = copy_rows(h, h->oK, 1, req->n_sims, nbins, res->K_sims)) ||
            (rc = copy_rows(h, h->oC, 1, req->n_sims, nbins, res->count_sims)))
            return rc;
    }
    CK(cudaStreamSynchronize(h->stream), "result copy");
    return STK_OK;
}

int stk_run(stk_handle* h, const stk_request* req, stk_result* res) {
    if (!h || !req || !res) return fail(STK_EINVAL, "handle, request and result must not be NULL");
    if (req->n_sims < 0 || req->n_sims > (1 << 24)) return fail(STK_EINVAL, "n_sims out of range");
    int R = 0;
    const int rc = run_job(h, req, true, default_plan(req), &R);
    if (rc) return rc;
    return download_result(h, req, res);
}

int stk_run_fused(stk_handle* const* hs, const stk_request* reqs, stk_result* results, int njobs,
                  int* pair_launches) {
    if (pair_launches) *pair_launches = 0;
    if (!hs || !reqs || !results || njobs < 1 || njobs > STK_MAX_FUSED_JOBS)
        return fail(STK_EINVAL, "handles, requests and results must not be NULL and njobs must "
                                "be in 1..%d", STK_MAX_FUSED_JOBS);
    for (int i = 0; i < njobs; ++i) {
        if (!hs[i]) return fail(STK_EINVAL, "handle %d is NULL", i);
        for (int k = 0; k < i; ++k)
            if (hs[k] == hs[i]) return fail(STK_EINVAL, "handle %d appears twice", i);
        if (reqs[i].n_sims < 0 || reqs[i].n_sims > (1 << 24))
            return fail(STK_EINVAL, "n_sims out of range (job %d)", i);
    }
    std::vector<SimPlan> plans(njobs);
    std::vector<FusePart> parts;
    for (int i = 0; i < njobs; ++i) {
        plans[i] = default_plan(&reqs[i]);
        parts.push_back({hs[i], &reqs[i], &plans[i]});
    }
    int launches = 0;
    int rc = run_plans_fused(parts, &launches);
    if (rc) return rc;
    for (int i = 0; i < njobs; ++i)
        if ((rc = download_result(hs[i], &reqs[i], &results[i]))) return rc;
    if (pair_launches) *pair_launches = launches;
    return STK_OK;
}

int stk_k(stk_handle* h, const double* s, int cs, const double* tt, int ct, int edge_mode,
          int prec, int norm, double* K, double* L, double* raw_sum, int64_t* pair_count) {
    stk_request q;
    memset(&q, 0, sizeof q);
    q.s = s;
    q.cs = cs;
    q.tt = tt;
    q.ct = ct;
    q.edge_mode = edge_mode;
    q.prec = prec;
    q.norm = norm;
    q.exec = STK_EXEC_BATCHED;
    stk_result r;
    memset(&r, 0, sizeof r);
    r.K = K;
    r.L = L;
    r.raw_sum = raw_sum;
    r.pair_count = pair_count;
    return stk_run(h, &q, &r);
}

int stk_envelope(stk_handle* h, const double* s, int cs, const double* tt, int ct, int edge_mode,
                 int prec, int norm, int n_sims, uint64_t seed, double* K_lo, double* K_hi,
                 double* L_lo, double* L_hi) {
    if (!h) return fail(STK_EINVAL, "handle is NULL");
    if (n_sims < 1) return fail(STK_EINVAL, "n_sims must be >= 1");
    stk_request q;
    memset(&q, 0, sizeof q);
    q.s = s;
    q.cs = cs;
    q.tt = tt;
    q.ct = ct;
    q.edge_mode = edge_mode;
    q.prec = prec;
    q.norm = norm;
    q.n_sims = n_sims;
    q.seed = seed;
    q.exec = STK_EXEC_BATCHED;
    if (n_sims > (1 << 24)) return fail(STK_EINVAL, "n_sims out of range");
    int R = 0;
    int rc = run_job(h, &q, false, default_plan(&q), &R);
    if (rc) return rc;
    const int nbins = cs * ct;
    if ((rc = copy_rows(h, h->env, 0, 1, nbins, K_lo)) || (rc = copy_rows(h, h->env, 1, 1, nbins, K_hi)) ||
        (rc = copy_rows(h, h->env, 2, 1, nbins, L_lo)) || (rc = copy_rows(h, h->env, 3, 1, nbins, L_hi)))
        return rc;
    CK(cudaStreamSynchronize(h->stream), "result copy");
    return STK_OK;
}

int stk_sim_points_polygon(const stk_box* box, const double* vx, const double* vy, int nv,
                           int64_t n, uint64_t seed, uint32_t sim, double* x, double* y,
                           double* t) {
    if (!x || !y || !t || !vx || !vy) return fail(STK_EINVAL, "arrays must not be NULL");
    if (n < 1 || n > ((int64_t)1 << 31) - 1) return fail(STK_EINVAL, "n out of range");
    if (nv < 3 || nv > kMaxPolyVertices)
        return fail(STK_EINVAL, "a polygon needs 3..%d vertices", kMaxPolyVertices);
    int rc = check_box(box);
    if (rc) return rc;
    Grid g;
    memset(&g, 0, sizeof g);
    g.nx = g.ny = g.nt = 1;
    g.ncells = 1;
    g.x0 = box->x0, g.x1 = box->x1, g.y0 = box->y0, g.y1 = box->y1, g.t0 = box->t0,
    g.t1 = box->t1;
    g.cw = box->x1 - box->x0, g.ch = box->y1 - box->y0, g.cd = box->t1 - box->t0;
    DevBuf bx, by, bt, bk, br, bc, bs, bp, be;
    DevBuf* all[] = {&bx, &by, &bt, &bk, &br, &bc, &bs, &bp, &be};
    auto release = [&]() {
        for (DevBuf* b : all) free_buf(*b);
    };
    const size_t b8 = 8 * (size_t)n, b4 = 4 * (size_t)n;
    if ((rc = ensure(bx, b8, "x")) || (rc = ensure(by, b8, "y")) || (rc = ensure(bt, b8, "t")) ||
        (rc = ensure(bk, b4, "keys")) || (rc = ensure(br, b4, "ranks")) ||
        (rc = ensure(bc, 16, "counts")) || (rc = ensure(bs, 16, "seed")) ||
        (rc = ensure(bp, 16 * (size_t)nv + (size_t)kPolyBands * kPolyBandBytes, "polygon")) ||
        (rc = ensure(be, 16, "status"))) {
        release();
        return rc;
    }
    struct {
        uint64_t seed;
        uint32_t sim, pad;
    } key_sim = {seed, sim, 0};
    std::vector<uint8_t> bands((size_t)kPolyBands * kPolyBandBytes, 0);
    Polygon poly;
    poly.vx = as<double>(bp);
    poly.vy = as<double>(bp) + nv;
    poly.nv = nv;
    poly.band = as<uint8_t>(bp) + 16 * (size_t)nv;
    build_poly_bands(vx, vy, nv, bands.data(), &poly.band_ylo, &poly.band_yhi);
    poly.band_inv = kPolyBands / (poly.band_yhi - poly.band_ylo);
    cudaStream_t st = nullptr;
    unsigned long long miss = 0;
    cudaError_t e = cudaMemcpyAsync(bp.p, vx, 8 * (size_t)nv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(as<double>(bp) + nv, vy, 8 * (size_t)nv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(as<uint8_t>(bp) + 16 * (size_t)nv, bands.data(), bands.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bc.p, 0, 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(be.p, 0, 16, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bs.p, &key_sim, sizeof key_sim, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_gen_csr(n, 1, as<uint64_t>(bs),
                           reinterpret_cast<const uint32_t*>(reinterpret_cast<char*>(bs.p) + 8),
                           g, as<double>(bx), as<double>(by), as<double>(bt), as<uint32_t>(bk),
                           as<uint32_t>(br), as<uint32_t>(bc), st, poly,
                           as<unsigned long long>(be));
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, bx.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, by.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t, bt.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&miss, be.p, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "CSR generation");
    if (miss) return fail(STK_EINVAL, "%llu points found no position inside the polygon", miss);
    return STK_OK;
}

int stk_sim_resample(const double* x0, const double* y0, const double* t0, int64_t n,
                     int method, uint64_t seed, uint32_t sim, double* x, double* y, double* t) {
    if (!x0 || !y0 || !t0 || !x || !y || !t) return fail(STK_EINVAL, "arrays must not be NULL");
    if (n < 1 || n > ((int64_t)1 << 31) - 1) return fail(STK_EINVAL, "n out of range");
    if (method != STK_SIM_PERMUTATION && method != STK_SIM_BOOTSTRAP)
        return fail(STK_EINVAL, "method must be STK_SIM_PERMUTATION or STK_SIM_BOOTSTRAP");
    // one cell holding everything: keys and ranks are by-products here
    Grid g;
    memset(&g, 0, sizeof g);
    g.nx = g.ny = g.nt = 1;
    g.ncells = 1;
    g.cw = g.ch = g.cd = 1.0;
    DevBuf bx0, by0, bt0, bx, by, bt, bk, br, bc, bs, be;
    const size_t b8 = 8 * (size_t)n, b4 = 4 * (size_t)n;
    DevBuf* all[] = {&bx0, &by0, &bt0, &bx, &by, &bt, &bk, &br, &bc, &bs, &be};
    auto release = [&]() {
        for (DevBuf* b : all) free_buf(*b);
    };
    int rc;
    if ((rc = ensure(bx0, b8, "x")) || (rc = ensure(by0, b8, "y")) || (rc = ensure(bt0, b8, "t")) ||
        (rc = ensure(bx, b8, "x")) || (rc = ensure(by, b8, "y")) || (rc = ensure(bt, b8, "t")) ||
        (rc = ensure(bk, b4, "keys")) || (rc = ensure(br, b4, "ranks")) ||
        (rc = ensure(bc, 16, "counts")) || (rc = ensure(bs, 16, "seed")) ||
        (rc = ensure(be, 16, "status"))) {
        release();
        return rc;
    }
    struct {
        uint64_t seed;
        uint32_t sim, pad;
    } key_sim = {seed, sim, 0};
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMemcpyAsync(bx0.p, x0, b8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(by0.p, y0, b8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bt0.p, t0, b8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bc.p, 0, 16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(be.p, 0, 16, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bs.p, &key_sim, sizeof key_sim, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_gen_resample(method, n, 1, as<uint64_t>(bs),
                                reinterpret_cast<const uint32_t*>(reinterpret_cast<char*>(bs.p) + 8),
                                g, as<double>(bx0), as<double>(by0), as<double>(bt0),
                                as<double>(bx), as<double>(by), as<double>(bt), as<uint32_t>(bk),
                                as<uint32_t>(br), as<uint32_t>(bc), as<unsigned long long>(be),
                                st);
    unsigned long long walk_err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, bx.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, by.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t, bt.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&walk_err, be.p, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "resampling");
    if (walk_err) return fail(STK_ECUDA, "internal consistency check failed (cycle walk)");
    return STK_OK;
}

int stk_sim_points(const stk_box* box, int64_t n, uint64_t seed, uint32_t sim, double* x,
                   double* y, double* t) {
    if (!x || !y || !t) return fail(STK_EINVAL, "output arrays must not be NULL");
    if (n < 1 || n > ((int64_t)1 << 31) - 1) return fail(STK_EINVAL, "n out of range");
    int rc = check_box(box);
    if (rc) return rc;
    const double b6[6] = {box->x0, box->x1, box->y0, box->y1, box->t0, box->t1};
    char err[128];
    Grid g;
    // one cell spanning the whole box: keys and ranks are by-products here
    if (build_grid(b6, box->x1 - box->x0, box->t1 - box->t0, n, 1, &g, err, sizeof err)) {
        g.nx = g.ny = g.nt = 1;
        g.ncells = 1;
        g.cw = box->x1 - box->x0;
        g.ch = box->y1 - box->y0;
        g.cd = box->t1 - box->t0;
    }
    DevBuf bx, by, bt, bk, br, bc, bs;
    const size_t b8 = 8 * (size_t)n, b4 = 4 * (size_t)n;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaSuccess;
    if ((rc = ensure(bx, b8, "x")) || (rc = ensure(by, b8, "y")) || (rc = ensure(bt, b8, "t")) ||
        (rc = ensure(bk, b4, "keys")) || (rc = ensure(br, b4, "ranks")) ||
        (rc = ensure(bc, 4 * (size_t)g.ncells, "counts")) || (rc = ensure(bs, 16, "seed"))) {
        free_buf(bx), free_buf(by), free_buf(bt), free_buf(bk), free_buf(br), free_buf(bc);
        free_buf(bs);
        return rc;
    }
    struct {
        uint64_t seed;
        uint32_t sim, pad;
    } key_sim = {seed, sim, 0};
    e = cudaMemsetAsync(bc.p, 0, 4 * (size_t)g.ncells, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bs.p, &key_sim, sizeof key_sim, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_gen_csr(n, 1, as<uint64_t>(bs),
                           reinterpret_cast<const uint32_t*>(reinterpret_cast<char*>(bs.p) + 8), g, as<double>(bx), as<double>(by), as<double>(bt), as<uint32_t>(bk),
                           as<uint32_t>(br), as<uint32_t>(bc), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, bx.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, by.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t, bt.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    free_buf(bx), free_buf(by), free_buf(bt), free_buf(bk), free_buf(br), free_buf(bc);
    free_buf(bs);
    if (e != cudaSuccess) return cuda_fail(e, "CSR generation");
    return STK_OK;
}

int stk_set_polygon(stk_handle* h, const double* vx, const double* vy, int nv) {
    if (!h) return fail(STK_EINVAL, "handle is NULL");
    if (nv == 0) {  // back to the rectangle
        free_buf(h->poly);
        h->nv = 0;
        h->area = (h->box[1] - h->box[0]) * (h->box[3] - h->box[2]);
        return STK_OK;
    }
    if (!vx || !vy) return fail(STK_EINVAL, "vertex arrays must not be NULL");
    if (h->inten.nix > 0)
        return fail(STK_EINVAL, "a polygon study area and an intensity cannot be combined");
    if (nv < 3 || nv > kMaxPolyVertices)
        return fail(STK_EINVAL, "a polygon needs 3..%d vertices", kMaxPolyVertices);
    double area2 = 0.0;
    for (int k = 0; k < nv; ++k) {
        if (!(vx[k] >= h->box[0] && vx[k] <= h->box[1] && vy[k] >= h->box[2] && vy[k] <= h->box[3]))
            return fail(STK_EINVAL, "polygon vertex %d is outside the handle's box", k);
        const int k1 = (k + 1) % nv;
        area2 += vx[k] * vy[k1] - vx[k1] * vy[k];
    }
    const double area = fabs(area2) * 0.5;
    const double box_area = (h->box[1] - h->box[0]) * (h->box[3] - h->box[2]);
    if (!(area > 0.0) || area * 64.0 < box_area)
        return fail(STK_EINVAL, "polygon area must be at least 1/64 of the box's");
    // edge bounding boxes in FP32 rounded outwards, for culling
    std::vector<float> ebox(4 * (size_t)nv);
    for (int k = 0; k < nv; ++k) {
        const int k1 = (k + 1) % nv;
        const double lo[2] = {fmin(vx[k], vx[k1]), fmin(vy[k], vy[k1])};
        const double hi[2] = {fmax(vx[k], vx[k1]), fmax(vy[k], vy[k1])};
        for (int c = 0; c < 2; ++c) {
            float l = (float)lo[c], u = (float)hi[c];
            if ((double)l > lo[c]) l = nextafterf(l, -INFINITY);
            if ((double)u < hi[c]) u = nextafterf(u, INFINITY);
            ebox[4 * (size_t)k + 2 * c] = l;
            ebox[4 * (size_t)k + 2 * c + 1] = u;
        }
    }
    // the FP32 polygon weight's edge table (poly_share_f32): per edge in the box frame the
    // start vertex, the unit direction and the normal's polar angle as pairs hi + lo of FP32
    // numbers (from FP64), the length, and the edge's box rounded outwards
    std::vector<float> pe32(16 * (size_t)nv, 0.0f);
    auto split = [](double v, float* o) {
        o[0] = (float)v;
        o[1] = (float)(v - (double)o[0]);
    };
    const double two_pi = 6.283185307179586;
    for (int k = 0; k < nv; ++k) {
        const int k1 = (k + 1) % nv;
        float* E = &pe32[16 * (size_t)k];
        const double ax = vx[k] - h->box[0], ay = vy[k] - h->box[2];
        const double bx = vx[k1] - h->box[0], by = vy[k1] - h->box[2];
        split(ax, E);
        split(ay, E + 2);
        const double dx = vx[k1] - vx[k], dy = vy[k1] - vy[k];
        const double len = sqrt(dx * dx + dy * dy);
        if (len > 0.0) {
            const double ux = dx / len, uy = dy / len;
            split(ux, E + 4);
            split(uy, E + 6);
            double phi = atan2(-ux, uy);
            if (phi < 0.0) phi += two_pi;
            split(phi, E + 8);
            E[10] = (float)len;
        }
        const double lo[2] = {fmin(ax, bx), fmin(ay, by)};
        const double hi[2] = {fmax(ax, bx), fmax(ay, by)};
        for (int c = 0; c < 2; ++c) {
            float l = (float)lo[c], u = (float)hi[c];
            if ((double)l > lo[c]) l = nextafterf(l, -INFINITY);
            if ((double)u < hi[c]) u = nextafterf(u, INFINITY);
            E[12 + 2 * c] = l;
            E[13 + 2 * c] = u;
        }
    }
    int rc;
    DevBuf pv;
    std::vector<uint8_t> bands((size_t)kPolyBands * kPolyBandBytes, 0);
    double band_ylo = 0.0, band_yhi = 0.0;
    build_poly_bands(vx, vy, nv, bands.data(), &band_ylo, &band_yhi);
    if ((rc = ensure(pv, poly_band_offset(nv) + bands.size(), "polygon"))) return rc;
    cudaStream_t st = h->stream;
    int bad = 0;
    DevBuf flag;
    if ((rc = ensure(flag, 16, "status"))) {
        free_buf(pv);
        return rc;
    }
    Polygon poly;
    poly.vx = as<double>(pv);
    poly.vy = as<double>(pv) + nv;
    poly.nv = nv;
    cudaError_t e = cudaMemcpyAsync(pv.p, vx, 8 * (size_t)nv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(as<double>(pv) + nv, vy, 8 * (size_t)nv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(as<double>(pv) + 2 * nv, ebox.data(), 16 * (size_t)nv,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(as<double>(pv) + 4 * nv, pe32.data(), 64 * (size_t)nv,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(as<uint8_t>(pv) + poly_band_offset(nv), bands.data(), bands.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag.p, 0, 4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // ebox and pe32 are read
    if (e == cudaSuccess) e = launch_poly_validate(h->d_x, h->d_y, h->n, poly, as<int>(flag), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, flag.p, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    free_buf(flag);
    if (e != cudaSuccess) {
        free_buf(pv);
        return cuda_fail(e, "polygon upload");
    }
    if (bad) {
        free_buf(pv);
        return fail(STK_EDOMAIN, "a point lies outside the polygon");
    }
    free_buf(h->poly);
    h->poly = pv;
    h->nv = nv;
    h->band_ylo = band_ylo;
    h->band_yhi = band_yhi;
    h->poly_bb[0] = *std::min_element(vx, vx + nv) - h->box[0];
    h->poly_bb[1] = *std::max_element(vx, vx + nv) - h->box[0];
    h->poly_bb[2] = *std::min_element(vy, vy + nv) - h->box[2];
    h->poly_bb[3] = *std::max_element(vy, vy + nv) - h->box[2];
    h->poly_span = std::max(h->poly_bb[1] - h->poly_bb[0], h->poly_bb[3] - h->poly_bb[2]);
    h->poly_ccw = area2 > 0.0 ? 1 : 0;
    h->area = area;
    return STK_OK;
}

}  // extern "C"

namespace {

// Host tables of a relative intensity: tab[0 .. cells) = mean(rho) / rho_c (0 where rho_c = 0)
// and tab[cells .. 2 cells) = rho_0 + ... + rho_c, added in cell order.  Checks the values and
// the range rule (every rho_c > 0 within 2^14 of the mean either way, which keeps a pair
// weight below 2^31).
int intensity_tables(const double* rho, int nix, int niy, int nit, std::vector<double>& tab,
                     Intensity* in, int* zero) {
    if (!rho) return fail(STK_EINVAL, "rho must not be NULL");
    if (nix < 1 || niy < 1 || nit < 1 || (int64_t)nix * niy * nit > ((int64_t)1 << 22))
        return fail(STK_EINVAL, "intensity grid must have 1..2^22 cells (nix, niy, nit >= 1)");
    const int cells = nix * niy * nit;
    double sum = 0.0;
    int last = -1;
    *zero = 0;
    tab.assign(2 * (size_t)cells, 0.0);
    for (int c = 0; c < cells; ++c) {
        const double r = rho[c];
        if (!(r >= 0.0) || !isfinite(r))
            return fail(STK_EINVAL, "rho[%d] must be finite and >= 0", c);
        sum += r;
        tab[(size_t)cells + c] = sum;
        if (r > 0.0)
            last = c;
        else
            *zero = 1;
    }
    if (last < 0 || !isfinite(sum)) return fail(STK_EINVAL, "rho must have a positive, finite sum");
    const double mean = sum / (double)cells;
    for (int c = 0; c < cells; ++c) {
        if (rho[c] == 0.0) continue;
        const double hc = mean / rho[c];
        if (!(hc <= 16384.0 && hc >= 1.0 / 16384.0))
            return fail(STK_EINVAL,
                        "rho[%d] is more than 2^14 times below or above the mean of rho", c);
        tab[(size_t)c] = hc;
    }
    in->nix = nix;
    in->niy = niy;
    in->nit = nit;
    in->total = tab[2 * (size_t)cells - 1];
    in->last_pos = last;
    return STK_OK;
}

}  // namespace

extern "C" {

int stk_set_intensity(stk_handle* h, const double* rho, int nix, int niy, int nit) {
    if (!h) return fail(STK_EINVAL, "handle is NULL");
    cudaStream_t st = h->stream;
    CK(cudaStreamSynchronize(st), "stream sync");  // no running job reads the old tables
    if (rho == nullptr || nix == 0) {  // back to the homogeneous estimator
        free_buf(h->inh);
        free_buf(h->inh_obs);
        h->inten = Intensity();
        h->inh_zero = 0;
        ++h->inh_gen;
        return STK_OK;
    }
    if (h->nv > 0)
        return fail(STK_EINVAL, "a polygon study area and an intensity cannot be combined");
    std::vector<double> tab;
    Intensity in;
    int zero = 0;
    int rc = intensity_tables(rho, nix, niy, nit, tab, &in, &zero);
    if (rc) return rc;
    const int cells = nix * niy * nit;
    DevBuf tb, ob, flag;
    if ((rc = ensure(tb, 16 * (size_t)cells, "intensity")) ||
        (rc = ensure(ob, 8 * (size_t)h->n, "intensity")) || (rc = ensure(flag, 16, "status"))) {
        free_buf(tb), free_buf(ob), free_buf(flag);
        return rc;
    }
    in.hcell = as<double>(tb);
    in.cum = as<double>(tb) + cells;
    unsigned long long bad = 0;
    cudaError_t e = cudaMemcpyAsync(tb.p, tab.data(), 16 * (size_t)cells, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag.p, 0, 8, st);
    if (e == cudaSuccess)
        e = launch_intensity_lookup(h->d_x, h->d_y, h->d_t, h->n, h->box, in, as<double>(ob),
                                    as<unsigned long long>(flag), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, flag.p, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // also: tab (pageable) was read
    free_buf(flag);
    if (e != cudaSuccess) {
        free_buf(tb), free_buf(ob);
        return cuda_fail(e, "intensity upload");
    }
    if (bad) {
        free_buf(tb), free_buf(ob);
        return fail(STK_EDOMAIN, "%llu observed points lie in cells with rho = 0", bad);
    }
    free_buf(h->inh);
    free_buf(h->inh_obs);
    h->inh = tb;
    h->inh_obs = ob;
    h->inten = in;
    h->inh_zero = zero;
    ++h->inh_gen;
    return STK_OK;
}

int stk_sim_points_inhom(const stk_box* box, const double* rho, int nix, int niy, int nit,
                         int64_t n, uint64_t seed, uint32_t sim, double* x, double* y,
                         double* t) {
    if (!x || !y || !t) return fail(STK_EINVAL, "output arrays must not be NULL");
    if (n < 1 || n > ((int64_t)1 << 31) - 1) return fail(STK_EINVAL, "n out of range");
    int rc = check_box(box);
    if (rc) return rc;
    std::vector<double> tab;
    Intensity in;
    int zero = 0;
    if ((rc = intensity_tables(rho, nix, niy, nit, tab, &in, &zero))) return rc;
    const int cells = nix * niy * nit;
    Grid g;  // one neighbour-grid cell: keys and ranks are by-products here
    memset(&g, 0, sizeof g);
    g.nx = g.ny = g.nt = 1;
    g.ncells = 1;
    g.x0 = box->x0, g.x1 = box->x1, g.y0 = box->y0, g.y1 = box->y1, g.t0 = box->t0,
    g.t1 = box->t1;
    g.cw = box->x1 - box->x0;
    g.ch = box->y1 - box->y0;
    g.cd = box->t1 - box->t0;
    DevBuf bx, by, bt, bh, bk, br, bc, bs, tb;
    const size_t b8 = 8 * (size_t)n, b4 = 4 * (size_t)n;
    auto release = [&]() {
        free_buf(bx), free_buf(by), free_buf(bt), free_buf(bh), free_buf(bk), free_buf(br);
        free_buf(bc), free_buf(bs), free_buf(tb);
    };
    if ((rc = ensure(bx, b8, "x")) || (rc = ensure(by, b8, "y")) || (rc = ensure(bt, b8, "t")) ||
        (rc = ensure(bh, b8, "h")) || (rc = ensure(bk, b4, "keys")) ||
        (rc = ensure(br, b4, "ranks")) || (rc = ensure(bc, 16, "counts")) ||
        (rc = ensure(bs, 16, "seed")) || (rc = ensure(tb, 16 * (size_t)cells, "intensity"))) {
        release();
        return rc;
    }
    in.hcell = as<double>(tb);
    in.cum = as<double>(tb) + cells;
    struct {
        uint64_t seed;
        uint32_t sim, pad;
    } key_sim = {seed, sim, 0};
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMemsetAsync(bc.p, 0, 16, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bs.p, &key_sim, sizeof key_sim, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tb.p, tab.data(), 16 * (size_t)cells, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_gen_inhom(n, 1, as<uint64_t>(bs),
                             reinterpret_cast<const uint32_t*>(reinterpret_cast<char*>(bs.p) + 8),
                             g, in, as<double>(bx), as<double>(by), as<double>(bt),
                             as<double>(bh), as<uint32_t>(bk), as<uint32_t>(br),
                             as<uint32_t>(bc), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(x, bx.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y, by.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t, bt.p, b8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_fail(e, "intensity-weighted generation");
    return STK_OK;
}

int stk_last_accumulators(stk_handle* h, int row0, int rows, uint64_t* out) {
    if (!h || !out) return fail(STK_EINVAL, "handle and out must not be NULL");
    if (h->last_rows < 1) return fail(STK_EINVAL, "no finished job on this handle");
    if (row0 < 0 || rows < 1 || row0 + rows > h->last_rows)
        return fail(STK_EINVAL, "rows %d .. %d are outside the last job's %d realizations", row0,
                    row0 + rows - 1, h->last_rows);
    const size_t per = 32 * (size_t)h->last_nbins;
    CK(cudaMemcpyAsync(out, reinterpret_cast<char*>(h->oA.p) + per * (size_t)row0,
                       per * (size_t)rows, cudaMemcpyDeviceToHost, h->stream),
       "accumulator copy");
    CK(cudaStreamSynchronize(h->stream), "accumulator copy");
    return STK_OK;
}

int stk_merge_grids(stk_handle* h, const stk_request* q, const uint64_t* acc, int rows, double* K,
                    double* L, double* raw_sum, int64_t* pair_count) {
    if (!h || !q || !acc) return fail(STK_EINVAL, "handle, request and acc must not be NULL");
    if (rows < 1 || rows > (1 << 24)) return fail(STK_EINVAL, "rows out of range");
    int rc = check_thresholds(h, q->s, q->cs, q->tt, q->ct);
    if (rc) return rc;
    if (q->n_sectors < 0 || q->n_sectors > kMaxSectors)
        return fail(STK_EINVAL, "n_sectors must be in 0..%d", kMaxSectors);
    if (q->norm != STK_NORM_N_NM1 && q->norm != STK_NORM_N2)
        return fail(STK_EINVAL, "unknown norm %d", q->norm);
    const int nsec = q->n_sectors > 1 ? q->n_sectors : 1;
    const int cs = q->cs, ct = q->ct, nb = cs * ct, nbins = nb * nsec;
    if (nbins > kMaxThr * kMaxThr)
        return fail(STK_EINVAL, "n_sectors * cs * ct must be at most %d", kMaxThr * kMaxThr);
    double coef = 0.0;
    if ((rc = job_coef(h, q, &coef))) return rc;
    // device: accumulators [4][rows][nbins], zero self pairs, thresholds, outputs
    const size_t cells = (size_t)rows * nbins;
    const size_t acc_b = 32 * cells, out_b = 32 * cells;
    DevBuf buf;
    if ((rc = ensure(buf, acc_b + out_b + 8 * (size_t)rows * nsec + 16 * kMaxThr, "merge")))
        return rc;
    unsigned char* base = reinterpret_cast<unsigned char*>(buf.p);
    unsigned long long* a = reinterpret_cast<unsigned long long*>(base);
    double* oK = reinterpret_cast<double*>(base + acc_b);
    double* oL = oK + cells;
    double* oS = oL + cells;
    int64_t* oC = reinterpret_cast<int64_t*>(oS + cells);
    int64_t* selfp = oC + cells;
    double* thr = reinterpret_cast<double*>(selfp + (size_t)rows * nsec);
    std::vector<double> hthr(2 * kMaxThr, 0.0);
    for (int i = 0; i < cs; ++i) hthr[(size_t)i] = q->s[i];
    for (int i = 0; i < ct; ++i) hthr[(size_t)kMaxThr + i] = q->tt[i];
    cudaStream_t st = h->stream;
    auto run = [&]() -> cudaError_t {
        const size_t w8 = 8 * (size_t)nbins;
        cudaError_t e = cudaSuccess;
        for (int c = 0; c < 4 && e == cudaSuccess; ++c)
            e = cudaMemcpy2DAsync(a + (size_t)c * cells, w8, acc + (size_t)c * nbins, 4 * w8, w8,
                                  (size_t)rows, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(selfp, 0, 8 * (size_t)rows * nsec, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(thr, hthr.data(), 16 * kMaxThr, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        Accum ac;
        ac.cnt = a;
        ac.exc_lo = a + cells;
        ac.exc_hi = a + 2 * cells;
        ac.stats = nullptr;
        ac.whole = h->inten.nix > 0 ? a + 3 * cells : nullptr;
        e = launch_finalize(rows * nsec, cs, ct, thr, thr + kMaxThr, coef, selfp, ac, oK, oL, oS,
                            oC, st, (double)nsec);
        double* outs[3] = {K, L, raw_sum};
        const double* srcs[3] = {oK, oL, oS};
        for (int c = 0; c < 3 && e == cudaSuccess; ++c)
            if (outs[c])
                e = cudaMemcpyAsync(outs[c], srcs[c], 8 * cells, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && pair_count)
            e = cudaMemcpyAsync(pair_count, oC, 8 * cells, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return e;
    };
    const cudaError_t e = run();
    free_buf(buf);
    if (e != cudaSuccess) return cuda_fail(e, "grid merge");
    return STK_OK;
}

int stk_envelope_merge(const double* K_rows, int rows, int cs, int ct, int n_sectors,
                       const double* s, const double* tt, double* K_lo, double* K_hi,
                       double* L_lo, double* L_hi) {
    if (!K_rows || !s || !tt) return fail(STK_EINVAL, "K_rows, s and tt must not be NULL");
    if (rows < 1 || rows > (1 << 24)) return fail(STK_EINVAL, "rows out of range");
    if (cs < 1 || cs > kMaxThr || ct < 1 || ct > kMaxThr)
        return fail(STK_EINVAL, "cs and ct must be in 1..%d", kMaxThr);
    if (n_sectors < 0 || n_sectors > kMaxSectors)
        return fail(STK_EINVAL, "n_sectors must be in 0..%d", kMaxSectors);
    const int nsec = n_sectors > 1 ? n_sectors : 1;
    const int nbins = nsec * cs * ct;
    if (nbins > kMaxThr * kMaxThr)
        return fail(STK_EINVAL, "n_sectors * cs * ct must be at most %d", kMaxThr * kMaxThr);
    for (int i = 0; i < cs; ++i)
        if (!isfinite(s[i])) return fail(STK_EINVAL, "spatial thresholds must be finite");
    for (int i = 0; i < ct; ++i)
        if (!(isfinite(tt[i]) && tt[i] > 0.0))
            return fail(STK_EINVAL, "temporal thresholds must be finite and > 0");
    int dev = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 != cudaSuccess) {
        cudaGetLastError();
        return fail(STK_ENODEV, "no CUDA device: %s", cudaGetErrorString(e0));
    }
    const size_t in_b = 8 * (size_t)rows * nbins;
    DevBuf buf;
    int rc = ensure(buf, in_b + 32 * (size_t)nbins + 16 * kMaxThr, "envelope merge");
    if (rc) return rc;
    double* dK = reinterpret_cast<double*>(buf.p);
    double* out = dK + (size_t)rows * nbins;  // K_lo, K_hi, L_lo, L_hi
    double* thr = out + 4 * (size_t)nbins;
    std::vector<double> hthr(2 * kMaxThr, 0.0);
    for (int i = 0; i < cs; ++i) hthr[(size_t)i] = s[i];
    for (int i = 0; i < ct; ++i) hthr[(size_t)kMaxThr + i] = tt[i];
    cudaStream_t st = nullptr;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "stream create");
    cudaError_t e = cudaMemcpyAsync(dK, K_rows, in_b, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(thr, hthr.data(), 16 * kMaxThr, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_envelope(rows, nbins, cs, ct, dK, thr, thr + kMaxThr, out, out + nbins,
                            out + 2 * nbins, out + 3 * nbins, st, (double)nsec);
    double* dst[4] = {K_lo, K_hi, L_lo, L_hi};
    for (int c = 0; c < 4 && e == cudaSuccess; ++c)
        if (dst[c])
            e = cudaMemcpyAsync(dst[c], out + (size_t)c * nbins, 8 * (size_t)nbins,
                                cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    free_buf(buf);
    if (e != cudaSuccess) return cuda_fail(e, "envelope merge");
    return STK_OK;
}

int stk_last_stats(const stk_handle* h, stk_stats* out) {
    if (!h || !out) return fail(STK_EINVAL, "handle and out must not be NULL");
    *out = h->last;
    return STK_OK;
}

void stk_destroy(stk_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_buf(h->poly);
    free_buf(h->inh);
    free_buf(h->inh_obs);
    free_buf(h->uh);
    free_buf(h->Hs);
    free_buf(h->acc_whole);
    DevBuf* bufs[] = {&h->xq_e, &h->xq_count, &h->ux, &h->uy, &h->ut, &h->key, &h->rank, &h->counts, &h->start,
                      &h->scan_tmp, &h->X, &h->Y, &h->T, &h->P, &h->Plo, &h->cell_start,
                      &h->chunks, &h->chunk_off, &h->items, &h->counter,
                      &h->acc_cnt, &h->acc_lo, &h->acc_hi, &h->stats, &h->pc, &h->thr,
                      &h->self_pairs, &h->mask_in, &h->mask_sorted, &h->oK, &h->oL, &h->oS,
                      &h->oC, &h->env, &h->simseed, &h->simid, &h->oA, &h->F, &h->stg, &h->fused, &h->obs};
    for (DevBuf* b : bufs) free_buf(*b);
    if (h->d_x) cudaFree(h->d_x);
    if (h->d_y) cudaFree(h->d_y);
    if (h->d_t) cudaFree(h->d_t);
    if (h->h_pc) cudaFreeHost(h->h_pc);
    if (h->h_thr) cudaFreeHost(h->h_thr);
    if (h->h_seed) cudaFreeHost(h->h_seed);
    if (h->h_id) cudaFreeHost(h->h_id);
    for (cudaGraphExec_t g : h->gexecs) cudaGraphExecDestroy(g);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

}  // extern "C"
