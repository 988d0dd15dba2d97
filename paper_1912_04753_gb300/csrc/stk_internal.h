// Internal declarations shared by the CUDA translation units of libstk.so.
//
// Data layout in HBM (one "realization" = the observed pattern or one CSR simulation):
//   - points sorted by grid cell (cell key = (ct*ny + cy)*nx + cx, x fastest), so the cells of
//     one (cy, ct) row are one contiguous run;
//   - per sorted point: FP64 x, y, t (SoA) for the exact FP64 steps; per realization [2n] float4:
//     the coordinate records (x_hi, y_hi, t_hi, cell x index) of all n points, then their edge
//     records (e_x, e_y, e_t, interior bound on d2), kept apart so that the edge records the
//     weight decisions read are dense; and a float2 (x_lo, y_lo): the coordinates are relative
//     to the point's own cell origin, hi parts multiples of a power-of-two quantum, so
//     differences of hi parts are exact in FP32, and hi + lo carries the offset to ~2^-45 of
//     the cell size -- except x_lo, which completes the filter's box-frame x hi part below;
//   - the pair filter's copy of the coordinates, structure of arrays per realization,
//     [3][nF] floats: -x_hi relative to the box's x0 (quantum Grid::qX), -y_hi and -t_hi in the
//     point's cell frame (the same values as above, negated), so four consecutive points load
//     as one float4 per axis;
//   - cell_start[ncells + 1] per realization (offsets into that realization's n points).
//   - work units: 32 consecutive centres of one (cy, ct) row, in realization order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "stk.h"

namespace stk {

constexpr int kMaxThr = 64;   // thresholds per axis
constexpr int kMaxPolyVertices = 128;  // vertices of a polygon study area
// bucket grid over a polygon's bounding box for the FP32 polygon weight: at most 64 x 64
// buckets, each a count (255: too many, scan every edge) and up to 47 edge indices
constexpr int kPolyBucketsMax = 64;
constexpr int kPolyBucketCap = 47;
constexpr int kPolyBucketBytes = 48;
constexpr int kMaxSectors = 64;        // direction sectors of the directional K
constexpr int kTab = 1024;    // bin-table entries per axis
constexpr int kBlock = 256;   // threads per pair-kernel block
constexpr int kUnit = 32;      // centres per work unit (one warp)

// Uniform grid over the study box.  Cell sides are >= s_max / fs (x, y) and >= t_max / ft (t)
// with fs, ft in {1, 2}, so every pair within the thresholds lies in the block of
// (2fs+1) x (2fs+1) x (2ft+1) cells around the centre's cell.
struct Grid {
    int nx, ny, nt;
    int fs, ft;
    int64_t ncells;
    double x0, x1, y0, y1, t0, t1;
    double cw, ch, cd;      // cell sides
    float qx, qy, qt;       // quantum of the FP32 hi parts (2^-22 x a power of two >= side)
    float cwq, chq, cdq;    // cell sides rounded to a multiple of the quantum (exact FP32)
    float cwl, chl, cdl;    // cell side minus its rounded value
    // quantum of the filter's x coordinates, which are taken relative to the box (x - x0,
    // rounded to a multiple of qX = 2^-24 x a power of two >= the box width: exact FP32
    // differences over the whole box, so one grid row is one coordinate frame)
    float qX;
};

// Everything the pair kernels need for one job, built on the host (see guard derivation in
// pair_setup.cpp).  The FP32 kernel copies the part before `s2` into shared memory.
struct PairConsts {
    Grid g;
    int cs, ct, nbins, edge;
    int64_t n;
    // FP32 bulk path: guard bands around each threshold, in d^2 and u.
    float s_lo[kMaxThr], s_hi[kMaxThr];
    float t_lo[kMaxThr], t_hi[kMaxThr];
    float s2_cut, u_cut;      // candidate filter (upper band edge of the last threshold)
    float inv_hs, inv_ht;     // bin-table index scale over d^2 and over u
    float tan_rel, tan_abs;   // tangency band |r - e| <= tan_rel*r + tan_abs -> FP64
    float fast_abs;           // interior fast path margin (hi-part error of r)
    float g_v;                // temporal-weight decision guard
    float r_acc_min;          // edge pairs with a smaller accurate r go to FP64
    uint8_t tab_s[kTab], tab_t[kTab];  // bit 7: entry meets a band; bits 0-6: first bin
    // evenly spaced thresholds: bins from value / spacing, exact outside +-tol of an integer
    int even_s, even_t;
    float inv_ds, inv_dt, tol_s, tol_t;
    float top_s, top_t;       // cs - tol_s, ct - tol_t: values at or above need FP64
    // cell index ranges [lo, hi] of points at least s_max from every spatial edge (x, y) and
    // t_max from both ends of the period (t): a pair of two such points has w = v = 1
    int deep_x[2], deep_y[2], deep_t[2];
    // failure-detection test hook (0 in normal use): a warp that should claim the next tile of
    // work units claims none and publishes nothing, so the block's other warps wait for a tile
    // that never comes until their bounded wait runs out
    int never_publish;
    // consecutive work units a block of the FP32 pair kernel claims at once (>= 1; the launch
    // shape's tile, kTileUnitsDefault unless tuned)
    uint32_t tile_units;
    // polygon study area (nv = 0: the rectangle); vertex arrays in device memory
    int nv;
    int pccw;                 // 1: vertices run counter-clockwise
    int poly_f32;             // 1: FP32-guarded weights in the FP32 kernel (else FP64 ones)
    float poly_eh;            // bound on the FP32 pair positions' error (box frame, length)
    float poly_span;          // larger side of the polygon's bounding box, rounded down
    const double* pvx;
    const double* pvy;
    const float4* pebox;      // per-edge bounding boxes, FP32 rounded outwards
    // per edge, 4 float4 in the box frame (coordinates minus (x0, y0)), each value a pair
    // hi + lo of FP32 numbers: (start vertex x, y), (unit direction x, y), (polar angle in
    // [0, 2 pi) of the normal (u_y, -u_x), length rounded to FP32, 0), and the edge's bounding
    // box (x_min, x_max, y_min, y_max) rounded outwards
    const float4* pe32;
    // bucket grid (box frame): bucket (i, j) = [pb_ox + i / pb_inv, ...) x [pb_oy + j / pb_inv,
    // ...), i < pb_nx, j < pb_ny; its edge list at pb_list + kPolyBucketBytes (j pb_nx + i)
    float pb_ox, pb_oy, pb_inv;
    float pb_rmax;            // the lists hold every edge circles up to this radius can meet
    int pb_nx, pb_ny;
    const uint8_t* pb_list;
    // the polygon's y-band lists (Polygon::band)
    const uint8_t* pband;
    double band_ylo, band_yhi, band_inv;
    // FP64 path: exact thresholds (s_a*s_a rounded once) and a table over d^2 and u.
    double s2[kMaxThr], tt[kMaxThr];
    double inv_hs2_64, inv_ht_64;
    uint8_t tab_s64[kTab], tab_t64[kTab];
    // directional K (FP64 kernel): nsec sectors, boundary m + 1 = (sec_bx[m], sec_by[m]);
    // histograms are [nsec][cs][ct] (nbins = nsec * cs * ct); edge 2 = translation weights
    // with the box's sides tw, th and period td
    int nsec;
    double sec_bx[kMaxSectors], sec_by[kMaxSectors];
    double tw, th, td;
    // the same in FP32 for the FP32-guarded directional kernel: boundaries rounded to FP32,
    // sides, and the guards of the sector test (|cross| <= sec_g, or |d_y| <= sec_gd near the
    // axis at angle 0 / pi: FP64 decides)
    float sec_bxf[kMaxSectors], sec_byf[kMaxSectors];
    float twf, thf, tdf;
    float sec_g, sec_gd;
};

// One unit of pair work for one warp: the centres [c_begin, c_begin + c_count) (at most 32,
// consecutive in sorted order, all in grid row `row` = ct * ny + cy) of realization `real`.
struct WorkItem {
    uint32_t real;
    uint32_t row;
    uint32_t c_begin;
    uint32_t c_count;
};

// Pointers to a batch of realizations laid out back to back ([m][n] and [m][ncells + 1]).
struct RealBatch {
    const float4* P;        // [realization][2n]: coordinate records, then edge records
    const float2* Plo;
    const double* X;
    const double* Y;
    const double* T;
    const uint32_t* cell_start;
    // sorted per-point role flags (bit 0: counts as a centre, bit 1: counts as a neighbour;
    // order (i, j) counts when i has bit 0 and j bit 1), or null (every order counts); of
    // realization 0 only, or of every realization (mask + k * n) when mask_all
    const uint8_t* mask;
    int64_t n;
    int64_t ncells;
    int mask_all = 0;
    // inhomogeneous K: per sorted point h = mean(rho) / rho(cell of the point), [m][n]; null
    // for the homogeneous estimator
    const double* H = nullptr;
    // the filter's coordinate arrays, [m][3][nF] (negated hi parts, see the layout above)
    const float* F = nullptr;
    int64_t nF = 0;
    // sharding of realization 0 of the launch (the observed pattern): its work units
    // [ubeg, uend) are split at grid-row starts into shard_count contiguous ranges of about
    // equal size and only range shard_index is evaluated (every unordered pair belongs to
    // exactly one range, see shard_units)
    int shard_count = 1;
    int shard_index = 0;
};

// Work-unit range [*b, *e) of realization k of a launch: the realization's units, or for
// realization 0 of a sharded launch its shard's share of them.  Shards are cut only at the first
// unit of a grid row (the smallest row start at or after an equal split of the unit count), so
// that every pair a row's units evaluate stays in one shard: which unit of a row owns a pair
// depends on the order of points inside a cell, which the counting sort does not fix from one
// run to the next, while pairs across rows always belong to the earlier row.
// unit_off: the launch's unit offsets [m * nrows + 1] (realization 0 first).
__device__ __forceinline__ uint32_t first_row_unit_at_or_after(const uint32_t* unit_off, int64_t nrows,
                                                      uint32_t target) {
    int64_t lo = 0, hi = nrows;  // unit_off[nrows] is the realization's end, >= target
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (unit_off[mid] >= target)
            hi = mid;
        else
            lo = mid + 1;
    }
    return unit_off[lo];
}

__device__ __forceinline__ void shard_units(const RealBatch& rb, const uint32_t* unit_off, int64_t nrows,
                                   int k, uint32_t* b, uint32_t* e) {
    if (k != 0 || rb.shard_count <= 1) return;
    const uint64_t u = (uint64_t)(*e - *b);
    const uint32_t tlo = *b + (uint32_t)(u * (uint64_t)rb.shard_index / (uint64_t)rb.shard_count);
    const uint32_t thi =
        *b + (uint32_t)(u * (uint64_t)(rb.shard_index + 1) / (uint64_t)rb.shard_count);
    const uint32_t lo = first_row_unit_at_or_after(unit_off, nrows, tlo);
    const uint32_t hi = first_row_unit_at_or_after(unit_off, nrows, thi);
    *b = lo;
    *e = hi;
}

// Per-realization accumulators: counts and the fixed-point (2^-32) sum of (w - 1), the latter
// split into the sums of the low and high 32-bit halves so that both are plain integer
// reductions without carries: excess = hi * 2^32 + lo (in units of 2^-32).
struct Accum {
    unsigned long long* cnt;     // [m][nbins]
    unsigned long long* exc_lo;  // [m][nbins]
    unsigned long long* exc_hi;  // [m][nbins]
    unsigned long long* stats;   // [0] candidates, [1] FP64 recomputes, [2] internal check
                                 // failures, [3] out-of-box flag, [4] bounded waits that ran
                                 // out (the job fails with STK_ETIMEOUT)
    // inhomogeneous K only (null otherwise): the pair weights themselves are accumulated, in
    // units of 2^-64: sum = whole * 2^64 + exc_hi * 2^32 + exc_lo; cnt still counts pairs
    unsigned long long* whole = nullptr;  // [m][nbins]
};

// Pairs the FP32 kernel hands to FP64: x = centre, y = neighbour (sorted indices local to the
// realization), z = realization, w = info: bit 0 = weight only (bins already counted),
// bit 1 = temporal weight 1/2, bits 2.. = bin (weight-only entries).
struct ExactQueue {
    uint4* e;
    unsigned int* count;  // entries pushed (may exceed cap; the excess ran in the pair kernel)
    unsigned int cap;
};

// One job of a fused FP32 pair launch (several jobs, each with its own point set, grid and
// thresholds, in one persistent launch; an array of these in device memory).
struct FusedJob {
    const PairConsts* pc;       // the job's whole constants (device)
    RealBatch rb;
    const WorkItem* units;
    const uint32_t* unit_off;   // [m * nrows + 1]
    uint32_t* counters;         // [m]
    Accum acc;
    ExactQueue xq;
    int m;                      // realizations
    int pad;
};

// ---------------------------------------------------------------- host-side launchers

cudaError_t launch_keys_observed(const double* x, const double* y, const double* t, int64_t n,
                                 const Grid& g, uint32_t* key, uint32_t* rank,
                                 uint32_t* cell_count, int* bad_flag, cudaStream_t st);
cudaError_t launch_validate(const double* x, const double* y, const double* t, int64_t n,
                            const double box[6], int* bad_flag, cudaStream_t st);
// Realization slot k (0..m-1) from the observed points x0, y0, t0 [n] (device): a random
// permutation of the timestamps or a bootstrap resample, keyed like the CSR generator;
// err counts cycle walks that ran out (never expected).
cudaError_t launch_gen_resample(int method, int64_t n, int m, const uint64_t* seeds,
                                const uint32_t* sims, const Grid& g, const double* x0,
                                const double* y0, const double* t0, double* x, double* y,
                                double* t, uint32_t* key, uint32_t* rank, uint32_t* cell_count,
                                unsigned long long* err, cudaStream_t st);
// A polygon study area: nv vertices in device memory (nv = 0: the grid's rectangle).
struct Polygon {
    const double* vx = nullptr;
    const double* vy = nullptr;
    int nv = 0;
    // optional y-band edge lists for the point-in-polygon test (poly_contains_banded):
    // kPolyBands bands of equal height over [band_ylo, band_yhi] (the vertices' y-range), band b
    // at band + b (1 + kMaxPolyVertices): its count, then the edges whose y-range meets the band
    // (widened by a margin); null: every edge is tested
    const uint8_t* band = nullptr;
    double band_ylo = 0.0, band_yhi = 0.0, band_inv = 0.0;
};
constexpr int kPolyBands = 32;
constexpr int kPolyBandBytes = 1 + kMaxPolyVertices;
// host: the band lists of a polygon (kPolyBands x kPolyBandBytes bytes) and the y-range
void build_poly_bands(const double* vx, const double* vy, int nv, uint8_t* out, double* ylo,
                      double* yhi);
// Relative intensity of the inhomogeneous K: rho on nix x niy x nit equal cells of the box
// ([nit][niy][nix], x fastest), in device memory.
struct Intensity {
    int nix = 0, niy = 0, nit = 0;  // 0: none
    const double* hcell = nullptr;  // [cells] mean(rho) / rho_c, 0 where rho_c = 0
    const double* cum = nullptr;    // [cells] rho_0 + ... + rho_c, added in cell order
    double total = 0.0;             // cum[cells - 1]
    int last_pos = 0;               // last cell with rho_c > 0
};
// h[i] = in.hcell[cell of (x[i], y[i], t[i])] for `count` points in the box; points in a cell
// with rho = 0 get 0 and are counted in *zero
cudaError_t launch_intensity_lookup(const double* x, const double* y, const double* t,
                                    int64_t count, const double box[6], Intensity in, double* h,
                                    unsigned long long* zero, cudaStream_t st);
// realization slot k (0..m-1): n points drawn with density proportional to rho (Philox
// realization sims[k] under key seeds[k]), h of each point from the cell it was drawn in
cudaError_t launch_gen_inhom(int64_t n, int m, const uint64_t* seeds, const uint32_t* sims,
                             const Grid& g, Intensity in, double* x, double* y, double* t,
                             double* h, uint32_t* key, uint32_t* rank, uint32_t* cell_count,
                             cudaStream_t st);
// realization slot k (0..m-1) is Philox realization sims[k] under key seeds[k] (device arrays);
// in a polygon, point i keeps the first of its attempts (Philox streams 32, 33, ...) that lies
// inside (err counts points that found none in the attempt limit)
cudaError_t launch_gen_csr(int64_t n, int m, const uint64_t* seeds, const uint32_t* sims,
                           const Grid& g, double* x, double* y, double* t, uint32_t* key,
                           uint32_t* rank, uint32_t* cell_count, cudaStream_t st,
                           Polygon poly = Polygon(), unsigned long long* err = nullptr);
// bucket lists of the FP32 polygon weight: in a grid of nx x ny buckets of side bs at (ox, oy)
// (box frame, the box's corner at (x0, y0)), bucket b lists the edges within `reach` of its
// centre (list[b kPolyBucketBytes] = count or 255, then the indices)
cudaError_t launch_poly_buckets(Polygon poly, double x0, double y0, double ox, double oy,
                                double bs, int nx, int ny, double reach, uint8_t* list,
                                cudaStream_t st);
// flags (bad = 1) any of the n points outside the polygon (closed)
cudaError_t launch_poly_validate(const double* x, const double* y, int64_t n, Polygon poly,
                                 int* bad, cudaStream_t st);
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t count,
                                  uint32_t* tmp, int64_t tmp_words, cudaStream_t st);
int64_t scan_tmp_words(int64_t count);
cudaError_t launch_scatter(int m, int64_t n, const Grid& g, const double* x, const double* y,
                           const double* t, const uint32_t* key, const uint32_t* rank,
                           const uint32_t* start_global, const uint8_t* mask_in,
                           double* X, double* Y, double* T, float4* P, float2* Plo,
                           uint8_t* mask_out, float tan_rel, float tan_abs, float fast_abs,
                           float* F, int64_t nF, double2* stage, cudaStream_t st,
                           Polygon poly = Polygon(), bool mask_all = false,
                           const double* h_in = nullptr, double* H = nullptr, int slot0 = 0);
// (slot0: the m realizations scattered are slots slot0 .. slot0 + m - 1 of the sorted arrays;
// the inputs x, y, t, key, rank, mask_in and h_in start at slot slot0's points.  stage:
// scratch of 32 bytes per scattered point, stage_bytes(m, n), 16-byte aligned)
inline size_t stage_bytes(int64_t m, int64_t n) { return 32 * (size_t)m * (size_t)n; }
// floats per realization and axis of the filter's coordinate arrays (n plus padding for the
// last four-point load, a multiple of 4 so that every axis starts 16-byte aligned)
inline int64_t filter_stride(int64_t n) { return (n + 8 + 3) & ~int64_t(3); }
cudaError_t launch_cell_starts(int m, int64_t n, int64_t ncells, const uint32_t* start_global,
                               uint32_t* cell_start, cudaStream_t st);
// units per (realization, row) -> counts[m * nrows] (+ a zero slot for the scan total)
cudaError_t launch_work_counts(int m, const Grid& g, const uint32_t* cell_start,
                               uint32_t* counts, cudaStream_t st);
// units[unit_off[k*nrows + r] ...] for every (k, r); unit_off has m * nrows + 1 entries
cudaError_t launch_work_fill(int m, const Grid& g, const uint32_t* cell_start,
                             const uint32_t* unit_off, WorkItem* units, cudaStream_t st);
// hpc: host copy of *d_pc, passed by value (its scalars are read from the constant bank).
// bps: the launch shape's blocks per SM (2, or 3 for the kernels pair_fp32_shape_tunable
// admits; grid = SMs x pair_fp32_blocks_per_sm(smem, bps))
cudaError_t launch_pair_fp32(const PairConsts& hpc, const PairConsts* d_pc, bool even, bool edge,
                             size_t smem, int reps,
                             int grid, int m, RealBatch rb, const WorkItem* units,
                             const uint32_t* unit_off, uint32_t* counters, Accum acc,
                             ExactQueue xq, cudaStream_t st, int bps = 2);
// One persistent launch over njobs jobs (d_jobs: device array) of one kernel class: even
// thresholds or not, edge correction or not (the plain rectangle estimator); smem and reps for
// the largest job's bin count nbins_max (pair_fp32_smem); grid = SMs x
// pair_fp32_fused_blocks_per_sm(smem).
cudaError_t launch_pair_fp32_fused(bool even, bool edge, size_t smem, int reps, int nbins_max,
                                   int grid, const FusedJob* d_jobs, int njobs, cudaStream_t st);
int pair_fp32_fused_blocks_per_sm(size_t smem);
// whether the FP32 pair kernel of a job has the 3-blocks-per-SM launch shape (the plain
// rectangle kernels: no polygon, no directional or inhomogeneous variant)
bool pair_fp32_shape_tunable(const PairConsts& hpc, bool inh);
constexpr uint32_t kTileUnitsDefault = 16;
cudaError_t launch_exact(const PairConsts* d_pc, int grid, RealBatch rb, Accum acc,
                         ExactQueue xq, cudaStream_t st, bool poly = false, bool dir = false);
cudaError_t launch_pair_fp64(const PairConsts* d_pc, size_t smem, int reps, int grid, int m,
                             RealBatch rb, const WorkItem* units, const uint32_t* unit_off,
                             uint32_t* counters, Accum acc, cudaStream_t st, bool poly = false,
                             bool inh = false, bool dir = false);
// dynamic shared memory a polygon job's FP32 kernel adds to pair_fp32_smem: its second
// histogram set (the realizations of either parity have their own)
size_t pair_fp32_poly_extra(int nbins, int reps);
size_t pair_fp32_smem(int nbins, int* replicas, bool inh = false);
size_t pair_fp64_smem(int nbins, int* replicas, bool inh = false);
cudaError_t pair_kernels_configure(size_t smem32, size_t smem64);
int pair_fp32_blocks_per_sm(size_t smem, int bps = 2);
int pair_fp64_blocks_per_sm(size_t smem, bool inh = false);
// m grids of cs x ct (a realization of a directional K holds nsec consecutive grids);
// L = sqrt(lfac K / (2 pi t)) - s (lfac = nsec, 1 for the plain estimator)
cudaError_t launch_finalize(int m, int cs, int ct, const double* s, const double* tt,
                            double coef, const int64_t* self_pairs, Accum acc, double* K,
                            double* L, double* S, int64_t* C, cudaStream_t st,
                            double lfac = 1.0);
// element-wise min / max over m rows of nbins (nbins a multiple of cs * ct)
cudaError_t launch_envelope(int m, int nbins, int cs, int ct, const double* K, const double* s,
                            const double* tt, double* K_lo, double* K_hi, double* L_lo,
                            double* L_hi, cudaStream_t st, double lfac = 1.0);

// Host: derive grid and guard constants for one job.  f_req = 0 lets the planner choose the
// refinement factor from the point density; 1 or 2 forces it.
int build_grid(const double box[6], double s_max, double t_max, int64_t n, int f_req, Grid* g,
               char* err, size_t errlen);
void build_pair_consts(const Grid& g, int64_t n, const double* s, int cs, const double* tt,
                       int ct, int edge, PairConsts* pc);
// Records `msg` as the calling thread's stk_last_error() text.
void stk_note_error(int code, const char* msg);

// Threshold rules of the C ABI (finite, > 0, strictly increasing, s_cs <= min(W, H) / 2).
int validate_thresholds(const double box[6], const double* s, int cs, const double* tt, int ct,
                        char* err, size_t errlen);

}  // namespace stk

#include <utility>
#include <vector>

namespace stk {

// Device bytes of a job: `per_real` for every realization resident in one wave, `fixed`
// for the rest (output rows, constants).
struct Footprint {
    size_t per_real = 0;
    size_t fixed = 0;
};

// Simulations of a job: realization r of the job is Philox realization id[r] under key
// seed[r]; groups are consecutive runs of realizations that form one envelope each.
struct SimPlan {
    std::vector<uint64_t> seed;
    std::vector<uint32_t> id;
    std::vector<std::pair<int, int>> groups;  // (first simulation, count)
};

// Runs the observed pattern (when include_obs) and the simulations of `plan` on h's stream.
int run_plan(stk_handle* h, const stk_request* q, const SimPlan& plan, bool include_obs);
// Jobs (observed pattern + plan) on several handles whose FP32 pair kernels run as one
// persistent launch per kernel class: each part's generation and grid index are built on its
// handle's stream, the fused launch runs on the first part's stream once all are built, then
// each part's FP64 queue, finalisation and envelopes follow on its own stream.  The results
// equal run_plan's bit for bit (exact fixed-point sums).  A part that turns out not to fit
// one wave runs alone afterwards.  fused_launches: pair launches issued for the fused parts.
struct FusePart {
    stk_handle* h;
    const stk_request* q;
    const SimPlan* plan;
};
// below this many point-realizations a job is small enough to share a launch
constexpr double kFuseMaxPointRealizations = 2.0e7;
bool fusable_job(const stk_handle* h, const stk_request* q, int64_t R);
int run_plans_fused(const std::vector<FusePart>& parts, int* fused_launches);
// Copies rows of the last job's grids to host: what = 0 K, 1 L, 2 raw sum, 3 count (int64),
// 4 envelope rows (K_lo, K_hi, L_lo, L_hi of each group, 4 rows per group).
int fetch_rows(stk_handle* h, int what, int row0, int rows, void* dst);
int handle_sync(stk_handle* h);
// Footprint of a job of R realizations and `groups` envelopes on h (builds the job's grid).
int job_footprint(stk_handle* h, const stk_request* q, int R, int groups, Footprint* out);
size_t handle_workspace_bytes(const stk_handle* h);
void handle_trim(stk_handle* h);  // frees the job workspace; the point set stays resident
// Device bytes the next jobs on h may hold (waves are sized to fit); 0 = a share of free memory.
void handle_set_wave_budget(stk_handle* h, size_t bytes);
int64_t handle_points(const stk_handle* h);

}  // namespace stk
