/*
 * stk.h -- C ABI of the GB300 space-time Ripley's K library (libstk.so).
 *
 * The library computes the edge-corrected space-time K function of Wang et al.,
 * "Optimizing and Accelerating Space-Time Ripley's K Function based on Apache
 * Spark" (Section 3):
 *
 *   K(s,t) = A*D / (n(n-1)) * sum_{i} sum_{j != i} I(d_ij <= s, u_ij <= t) / (w_ij v_ij)   (Eq. 2, 3)
 *   L(s,t) = sqrt(K(s,t) / (2 pi t)) - s                                                    (Eq. 4)
 *
 * over a grid of spatial thresholds s_1 < ... < s_cs and temporal thresholds
 * t_1 < ... < t_ct, together with Monte Carlo CSR simulation envelopes
 * (Section 3: envelopes from simulated complete spatio-temporal randomness).
 * w_ij is the proportion of the circumference of the circle centred at i with
 * radius d_ij that lies inside the study rectangle, v_ij is 1 when
 * [t_i - u_ij, t_i + u_ij] lies inside the study period and 1/2 otherwise
 * (Section 3, isotropic correction); u_ij = |t_i - t_j|.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status (enum stk_status) and never aborts.
 *     On failure stk_last_error() describes the cause (thread-local string).
 *   - Input arrays are read during the call and never retained: the library
 *     copies what it needs.  Output arrays are owned by the caller.
 *   - Grids are row-major [cs][ct] with cs, ct in [1, STK_MAX_THRESHOLDS];
 *     entry (a, b) is cumulative: it covers every ordered pair with
 *     d_ij <= s_a and u_ij <= t_b.
 *   - Thresholds must be finite, > 0 and strictly increasing, and
 *     s_cs <= min(x1-x0, y1-y0)/2 (so a circle crosses at most one x-edge and
 *     one y-edge and 1/(w v) <= 8).  Points must be finite and inside the
 *     closed box.  n >= 2.
 *   - A handle is not thread-safe; distinct handles may be used from distinct
 *     threads.  All device work of a handle runs on its stream (see
 *     stk_set_stream); functions that return host results synchronise it.
 *   - Parity contract with the FP64 reference definition: pair counts are
 *     exact in both precisions; K, L and raw sums agree to relative 1e-9 in
 *     STK_PREC_FP64 and 1e-6 in STK_PREC_FP32_GUARDED.
 */
#ifndef STK_H
#define STK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STK_MAX_THRESHOLDS 64
#define STK_MAX_FUSED_JOBS 256

typedef struct stk_handle stk_handle;

/* Study area (rectangle) and study period; a closed box with x0<x1, y0<y1, t0<t1. */
typedef struct {
    double x0, x1, y0, y1, t0, t1;
} stk_box;

enum stk_status {
    STK_OK = 0,
    STK_EINVAL = 1,   /* malformed argument (sizes, NULL, thresholds, n < 2) */
    STK_EDOMAIN = 2,  /* a point lies outside the closed study box, or is not finite */
    STK_ENOMEM = 3,   /* device or host allocation failed */
    STK_ECUDA = 4,    /* a CUDA call failed; the message names it */
    STK_ETIMEOUT = 5, /* a bounded device or host wait ran out */
    STK_EBUSY = 6,    /* the server cannot take the request now */
    STK_ENODEV = 7    /* no usable CUDA device */
};

/* NONE: weight 1.  ISOTROPIC: Section 3 (proportion of the circle's circumference inside the
 * study area, temporal weight 1 or 1/2).  TRANSLATION: the translation correction, pair weight
 * W H / ((W - |dx|)(H - |dy|)) * D / (D - u) (|A| over the area of the box intersected with
 * its copy shifted by the pair's offset, likewise in time; rectangle only; needs
 * t_ct <= (t1 - t0) / 2 so that the weight stays <= 8): unbiased for every direction, so the
 * one the directional K (n_sectors > 1) takes. */
enum { STK_EDGE_NONE = 0, STK_EDGE_ISOTROPIC = 1, STK_EDGE_TRANSLATION = 2 };
/* FP64: every pair in IEEE double, bit-compatible with the reference definition.
 * FP32_GUARDED: pairs in FP32 with cell-relative coordinates; any pair whose
 * bin, temporal weight or spatial-weight branch FP32 cannot decide with a
 * proven error bound is recomputed in FP64, so counts stay exact. */
enum { STK_PREC_FP64 = 0, STK_PREC_FP32_GUARDED = 1 };
/* Eq. 2 prints A*D/n^2; A*D/(n(n-1)) makes E[K] = 2 pi s^2 t exact under CSR. */
enum { STK_NORM_N_NM1 = 0, STK_NORM_N2 = 1 };
/* Execution form for jobs with simulations. */
enum { STK_EXEC_BATCHED = 0, STK_EXEC_PLAIN = 1 };
/* Simulation method (Section 3): Monte Carlo CSR (points uniform in the box and period),
 * random permutation (the observed points with their timestamps exchanged by a keyed
 * pseudo-random bijection: a 4-round Feistel network on Philox round functions, streams
 * 16-19, restricted to [0, n) by cycle walking), bootstrapping (n draws with replacement from
 * the observed points: source floor(u n), u the 53-bit uniform of Philox stream 4). */
enum { STK_SIM_CSR = 0, STK_SIM_PERMUTATION = 1, STK_SIM_BOOTSTRAP = 2 };

/* Create a handle over n points (host arrays, FP64).  The points are copied to
 * the device.  Errors: STK_EINVAL (NULL, n < 2, bad box), STK_EDOMAIN (point
 * outside the box or not finite), STK_ENOMEM, STK_ENODEV, STK_ECUDA. */
int stk_create(const double* x, const double* y, const double* t, int64_t n, const stk_box* box,
               stk_handle** out);

/* Same, from device-resident FP64 arrays (copied device-to-device on `stream`,
 * a cudaStream_t or NULL for the library's own stream).  Points are validated
 * on the device. */
int stk_create_device(const double* d_x, const double* d_y, const double* d_t, int64_t n,
                      const stk_box* box, void* stream, stk_handle** out);

/* Polygon study area (the paper's experiments use an 85-vertex outline, Sections 3 and 6):
 * subsequent jobs on h take the closed simple polygon of nv vertices (vx[k], vy[k]), either
 * orientation, as the study region: A in Eq. 2 is its area, the spatial weight is the
 * proportion of the circle's circumference inside it (whenever the circle reaches the
 * boundary: in FP64 on the FP64 path; on the FP32-guarded path in FP32 with an error bound
 * per circle, FP64 for what that bound cannot decide), and CSR simulations are uniform in it
 * (each point the first of its draws in the bounding box, Philox streams 32, 33, ..., that
 * falls inside).  The period stays the box's.  Requires 3 <= nv <= 128, every vertex inside the handle's box, an area of at
 * least 1/64 of the box's, and every point of the handle inside the polygon (else
 * STK_EDOMAIN, the study area unchanged).  nv = 0 restores the box.  Errors: STK_EINVAL,
 * STK_EDOMAIN, STK_ENOMEM, STK_ECUDA. */
int stk_set_polygon(stk_handle* h, const double* vx, const double* vy, int nv);

/* Inhomogeneous K (the variant Section 7 lists as future work): subsequent jobs on h divide
 * every ordered pair by the intensities at both of its points.  rho is a caller-owned host
 * array of nix * niy * nit relative intensities, piecewise constant on that many equal cells
 * of the box, row-major [nit][niy][nix] (x fastest); only its shape matters: the intensity is
 * lambda_c = n rho_c / sum_c(rho_c V), V the cell volume, so that it integrates to n.  A
 * point (x, y, t) lies in cell floor(((x - x0) / (x1 - x0)) * nix) (each operation rounded
 * separately, clamped to [0, nix - 1]), and likewise along y and t.  The estimator is
 *   K_I(s, t) = n / ((n - 1) A D) * sum_{i != j} I(d_ij <= s, u_ij <= t) / (w_ij v_ij lambda_i lambda_j)
 * (1 / (A D) with STK_NORM_N2), Eq. 2 when rho is constant; raw_sum reports that sum times
 * (n / (A D))^2, so K = raw_sum * A D / (n (n - 1)) as in Eq. 2, and L follows Eq. 4.  Both
 * precisions apply (counts exact; the weighted sums, each pair's weight times h_i h_j, are
 * kept in 2^-64 fixed point).  Simulations: STK_SIM_CSR draws n points independently with density
 * proportional to rho (cell i of a point: the first whose running sum of rho exceeds u times
 * the total, u from Philox block (i, sim, 40, i >> 32); the position inside the cell from the
 * CSR streams 0, 1, 2: x = x0 + (x1 - x0) * ((cell x index + u_x) / nix)), and each point
 * takes the intensity of its cell; with one cell this is the CSR realization.  Bootstrap and
 * permutation realizations take the intensity of the cell each point lies in; permutations
 * need rho > 0 in every cell.  Requires rho finite and >= 0 with a positive sum, every
 * positive rho_c within 2^14 times the mean of rho either way, 1 <= cells <= 2^22, and every
 * observed point in a cell with rho > 0 (else STK_EDOMAIN, the handle unchanged).  Cannot be
 * combined with a polygon study area or with labels (cross K).  rho = NULL or nix = 0
 * restores the homogeneous estimator.  Errors: STK_EINVAL, STK_EDOMAIN, STK_ENOMEM,
 * STK_ECUDA. */
int stk_set_intensity(stk_handle* h, const double* rho, int nix, int niy, int nit);

/* Run this handle's device work on `stream` (a cudaStream_t); NULL restores
 * the handle's own stream. */
int stk_set_stream(stk_handle* h, void* stream);

/* Observed K over the threshold grid (Eq. 2-4).  Each output is a caller-owned
 * [cs*ct] row-major array or NULL to skip it.  raw_sum is the cumulative
 * weighted pair sum before normalisation, pair_count the cumulative number of
 * ordered pairs. */
int stk_k(stk_handle* h, const double* s, int cs, const double* tt, int ct, int edge_mode,
          int prec, int norm, double* K, double* L, double* raw_sum, int64_t* pair_count);

/* Monte Carlo CSR envelope (Section 3): n_sims realizations of n points,
 * uniform in the handle's box, drawn with Philox4x32-10 under key (seed low
 * word, seed high word) and counter (i low word, realization, stream 0/1/2 for
 * x/y/t, i high word); u = ((w0>>5)*2^26 + (w1>>6)) * 2^-53, coordinate =
 * min(lo + (hi-lo)*u, hi).  Outputs: element-wise min / max of K over the
 * realizations, and L of those.  Any output may be NULL. */
int stk_envelope(stk_handle* h, const double* s, int cs, const double* tt, int ct, int edge_mode,
                 int prec, int norm, int n_sims, uint64_t seed, double* K_lo, double* K_hi,
                 double* L_lo, double* L_hi);

/* A whole analysis job: observed K plus an n_sims CSR envelope.
 * exec = STK_EXEC_BATCHED runs the observed pattern and every realization
 * through one index build and one persistent pair launch (memory permitting;
 * otherwise in waves); STK_EXEC_PLAIN runs one launch per realization. */
typedef struct {
    const double* s;
    int cs;
    const double* tt;
    int ct;
    int edge_mode;
    int prec;
    int norm;
    int n_sims;          /* 0 = observed K only */
    uint64_t seed;
    int exec;
    const uint8_t* centre_mask; /* optional host [n]: only centres with mask != 0
                                   contribute to the OBSERVED grids (sampled-centre
                                   checking mode); NULL = all */
    int sim_method;      /* STK_SIM_*; the envelope is over realizations of this method */
    uint32_t first_sim;  /* simulations are realizations first_sim .. first_sim+n_sims-1 of
                            the counter-based generator, so a long envelope job can run (or
                            resume after an interruption) in chunks: the union of the chunks'
                            realizations equals the whole job's, bit for bit */
    /* Bivariate (cross) K, the variant the paper names as future work: with labels (host
     * [n], copied) every grid is over ordered pairs from centres labelled cross_a to
     * neighbours labelled cross_b, weights centred at the centre, normalised by
     * n_a * n_b (the subset's univariate normalisation when cross_a == cross_b).  Simulated
     * point i keeps the label of observed point i (CSR and permutation; not bootstrap).
     * NULL = univariate.  Not combined with centre_mask, a polygon study area or an
     * intensity. */
    const uint8_t* labels;
    int cross_a;
    int cross_b;
    /* Directional (sector) K, the anisotropic analysis the paper names as future work:
     * n_sectors in 2..64 splits the pairs by the axial direction of their offset into
     * n_sectors equal sectors of [0, pi) (sector k: angles [k pi / n, (k + 1) pi / n); the
     * offset turned into the upper half plane, then counted against the boundaries
     * (cos(m pi / n), sin(m pi / n)) by the sign of b_x d_y - b_y d_x >= 0, each operation
     * rounded separately; coincident points in sector 0).  Every grid output then holds
     * n_sectors grids, [n_sectors][cs][ct], with n_sectors * cs * ct <= 4096; L of a sector is
     * sqrt(n_sectors K / (2 pi t)) - s (zero in expectation under CSR, like Eq. 4).  Needs
     * edge_mode NONE or TRANSLATION, the rectangle, no intensity and no labels.
     * 0 or 1: no split. */
    int n_sectors;
    /* Sharding of the OBSERVED pattern across processes (one GPU each; the paper partitions the
     * points over Spark workers, Section 4.4).  With shard_count > 1 this call evaluates only
     * shard shard_index (0 .. shard_count - 1) of the observed pattern's pairs: its work units
     * (32 centres of one grid row each, in time-major row order) are split into shard_count
     * contiguous ranges of whole grid rows with about equal unit counts, and each unordered
     * pair belongs to exactly one range whatever the order of points inside a cell.  The observed grids returned then hold that shard's share only; the integer
     * accumulators of all shards (stk_last_accumulators) summed element-wise equal the whole
     * pattern's bit for bit, and stk_merge_grids turns the sum into K, L, raw sums and counts.
     * Simulations are not affected (shard them with first_sim / n_sims).  0 or 1: no split. */
    int shard_count;
    int shard_index;
} stk_request;

typedef struct {
    /* observed pattern, each [cs*ct] (times n_sectors for a directional K) or NULL */
    double* K;
    double* L;
    double* raw_sum;
    int64_t* pair_count;
    /* envelope, each [cs*ct] or NULL (ignored when n_sims == 0) */
    double* K_lo;
    double* K_hi;
    double* L_lo;
    double* L_hi;
    /* optional per-realization grids [n_sims][cs*ct] */
    double* K_sims;
    int64_t* count_sims;
} stk_result;

/* Statistics of the last job run on a handle. */
typedef struct {
    int64_t qualifying_pairs;  /* ordered pairs with d <= s_cs and u <= t_ct, all realizations */
    int64_t candidate_pairs;   /* ordered pairs examined by the pair kernel */
    int64_t fp64_recomputed;   /* FP32_GUARDED: pairs decided in FP64 */
    int64_t work_items;
    int32_t realizations;
    int32_t waves;
    double ms_total;           /* host wall time of the job */
    double ms_pair;            /* device time of the pair kernel launches */
    int64_t kernel_launches;   /* CUDA kernels this library launched for the job */
    int64_t internal_errors;   /* consistency checks that failed inside the kernels (0 expected) */
    int32_t grid_refinement;   /* fs: grid cells of s_max/fs x s_max/fs (1..3) */
    int32_t graph_replays;     /* waves replayed from a captured CUDA graph */
    int32_t grid_refinement_t; /* ft: grid cells of t_max/ft in time (1..3) */
    int32_t obs_index_reused;  /* 1: the observed pattern's sorted grid index was resident (the
                                  last job on h had the same grid), not rebuilt */
    int32_t tile_units;        /* launch shape of the FP32 pair kernel: work units a block
                                  claims at once (the launch-shape tuner's choice for the
                                  job's problem shape, made by its first job; 16 untuned) */
    int32_t blocks_per_sm;     /* resident blocks per SM of the pair kernel's launch (the FP32
                                  kernel: 2, or 3 where the tuner chose its 85-register build) */
} stk_stats;

int stk_run(stk_handle* h, const stk_request* req, stk_result* res);

/* Several jobs, each on its own handle (point set), whose FP32 pair kernels run as ONE
 * persistent launch (the batched path of Section 3's envelope over small problems at once):
 * job i is reqs[i] on hs[i] with results into results[i], exactly as stk_run(hs[i], &reqs[i],
 * &results[i]) would compute them (bit for bit: the sums are exact fixed-point integers, and a
 * job takes its problem shape's tuned launch shape either way).  Each job's
 * simulation generation and grid index run on its handle's stream; the fused pair launch runs
 * on hs[0]'s stream (or the first fused job's) once every index is built, with each job's
 * constants, grid and accumulators taken from a per-job descriptor; each job's FP64 queue,
 * finalisation and envelope follow on its own stream.  Jobs that cannot share the launch run
 * alone, in order, after it: FP64 precision, the translation correction or sectors, labels, a
 * centre mask, shards, a polygon or an intensity on the handle, more than 2e7
 * point-realizations (n x (1 + n_sims)), or too large to fit one wave.  Jobs whose thresholds
 * differ in kind (evenly spaced or not, edge correction or not) share one launch per kind.
 * hs: njobs distinct handles (1 <= njobs <= STK_MAX_FUSED_JOBS); reqs, results: njobs each,
 * caller-owned, result pointers as for stk_run.  pair_launches (may be NULL): pair-kernel
 * launches the fused jobs took (1 when all share one kind).  Errors: STK_EINVAL (NULL arrays,
 * a repeated handle, njobs or n_sims out of range, any request error of stk_run), STK_ENOMEM,
 * STK_ECUDA, STK_EDOMAIN, STK_ETIMEOUT; on an error the jobs' results are unspecified and
 * every handle remains usable. */
int stk_run_fused(stk_handle* const* hs, const stk_request* reqs, stk_result* results, int njobs,
                  int* pair_launches);

/* ---- Partial results and their exact merge (multi-process jobs; Section 3, Eq. 2-4) ------
 * A job split across processes (realizations k in blocks via first_sim / n_sims, the observed
 * pattern via shard_count / shard_index) is merged from two kinds of partial results:
 *   - the raw integer accumulators of a realization, which add exactly: per histogram bin
 *     (s_bin, t_bin), NOT cumulative, the count of ordered pairs and the fixed-point sum of
 *     their weights, as four uint64 rows [4][nbins]: count, low and high 32-bit halves of the
 *     sum of (w - 1) in units of 2^-32 (the weight excess of Eq. 2's 1 / (w v) over 1), and a
 *     whole part (inhomogeneous K only: its sum of h_i h_j / (w v) is kept as
 *     whole * 2^64 + high * 2^32 + low in units of 2^-64; zero otherwise).  Element-wise
 *     sums over shards are the whole job's accumulators, whatever the order;
 *   - per-realization K grids, whose envelope (element-wise min / max) is exact and
 *     order-free, so local envelopes merge by a min / max reduction.
 * nbins = n_sectors * cs * ct (n_sectors >= 1). */

/* Raw accumulators of realizations row0 .. row0 + rows - 1 of the last job on h (row 0 is the
 * observed pattern when the job had one, then the simulations in order), copied to the
 * caller-owned host array out [rows][4][nbins] (uint64).  Errors: STK_EINVAL (NULL, rows out of
 * range of the last job). */
int stk_last_accumulators(stk_handle* h, int row0, int rows, uint64_t* out);

/* Turns `rows` merged accumulator sets acc [rows][4][nbins] (host, as stk_last_accumulators
 * writes them) into the cumulative grids of Eq. 2-4 with the normalisation the request q would
 * use on h (A and D of h's study area, n or the label counts of a cross K, q->norm; L scaled by
 * n_sectors for a directional K): K, L, raw_sum [rows][nbins] (double) and pair_count
 * [rows][nbins] (int64), caller-owned host arrays, each may be NULL.  Computed on the device
 * (the cumulation in 128-bit fixed point), so a merged job equals the single-process job bit
 * for bit.  Errors: STK_EINVAL (NULL, bad sizes, request rules of stk_run), STK_ENOMEM,
 * STK_ECUDA. */
int stk_merge_grids(stk_handle* h, const stk_request* q, const uint64_t* acc, int rows, double* K,
                    double* L, double* raw_sum, int64_t* pair_count);

/* Envelope of `rows` K grids (host array K_rows [rows][n_sectors][cs][ct], e.g. the
 * per-realization grids of several chunks of a job, or the local K_lo and K_hi of several
 * processes stacked): element-wise min and max over the rows (Section 3 envelopes) and L of
 * those (Eq. 4, sqrt(n_sectors K / (2 pi t)) - s for a directional K, n_sectors = 1 otherwise),
 * into caller-owned host arrays [n_sectors][cs][ct], each may be NULL.  Computed on the current
 * device.  Errors: STK_EINVAL (NULL input, rows < 1, bad sizes or thresholds), STK_ENOMEM,
 * STK_ECUDA, STK_ENODEV. */
int stk_envelope_merge(const double* K_rows, int rows, int cs, int ct, int n_sectors,
                       const double* s, const double* tt, double* K_lo, double* K_hi,
                       double* L_lo, double* L_hi);

/* Statistics of the last job on h.  With the environment variable STK_JOB_LOG naming a file,
 * every job also appends them, with its parameters, to that file as one JSON line. */
int stk_last_stats(const stk_handle* h, stk_stats* out);

/* One CSR realization generated by the device generator that stk_envelope
 * uses (same Philox contract), copied to caller-owned host arrays x, y, t [n].
 * Exposes step "CSR simulation generation" for checking. */
int stk_sim_points(const stk_box* box, int64_t n, uint64_t seed, uint32_t sim, double* x,
                   double* y, double* t);

/* One CSR realization in the polygon (vx, vy, nv) (as in jobs after stk_set_polygon), with
 * the period of `box`, whose x/y range is the rectangle the draws are taken in; copied to
 * caller-owned host arrays x, y, t [n].  Errors: STK_EINVAL. */
int stk_sim_points_polygon(const stk_box* box, const double* vx, const double* vy, int nv,
                           int64_t n, uint64_t seed, uint32_t sim, double* x, double* y,
                           double* t);

/* One realization of the intensity-weighted simulation of stk_set_intensity (n points with
 * density proportional to rho over `box`), generated by the device generator the jobs use,
 * copied to caller-owned host arrays x, y, t [n].  Errors: STK_EINVAL. */
int stk_sim_points_inhom(const stk_box* box, const double* rho, int nix, int niy, int nit,
                         int64_t n, uint64_t seed, uint32_t sim, double* x, double* y,
                         double* t);

/* One random-permutation or bootstrap realization (method STK_SIM_PERMUTATION or
 * STK_SIM_BOOTSTRAP, Section 3) of the observed host points x0, y0, t0 [n], generated by
 * the device generator the jobs use, copied to caller-owned host arrays x, y, t [n].
 * Exposes step "simulation generation" for checking.  Errors: STK_EINVAL. */
int stk_sim_resample(const double* x0, const double* y0, const double* t0, int64_t n,
                     int method, uint64_t seed, uint32_t sim, double* x, double* y, double* t);

/* Observed K of one pattern without allocating memory.  Not part of the paper's method: an
 * interface for callers that cannot call cudaMalloc where they need K (a region where
 * cudaMalloc / cudaFree would synchronise the device and stall pipelined work, a caching
 * allocator's reserved pool, an embedding that owns every buffer).  Inputs d_x, d_y, d_t
 * [n] and outputs d_K, d_L, d_S (double) and d_C (int64) [cs*ct] are caller-owned DEVICE
 * arrays; thresholds are host arrays; FP32_GUARDED precision, A*D/(n(n-1)) normalisation.
 * Every intermediate buffer lives in one static device array of 64 MiB inside the library,
 * held on every GPU that loads it until the process exits; patterns up to 262,144 points
 * and grids up to 2^20 cells are accepted, larger ones fail with STK_EINVAL, as do NULL
 * pointers.  STK_EDOMAIN: a point outside the box; STK_ETIMEOUT: a bounded wait inside the
 * pair kernel ran out (outputs incomplete; the next call starts afresh).  The first call
 * on a device looks up the array's address (once per device): make it before any stream
 * capture.  All calls share the array, so calls that overlap on the GPU race; the caller
 * serialises them.  `stream` is a cudaStream_t or NULL; the call synchronises it.  Calls no
 * cudaMalloc, cudaFree or allocating library routine. */
int stk_k_noalloc(const double* d_x, const double* d_y, const double* d_t, int64_t n,
                  const stk_box* box, const double* s, int cs, const double* tt, int ct,
                  int edge_mode, double* d_K, double* d_L, double* d_S, int64_t* d_C,
                  void* stream);

/* ---- Serving loop ---------------------------------------------------------------------
 * The paper serves K and envelope jobs to a web front end through a job-submission tier
 * (Section 5); this is the single-GPU counterpart.  A server keeps registered point sets
 * resident on one device and runs jobs submitted from any thread:
 *   - `slots` worker threads, each driving its own CUDA stream, take queued jobs in arrival
 *     order; a job whose point set is busy in another slot waits for it, later jobs on other
 *     point sets go ahead, so the work of different requests overlaps on the GPU;
 *   - admission by device memory: point sets plus the workspaces of running and idle jobs
 *     stay within mem_budget_bytes; a job starts when its minimum footprint (one realization
 *     resident at a time) fits, after idle workspaces have been released if needed, and
 *     runs its realizations in waves sized to what it was granted;
 *   - continuous batching: when a slot takes a job it also takes every queued job on the
 *     same point set with the same thresholds, edge mode, precision and normalisation (up to
 *     max_batch_sims simulations in total).  The observed pattern is computed once and all
 *     their simulations go through the same launches, each job's under its own seed:
 *     realization k of a job is Philox realization k under the job's seed, exactly as in
 *     stk_envelope, and every realization is accumulated on its own, so a job's results do
 *     not depend on the jobs it ran with;
 *   - fused launches (cfg.fuse): when a slot takes a small batch (FP32-guarded, rectangle,
 *     isotropic or no edge correction, no sectors, below 2e7 point-realizations) it also takes
 *     the next admissible such batches on other idle point sets (up to 16, 2e7
 *     point-realizations in all) and runs their pair kernels as one persistent launch, as
 *     stk_run_fused does; each job's results are those it would have alone, bit for bit.  It
 *     pays where launches and host work dominate (streams of tiny jobs); where the slots'
 *     concurrent streams already keep the GPU busy it adds latency (a group finishes
 *     together), so it is off by default.
 * A server is thread-safe; handles created with stk_create are unaffected by it. */
typedef struct stk_server stk_server;

typedef struct {
    int device;               /* CUDA device ordinal */
    int slots;                /* concurrent jobs (worker threads, one stream each); 0 = 4 */
    int64_t mem_budget_bytes; /* device bytes for point sets and job workspaces;
                                 0 = 80% of the device's free memory at creation */
    int max_batch_sims;       /* most simulations merged into one batched job; 0 = 8192 */
    int max_queue;            /* queued jobs beyond which stk_submit returns STK_EBUSY;
                                 0 = 65536 */
    int no_merge;             /* 1: run every job on its own (no continuous batching) */
    int fuse;                 /* 1: let small batches on different point sets share a pair
                                 launch (see stk_run_fused); 0: every batch launches its own */
} stk_server_config;

typedef struct {
    uint64_t dataset;    /* from stk_server_register */
    const double* s;     /* thresholds, copied at submission (same rules as stk_k) */
    int cs;
    const double* tt;
    int ct;
    int edge_mode;
    int prec;
    int norm;
    int n_sims;          /* 0 = observed K only */
    uint64_t seed;
    int want_sims;       /* 1: keep per-realization K and counts for stk_poll */
    int sim_method;      /* STK_SIM_* */
    int n_sectors;       /* directional K (as stk_request.n_sectors); grids [n_sectors][cs][ct] */
} stk_job;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t queued, running;      /* now */
    int64_t max_queue_depth;
    int64_t batches;              /* batched jobs run on the device */
    int64_t merged_jobs;          /* jobs that shared their batch with another job */
    int64_t simulations;          /* realizations of completed jobs, observed excluded */
    int64_t qualifying_pairs;     /* over all completed batches and realizations */
    double p50_ms, p99_ms, max_ms, mean_ms; /* submission -> result ready, completed jobs */
    double wall_s;                /* first submission -> last completion */
    double jobs_per_s, sims_per_s;
    int64_t resident_bytes;       /* point sets + workspaces held now */
    int64_t peak_bytes;           /* most held (accounted) at once */
    int64_t budget_bytes;
    int64_t kernel_launches;      /* CUDA kernels the batches launched (graph replays included) */
    int64_t fused_jobs;           /* jobs whose pair kernel ran in one launch with jobs on other
                                     point sets */
} stk_serve_stats;

/* Errors: STK_EINVAL (bad config), STK_ENODEV, STK_ECUDA, STK_ENOMEM. */
int stk_server_create(const stk_server_config* cfg, stk_server** out);
/* Copies a point set to the device and keeps it there until stk_server_unregister or
 * stk_server_destroy.  Same argument rules and errors as stk_create; STK_ENOMEM when the
 * point set does not fit the server's budget. */
int stk_server_register(stk_server* sv, const double* x, const double* y, const double* t,
                        int64_t n, const stk_box* box, uint64_t* dataset);
/* Releases a point set; STK_EBUSY while jobs on it are queued or running. */
int stk_server_unregister(stk_server* sv, uint64_t dataset);
/* A polygon study area or a relative intensity for a registered point set, as
 * stk_set_polygon / stk_set_intensity on a handle; later jobs on it use them (jobs on one point
 * set share them, so merged jobs agree).  Errors: those of the handle functions, STK_EINVAL
 * (unknown dataset), STK_EBUSY while jobs on the point set are queued or running. */
int stk_server_set_polygon(stk_server* sv, uint64_t dataset, const double* vx, const double* vy,
                           int nv);
int stk_server_set_intensity(stk_server* sv, uint64_t dataset, const double* rho, int nix,
                             int niy, int nit);
/* Queues a job; its thresholds are checked and copied here.  Errors: STK_EINVAL (unknown
 * dataset, bad thresholds or modes, n_sims < 0), STK_EBUSY (queue full). */
int stk_submit(stk_server* sv, const stk_job* job, uint64_t* ticket);
/* Waits up to wait_ms milliseconds (< 0: without limit) for a job.  STK_OK: the result is
 * copied into `res` (its pointers as in stk_run; K_sims / count_sims need want_sims) and the
 * ticket is released; latency_ms (may be NULL) receives submission -> completion time.
 * STK_ETIMEOUT: not finished yet, the ticket stays valid.  The job's own error code when it
 * failed (ticket released, message in stk_last_error).  STK_EINVAL: unknown ticket. */
int stk_poll(stk_server* sv, uint64_t ticket, stk_result* res, int wait_ms, double* latency_ms);
int stk_server_stats(stk_server* sv, stk_serve_stats* out);
/* Clears latency and throughput counters (not the queue). */
int stk_server_reset_stats(stk_server* sv);
/* Finishes running jobs, fails queued ones with STK_EBUSY, frees everything. */
void stk_server_destroy(stk_server* sv);

void stk_destroy(stk_handle* h);
const char* stk_last_error(void);
const char* stk_version(void);

#ifdef __cplusplus
}
#endif
#endif /* STK_H */
