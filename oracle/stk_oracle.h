/*
 * Oracle for the edge-corrected space-time Ripley's K estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64
 * restatement of the paper's estimator (Section 3, Eq. 2-4) used to check the
 * CUDA path.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline / reference arm may load it.  It shares no code, header, table or
 * constant with the CUDA library, and the CUDA library never calls it.
 *
 * Conventions (readings of the paper where it is silent or ambiguous):
 *   - ordered pairs (i, j), i != j, O(n^2), no index (Eq. 2 double sum);
 *   - indicator I = [d_ij <= s] * [u_ij <= t], both inclusive (Eq. 3);
 *     d2 = dx*dx + dy*dy with every operation rounded separately (no FMA),
 *     compared against s*s, so no square root enters the count;
 *   - u_ij = |t_i - t_j| (cylinder of height 2t, Section 3);
 *   - spatial weight = fraction of the circumference of the circle centred at
 *     i through j that lies inside the study rectangle (Section 3, isotropic
 *     correction); temporal weight = 1 if [t_i - u, t_i + u] lies inside the
 *     study period (closed), else 1/2 (Section 3);
 *   - normalisation A*D/(n(n-1)) by default, A*D/n^2 on request (Eq. 2 prints
 *     n^2; see the design notes);
 *   - L = sqrt(K / (2 pi t)) - s (Eq. 4);
 *   - CSR simulations: n points uniform in the box and window, drawn with
 *     Philox4x32-10 (Salmon et al., SC'11) under counter (i, sim, stream, 0),
 *     key (seed lo, seed hi) (Section 3, Monte Carlo simulation);
 *   - bootstrap and random-permutation simulations (Section 3) draw from the
 *     same generator (streams 4 and 16..19), see their declarations.
 *
 * Grids are row-major [cs][ct]; bins are non-cumulative in *_hist and
 * cumulative (d <= s_a and u <= t_b) everywhere else.
 */
#ifndef STK_ORACLE_H
#define STK_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 block function: out = philox(ctr, key). */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* 53-bit uniform in [0,1) from two 32-bit words: ((w0>>5)*2^26 + (w1>>6)) * 2^-53. */
double oracle_u01(uint32_t w0, uint32_t w1);

/* One CSR realization `sim` of n points in box[6] = {x0,x1,y0,y1,t0,t1}. */
void oracle_csr_points(int64_t n, const double box[6], uint64_t seed, uint32_t sim,
                       double* x, double* y, double* t);

/* Finalize with an explicit study-area measure A and period length D. */
void oracle_finalize_area(int64_t n, double area, double dur, const double* s, int cs,
                          const double* tt, int ct, int norm, const int64_t* cnt,
                          const double* wsum, int64_t* C, double* S, double* K, double* L);

/* Polygon study areas (simple polygon, either orientation, closed). */
double oracle_polygon_area(const double* vx, const double* vy, int nv);
int oracle_point_in_polygon(double px, double py, const double* vx, const double* vy, int nv);
double oracle_polygon_weight(double xi, double yi, double r, const double* vx, const double* vy,
                             int nv);
int64_t oracle_pair_hist_polygon(int64_t n, const double* x, const double* y, const double* t,
                                 const double box[6], const double* vx, const double* vy,
                                 int nv, const double* s, int cs, const double* tt, int ct,
                                 int edge_mode, int64_t* cnt, double* wsum);
int oracle_csr_polygon_points(int64_t n, const double box[6], const double* vx,
                              const double* vy, int nv, uint64_t seed, uint32_t sim,
                              int max_attempts, double* x, double* y, double* t);

/* Bivariate (cross) K: centres labelled a, neighbours labelled b (see the source). */
int64_t oracle_k_cross(int64_t n, const double* x, const double* y, const double* t,
                       const uint8_t* labels, int a, int b, const double box[6], const double* s,
                       int cs, const double* tt, int ct, int edge_mode, int norm, int64_t* C,
                       double* S, double* K, double* L);

/* Bootstrapping (Section 3): source index of point i of realization `sim`
 * (uniform draw with replacement), and the whole resampled realization. */
int64_t oracle_bootstrap_index(int64_t n, uint64_t seed, uint32_t sim, int64_t i);
void oracle_bootstrap_points(const double* x, const double* y, const double* t, int64_t n,
                             uint64_t seed, uint32_t sim, double* ox, double* oy, double* ot);

/* Random permutation (Section 3): pi(i) of realization `sim`, the keyed Feistel
 * bijection on b = oracle_feistel_bits(n) bits it is built from, and the
 * realization (x, y kept, t_i <- t_pi(i)). */
int oracle_feistel_bits(int64_t n);
uint64_t oracle_feistel(uint64_t v, int b, uint64_t seed, uint32_t sim);
int64_t oracle_permutation_index(int64_t n, uint64_t seed, uint32_t sim, int64_t i);
void oracle_permutation_points(const double* x, const double* y, const double* t, int64_t n,
                               uint64_t seed, uint32_t sim, double* ox, double* oy, double* ot);

/* Spatial isotropic weight: proportion of the circumference of the circle of
 * radius r centred at (xi, yi) that lies inside the rectangle.  Computed as
 * 1 - |union of outside arcs| / (2 pi) for any r, by sorting the arcs. */
double oracle_spatial_weight(double xi, double yi, double r, const double box[6]);

/* Temporal weight: 1 if t_i - u >= t0 and t_i + u <= t1, else 0.5. */
double oracle_temporal_weight(double ti, double u, double t0, double t1);

/* Non-cumulative pair histogram over ordered pairs.  cnt[cs*ct] (int64) and
 * wsum[cs*ct] (FP64, compensated) are overwritten.  If centre_mask is not
 * NULL only centres i with centre_mask[i] != 0 contribute (sampled-centre
 * mode; j still runs over all n).  edge_mode 0 = no correction (weight 1),
 * 1 = isotropic.  Returns the number of qualifying ordered pairs. */
int64_t oracle_pair_hist(int64_t n, const double* x, const double* y, const double* t,
                         const double box[6], const double* s, int cs, const double* tt,
                         int ct, int edge_mode, const uint8_t* centre_mask,
                         int64_t* cnt, double* wsum);

/* Cumulative grids from a non-cumulative histogram, then K and L.
 * norm 0: A*D/(n(n-1)); norm 1: A*D/n^2.  Any output may be NULL. */
void oracle_finalize(int64_t n, const double box[6], const double* s, int cs,
                     const double* tt, int ct, int norm, const int64_t* cnt,
                     const double* wsum, int64_t* C, double* S, double* K, double* L);

/* Full estimator: pair histogram + finalize.  Returns qualifying pairs. */
int64_t oracle_k(int64_t n, const double* x, const double* y, const double* t,
                 const double box[6], const double* s, int cs, const double* tt, int ct,
                 int edge_mode, int norm, int64_t* C, double* S, double* K, double* L);

/* Monte Carlo CSR envelope: n_sims realizations of n points, element-wise
 * min / max of K; L envelopes are L(K_lo), L(K_hi).  K_all, if not NULL,
 * receives every realization's K as [n_sims][cs*ct]. */
int oracle_envelope(int64_t n, const double box[6], const double* s, int cs,
                    const double* tt, int ct, int edge_mode, int norm, int n_sims,
                    uint64_t seed, double* K_lo, double* K_hi, double* L_lo,
                    double* L_hi, double* K_all);

/* Inhomogeneous K (Section 7 future work): relative intensity rho on
 * nix x niy x nit equal cells of the box ([nit][niy][nix], x fastest), scaled
 * to integrate to n; see the source for the estimator and its readings. */
int oracle_intensity_cell(const double box[6], int nix, int niy, int nit, double x, double y,
                          double t);
void oracle_intensity_lambda(const double* rho, int nix, int niy, int nit, const double box[6],
                             int64_t n, double* lam_cell);
void oracle_inhom_points(int64_t n, const double box[6], const double* rho, int nix, int niy,
                         int nit, uint64_t seed, uint32_t sim, double* x, double* y, double* t,
                         int32_t* cell);
int64_t oracle_pair_hist_inhom(int64_t n, const double* x, const double* y, const double* t,
                               const double* lam, const double box[6], const double* s, int cs,
                               const double* tt, int ct, int edge_mode,
                               const uint8_t* centre_mask, int64_t* cnt, double* wsum);
void oracle_finalize_inhom(int64_t n, const double box[6], const double* s, int cs,
                           const double* tt, int ct, int norm, const int64_t* cnt,
                           const double* wsum, int64_t* C, double* S, double* K, double* L);

/* Directional (sector) K with translation edge correction (Section 7 future
 * work, anisotropic analysis); see the source for the estimator. */
double oracle_translation_weight(double dx, double dy, double u, const double box[6]);
int oracle_sector(double dx, double dy, int n_sec);
int64_t oracle_pair_hist_dir(int64_t n, const double* x, const double* y, const double* t,
                             const double box[6], const double* s, int cs, const double* tt,
                             int ct, int n_sec, int edge_mode, const uint8_t* centre_mask,
                             int64_t* cnt, double* wsum);

/* oracle_pair_hist restricted to pairs in adjacent cells of a uniform grid wider
 * than the largest thresholds, centres split over n_threads threads (pthreads):
 * the same pairs and per-pair arithmetic, for whole grids at large n. */
int64_t oracle_pair_hist_grid(int64_t n, const double* x, const double* y, const double* t,
                              const double box[6], const double* s, int cs, const double* tt,
                              int ct, int edge_mode, const uint8_t* centre_mask, int n_threads,
                              int64_t* cnt, double* wsum);

#ifdef __cplusplus
}
#endif
#endif
