/*
 * Oracle for the edge-corrected space-time Ripley's K estimator.
 *
 * TEST INFRASTRUCTURE ONLY: a plain single-threaded FP64 restatement of the
 * paper's Section 3 (Eq. 2, 3, 4 and the Monte Carlo envelope), written for
 * readability, not speed.  Only tests, the smoke check and the benchmark's
 * CPU-baseline / reference legs may call it.  It shares no code with the CUDA
 * library.  Build with -O2 -ffp-contract=off so that every floating-point
 * operation is rounded separately, as the pair predicate below assumes.
 */
#include "stk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Each round multiplies words 0 and 2 by the two
 * round multipliers, then mixes the high halves with the other words and the
 * key; the key is advanced by the two Weyl increments between rounds.
 * Used by the Monte Carlo CSR simulation of Section 3.
 * ------------------------------------------------------------------------- */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

double oracle_u01(uint32_t w0, uint32_t w1) {
    const double hi = (double)(w0 >> 5); /* 27 bits */
    const double lo = (double)(w1 >> 6); /* 26 bits */
    return (hi * 67108864.0 + lo) * (1.0 / 9007199254740992.0);
}

/* One coordinate of point i of realization `sim`: stream 0 = x, 1 = y, 2 = t. */
static double csr_coord(uint64_t seed, uint32_t sim, int64_t i, uint32_t stream, double lo,
                        double hi) {
    const uint32_t ctr[4] = {(uint32_t)i, sim, stream, (uint32_t)((uint64_t)i >> 32)};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    const double u = oracle_u01(w[0], w[1]);
    const double span = hi - lo;
    double v = lo + span * u;
    if (v > hi) v = hi; /* closed box: rounding may not leave it */
    return v;
}

/* Section 3, Monte Carlo method: points uniform in the spatio-temporal box. */
void oracle_csr_points(int64_t n, const double box[6], uint64_t seed, uint32_t sim, double* x,
                       double* y, double* t) {
    for (int64_t i = 0; i < n; ++i) {
        x[i] = csr_coord(seed, sim, i, 0u, box[0], box[1]);
        y[i] = csr_coord(seed, sim, i, 1u, box[2], box[3]);
        t[i] = csr_coord(seed, sim, i, 2u, box[4], box[5]);
    }
}

/* Section 3, bootstrapping: point i of realization `sim` is observed point
 * src = floor(u * n), u the 53-bit uniform of Philox block (i, sim, 4, i>>32)
 * under key (seed lo, seed hi); the product is rounded once and a result that
 * rounds up to n is taken as n - 1. */
int64_t oracle_bootstrap_index(int64_t n, uint64_t seed, uint32_t sim, int64_t i) {
    const uint32_t ctr[4] = {(uint32_t)i, sim, 4u, (uint32_t)((uint64_t)i >> 32)};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    oracle_philox4x32_10(ctr, key, w);
    const double u = oracle_u01(w[0], w[1]);
    int64_t src = (int64_t)(u * (double)n);
    if (src >= n) src = n - 1;
    return src;
}

void oracle_bootstrap_points(const double* x, const double* y, const double* t, int64_t n,
                             uint64_t seed, uint32_t sim, double* ox, double* oy, double* ot) {
    for (int64_t i = 0; i < n; ++i) {
        const int64_t src = oracle_bootstrap_index(n, seed, sim, i);
        ox[i] = x[src];
        oy[i] = y[src];
        ot[i] = t[src];
    }
}

/* Section 3, random permutation: the timestamps are exchanged among the points
 * by a pseudo-random bijection pi of [0, n) (t_i <- t_pi(i), x and y kept).
 * pi is a balanced 4-round Feistel network on b-bit values (b the smallest even
 * number >= 2 with 2^b >= n), round r mixing the right half into the left with
 * the low half-width bits of word 0 of Philox block (right, sim, 16 + r, 0)
 * under key (seed lo, seed hi) (Luby-Rackoff construction), restricted to
 * [0, n) by cycle walking: apply the network again until the value is below n
 * (Black and Rogaway, "Ciphers with arbitrary finite domains", 2002). */
int oracle_feistel_bits(int64_t n) {
    int b = 2;
    while (((int64_t)1 << b) < n) b += 2;
    return b;
}

uint64_t oracle_feistel(uint64_t v, int b, uint64_t seed, uint32_t sim) {
    const int half = b / 2;
    const uint64_t mask = ((uint64_t)1 << half) - 1;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t left = v >> half, right = v & mask;
    for (uint32_t r = 0; r < 4; ++r) {
        const uint32_t ctr[4] = {(uint32_t)right, sim, 16u + r, 0u};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        const uint64_t f = (uint64_t)w[0] & mask;
        const uint64_t next_right = left ^ f;
        left = right;
        right = next_right;
    }
    return (left << half) | right;
}

int64_t oracle_permutation_index(int64_t n, uint64_t seed, uint32_t sim, int64_t i) {
    const int b = oracle_feistel_bits(n);
    uint64_t v = oracle_feistel((uint64_t)i, b, seed, sim);
    while (v >= (uint64_t)n) v = oracle_feistel(v, b, seed, sim);
    return (int64_t)v;
}

void oracle_permutation_points(const double* x, const double* y, const double* t, int64_t n,
                               uint64_t seed, uint32_t sim, double* ox, double* oy, double* ot) {
    for (int64_t i = 0; i < n; ++i) {
        ox[i] = x[i];
        oy[i] = y[i];
        ot[i] = t[oracle_permutation_index(n, seed, sim, i)];
    }
}

/* ---------------------------------------------------------------------------
 * Section 3, spatial isotropic edge correction: the weight is the proportion
 * of the circumference of the circle centred at point i with radius d_ij that
 * lies inside the study area.  For a rectangle, the part of the circle beyond
 * an edge at distance e < r is the arc of half-angle acos(e/r) around that
 * edge's outward normal.  The outside length is the measure of the union of
 * those arcs (they can overlap near a corner), found here by sorting.
 * ------------------------------------------------------------------------- */
typedef struct {
    double lo, hi;
} arc_t;

static int arc_cmp(const void* a, const void* b) {
    const double x = ((const arc_t*)a)->lo, y = ((const arc_t*)b)->lo;
    return (x > y) - (x < y);
}

double oracle_spatial_weight(double xi, double yi, double r, const double box[6]) {
    if (r == 0.0) return 1.0; /* coincident points: the circle degenerates */
    /* distances to the right, top, left and bottom edges */
    const double e[4] = {box[1] - xi, box[3] - yi, xi - box[0], yi - box[2]};
    /* outward normals of the right, top, left and bottom edges */
    const double normal[4] = {0.0, 0.5 * ORACLE_PI, ORACLE_PI, 1.5 * ORACLE_PI};
    arc_t arcs[8];
    int na = 0;
    for (int k = 0; k < 4; ++k) {
        if (e[k] < r) {
            const double alpha = acos(e[k] / r);
            double lo = normal[k] - alpha, hi = normal[k] + alpha;
            if (lo < 0.0) { /* wraps through angle 0: split */
                arcs[na].lo = lo + 2.0 * ORACLE_PI;
                arcs[na].hi = 2.0 * ORACLE_PI;
                ++na;
                lo = 0.0;
            }
            arcs[na].lo = lo;
            arcs[na].hi = hi;
            ++na;
        }
    }
    if (na == 0) return 1.0;
    qsort(arcs, (size_t)na, sizeof(arc_t), arc_cmp);
    double outside = 0.0, cur_lo = arcs[0].lo, cur_hi = arcs[0].hi;
    for (int k = 1; k < na; ++k) {
        if (arcs[k].lo <= cur_hi) {
            if (arcs[k].hi > cur_hi) cur_hi = arcs[k].hi;
        } else {
            outside += cur_hi - cur_lo;
            cur_lo = arcs[k].lo;
            cur_hi = arcs[k].hi;
        }
    }
    outside += cur_hi - cur_lo;
    return 1.0 - outside / (2.0 * ORACLE_PI);
}

/* Section 3, temporal edge correction: 1 if both ends of the interval of
 * length 2u centred at t_i lie within the study period (closed), else 1/2. */
double oracle_temporal_weight(double ti, double u, double t0, double t1) {
    return (ti - u >= t0 && ti + u <= t1) ? 1.0 : 0.5;
}

/* ---------------------------------------------------------------------------
 * Eq. 2 and Eq. 3: the double sum over ordered pairs i != j of
 * I(d_ij <= s, u_ij <= t) / (w_ij v_ij), kept as a histogram over the
 * threshold grid: pair (i, j) falls in bin (a, b) with a the first spatial
 * threshold with d_ij <= s_a and b the first temporal threshold with
 * u_ij <= t_b.  Cumulating the histogram gives the sum at every (s_a, t_b).
 * ------------------------------------------------------------------------- */
int64_t oracle_pair_hist(int64_t n, const double* x, const double* y, const double* t,
                         const double box[6], const double* s, int cs, const double* tt,
                         int ct, int edge_mode, const uint8_t* centre_mask, int64_t* cnt,
                         double* wsum) {
    const int nb = cs * ct;
    double* s2 = (double*)malloc(sizeof(double) * (size_t)cs);
    double* comp = (double*)calloc((size_t)nb, sizeof(double));
    for (int a = 0; a < cs; ++a) s2[a] = s[a] * s[a];
    for (int k = 0; k < nb; ++k) {
        cnt[k] = 0;
        wsum[k] = 0.0;
    }
    const double s2max = s2[cs - 1], tmax = tt[ct - 1];
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (centre_mask && !centre_mask[i]) continue;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = x[i] - x[j];
            const double dy = y[i] - y[j];
            const double d2 = dx * dx + dy * dy;
            if (d2 > s2max) continue;
            const double u = fabs(t[i] - t[j]);
            if (u > tmax) continue;
            int a = 0;
            while (d2 > s2[a]) ++a;
            int b = 0;
            while (u > tt[b]) ++b;
            double w = 1.0;
            if (edge_mode == 1) {
                const double om = oracle_spatial_weight(x[i], y[i], sqrt(d2), box);
                const double v = oracle_temporal_weight(t[i], u, box[4], box[5]);
                w = 1.0 / (om * v);
            }
            const int k = a * ct + b;
            cnt[k] += 1;
            /* compensated (Kahan) accumulation keeps the oracle's own
             * rounding error far below the 1e-9 parity tolerance */
            const double yk = w - comp[k];
            const double tk = wsum[k] + yk;
            comp[k] = (tk - wsum[k]) - yk;
            wsum[k] = tk;
            ++total;
        }
    }
    free(s2);
    free(comp);
    return total;
}

/* Eq. 2 normalisation and Eq. 4 L transform over the cumulative grids. */
void oracle_finalize(int64_t n, const double box[6], const double* s, int cs, const double* tt,
                     int ct, int norm, const int64_t* cnt, const double* wsum, int64_t* C,
                     double* S, double* K, double* L) {
    const double area = (box[1] - box[0]) * (box[3] - box[2]);
    oracle_finalize_area(n, area, box[5] - box[4], s, cs, tt, ct, norm, cnt, wsum, C, S, K, L);
}

void oracle_finalize_area(int64_t n, double area, double dur, const double* s, int cs,
                          const double* tt, int ct, int norm, const int64_t* cnt,
                          const double* wsum, int64_t* C, double* S, double* K, double* L) {
    const int nb = cs * ct;
    int64_t* Cc = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    double* Sc = (double*)malloc(sizeof(double) * (size_t)nb);
    for (int a = 0; a < cs; ++a) {
        for (int b = 0; b < ct; ++b) {
            int64_t c = 0;
            double w = 0.0;
            for (int a2 = 0; a2 <= a; ++a2) {
                for (int b2 = 0; b2 <= b; ++b2) {
                    c += cnt[a2 * ct + b2];
                    w += wsum[a2 * ct + b2];
                }
            }
            Cc[a * ct + b] = c;
            Sc[a * ct + b] = w;
        }
    }
    const double nn = (double)n;
    const double denom = (norm == 1) ? nn * nn : nn * (nn - 1.0);
    const double coef = area * dur / denom;
    for (int a = 0; a < cs; ++a) {
        for (int b = 0; b < ct; ++b) {
            const int k = a * ct + b;
            const double kv = coef * Sc[k];
            if (C) C[k] = Cc[k];
            if (S) S[k] = Sc[k];
            if (K) K[k] = kv;
            if (L) L[k] = sqrt(kv / (2.0 * ORACLE_PI * tt[b])) - s[a];
        }
    }
    free(Cc);
    free(Sc);
}

int64_t oracle_k(int64_t n, const double* x, const double* y, const double* t,
                 const double box[6], const double* s, int cs, const double* tt, int ct,
                 int edge_mode, int norm, int64_t* C, double* S, double* K, double* L) {
    const int nb = cs * ct;
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)nb);
    double* wsum = (double*)malloc(sizeof(double) * (size_t)nb);
    const int64_t q =
        oracle_pair_hist(n, x, y, t, box, s, cs, tt, ct, edge_mode, NULL, cnt, wsum);
    oracle_finalize(n, box, s, cs, tt, ct, norm, cnt, wsum, C, S, K, L);
    free(cnt);
    free(wsum);
    return q;
}

/* Section 3: envelopes from the K values of simulated CSR patterns; the
 * observed pattern is not part of the envelope. */
int oracle_envelope(int64_t n, const double box[6], const double* s, int cs, const double* tt,
                    int ct, int edge_mode, int norm, int n_sims, uint64_t seed, double* K_lo,
                    double* K_hi, double* L_lo, double* L_hi, double* K_all) {
    const int nb = cs * ct;
    if (n_sims < 1) return 1;
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* t = (double*)malloc(sizeof(double) * (size_t)n);
    double* K = (double*)malloc(sizeof(double) * (size_t)nb);
    for (int k = 0; k < n_sims; ++k) {
        oracle_csr_points(n, box, seed, (uint32_t)k, x, y, t);
        oracle_k(n, x, y, t, box, s, cs, tt, ct, edge_mode, norm, NULL, NULL, K, NULL);
        for (int c = 0; c < nb; ++c) {
            if (k == 0 || K[c] < K_lo[c]) K_lo[c] = K[c];
            if (k == 0 || K[c] > K_hi[c]) K_hi[c] = K[c];
        }
        if (K_all) memcpy(K_all + (size_t)k * (size_t)nb, K, sizeof(double) * (size_t)nb);
    }
    for (int a = 0; a < cs; ++a) {
        for (int b = 0; b < ct; ++b) {
            const int c = a * ct + b;
            if (L_lo) L_lo[c] = sqrt(K_lo[c] / (2.0 * ORACLE_PI * tt[b])) - s[a];
            if (L_hi) L_hi[c] = sqrt(K_hi[c] / (2.0 * ORACLE_PI * tt[b])) - s[a];
        }
    }
    free(x);
    free(y);
    free(t);
    free(K);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Polygon study areas (the paper's experiments use an 85-vertex outline,
 * Sections 3 and 6): a simple polygon of nv vertices in either orientation,
 * closed (its boundary belongs to it).
 * ------------------------------------------------------------------------- */

/* Shoelace formula, absolute value. */
double oracle_polygon_area(const double* vx, const double* vy, int nv) {
    double a = 0.0;
    for (int k = 0; k < nv; ++k) {
        const int k1 = (k + 1) % nv;
        a += vx[k] * vy[k1] - vx[k1] * vy[k];
    }
    return fabs(a) * 0.5;
}

/* 1 if (px, py) lies on the segment a-b: zero cross product and inside the
 * segment's bounding box. */
static int on_segment(double px, double py, double ax, double ay, double bx, double by) {
    const double cross = (bx - ax) * (py - ay) - (by - ay) * (px - ax);
    if (cross != 0.0) return 0;
    return px >= fmin(ax, bx) && px <= fmax(ax, bx) && py >= fmin(ay, by) && py <= fmax(ay, by);
}

/* Closed point-in-polygon: boundary points are inside; otherwise the parity of
 * the crossings of the ray from (px, py) towards +x with the edges, an edge
 * counting when it straddles the ray's height (upper end exclusive). */
int oracle_point_in_polygon(double px, double py, const double* vx, const double* vy, int nv) {
    int inside = 0;
    for (int k = 0; k < nv; ++k) {
        const int k1 = (k + 1) % nv;
        const double ax = vx[k], ay = vy[k], bx = vx[k1], by = vy[k1];
        if (on_segment(px, py, ax, ay, bx, by)) return 1;
        if ((ay > py) != (by > py)) {
            const double xc = ax + (py - ay) * (bx - ax) / (by - ay);
            if (px < xc) inside = !inside;
        }
    }
    return inside;
}

static int cmp_double(const void* a, const void* b) {
    const double x = *(const double*)a, y = *(const double*)b;
    return x < y ? -1 : x > y ? 1 : 0;
}

/* Isotropic spatial weight for a polygon: proportion of the circumference of
 * the circle of radius r centred at (xi, yi) inside the polygon.  The circle
 * meets the edges at the roots of |a + s (b - a) - c|^2 = r^2, 0 <= s <= 1;
 * between consecutive crossing angles an arc is wholly inside or outside, and
 * its midpoint decides which. */
double oracle_polygon_weight(double xi, double yi, double r, const double* vx, const double* vy,
                             int nv) {
    if (r <= 0.0) return 1.0;
    double* ang = (double*)malloc(sizeof(double) * (size_t)(2 * nv + 1));
    int na = 0;
    for (int k = 0; k < nv; ++k) {
        const int k1 = (k + 1) % nv;
        const double ax = vx[k], ay = vy[k];
        const double dx = vx[k1] - ax, dy = vy[k1] - ay;
        const double fx = ax - xi, fy = ay - yi;
        const double A = dx * dx + dy * dy;
        if (A == 0.0) continue;
        const double B = 2.0 * (fx * dx + fy * dy);
        const double C = fx * fx + fy * fy - r * r;
        const double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) continue;
        const double sq = sqrt(disc);
        const double roots[2] = {(-B - sq) / (2.0 * A), (-B + sq) / (2.0 * A)};
        for (int q = 0; q < 2; ++q) {
            const double sr = roots[q];
            if (sr < 0.0 || sr > 1.0) continue;
            ang[na++] = atan2(fy + sr * dy, fx + sr * dx);
        }
    }
    double w;
    if (na == 0) {
        w = oracle_point_in_polygon(xi + r, yi, vx, vy, nv) ? 1.0 : 0.0;
    } else {
        qsort(ang, (size_t)na, sizeof(double), cmp_double);
        double inside = 0.0;
        for (int k = 0; k < na; ++k) {
            const double a0 = ang[k];
            const double a1 = (k + 1 < na) ? ang[k + 1] : ang[0] + 2.0 * ORACLE_PI;
            if (!(a1 > a0)) continue;
            const double mid = 0.5 * (a0 + a1);
            if (oracle_point_in_polygon(xi + r * cos(mid), yi + r * sin(mid), vx, vy, nv))
                inside += a1 - a0;
        }
        w = inside / (2.0 * ORACLE_PI);
    }
    free(ang);
    return w;
}

/* Pair histogram with the polygon weight (otherwise as oracle_pair_hist); the
 * temporal window is box[4]..box[5]. */
int64_t oracle_pair_hist_polygon(int64_t n, const double* x, const double* y, const double* t,
                                 const double box[6], const double* vx, const double* vy,
                                 int nv, const double* s, int cs, const double* tt, int ct,
                                 int edge_mode, int64_t* cnt, double* wsum) {
    const int nb = cs * ct;
    double* s2 = (double*)malloc(sizeof(double) * (size_t)cs);
    double* comp = (double*)calloc((size_t)nb, sizeof(double));
    for (int a = 0; a < cs; ++a) s2[a] = s[a] * s[a];
    for (int k = 0; k < nb; ++k) {
        cnt[k] = 0;
        wsum[k] = 0.0;
    }
    const double s2max = s2[cs - 1], tmax = tt[ct - 1];
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = x[i] - x[j];
            const double dy = y[i] - y[j];
            const double d2 = dx * dx + dy * dy;
            if (d2 > s2max) continue;
            const double u = fabs(t[i] - t[j]);
            if (u > tmax) continue;
            int a = 0;
            while (d2 > s2[a]) ++a;
            int b = 0;
            while (u > tt[b]) ++b;
            double w = 1.0;
            if (edge_mode == 1) {
                const double om = oracle_polygon_weight(x[i], y[i], sqrt(d2), vx, vy, nv);
                const double v = oracle_temporal_weight(t[i], u, box[4], box[5]);
                w = 1.0 / (om * v);
            }
            const int k = a * ct + b;
            cnt[k] += 1;
            const double yk = w - comp[k];
            const double tk = wsum[k] + yk;
            comp[k] = (tk - wsum[k]) - yk;
            wsum[k] = tk;
            ++total;
        }
    }
    free(s2);
    free(comp);
    return total;
}

/* CSR in a polygon (Section 3, Monte Carlo method): point i of realization
 * `sim` takes the first of the attempts k = 0, 1, ... whose position lies in
 * the polygon, attempt k drawing x from words 0-1 and y from words 2-3 of
 * Philox block (i, sim, 32 + k, i >> 32) uniformly in the bounding rectangle
 * box[0..3]; t as for the box (stream 2).  Returns 0, or -1 when some point
 * found no position in max_attempts attempts. */
int oracle_csr_polygon_points(int64_t n, const double box[6], const double* vx,
                              const double* vy, int nv, uint64_t seed, uint32_t sim,
                              int max_attempts, double* x, double* y, double* t) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) {
        int found = 0;
        for (int k = 0; k < max_attempts && !found; ++k) {
            const uint32_t ctr[4] = {(uint32_t)i, sim, 32u + (uint32_t)k,
                                     (uint32_t)((uint64_t)i >> 32)};
            uint32_t w[4];
            oracle_philox4x32_10(ctr, key, w);
            double px = box[0] + (box[1] - box[0]) * oracle_u01(w[0], w[1]);
            double py = box[2] + (box[3] - box[2]) * oracle_u01(w[2], w[3]);
            if (px > box[1]) px = box[1];
            if (py > box[3]) py = box[3];
            if (oracle_point_in_polygon(px, py, vx, vy, nv)) {
                x[i] = px;
                y[i] = py;
                found = 1;
            }
        }
        if (!found) return -1;
        t[i] = csr_coord(seed, sim, i, 2u, box[4], box[5]);
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * Bivariate (cross) K between the points labelled a (centres) and the points
 * labelled b (neighbours), the bivariate variant the paper names as future
 * work: ordered pairs (i, j), i != j, labels[i] == a, labels[j] == b, weights
 * centred at i; K = A*D/(n_a n_b) * sum (a != b), and for a == b the
 * univariate estimator of that subset (n_a (n_a - 1), or n_a^2 with norm 1).
 * ------------------------------------------------------------------------- */
int64_t oracle_k_cross(int64_t n, const double* x, const double* y, const double* t,
                       const uint8_t* labels, int a, int b, const double box[6], const double* s,
                       int cs, const double* tt, int ct, int edge_mode, int norm, int64_t* C,
                       double* S, double* K, double* L) {
    const int nb = cs * ct;
    int64_t* cnt = (int64_t*)calloc((size_t)nb, sizeof(int64_t));
    double* wsum = (double*)calloc((size_t)nb, sizeof(double));
    double* comp = (double*)calloc((size_t)nb, sizeof(double));
    double* s2 = (double*)malloc(sizeof(double) * (size_t)cs);
    for (int q = 0; q < cs; ++q) s2[q] = s[q] * s[q];
    const double s2max = s2[cs - 1], tmax = tt[ct - 1];
    int64_t na = 0, nbb = 0, total = 0;
    for (int64_t i = 0; i < n; ++i) {
        na += labels[i] == a;
        nbb += labels[i] == b;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (labels[i] != a) continue;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i || labels[j] != b) continue;
            const double dx = x[i] - x[j];
            const double dy = y[i] - y[j];
            const double d2 = dx * dx + dy * dy;
            if (d2 > s2max) continue;
            const double u = fabs(t[i] - t[j]);
            if (u > tmax) continue;
            int ai = 0;
            while (d2 > s2[ai]) ++ai;
            int bi = 0;
            while (u > tt[bi]) ++bi;
            double w = 1.0;
            if (edge_mode == 1) {
                const double om = oracle_spatial_weight(x[i], y[i], sqrt(d2), box);
                const double v = oracle_temporal_weight(t[i], u, box[4], box[5]);
                w = 1.0 / (om * v);
            }
            const int k = ai * ct + bi;
            cnt[k] += 1;
            const double yk = w - comp[k];
            const double tk = wsum[k] + yk;
            comp[k] = (tk - wsum[k]) - yk;
            wsum[k] = tk;
            ++total;
        }
    }
    /* cumulative grids and the normalisation of Eq. 2 with the cross denominator */
    const double area = (box[1] - box[0]) * (box[3] - box[2]);
    const double dur = box[5] - box[4];
    const double fa = (double)na, fb = (double)nbb;
    const double denom = (a != b) ? fa * fb : (norm == 1 ? fa * fa : fa * (fa - 1.0));
    for (int p = 0; p < cs; ++p) {
        for (int q = 0; q < ct; ++q) {
            int64_t c = 0;
            double wsumc = 0.0;
            for (int p2 = 0; p2 <= p; ++p2)
                for (int q2 = 0; q2 <= q; ++q2) {
                    c += cnt[p2 * ct + q2];
                    wsumc += wsum[p2 * ct + q2];
                }
            const int k = p * ct + q;
            const double kv = area * dur / denom * wsumc;
            if (C) C[k] = c;
            if (S) S[k] = wsumc;
            if (K) K[k] = kv;
            if (L) L[k] = sqrt(kv / (2.0 * ORACLE_PI * tt[q])) - s[p];
        }
    }
    free(cnt);
    free(wsum);
    free(comp);
    free(s2);
    return total;
}


/* ---------------------------------------------------------------------------
 * Inhomogeneous K, the variant Section 7 names as future work, in the
 * second-order intensity-reweighted form: every ordered pair is divided by the
 * product of the intensities at its two points.
 *
 * The caller gives a relative intensity rho, piecewise constant on
 * nix x niy x nit equal cells of the box (row-major [nit][niy][nix], x
 * fastest).  The intensity is rho scaled to integrate to n over the box:
 * lambda_c = n rho_c / sum_c (rho_c V), V = A D / (nix niy nit).
 *   K_I(s, t) = n / ((n - 1) A D) * sum_{i != j} I(d <= s, u <= t) / (w v lambda_i lambda_j)
 * (1 / (A D) with norm 1).  With rho constant, lambda = n / (A D) and K_I is
 * Eq. 2; for n points drawn independently with density proportional to rho
 * (rho > 0 everywhere) its expectation is 2 pi s^2 t, as for Eq. 2 under CSR.
 * The raw sum S reported beside K is sum I / (w v lambda_i lambda_j) times
 * (n / (A D))^2, so that K = S * A D / (n (n - 1)) in both modes.
 * ------------------------------------------------------------------------- */

/* Cell of v along one axis of the intensity grid: floor(((v - lo) / (hi - lo)) * nc),
 * each operation rounded separately, clamped into [0, nc - 1]. */
static int axis_cell(double v, double lo, double hi, int nc) {
    double f = floor(((v - lo) / (hi - lo)) * (double)nc);
    if (f < 0.0) f = 0.0;
    if (f > (double)(nc - 1)) f = (double)(nc - 1);
    return (int)f;
}

int oracle_intensity_cell(const double box[6], int nix, int niy, int nit, double x, double y,
                          double t) {
    const int ix = axis_cell(x, box[0], box[1], nix);
    const int iy = axis_cell(y, box[2], box[3], niy);
    const int it = axis_cell(t, box[4], box[5], nit);
    return (it * niy + iy) * nix + ix;
}

void oracle_intensity_lambda(const double* rho, int nix, int niy, int nit, const double box[6],
                             int64_t n, double* lam_cell) {
    const int nc = nix * niy * nit;
    const double vol = (box[1] - box[0]) * (box[3] - box[2]) * (box[5] - box[4]) / (double)nc;
    double mass = 0.0;
    for (int c = 0; c < nc; ++c) mass += rho[c] * vol;
    for (int c = 0; c < nc; ++c) lam_cell[c] = (double)n * rho[c] / mass;
}

/* Realization `sim` of n points drawn independently with density proportional
 * to rho.  Point i: a cell with probability rho_c / sum rho (cells have equal
 * volumes), then a uniform position inside it.  The cell is the first c whose
 * running sum cum_c = rho_0 + ... + rho_c (added in cell order) exceeds
 * u * cum_last, u the 53-bit uniform of Philox block (i, sim, 40, i >> 32); if
 * rounding leaves no such c, the last cell with rho > 0.  Inside cell
 * (ix, iy, it): x = x0 + (x1 - x0) * ((ix + u_x) / nix), clamped to x1, u_x
 * the uniform of stream 0 (y: stream 1, t: stream 2), as the CSR coordinates.
 * With one cell this is exactly the CSR realization. */
void oracle_inhom_points(int64_t n, const double box[6], const double* rho, int nix, int niy,
                         int nit, uint64_t seed, uint32_t sim, double* x, double* y, double* t,
                         int32_t* cell) {
    const int nc = nix * niy * nit;
    double* cum = (double*)malloc(sizeof(double) * (size_t)nc);
    double run = 0.0;
    int last_pos = 0;
    for (int c = 0; c < nc; ++c) {
        run += rho[c];
        cum[c] = run;
        if (rho[c] > 0.0) last_pos = c;
    }
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t i = 0; i < n; ++i) {
        uint32_t w[4];
        const uint32_t ctr[4] = {(uint32_t)i, sim, 40u, (uint32_t)((uint64_t)i >> 32)};
        oracle_philox4x32_10(ctr, key, w);
        const double target = oracle_u01(w[0], w[1]) * cum[nc - 1];
        int c = last_pos;
        for (int q = 0; q < nc; ++q) {
            if (cum[q] > target) {
                c = q;
                break;
            }
        }
        const int ix = c % nix, iy = (c / nix) % niy, it = c / (nix * niy);
        const double lo[3] = {box[0], box[2], box[4]}, hi[3] = {box[1], box[3], box[5]};
        const int idx[3] = {ix, iy, it}, cnt[3] = {nix, niy, nit};
        double out[3];
        for (int a = 0; a < 3; ++a) {
            const uint32_t ctr2[4] = {(uint32_t)i, sim, (uint32_t)a, (uint32_t)((uint64_t)i >> 32)};
            oracle_philox4x32_10(ctr2, key, w);
            const double u = oracle_u01(w[0], w[1]);
            double v = lo[a] + (hi[a] - lo[a]) * (((double)idx[a] + u) / (double)cnt[a]);
            if (v > hi[a]) v = hi[a];
            out[a] = v;
        }
        x[i] = out[0];
        y[i] = out[1];
        t[i] = out[2];
        if (cell) cell[i] = c;
    }
    free(cum);
}

/* Non-cumulative histograms of the inhomogeneous double sum: cnt as in
 * oracle_pair_hist, wsum of I / (w v lambda_i lambda_j) with lam[i] the
 * intensity at point i.  centre_mask as in oracle_pair_hist. */
int64_t oracle_pair_hist_inhom(int64_t n, const double* x, const double* y, const double* t,
                               const double* lam, const double box[6], const double* s, int cs,
                               const double* tt, int ct, int edge_mode,
                               const uint8_t* centre_mask, int64_t* cnt, double* wsum) {
    const int nb = cs * ct;
    double* s2 = (double*)malloc(sizeof(double) * (size_t)cs);
    double* comp = (double*)calloc((size_t)nb, sizeof(double));
    for (int a = 0; a < cs; ++a) s2[a] = s[a] * s[a];
    for (int k = 0; k < nb; ++k) {
        cnt[k] = 0;
        wsum[k] = 0.0;
    }
    const double s2max = s2[cs - 1], tmax = tt[ct - 1];
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (centre_mask && !centre_mask[i]) continue;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = x[i] - x[j];
            const double dy = y[i] - y[j];
            const double d2 = dx * dx + dy * dy;
            if (d2 > s2max) continue;
            const double u = fabs(t[i] - t[j]);
            if (u > tmax) continue;
            int a = 0;
            while (d2 > s2[a]) ++a;
            int b = 0;
            while (u > tt[b]) ++b;
            double om = 1.0, v = 1.0;
            if (edge_mode == 1) {
                om = oracle_spatial_weight(x[i], y[i], sqrt(d2), box);
                v = oracle_temporal_weight(t[i], u, box[4], box[5]);
            }
            const double w = 1.0 / (om * v * lam[i] * lam[j]);
            const int k = a * ct + b;
            cnt[k] += 1;
            const double yk = w - comp[k];
            const double tk = wsum[k] + yk;
            comp[k] = (tk - wsum[k]) - yk;
            wsum[k] = tk;
            ++total;
        }
    }
    free(s2);
    free(comp);
    return total;
}

/* Cumulative grids of the inhomogeneous estimator from its non-cumulative
 * histograms; S and K as described above, L by Eq. 4. */
void oracle_finalize_inhom(int64_t n, const double box[6], const double* s, int cs,
                           const double* tt, int ct, int norm, const int64_t* cnt,
                           const double* wsum, int64_t* C, double* S, double* K, double* L) {
    const double ad = (box[1] - box[0]) * (box[3] - box[2]) * (box[5] - box[4]);
    const double nn = (double)n;
    const double kcoef = (norm == 1) ? 1.0 / ad : nn / ((nn - 1.0) * ad);
    const double lbar = nn / ad;
    for (int a = 0; a < cs; ++a) {
        for (int b = 0; b < ct; ++b) {
            int64_t c = 0;
            double w = 0.0;
            for (int a2 = 0; a2 <= a; ++a2)
                for (int b2 = 0; b2 <= b; ++b2) {
                    c += cnt[a2 * ct + b2];
                    w += wsum[a2 * ct + b2];
                }
            const int k = a * ct + b;
            const double kv = kcoef * w;
            if (C) C[k] = c;
            if (S) S[k] = w * lbar * lbar;
            if (K) K[k] = kv;
            if (L) L[k] = sqrt(kv / (2.0 * ORACLE_PI * tt[b])) - s[a];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Directional (sector) K with translation edge correction: the anisotropic
 * analysis Section 7 names as future work.  The ordered pairs of Eq. 2 are
 * further split by the axial direction of the vector between the two points
 * (a direction and its opposite are the same axis) into n_sec equal sectors of
 * [0, pi): sector k holds the axes with angle in [k pi / n_sec, (k+1) pi / n_sec).
 * The isotropic weight of Section 3 corrects for the whole circle and is not
 * unbiased direction by direction, so this estimator uses the translation
 * correction (Ohser and Stoyan): a pair at offset (dx, dy, u) is weighted by
 * |A| / |A intersected with A shifted by (dx, dy)| = W H / ((W - |dx|)(H - |dy|))
 * in space and D / (D - u) in time.  Under CSR its expectation is
 * 2 pi s^2 t / n_sec in every sector (the shifted-window identity makes the
 * weighted pair sum an integral over offsets).
 *
 * Sector of a pair: the offset d = (x_i - x_j, y_i - y_j) is turned into the
 * upper half plane (d is kept when d_y > 0, or d_y = 0 and d_x > 0, else
 * negated), so both orders of a pair share it; the sector index is then the
 * number of boundaries b_m = (cos(m pi / n_sec), sin(m pi / n_sec)),
 * m = 1 .. n_sec - 1, with b_mx d_y - b_my d_x >= 0 (every operation rounded
 * separately).  Coincident points (d = 0) go to sector 0.
 * ------------------------------------------------------------------------- */

double oracle_translation_weight(double dx, double dy, double u, const double box[6]) {
    const double w = box[1] - box[0], h = box[3] - box[2], dur = box[5] - box[4];
    const double es = (w * h) / ((w - fabs(dx)) * (h - fabs(dy)));
    const double et = dur / (dur - u);
    return es * et;
}

int oracle_sector(double dx, double dy, int n_sec) {
    if (dx == 0.0 && dy == 0.0) return 0;
    if (!(dy > 0.0 || (dy == 0.0 && dx > 0.0))) {
        dx = -dx;
        dy = -dy;
    }
    int k = 0;
    for (int m = 1; m < n_sec; ++m) {
        const double ang = (double)m * ORACLE_PI / (double)n_sec;
        const double bx = cos(ang), by = sin(ang);
        const double cr = bx * dy - by * dx;
        if (cr >= 0.0) ++k;
    }
    return k;
}

/* Non-cumulative histograms [n_sec][cs][ct] of the directional estimator.
 * edge_mode 0: weight 1; 2: translation correction.  centre_mask as in
 * oracle_pair_hist. */
int64_t oracle_pair_hist_dir(int64_t n, const double* x, const double* y, const double* t,
                             const double box[6], const double* s, int cs, const double* tt,
                             int ct, int n_sec, int edge_mode, const uint8_t* centre_mask,
                             int64_t* cnt, double* wsum) {
    const int nb = cs * ct * n_sec;
    double* s2 = (double*)malloc(sizeof(double) * (size_t)cs);
    double* comp = (double*)calloc((size_t)nb, sizeof(double));
    for (int a = 0; a < cs; ++a) s2[a] = s[a] * s[a];
    for (int k = 0; k < nb; ++k) {
        cnt[k] = 0;
        wsum[k] = 0.0;
    }
    const double s2max = s2[cs - 1], tmax = tt[ct - 1];
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (centre_mask && !centre_mask[i]) continue;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            const double dx = x[i] - x[j];
            const double dy = y[i] - y[j];
            const double d2 = dx * dx + dy * dy;
            if (d2 > s2max) continue;
            const double u = fabs(t[i] - t[j]);
            if (u > tmax) continue;
            int a = 0;
            while (d2 > s2[a]) ++a;
            int b = 0;
            while (u > tt[b]) ++b;
            const double w = edge_mode == 2 ? oracle_translation_weight(dx, dy, u, box) : 1.0;
            const int k = (oracle_sector(dx, dy, n_sec) * cs + a) * ct + b;
            cnt[k] += 1;
            const double yk = w - comp[k];
            const double tk = wsum[k] + yk;
            comp[k] = (tk - wsum[k]) - yk;
            wsum[k] = tk;
            ++total;
        }
    }
    free(s2);
    free(comp);
    return total;
}

/* ---------------------------------------------------------------------------
 * Grid-accelerated, multithreaded restatement of oracle_pair_hist, for checking
 * whole grids at sizes where the O(n^2) loop is out of reach.  Every pair it
 * evaluates goes through the same steps as oracle_pair_hist (the same
 * separately rounded d2 and u, the same bin search, the same weight
 * functions); it only skips pairs that cannot qualify: points are binned into
 * a uniform grid whose cells are wider than s_max (x, y) and t_max (t), so a
 * qualifying pair lies in the same or adjacent cells.  Centres are split over
 * threads, each with its own compensated histograms, added in thread order.
 * Trusted only after matching oracle_pair_hist on small inputs (tests).
 * ------------------------------------------------------------------------- */
#include <pthread.h>

typedef struct {
    int64_t n;
    const double *x, *y, *t;
    const double* box;
    const double *s, *s2, *tt;
    int cs, ct, edge_mode;
    const uint8_t* centre_mask;
    int nx, ny, nt;
    const int64_t* start; /* [cells + 1] */
    const int64_t* order; /* point indices sorted by cell */
    const int* cell;      /* cell of each point */
    int64_t i0, i1;       /* centres of this thread: order[i0 .. i1) */
    int64_t* cnt;
    double *wsum, *comp;
    int64_t total;
} grid_job;

static int grid_axis(double v, double lo, double side, int nc) {
    double f = floor((v - lo) / side);
    if (f < 0.0) f = 0.0;
    if (f > (double)(nc - 1)) f = (double)(nc - 1);
    return (int)f;
}

static void* grid_worker(void* arg) {
    grid_job* g = (grid_job*)arg;
    const double s2max = g->s2[g->cs - 1], tmax = g->tt[g->ct - 1];
    for (int64_t oi = g->i0; oi < g->i1; ++oi) {
        const int64_t i = g->order[oi];
        if (g->centre_mask && !g->centre_mask[i]) continue;
        const int c = g->cell[i];
        const int cx = c % g->nx, cy = (c / g->nx) % g->ny, ct = c / (g->nx * g->ny);
        for (int dz = -1; dz <= 1; ++dz) {
            const int zz = ct + dz;
            if (zz < 0 || zz >= g->nt) continue;
            for (int dyy = -1; dyy <= 1; ++dyy) {
                const int yy = cy + dyy;
                if (yy < 0 || yy >= g->ny) continue;
                for (int dxx = -1; dxx <= 1; ++dxx) {
                    const int xx = cx + dxx;
                    if (xx < 0 || xx >= g->nx) continue;
                    const int nc = (zz * g->ny + yy) * g->nx + xx;
                    for (int64_t oj = g->start[nc]; oj < g->start[nc + 1]; ++oj) {
                        const int64_t j = g->order[oj];
                        if (j == i) continue;
                        const double dx = g->x[i] - g->x[j];
                        const double dy = g->y[i] - g->y[j];
                        const double d2 = dx * dx + dy * dy;
                        if (d2 > s2max) continue;
                        const double u = fabs(g->t[i] - g->t[j]);
                        if (u > tmax) continue;
                        int a = 0;
                        while (d2 > g->s2[a]) ++a;
                        int b = 0;
                        while (u > g->tt[b]) ++b;
                        double w = 1.0;
                        if (g->edge_mode == 1) {
                            const double om = oracle_spatial_weight(g->x[i], g->y[i], sqrt(d2),
                                                                    g->box);
                            const double v =
                                oracle_temporal_weight(g->t[i], u, g->box[4], g->box[5]);
                            w = 1.0 / (om * v);
                        }
                        const int k = a * g->ct + b;
                        g->cnt[k] += 1;
                        const double yk = w - g->comp[k];
                        const double tk = g->wsum[k] + yk;
                        g->comp[k] = (tk - g->wsum[k]) - yk;
                        g->wsum[k] = tk;
                        ++g->total;
                    }
                }
            }
        }
    }
    return NULL;
}

int64_t oracle_pair_hist_grid(int64_t n, const double* x, const double* y, const double* t,
                              const double box[6], const double* s, int cs, const double* tt,
                              int ct, int edge_mode, const uint8_t* centre_mask, int n_threads,
                              int64_t* cnt, double* wsum) {
    const int nb = cs * ct;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    /* cells strictly wider than the largest thresholds (a margin of 2^-20 absorbs the rounding
     * of the cell index), at most 2^24 of them */
    const double w = box[1] - box[0], h = box[3] - box[2], d = box[5] - box[4];
    const double side_s = s[cs - 1] * (1.0 + 1.0 / 1048576.0);
    const double side_t = tt[ct - 1] * (1.0 + 1.0 / 1048576.0);
    int nx = (int)fmin(fmax(floor(w / side_s), 1.0), 4096.0);
    int ny = (int)fmin(fmax(floor(h / side_s), 1.0), 4096.0);
    int nt = (int)fmin(fmax(floor(d / side_t), 1.0), 4096.0);
    while ((int64_t)nx * ny * nt > ((int64_t)1 << 24)) {
        nx = nx > 1 ? nx / 2 : 1;
        ny = ny > 1 ? ny / 2 : 1;
        nt = nt > 1 ? nt / 2 : 1;
    }
    const double cw = w / nx, ch = h / ny, cd = d / nt;
    const int64_t cells = (int64_t)nx * ny * nt;
    int* cell = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int64_t* start = (int64_t*)calloc((size_t)cells + 1, sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)cells, sizeof(int64_t));
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double* s2 = (double*)malloc(sizeof(double) * (size_t)cs);
    for (int a = 0; a < cs; ++a) s2[a] = s[a] * s[a];
    for (int64_t i = 0; i < n; ++i) {
        const int c = (grid_axis(t[i], box[4], cd, nt) * ny + grid_axis(y[i], box[2], ch, ny)) *
                          nx +
                      grid_axis(x[i], box[0], cw, nx);
        cell[i] = c;
        start[c + 1] += 1;
    }
    for (int64_t c = 0; c < cells; ++c) start[c + 1] += start[c];
    for (int64_t i = 0; i < n; ++i) order[start[cell[i]] + fill[cell[i]]++] = i;
    grid_job* jobs = (grid_job*)calloc((size_t)n_threads, sizeof(grid_job));
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int k = 0; k < n_threads; ++k) {
        grid_job* g = &jobs[k];
        g->n = n, g->x = x, g->y = y, g->t = t, g->box = box, g->s = s, g->s2 = s2, g->tt = tt;
        g->cs = cs, g->ct = ct, g->edge_mode = edge_mode, g->centre_mask = centre_mask;
        g->nx = nx, g->ny = ny, g->nt = nt, g->start = start, g->order = order, g->cell = cell;
        g->i0 = n * k / n_threads;
        g->i1 = n * (k + 1) / n_threads;
        g->cnt = (int64_t*)calloc((size_t)nb, sizeof(int64_t));
        g->wsum = (double*)calloc((size_t)nb, sizeof(double));
        g->comp = (double*)calloc((size_t)nb, sizeof(double));
        g->total = 0;
        if (n_threads == 1 || pthread_create(&th[k], NULL, grid_worker, g) != 0) {
            th[k] = 0;
            grid_worker(g); /* run inline when a thread cannot be started */
        }
    }
    int64_t total = 0;
    for (int k = 0; k < nb; ++k) {
        cnt[k] = 0;
        wsum[k] = 0.0;
    }
    for (int k = 0; k < n_threads; ++k) {
        if (th[k]) pthread_join(th[k], NULL);
        for (int q = 0; q < nb; ++q) {
            cnt[q] += jobs[k].cnt[q];
            wsum[q] += jobs[k].wsum[q];
        }
        total += jobs[k].total;
        free(jobs[k].cnt);
        free(jobs[k].wsum);
        free(jobs[k].comp);
    }
    free(jobs);
    free(th);
    free(cell);
    free(start);
    free(fill);
    free(order);
    free(s2);
    return total;
}
