// Host-side set-up of a job: the uniform grid and the constants of the pair kernels.
//
// Guard derivation for the FP32 bulk path.  Every point is stored relative to the origin of
// its own cell as hi + lo, with hi a multiple of the quantum q = 2^-22 * P (P the smallest
// power of two >= the cell side).  The centre is moved into each neighbour cell's frame
// (at most fs <= 3 cells away), so it lies in [-3P, 4P]: hi parts stay exact multiples of q
// below 2^24 q = 4P and the FP32 difference of two hi parts is exact; it differs
// from the true coordinate difference by at most eps = 2q (+ FP64 rounding of the cell
// origins, 2^-50 |box|).  The filter takes x instead relative to the box (quantum qX, see
// Grid), so one grid row is one frame; there eps_x = qX.  From that:
//   d2_hi = fl(fma(dx, dx, fl(dy*dy))) satisfies |d2_hi - d2| <= 2 r (eps_x + eps_y)
//           + eps_x^2 + eps_y^2 + 2^-22 r^2;
//   u_hi  = |dt_hi| satisfies |u_hi - u| <= eps_t.
// The reference predicates compare FP64 values (d2 rounded three times, s*s rounded once),
// which differ from the real ones by < 2^-50 of their size.  A band of twice the combined
// bound around each threshold therefore contains every pair whose FP32 decision could differ
// from the FP64 decision; such pairs are recomputed in FP64 by the kernel.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>

#include "stk_internal.h"

namespace stk {

static float round_down(double v) {
    float f = (float)v;
    if ((double)f > v) f = nextafterf(f, -INFINITY);
    return f;
}

static float round_up(double v) {
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return f;
}

static double pow2_at_least(double v) {
    int e;
    const double m = frexp(v, &e);  // v = m * 2^e, m in [0.5, 1)
    return m == 0.5 ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

static int cells_along(double extent, double thr) {
    // largest count whose cell side stays above thr with a relative margin, so that rounding
    // in the cell assignment can never put a qualifying pair one cell too far apart
    const double want = thr * (1.0 + 1e-9);
    long long n = (long long)floor(extent / want);
    if (n < 1) n = 1;
    while (n > 1 && extent / (double)n < want) --n;
    return (int)std::min<long long>(n, 1 << 20);
}

static void grid_counts(double W, double H, double D, double s_max, double t_max, int fs, int ft,
                        int* nx, int* ny, int* nt) {
    *nx = cells_along(W, s_max / fs);
    *ny = cells_along(H, s_max / fs);
    *nt = cells_along(D, t_max / ft);
    // keep the cell table modest: coarsen the largest axis until the grid fits
    const long long kMaxCells = 1ll << 26;
    while ((long long)*nx * *ny * *nt > kMaxCells) {
        if (*nx >= *ny && *nx >= *nt)
            *nx = (*nx + 1) / 2;
        else if (*ny >= *nt)
            *ny = (*ny + 1) / 2;
        else
            *nt = (*nt + 1) / 2;
    }
}

int build_grid(const double box[6], double s_max, double t_max, int64_t n, int f_req, Grid* g,
               char* err, size_t errlen) {
    memset(g, 0, sizeof(*g));
    g->x0 = box[0];
    g->x1 = box[1];
    g->y0 = box[2];
    g->y1 = box[3];
    g->t0 = box[4];
    g->t1 = box[5];
    const double W = box[1] - box[0], H = box[3] - box[2], D = box[5] - box[4];
    // Refinement fs (space) and ft (time), each 1..3: cells of s_max/fs and t_max/ft shrink
    // the examined neighbourhood ((2fs+1)^2 (ft+1) cells of volume 1/(fs^2 ft) threshold-cells:
    // 18, 9.4, 7.3 for fs = ft = 1, 2, 3) but visit more, smaller cells.  f_req = fs | ft << 8
    // (ft = 0: ft = fs).  Without a request (fs outside 1..3) the planner takes fs = ft = 2
    // once a cell of s_max/2 holds a few points, else 1; the job runner's tuner requests the
    // pair it measured fastest.  Up to 3 keeps hi-part differences exact (centre coordinates in
    // a neighbour's cell frame stay below 4 cells < 2^24 quanta).
    int fs = f_req & 0xff, ft = (f_req >> 8) & 0xff;
    if (fs < 1 || fs > 3) {
        int nx2, ny2, nt2;
        grid_counts(W, H, D, s_max, t_max, 2, 2, &nx2, &ny2, &nt2);
        const double per_cell = (double)n / ((double)nx2 * ny2 * nt2);
        fs = ft = per_cell >= 8.0 ? 2 : 1;
    }
    if (ft == 0) ft = fs;
    if (ft < 1 || ft > 3) {
        snprintf(err, errlen, "temporal grid refinement must be 1..3");
        return 1;
    }
    int nx, ny, nt;
    grid_counts(W, H, D, s_max, t_max, fs, ft, &nx, &ny, &nt);
    g->fs = fs;
    g->ft = ft;
    g->nx = nx;
    g->ny = ny;
    g->nt = nt;
    g->ncells = (int64_t)nx * ny * nt;
    g->cw = W / nx;
    g->ch = H / ny;
    g->cd = D / nt;
    if (!(g->cw * fs >= s_max && g->ch * fs >= s_max && g->cd * ft >= t_max)) {
        snprintf(err, errlen, "grid cells smaller than the thresholds");
        return 1;
    }
    const double px = pow2_at_least(g->cw), py = pow2_at_least(g->ch), pt = pow2_at_least(g->cd);
    g->qx = (float)ldexp(px, -22);
    g->qy = (float)ldexp(py, -22);
    g->qt = (float)ldexp(pt, -22);
    const double cwq = nearbyint(g->cw / g->qx) * g->qx;
    const double chq = nearbyint(g->ch / g->qy) * g->qy;
    const double cdq = nearbyint(g->cd / g->qt) * g->qt;
    g->cwq = (float)cwq;
    g->chq = (float)chq;
    g->cdq = (float)cdq;
    g->cwl = (float)(g->cw - cwq);
    g->chl = (float)(g->ch - chq);
    g->cdl = (float)(g->cd - cdq);
    g->qX = (float)ldexp(pow2_at_least(W), -24);
    return 0;
}

int validate_thresholds(const double box[6], const double* s, int cs, const double* tt, int ct,
                        char* err, size_t errlen) {
    if (!s || !tt) {
        snprintf(err, errlen, "threshold arrays must not be NULL");
        return 1;
    }
    if (cs < 1 || cs > kMaxThr || ct < 1 || ct > kMaxThr) {
        snprintf(err, errlen, "cs and ct must be in [1, %d]", kMaxThr);
        return 1;
    }
    for (int a = 0; a < cs; ++a) {
        if (!std::isfinite(s[a]) || s[a] <= 0.0) {
            snprintf(err, errlen, "spatial threshold %d must be finite and > 0", a);
            return 1;
        }
        if (a > 0 && !(s[a] > s[a - 1])) {
            snprintf(err, errlen, "spatial thresholds must be strictly increasing");
            return 1;
        }
    }
    for (int b = 0; b < ct; ++b) {
        if (!std::isfinite(tt[b]) || tt[b] <= 0.0) {
            snprintf(err, errlen, "temporal threshold %d must be finite and > 0", b);
            return 1;
        }
        if (b > 0 && !(tt[b] > tt[b - 1])) {
            snprintf(err, errlen, "temporal thresholds must be strictly increasing");
            return 1;
        }
    }
    const double W = box[1] - box[0], H = box[3] - box[2];
    if (s[cs - 1] > 0.5 * (W < H ? W : H)) {
        snprintf(err, errlen, "largest spatial threshold exceeds half the shorter box side");
        return 1;
    }
    return 0;
}

// Cells c of an axis (side `w`, nc cells from the box's lower bound) whose points lie at
// least `req` from both ends of the axis.  A point of cell c has v - v0 >= c*w and
// v1 - v >= (v1 - v0) - (c+1)*w up to the rounding of its cell index (a relative 2^-50 at
// most, covered by the 1e-12 factors); the last cell also takes clamped points and is never
// deep.  Returns lo > hi when no cell qualifies.
void deep_range(double w, int nc, double extent, double req, int out[2]) {
    int lo = 0;
    while (lo < nc && (double)lo * w * (1.0 - 1e-12) < req) ++lo;
    int hi = nc - 2;
    while (hi >= 0 && extent - (double)(hi + 1) * w * (1.0 + 1e-12) < req) --hi;
    out[0] = lo;
    out[1] = hi;
}

void build_pair_consts(const Grid& g, int64_t n, const double* s, int cs, const double* tt,
                       int ct, int edge, PairConsts* pc) {
    memset(pc, 0, sizeof(*pc));
    pc->tile_units = kTileUnitsDefault;
    pc->g = g;
    pc->cs = cs;
    pc->ct = ct;
    pc->nbins = cs * ct;
    pc->edge = edge;
    pc->n = n;
    // x: the filter's box-frame hi parts (each within qX / 2 of x - x0, which FP64 gives to
    // 2^-53 of the box), so a difference of two is within qX of dx
    const double ex = (double)g.qX + ldexp(fabs(g.x0) + fabs(g.x1), -50);
    const double ey = 2.0 * g.qy + ldexp(fabs(g.y0) + fabs(g.y1), -50);
    const double et = 2.0 * g.qt + ldexp(fabs(g.t0) + fabs(g.t1), -50);
    for (int a = 0; a < cs; ++a) {
        const double s2 = s[a] * s[a];
        const double sp = s[a] * (1.0 + 1e-6) + ex + ey;
        const double G = 2.0 * (2.0 * sp * (ex + ey) + ex * ex + ey * ey + ldexp(sp * sp, -22)) +
                         ldexp(sp * sp, -48);
        pc->s2[a] = s2;
        pc->s_lo[a] = s2 - G > 0.0 ? round_down(s2 - G) : -1.0f;
        pc->s_hi[a] = round_up(s2 + G);
    }
    for (int b = 0; b < ct; ++b) {
        const double G = 2.0 * et + ldexp(tt[b], -48);
        pc->tt[b] = tt[b];
        pc->t_lo[b] = tt[b] - G > 0.0 ? round_down(tt[b] - G) : -1.0f;
        pc->t_hi[b] = round_up(tt[b] + G);
    }
    pc->s2_cut = pc->s_hi[cs - 1];
    pc->u_cut = pc->t_hi[ct - 1];
    {
        const double sreq = s[cs - 1] * (1.0 + 1e-9), treq = tt[ct - 1] * (1.0 + 1e-9);
        deep_range(g.cw, g.nx, g.x1 - g.x0, sreq, pc->deep_x);
        deep_range(g.ch, g.ny, g.y1 - g.y0, sreq, pc->deep_y);
        deep_range(g.cd, g.nt, g.t1 - g.t0, treq, pc->deep_t);
    }

    // bin tables over d2 and over u: entry k holds the first bin any value in it can fall
    // into, and a flag when some guard band meets the entry.  The index (int)(v * inv_h) is
    // computed in FP32, so each entry is widened by a relative 2^-21 on both sides.
    const double dmax = (double)pc->s2_cut * (1.0 + 1e-6);
    pc->inv_hs = (float)(kTab / dmax);
    const double hs = 1.0 / (double)pc->inv_hs;
    for (int k = 0; k < kTab; ++k) {
        const double dlo = (double)k * hs * (1.0 - ldexp(1.0, -21));
        const double dhi = (k == kTab - 1) ? INFINITY : (double)(k + 1) * hs * (1.0 + ldexp(1.0, -21));
        int first = 0;
        while (first < cs && (double)pc->s_hi[first] < dlo) ++first;
        bool dirty = false;
        for (int a = 0; a < cs; ++a)
            if ((double)pc->s_lo[a] <= dhi && (double)pc->s_hi[a] >= dlo) dirty = true;
        if (first >= cs) {
            first = cs - 1;
            dirty = true;
        }
        pc->tab_s[k] = (uint8_t)(first | (dirty ? 0x80 : 0));
    }
    const double umax = (double)pc->u_cut * (1.0 + 1e-6);
    pc->inv_ht = (float)(kTab / umax);
    const double ht = 1.0 / (double)pc->inv_ht;
    for (int k = 0; k < kTab; ++k) {
        const double vlo = (double)k * ht * (1.0 - ldexp(1.0, -21));
        const double vhi = (k == kTab - 1) ? INFINITY : (double)(k + 1) * ht * (1.0 + ldexp(1.0, -21));
        int first = 0;
        while (first < ct && (double)pc->t_hi[first] < vlo) ++first;
        bool dirty = false;
        for (int b = 0; b < ct; ++b)
            if ((double)pc->t_lo[b] <= vhi && (double)pc->t_hi[b] >= vlo) dirty = true;
        if (first >= ct) {
            first = ct - 1;
            dirty = true;
        }
        pc->tab_t[k] = (uint8_t)(first | (dirty ? 0x80 : 0));
    }

    // evenly spaced thresholds (s_a ~ a * ds): bin = ceil(r / ds) - 1, decided in FP32 unless
    // r / ds lies within tol of an integer.  tol covers the d2 error above (divided by the
    // distance), the rsqrt / multiply rounding (5 * 2^-24 relative), and the largest deviation
    // of a threshold from its grid value.
    {
        const double ds = s[cs - 1] / cs;
        double dev = 0.0;
        for (int a = 0; a < cs; ++a) dev = std::max(dev, fabs(s[a] - (a + 1) * ds));
        const double tol = 2.0 * ((ex + ey) / ds + (ex * ex + ey * ey) / (ds * ds)) +
                           ldexp((double)(cs + 1), -19) + dev / ds + 1e-9 * cs;
        pc->even_s = tol < 1e-3;
        pc->inv_ds = (float)(1.0 / ds);
        pc->tol_s = round_up(tol);
        const double dt = tt[ct - 1] / ct;
        double devt = 0.0;
        for (int b = 0; b < ct; ++b) devt = std::max(devt, fabs(tt[b] - (b + 1) * dt));
        const double tolt = 2.0 * et / dt + ldexp((double)(ct + 1), -20) + devt / dt + 1e-9 * ct;
        pc->even_t = tolt < 1e-3;
        pc->inv_dt = (float)(1.0 / dt);
        pc->tol_t = round_up(tolt);
        pc->top_s = round_down((double)cs - (double)pc->tol_s);
        pc->top_t = round_down((double)ct - (double)pc->tol_t);
    }

    // weights: accurate hi + lo differences are within acc of the truth (absolute part); x's
    // hi part is the filter's box-frame one (quantum qX), its low part below qX / 2 rounded to
    // FP32 (2^-25 qX each)
    const double acc_x = ldexp((double)g.qX, -24) + ldexp(fabs(g.x0) + fabs(g.x1), -50);
    const double acc_y = ldexp((double)g.qy, -22) + ldexp(fabs(g.y0) + fabs(g.y1), -50);
    pc->tan_rel = 1e-3f;
    pc->tan_abs = round_up(4.0 * (acc_x + acc_y));
    pc->r_acc_min = round_up(ldexp(acc_x + acc_y, 22));
    const double rcut = sqrt((double)pc->s2_cut);
    pc->fast_abs = round_up(3.0 * (ex + ey) + ldexp(rcut, -21));
    pc->g_v = round_up(2.0 * (et + ldexp((double)pc->u_cut + et, -23)) +
                       ldexp(fabs(g.t0) + fabs(g.t1), -48));

    // FP64 path tables over d2 and u (start bins; exact comparisons finish the job)
    pc->inv_hs2_64 = kTab / pc->s2[cs - 1];
    pc->inv_ht_64 = kTab / pc->tt[ct - 1];
    for (int k = 0; k < kTab; ++k) {
        const double dlo = (double)k / pc->inv_hs2_64 * (1.0 - 1e-12);
        int first = 0;
        while (first < cs - 1 && pc->s2[first] < dlo) ++first;
        pc->tab_s64[k] = (uint8_t)first;
        const double vlo = (double)k / pc->inv_ht_64 * (1.0 - 1e-12);
        first = 0;
        while (first < ct - 1 && pc->tt[first] < vlo) ++first;
        pc->tab_t64[k] = (uint8_t)first;
    }
}

}  // namespace stk
