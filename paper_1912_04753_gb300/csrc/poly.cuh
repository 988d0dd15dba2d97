// Polygon study areas on the device: closed point-in-polygon, distance to the boundary and the
// isotropic circumference weight, all in FP64 with every operation rounded separately (the
// point-in-polygon decisions decide which CSR draws are kept, so they are reproducible).
// A polygon is nv vertices (vx[k], vy[k]) in either orientation, simple, closed.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "stk_internal.h"

namespace stk {

// (px, py) on the segment a-b: zero cross product and inside the segment's bounding box.
static __device__ __forceinline__ bool poly_on_segment(double px, double py, double ax,
                                                       double ay, double bx, double by) {
    const double cross = __dsub_rn(__dmul_rn(__dsub_rn(bx, ax), __dsub_rn(py, ay)),
                                   __dmul_rn(__dsub_rn(by, ay), __dsub_rn(px, ax)));
    if (cross != 0.0) return false;
    return px >= fmin(ax, bx) && px <= fmax(ax, bx) && py >= fmin(ay, by) && py <= fmax(ay, by);
}

// Boundary points are inside; otherwise the parity of the crossings of the ray towards +x
// with the edges that straddle the ray's height (upper end exclusive).
static __device__ __forceinline__ bool poly_contains(double px, double py, const double* vx,
                                                     const double* vy, int nv) {
    bool inside = false;
    for (int k = 0; k < nv; ++k) {
        const int k1 = k + 1 < nv ? k + 1 : 0;
        const double ax = vx[k], ay = vy[k], bx = vx[k1], by = vy[k1];
        if (poly_on_segment(px, py, ax, ay, bx, by)) return true;
        if ((ay > py) != (by > py)) {
            const double xc = __dadd_rn(
                ax, __ddiv_rn(__dmul_rn(__dsub_rn(py, ay), __dsub_rn(bx, ax)), __dsub_rn(by, ay)));
            if (px < xc) inside = !inside;
        }
    }
    return inside;
}

// poly_contains over the edges of py's band only (Polygon::band): the same decisions, since
// an edge whose y-range misses py neither holds the point nor straddles the ray's height, and
// a point outside the vertices' y-range meets no edge at all.
static __device__ __forceinline__ bool poly_contains_banded(double px, double py,
                                                            const Polygon& poly) {
    if (!(py >= poly.band_ylo && py <= poly.band_yhi)) return false;
    const int b = min(max((int)((py - poly.band_ylo) * poly.band_inv), 0), kPolyBands - 1);
    const uint8_t* L = poly.band + (size_t)b * kPolyBandBytes;
    const int cnt = L[0];
    bool inside = false;
    for (int i = 0; i < cnt; ++i) {
        const int k = L[1 + i];
        const int k1 = k + 1 < poly.nv ? k + 1 : 0;
        const double ax = poly.vx[k], ay = poly.vy[k], bx = poly.vx[k1], by = poly.vy[k1];
        if (poly_on_segment(px, py, ax, ay, bx, by)) return true;
        if ((ay > py) != (by > py)) {
            const double xc = __dadd_rn(
                ax, __ddiv_rn(__dmul_rn(__dsub_rn(py, ay), __dsub_rn(bx, ax)), __dsub_rn(by, ay)));
            if (px < xc) inside = !inside;
        }
    }
    return inside;
}

// Distance from (px, py) to the polygon's boundary (the root of the least squared distance:
// the same value as the least root, the rounded root being monotone).
static __device__ __forceinline__ double poly_boundary_distance(double px, double py,
                                                                const double* vx,
                                                                const double* vy, int nv) {
    double best = INFINITY;
    for (int k = 0; k < nv; ++k) {
        const int k1 = k + 1 < nv ? k + 1 : 0;
        const double ax = vx[k], ay = vy[k];
        const double dx = vx[k1] - ax, dy = vy[k1] - ay;
        const double fx = px - ax, fy = py - ay;
        const double len2 = dx * dx + dy * dy;
        double s = len2 > 0.0 ? (fx * dx + fy * dy) / len2 : 0.0;
        s = fmin(1.0, fmax(0.0, s));
        const double ex = fx - s * dx, ey = fy - s * dy;
        best = fmin(best, ex * ex + ey * ey);
    }
    return sqrt(best);
}


// Proportion of the circumference of the circle of radius r centred at (xi, yi) inside the
// polygon: the crossings with the edges (edges whose bounding box misses the circle's are
// skipped) split the circle into arcs that are wholly inside or outside; a midpoint test
// decides each.
constexpr int kMaxCross = 32;  // crossings of one circle with the boundary

static __device__ __noinline__ double poly_weight(double xi, double yi, double r,
                                                  const double* vx, const double* vy, int nv) {
    if (r <= 0.0) return 1.0;
    double ang[kMaxCross];
    int na = 0;
    for (int k = 0; k < nv; ++k) {
        const int k1 = k + 1 < nv ? k + 1 : 0;
        const double ax = vx[k], ay = vy[k], bx = vx[k1], by = vy[k1];
        if (fmin(ax, bx) > xi + r || fmax(ax, bx) < xi - r || fmin(ay, by) > yi + r ||
            fmax(ay, by) < yi - r)
            continue;
        const double dx = bx - ax, dy = by - ay;
        const double fx = ax - xi, fy = ay - yi;
        const double A = dx * dx + dy * dy;
        if (A == 0.0) continue;
        const double B = 2.0 * (fx * dx + fy * dy);
        const double C = fx * fx + fy * fy - r * r;
        const double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) continue;
        const double sq = sqrt(disc);
        const double r0 = (-B - sq) / (2.0 * A), r1 = (-B + sq) / (2.0 * A);
        for (int q = 0; q < 2; ++q) {
            const double sr = q ? r1 : r0;
            if (sr < 0.0 || sr > 1.0) continue;
            if (na == kMaxCross) return -2.0;  // more crossings than supported
            ang[na++] = atan2(fy + sr * dy, fx + sr * dx);
        }
    }
    if (na == 0) return poly_contains(xi + r, yi, vx, vy, nv) ? 1.0 : 0.0;
    for (int a = 1; a < na; ++a) {  // insertion sort: a handful of crossings in practice
        const double v = ang[a];
        int b = a - 1;
        while (b >= 0 && ang[b] > v) {
            ang[b + 1] = ang[b];
            --b;
        }
        ang[b + 1] = v;
    }
    const double two_pi = 6.283185307179586;
    double inside = 0.0;
    for (int k = 0; k < na; ++k) {
        const double a0 = ang[k];
        const double a1 = k + 1 < na ? ang[k + 1] : ang[0] + two_pi;
        if (!(a1 > a0)) continue;
        const double mid = 0.5 * (a0 + a1);
        if (poly_contains(xi + r * cos(mid), yi + r * sin(mid), vx, vy, nv)) inside += a1 - a0;
    }
    return inside / two_pi;
}

// The same weight from the crossings' directions (no point-in-polygon test per arc, one FP32
// arctangent per inside arc): along a
// crossed edge a -> b the segment enters the disc at the smaller root of
// |a + s (b - a) - c|^2 = r^2 and leaves it at the larger, and at the larger root the circle,
// run counter-clockwise, passes to the left of the edge, i.e. into the polygon when its
// vertices run counter-clockwise (ccw = 1; the other way round for ccw = 0).  Crossings are
// taken for 0 <= s < 1 (a vertex belongs to the edge it starts).  Inside arcs run from an
// entering crossing to the next.  ebox[k] is edge k's bounding box in FP32 rounded outwards
// (x_min, x_max, y_min, y_max), for culling.  Returns -1 when a crossing is too close to a
// tangency to call or the crossings do not alternate (a vertex on the circle): the caller
// then uses poly_weight.
// F64: arc lengths in FP64 (the FP64 paths); else in FP32 from FP64 end vectors (relative
// error ~1e-7 of each arc: the FP32-guarded path).
// `list` (ne increasing edge indices, or null: every edge) restricts the scan to the edges that
// can meet the circle (a bucket list): the same crossings in the same order.  The no-crossing
// case tests a point of the circle with poly_contains_banded.
template <bool F64>
static __device__ __noinline__ double poly_weight_fast(double xi, double yi, double r,
                                                       const Polygon& poly, const float4* ebox,
                                                       int ccw, const uint8_t* list, int ne) {
    const double* vx = poly.vx;
    const double* vy = poly.vy;
    const int nv = poly.nv;
    if (r <= 0.0) return 1.0;
    // crossing points relative to the centre (FP64), an FP32 angle to sort them by, and
    // whether the circle enters the polygon there
    double cpx[kMaxCross], cpy[kMaxCross];
    float key[kMaxCross];
    bool enter[kMaxCross];
    int na = 0;
    const float m = (float)(r * 1e-4) + 1e-6f * (fabsf((float)xi) + fabsf((float)yi)) + 1e-30f;
    const float x0 = (float)(xi - r) - m, x1 = (float)(xi + r) + m;
    const float y0 = (float)(yi - r) - m, y1 = (float)(yi + r) + m;
    const double r2 = r * r;
    for (int i = 0; i < ne; ++i) {
        const int k = list ? (int)list[i] : i;
        const float4 eb = ebox[k];
        if (eb.x > x1 || eb.y < x0 || eb.z > y1 || eb.w < y0) continue;
        const int k1 = k + 1 < nv ? k + 1 : 0;
        const double ax = vx[k], ay = vy[k];
        const double dx = vx[k1] - ax, dy = vy[k1] - ay;
        const double fx = ax - xi, fy = ay - yi;
        const double A = dx * dx + dy * dy;
        if (A == 0.0) continue;
        const double hb = fx * dx + fy * dy;  // B / 2
        const double C = fx * fx + fy * fy - r2;
        const double disc = hb * hb - A * C;   // (B^2 - 4AC) / 4
        if (disc <= 0.0) continue;             // no crossing, or a touching
        const double sq = sqrt(disc);
        if (sq <= 1e-9 * A * r) return -1.0;   // nearly tangent: direction too close to call
        const double s0 = (-hb - sq) / A, s1 = (-hb + sq) / A;
        for (int q = 0; q < 2; ++q) {
            const double sr = q ? s1 : s0;
            if (sr < 0.0 || sr >= 1.0) continue;
            if (na == kMaxCross) return -2.0;  // more crossings than supported
            cpx[na] = fx + sr * dx;
            cpy[na] = fy + sr * dy;
            key[na] = atan2f((float)cpy[na], (float)cpx[na]);
            enter[na++] = (q == 1) == (ccw != 0);
        }
    }
    if (na == 0) return poly_contains_banded(xi + r, yi, poly) ? 1.0 : 0.0;
    if (na & 1) return -1.0;
    for (int a = 1; a < na; ++a) {  // insertion sort by angle: a handful of crossings
        const float kv = key[a];
        const double px = cpx[a], py = cpy[a];
        const bool e = enter[a];
        int b = a - 1;
        while (b >= 0 && key[b] > kv) {
            key[b + 1] = key[b];
            cpx[b + 1] = cpx[b];
            cpy[b + 1] = cpy[b];
            enter[b + 1] = enter[b];
            --b;
        }
        key[b + 1] = kv;
        cpx[b + 1] = px;
        cpy[b + 1] = py;
        enter[b + 1] = e;
    }
    // inside arcs run from an entering crossing to the next one, counter-clockwise; each
    // length is the angle between its end vectors, from their cross and dot products in FP64
    // (relative accuracy of the short arcs), then atan2 in FP32
    const double two_pi = 6.283185307179586;
    double inside = 0.0;
    for (int k = 0; k < na; ++k) {
        const int k1 = k + 1 < na ? k + 1 : 0;
        if (enter[k] == enter[k1]) return -1.0;  // crossings must alternate
        if (!enter[k]) continue;
        const double cr = cpx[k] * cpy[k1] - cpy[k] * cpx[k1];
        const double dt = cpx[k] * cpx[k1] + cpy[k] * cpy[k1];
        double da = F64 ? atan2(cr, dt) : (double)atan2f((float)cr, (float)dt);
        if (da < 0.0 || (da == 0.0 && dt < 0.0)) da += two_pi;
        inside += da;
    }
    return inside / two_pi;
}

}  // namespace stk
