// Fused pair kernels: the hot loop of the space-time K estimator (Section 3, Eq. 2 and 3).
//
// Replaces the paper's per-point cylinder range query on an R-tree (Section 4.2) and its
// 2-tier weight cache (Section 4.3): every (centre, neighbour) candidate from the grid cells
// around a centre is evaluated once, and each qualifying ordered pair is added to a
// block-private (s_bin, t_bin) histogram: the first spatial threshold s_a with d <= s_a and the
// first temporal threshold t_b with u <= t_b.  Cumulating the histogram over (a, b) gives the
// indicator sum of Eq. 2 at every threshold pair.  Weights enter as fixed-point
// (w - 1) * 2^32, so all sums are order-independent integers.
//
// Two precisions:
//   * pair_fp32: filter, bins and weights in FP32 on cell-relative coordinates.  Every decision
//     FP32 cannot make with a proven error bound (a squared distance or a time lag inside the
//     guard band of a threshold, a temporal weight near its switch, a circle nearly tangent
//     to an edge) is recomputed in FP64 with the reference arithmetic, so counts are exact.
//   * pair_fp64: the same traversal with every pair in FP64 (the plain comparison path).
//
// Both come in variants (template parameters): a polygon study area; the directional (sector)
// K with the translation correction, whose histograms gain a sector axis; and the
// inhomogeneous K, whose pair weights h_i h_j / (w v) are accumulated in 2^-64 fixed point
// (whole part + two 32-bit fraction halves) because they are not >= 1.
//
// This is CUDA-core work (no dense contraction), bound by instruction issue.
#include <stddef.h>
#include <algorithm>

#include "stk_internal.h"
#include "poly.cuh"

#include <math.h>

namespace stk {
namespace {

constexpr int kWarps = kBlock / 32;
// variants of the FP32-guarded kernel and of its FP64 queue
constexpr int kVarPlain = 0;  // Eq. 2 (isotropic correction or none, rectangle or polygon)
constexpr int kVarDir = 1;    // directional K / translation correction
constexpr int kVarInh = 2;    // inhomogeneous K

// ---------------------------------------------------------------- exact FP64 pair (reference)

// The job's polygon with its band lists.
__device__ __forceinline__ Polygon poly_of(const PairConsts& pc) {
    Polygon p;
    p.vx = pc.pvx;
    p.vy = pc.pvy;
    p.nv = pc.nv;
    p.band = pc.pband;
    p.band_ylo = pc.band_ylo;
    p.band_yhi = pc.band_yhi;
    p.band_inv = pc.band_inv;
    return p;
}

// The edges a circle of radius r around (xi, yi) can meet: its centre's bucket list (ne
// indices), or null (every edge, ne = nv) when the radius is beyond the lists' reach or the
// list overflowed.  The bucket index comes from the FP32 box-frame position; the lists' margin
// covers its rounding.
__device__ __forceinline__ const uint8_t* poly_edges_of(const PairConsts& pc, double xi,
                                                        double yi, double r, int& ne) {
    ne = pc.nv;
    if (!(r <= (double)pc.pb_rmax)) return nullptr;
    const float fx = (float)__dsub_rn(xi, pc.g.x0), fy = (float)__dsub_rn(yi, pc.g.y0);
    const int bi = min(max((int)((fx - pc.pb_ox) * pc.pb_inv), 0), pc.pb_nx - 1);
    const int bj = min(max((int)((fy - pc.pb_oy) * pc.pb_inv), 0), pc.pb_ny - 1);
    const uint8_t* L = pc.pb_list + kPolyBucketBytes * (bj * pc.pb_nx + bi);
    const int lc = L[0];
    if (lc > kPolyBucketCap) return nullptr;
    ne = lc;
    return L + 1;
}

// Section 3 isotropic weight for a rectangle when the radius is at most half of each side:
// at most one x-edge and one y-edge cut the circle.  An edge at distance e < r removes an arc
// of half-angle acos(e/r) around its normal; when the corner lies inside the circle the two
// arcs overlap and the outside part is alpha_x + alpha_y + pi/2 (out of 2 pi).
// POLY: the study area may be a polygon (pc.nv > 0); kernels for the rectangle are compiled
// without the polygon code so that it costs them no registers.
template <bool POLY>
__device__ __forceinline__ double omega64(const PairConsts& pc, double xi, double yi,
                                          double r) {
    if (r == 0.0) return 1.0;
    if (POLY && pc.nv > 0) {
        int ne;
        const uint8_t* list = poly_edges_of(pc, xi, yi, r, ne);
        const double w = poly_weight_fast<true>(xi, yi, r, poly_of(pc), pc.pebox, pc.pccw,
                                                list, ne);
        return w >= 0.0 ? w : poly_weight(xi, yi, r, pc.pvx, pc.pvy, pc.nv);
    }
    const double ex = fmin(__dsub_rn(xi, pc.g.x0), __dsub_rn(pc.g.x1, xi));
    const double ey = fmin(__dsub_rn(yi, pc.g.y0), __dsub_rn(pc.g.y1, yi));
    const double ax = ex < r ? acos(ex / r) : 0.0;
    const double ay = ey < r ? acos(ey / r) : 0.0;
    double outside;
    if (ex < r && ey < r && __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)) < __dmul_rn(r, r))
        outside = ax + ay + 0.5 * 3.141592653589793;
    else
        outside = 2.0 * (ax + ay);
    return 1.0 - outside / (2.0 * 3.141592653589793);
}

// Section 3 temporal weight: 1 if [t_i - u, t_i + u] lies in the closed study period.
__device__ __forceinline__ double v64(const PairConsts& pc, double ti, double u) {
    return (__dsub_rn(ti, u) >= pc.g.t0 && __dadd_rn(ti, u) <= pc.g.t1) ? 1.0 : 0.5;
}

__device__ __forceinline__ unsigned long long excess_fixed64(double w) {
    const double e = w - 1.0;
    return e > 0.0 ? __double2ull_rn(e * 4294967296.0) : 0ull;
}

// excess_fixed64(1 / (om v)) without the division when om = 1 (v is 1 or 1/2: the weight is
// exactly 1 or 2, as the division gives it)
__device__ __forceinline__ unsigned long long excess_of_weights(double om, double v) {
    if (om == 1.0) return v == 1.0 ? 0ull : 4294967296ull;
    return excess_fixed64(1.0 / (om * v));
}

// Exact evaluation of the unordered pair {i, j} with the reference rounding (every operation
// rounded separately): its bin and the fixed-point excess of both ordered pairs (i, j), with
// centre i, and (j, i), with centre j.  d2 and u are the same for both orders (the FP64
// difference of two numbers is exactly the negation of the reversed difference).  Returns
// false when the pair does not qualify.
template <bool POLY, int CALLER = 0>
__device__ __noinline__ bool pair_exact(const PairConsts& pc, double xi, double yi, double ti,
                                        double xj, double yj, double tj, int& a, int& b,
                                        unsigned long long& exc_i, unsigned long long& exc_j) {
    const double dx = __dsub_rn(xi, xj);
    const double dy = __dsub_rn(yi, yj);
    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (d2 > pc.s2[pc.cs - 1]) return false;
    const double u = fabs(__dsub_rn(ti, tj));
    if (u > pc.tt[pc.ct - 1]) return false;
    // bins: the tables' start (never past the answer) and exact comparisons from there
    int ks = (int)(d2 * pc.inv_hs2_64);
    ks = ks < kTab - 1 ? ks : kTab - 1;
    a = pc.tab_s64[ks];
    while (a < pc.cs - 1 && d2 > pc.s2[a]) ++a;
    int kt = (int)(u * pc.inv_ht_64);
    kt = kt < kTab - 1 ? kt : kTab - 1;
    b = pc.tab_t64[kt];
    while (b < pc.ct - 1 && u > pc.tt[b]) ++b;
    exc_i = 0;
    exc_j = 0;
    if (pc.edge) {
        const double r = __dsqrt_rn(d2);
        exc_i = excess_of_weights(omega64<POLY>(pc, xi, yi, r), v64(pc, ti, u));
        exc_j = excess_of_weights(omega64<POLY>(pc, xj, yj, r), v64(pc, tj, u));
    }
    return true;
}

// ---------------------------------------------------------------- histogram flush

// Adds the block's histograms to the realization's global accumulators and clears them.
// hh (optional) counts pairs whose excess is exactly 1, i.e. 2^32 units: they go straight to
// the high half.
__device__ __forceinline__ void flush_hist(int real, int nbins, int reps, uint32_t* hc,
                                           unsigned long long* he, const Accum& acc,
                                           uint32_t* hh = nullptr) {
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += kBlock) {
        uint32_t c = 0, h = 0;
        unsigned long long e = 0;
        for (int r = 0; r < reps; ++r) {
            c += hc[r * nbins + b];
            e += he[r * nbins + b];
            hc[r * nbins + b] = 0;
            he[r * nbins + b] = 0;
            if (hh) {
                h += hh[r * nbins + b];
                hh[r * nbins + b] = 0;
            }
        }
        const int64_t o = (int64_t)real * nbins + b;
        if (c) atomicAdd(&acc.cnt[o], (unsigned long long)c);
        if (e & 0xffffffffull) atomicAdd(&acc.exc_lo[o], e & 0xffffffffull);
        if ((e >> 32) + h) atomicAdd(&acc.exc_hi[o], (e >> 32) + h);
    }
    __syncthreads();
}

// A warp moves its histogram replica to the global accumulators without stopping the other
// warps that share the replica: atomicExch takes each bin's value and zeroes it, so adds that
// race with it either make this flush or the next one.  Called after a warp has added
// kWarpFlush candidates, which keeps every u32 count and u64 excess of a replica far from
// overflow (at most kWarps * kWarpFlush candidates, each excess < 2^35, reach a bin between
// two flushes).
constexpr uint64_t kWarpFlush = 1ull << 26;

__device__ __forceinline__ void warp_flush(int real, int nbins, uint32_t* hc, uint32_t* hh,
                                           unsigned long long* he, const Accum& acc, int lane) {
    for (int b = lane; b < nbins; b += 32) {
        const uint32_t c = atomicExch(&hc[b], 0u);
        const uint32_t h = hh ? atomicExch(&hh[b], 0u) : 0u;
        const unsigned long long e = atomicExch(&he[b], 0ull);
        const int64_t o = (int64_t)real * nbins + b;
        if (c) atomicAdd(&acc.cnt[o], (unsigned long long)c);
        if (e & 0xffffffffull) atomicAdd(&acc.exc_lo[o], e & 0xffffffffull);
        if ((e >> 32) + h) atomicAdd(&acc.exc_hi[o], (e >> 32) + h);
    }
}

// Inhomogeneous K: a pair weight W = h_i h_j / (w v) in fixed point, split so that every part is
// a plain integer sum: the whole part, and the fraction in units of 2^-64 as two 32-bit halves.
// W < 2^32 (h is at most 2^14 and 1 / (w v) at most 8).
struct Fix96 {
    unsigned long long whole = 0, lo = 0, hi = 0;
};

__device__ __forceinline__ void add_fix96(double W, Fix96& f) {
    const double wh = floor(W);
    const unsigned long long m = __double2ull_rn(__dsub_rn(W, wh) * 18446744073709551616.0);
    f.whole += (unsigned long long)wh;
    f.lo += m & 0xffffffffull;
    f.hi += m >> 32;
}

// Adds a replica's sums to the global accumulators: lo (2^-64 units) and hi (2^-32 units) are
// re-split so that each global add is below 2^32 (no overflow however many flushes).
__device__ __forceinline__ void add_fix96_global(const Accum& acc, int64_t o,
                                                 unsigned long long whole,
                                                 unsigned long long lo,
                                                 unsigned long long hi) {
    const unsigned long long g_lo = lo & 0xffffffffull;
    const unsigned long long g_hi = (lo >> 32) + (hi & 0xffffffffull);
    const unsigned long long g_whole = whole + (hi >> 32);
    if (g_lo) atomicAdd(&acc.exc_lo[o], g_lo);
    if (g_hi) atomicAdd(&acc.exc_hi[o], g_hi);
    if (g_whole) atomicAdd(&acc.whole[o], g_whole);
}

// Inhomogeneous K: flushes of the three fixed-point sums (see flush_hist and warp_flush).
__device__ __forceinline__ void flush_hist_inh(int real, int nbins, int reps, uint32_t* hc,
                                               unsigned long long* he, unsigned long long* hf,
                                               unsigned long long* hw, const Accum& acc) {
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += kBlock) {
        uint32_t c = 0;
        unsigned long long lo = 0, hi = 0, wh = 0;
        for (int r = 0; r < reps; ++r) {
            const int i = r * nbins + b;
            c += hc[i];
            lo += he[i];
            hi += hf[i];
            wh += hw[i];
            hc[i] = 0;
            he[i] = 0;
            hf[i] = 0;
            hw[i] = 0;
        }
        const int64_t o = (int64_t)real * nbins + b;
        if (c) atomicAdd(&acc.cnt[o], (unsigned long long)c);
        add_fix96_global(acc, o, wh, lo, hi);
    }
    __syncthreads();
}

__device__ __forceinline__ void warp_flush_inh(int real, int nbins, uint32_t* hc,
                                               unsigned long long* he, unsigned long long* hf,
                                               unsigned long long* hw, const Accum& acc,
                                               int lane) {
    for (int b = lane; b < nbins; b += 32) {
        const uint32_t c = atomicExch(&hc[b], 0u);
        const unsigned long long lo = atomicExch(&he[b], 0ull);
        const unsigned long long hi = atomicExch(&hf[b], 0ull);
        const unsigned long long wh = atomicExch(&hw[b], 0ull);
        const int64_t o = (int64_t)real * nbins + b;
        if (c) atomicAdd(&acc.cnt[o], (unsigned long long)c);
        add_fix96_global(acc, o, wh, lo, hi);
    }
}

__device__ __forceinline__ int bin_fp32(float v, float inv_h, const uint8_t* tab,
                                        const float* lo, const float* hi, int nthr, bool& amb) {
    int k = (int)(v * inv_h);
    k = k < kTab - 1 ? k : kTab - 1;
    k = k > 0 ? k : 0;  // also keeps lanes without an entry inside the table
    const uint32_t e = tab[k];
    int a = (int)(e & 0x7fu);
    if (e & 0x80u) {
        while (a < nthr - 1 && v > hi[a]) ++a;
        if (v >= lo[a]) amb = true;
    }
    return a;
}


// Bin of value/spacing for evenly spaced thresholds at 1, 2, ..., nthr (in spacing units):
// ceil(t) - 1, clamped, with `amb` set when t lies within tol of a threshold.  rint is taken
// with the 1.5 * 2^23 shift, exact for 0 <= t < 2^22.
__device__ __forceinline__ int bin_even(float t, float tol, float top, int nthr, bool& amb) {
    const float kShift = 12582912.0f;
    const float ts = t + kShift;
    const float kf = ts - kShift;
    const int k = __float_as_int(ts) - 0x4B400000;
    const float fr = t - kf;
    amb |= (fabsf(fr) <= tol && k >= 1) || t >= top;
    int a = k + (fr > 0.0f ? 1 : 0) - 1;
    a = a < 0 ? 0 : a;
    return a < nthr - 1 ? a : nthr - 1;
}

// Directional K: sector of the pair offset (dx, dy) among pc.nsec equal axial sectors of
// [0, pi): the offset turned into the upper half plane (both orders of a pair agree), then the
// number of boundaries b with b_x d_y - b_y d_x >= 0, each operation rounded separately;
// coincident points in sector 0.
__device__ __forceinline__ int sector_of(const PairConsts& pc, double dx, double dy) {
    if (dx == 0.0 && dy == 0.0) return 0;
    if (!(dy > 0.0 || (dy == 0.0 && dx > 0.0))) {
        dx = -dx;
        dy = -dy;
    }
    int k = 0;
    for (int m = 0; m < pc.nsec - 1; ++m)
        k += __dsub_rn(__dmul_rn(pc.sec_bx[m], dy), __dmul_rn(pc.sec_by[m], dx)) >= 0.0 ? 1 : 0;
    return k;
}

// Translation correction of a pair at offset (dx, dy) and lag u: |A| / |A intersected with A
// shifted by (dx, dy)| in space times D / (D - u) in time (at most 4 * 2 for thresholds within
// half the sides and half the period).
__device__ __forceinline__ double translation_weight(const PairConsts& pc, double dx, double dy,
                                                     double u) {
    const double es = (pc.tw * pc.th) / ((pc.tw - fabs(dx)) * (pc.th - fabs(dy)));
    return es * (pc.td / (pc.td - u));
}

// Evaluates one queued entry in FP64.  Full entries (w bit 0 clear) are unordered pairs
// {x, y}: bins, a count of (w bit 1) + (w bit 2) ordered pairs (the centre of each order may
// be masked out) and the excess of those orders.  Weight-only entries (w bit 0 set) carry the
// bin in w >> 2 and add the excess of the single ordered pair with centre x.
// kVarDir: the directional / translation-corrected estimator (full entries only): the bin
// takes the pair's sector, both orders the translation weight.  kVarInh: the inhomogeneous K
// (full entries only): the weights of both orders times h_i h_j, returned in *fx.
template <bool POLY, int VAR = kVarPlain, int CALLER = 0>
__device__ __forceinline__ bool exact_eval(const PairConsts& pc, const RealBatch& rb, uint4 q,
                                           int& bin, uint32_t& counts,
                                           unsigned long long& exc, Fix96* fx = nullptr) {
    const int64_t base = (int64_t)q.z * rb.n;
    const double xi = rb.X[base + q.x], yi = rb.Y[base + q.x], ti = rb.T[base + q.x];
    const double xj = rb.X[base + q.y], yj = rb.Y[base + q.y], tj = rb.T[base + q.y];
    if (VAR == kVarInh) {
        int a, b;
        unsigned long long ei, ej;
        if (!pair_exact<false, CALLER>(pc, xi, yi, ti, xj, yj, tj, a, b, ei, ej)) return false;
        const bool act_i = (q.w >> 1) & 1u, act_j = (q.w >> 2) & 1u;
        bin = a * pc.ct + b;
        counts = (uint32_t)act_i + (uint32_t)act_j;
        exc = 0;
        const double hh = __dmul_rn(rb.H[base + q.x], rb.H[base + q.y]);
        double wi = 1.0, wj = 1.0;
        if (pc.edge) {
            const double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj);
            const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
            const double u = fabs(__dsub_rn(ti, tj));
            wi = 1.0 / (omega64<false>(pc, xi, yi, r) * v64(pc, ti, u));
            wj = 1.0 / (omega64<false>(pc, xj, yj, r) * v64(pc, tj, u));
        }
        Fix96 f;
        if (act_i) add_fix96(__dmul_rn(wi, hh), f);
        if (act_j) add_fix96(__dmul_rn(wj, hh), f);
        *fx = f;
        return true;
    }
    if (VAR == kVarDir) {
        const double dx = __dsub_rn(xi, xj);
        const double dy = __dsub_rn(yi, yj);
        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        const double u = fabs(__dsub_rn(ti, tj));
        if (d2 > pc.s2[pc.cs - 1] || u > pc.tt[pc.ct - 1]) return false;
        int a = 0;
        while (a < pc.cs - 1 && d2 > pc.s2[a]) ++a;
        int b = 0;
        while (b < pc.ct - 1 && u > pc.tt[b]) ++b;
        const bool act_i = (q.w >> 1) & 1u, act_j = (q.w >> 2) & 1u;
        bin = (sector_of(pc, dx, dy) * pc.cs + a) * pc.ct + b;
        counts = (uint32_t)act_i + (uint32_t)act_j;
        const unsigned long long e =
            pc.edge == STK_EDGE_TRANSLATION ? excess_fixed64(translation_weight(pc, dx, dy, u))
                                            : 0ull;
        exc = (act_i ? e : 0ull) + (act_j ? e : 0ull);
        return true;
    }
    if ((q.w & 1u) == 0u) {
        int a, b;
        unsigned long long ei, ej;
        if (!pair_exact<POLY, CALLER>(pc, xi, yi, ti, xj, yj, tj, a, b, ei, ej)) return false;
        const bool act_i = (q.w >> 1) & 1u, act_j = (q.w >> 2) & 1u;
        bin = a * pc.ct + b;
        counts = (uint32_t)act_i + (uint32_t)act_j;
        exc = (act_i ? ei : 0ull) + (act_j ? ej : 0ull);
    } else {
        bin = (int)(q.w >> 2);
        counts = 0;
        const double dx = __dsub_rn(xi, xj);
        const double dy = __dsub_rn(yi, yj);
        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        const double u = fabs(__dsub_rn(ti, tj));
        exc = excess_fixed64(1.0 / (omega64<POLY>(pc, xi, yi, __dsqrt_rn(d2)) * v64(pc, ti, u)));
    }
    return true;
}

// ---------------------------------------------------------------- FP32 guarded kernel
//
// Each unordered pair {i, j} is evaluated once: a centre i only scans neighbours j with a
// larger sorted index (rows of the grid before i's row are skipped; within i's own row, a
// single index compare), the pair's bin is found once, and both ordered pairs (i, j) and
// (j, i) are added: the count by 2, the weight excess of each order with its own centre.
//
// One warp processes one work unit (32 consecutive centres of a grid row) at a time, in three
// phases that keep the expensive work on full warps:
//   A (filter): the warp walks the neighbour cells of its centres (reading the sorted points
//     from L2 / L1, every lane the same address), moves its centres into each neighbour
//     cell's frame, and tests every candidate with paired FP32 arithmetic.  Candidates inside
//     the s_max / t_max bands are appended, with their d2 and u, to a per-warp queue by ballot
//     compaction.
//   B (bin): 64 queued pairs at a time (two per lane): spatial and temporal bins, the counts,
//     the temporal weights and the interior tests of both orders.  Orders whose spatial weight
//     is not 1 go to queue 2; pairs or orders FP32 cannot decide go to the global FP64 queue.
//   C (weight): 32 orders of queue 2 at a time: accurate distance from the hi + lo parts and
//     the isotropic weight of the (at most two) cutting edges; near-tangent circles go to
//     the FP64 queue.
// The directional and inhomogeneous variants take every pair's sector and weights in phase B
// itself (no queue 2); what FP32 cannot decide there goes to the FP64 queue as a whole pair.
// Entries of the FP64 queue are evaluated with the reference arithmetic by exact_kernel.
// FP64 runs at 1/64 of the FP32 rate on this part: a handful of such pairs inside this
// kernel would hold a whole warp for thousands of cycles.

constexpr int kRing = 192;   // per-warp queue of candidate pairs (linear, compacted on drain)
constexpr int kDrain = 64;   // phase-B batch: two pairs per lane
constexpr int kQ2 = 32 + 4 * 32;  // per-warp queue of orders needing the spatial weight:
                                  // under 32 left over + up to 4 orders per lane of a pass
static_assert(kDrain - 1 + 4 * 32 <= kRing, "queue must hold a batch plus one step");

struct WarpSm {
    float4 cen_a[32];   // x_hi (box frame), y_hi, t_hi (own cell frame), interior bound on d2
    float4 cen_b[32];   // x_lo (box frame), y_lo, e_x, e_y
    float cen_te[32];   // distance to the nearer end of the study period
    float cen_h[32];    // inhomogeneous K: h of the centres
    uint4 ring[kRing + 1];  // (d2 bits, u bits, meta, neighbour)  meta: lane | (fs + dcy) << 8,
                            // dcy = centre's y cell - neighbour's y cell
    uint2 q2[kQ2];      // (meta | order << 11 | vhalf << 12 | bin << 13, neighbour)
};

struct Smem32 {
    PairConsts pc;      // the single-job kernel copies only the part before `s2`
    WarpSm w[kWarps];
    unsigned long long cursor;  // (tile << 32) | next index in the tile, see next_unit
    // polygon study areas (no block barrier between realizations): the cursors of realizations
    // of either parity, the warps done with the realization in each slot, and the realization
    // each slot is ready for
    unsigned long long pcur[2];
    int pdone[2], pready[2];
    // histograms follow (dynamic size)
};

constexpr uint32_t kNoUnit = 0xffffffffu;
constexpr int kSpinLimit = 1 << 20;

// Next work unit of the current realization for the calling warp, or kNoUnit when none is
// left.  The block claims tiles of `tile` consecutive units (neighbouring centres of one row,
// so its warps walk the same neighbour cells and share them in L1; `ntiles` tiles in
// [ubeg, uend)) from the realization's global counter; its warps draw units from the current
// tile through a shared cursor, with no block barrier, so a warp with a cheap unit never waits
// for one with a dear unit.  The warp that draws index `tile` claims the next tile; warps that
// draw past it wait (bounded) for the new tile.  Lane 0 works, the result is broadcast.
__device__ __forceinline__ uint32_t next_unit(unsigned long long* cursor, uint32_t* counter,
                                              uint32_t ubeg, uint32_t uend, uint32_t tile,
                                              uint32_t ntiles, int lane,
                                              unsigned long long* stats, bool never_publish) {
    uint32_t ui = kNoUnit;
    if (lane == 0) {
        int spin = 0;
        bool stuck = false;
        while (!stuck) {
            const unsigned long long old = atomicAdd(cursor, 1ull);
            const uint32_t t = (uint32_t)(old >> 32), idx = (uint32_t)old;  // tile index
            if (t >= ntiles) break;
            if (idx < tile) {
                const uint32_t u = ubeg + t * tile + idx;
                if (u < uend) {
                    ui = u;
                    break;
                }
                continue;  // past the end of the last tile: draw until someone claims anew
            }
            if (idx == tile) {
                if (never_publish) break;  // test hook: the waiting warps' waits run out
                const uint32_t nt = atomicAdd(counter, 1u);
                atomicExch(cursor, ((unsigned long long)nt << 32) | 1ull);  // index 0 is ours
                if (nt >= ntiles) break;
                ui = ubeg + nt * tile;  // < uend: nt < ntiles
                break;
            }
            while ((uint32_t)(*reinterpret_cast<volatile unsigned long long*>(cursor) >> 32) ==
                   t) {
                if (++spin > kSpinLimit) {
                    atomicAdd(&stats[4], 1ull);  // never expected: the claimer is resident
                    stuck = true;
                    break;
                }
                __nanosleep(32);
            }
        }
    }
    return __shfl_sync(0xffffffffu, ui, 0);
}

struct WarpCtx {
    uint32_t* hc;             // this warp's histogram replica: counts
    uint32_t* hh;             //   orders whose weight is exactly 2 (excess 1)
    unsigned long long* he;   //   other excess, 2^-32 units
    const float4* Pk;         // coordinate records of the current realization
    const float4* Ek;         // edge records of the current realization
    const float* NX;          // the filter's x and y arrays (negated hi parts)
    const float* NY;
    const uint8_t* mk;        // centre mask of the current realization, or null
    uint32_t real;
    uint32_t c_begin;
    int cy;                   // the unit's cell row (set in polygon study areas only)
    // polygon study areas: the global excess accumulators, for weights above 8
    unsigned long long* exlo;
    unsigned long long* exhi;
    uint32_t onA, onB;        // lanes whose centre counts as a centre / as a neighbour
    int q2n;                  // queue 2 fill (warp-uniform)
    bool deep;                // every point the unit meets has w = v = 1 for counted pairs
    const PairConsts* pa;     // shared-memory copy (indexed tables and bands)
    // inhomogeneous K: the weights' fraction high halves and whole parts (`he` holds the low
    // halves), and h and the low parts of the current realization's points
    unsigned long long* hf;
    unsigned long long* hw;
    const double* H;
    const float2* Plok;
};

// Evaluates an entry in FP64 inside the pair kernel (only when the FP64 queue is full).
// CALLER: 0 for the single-job kernels, 1 for the fused kernel, which gets its own instances of
// the out-of-line helpers (a callee shared with the fused kernel changed the single-job
// kernel's register allocation and cost it 2%).
template <bool POLY, int VAR = kVarPlain, int CALLER = 0>
__device__ __noinline__ void exact_inline(const PairConsts* gpc, RealBatch rb, uint4 entry,
                                          uint32_t* hc, unsigned long long* he,
                                          unsigned long long* hf, unsigned long long* hw) {
    int bin;
    uint32_t counts;
    unsigned long long exc;
    Fix96 f;
    if (exact_eval<POLY, VAR, CALLER>(*gpc, rb, entry, bin, counts, exc, &f)) {
        if (counts) atomicAdd(&hc[bin], counts);
        if (exc) atomicAdd(&he[bin], exc);
        if (VAR == kVarInh) {
            if (f.lo) atomicAdd(&he[bin], f.lo);
            if (f.hi) atomicAdd(&hf[bin], f.hi);
            if (f.whole) atomicAdd(&hw[bin], f.whole);
        }
    }
}

// Appends the flagged lanes' entries to the global FP64 queue.  If the queue is full the entry
// is evaluated here instead (correct, only slower).
template <bool POLY, int VAR = kVarPlain, int CALLER = 0>
__device__ __forceinline__ void push_exact(const PairConsts* gpc, const RealBatch& rb,
                                           const ExactQueue& xq, bool flag, uint4 entry,
                                           int lane, uint32_t lt, uint32_t* hc,
                                           unsigned long long* he,
                                           unsigned long long* hf = nullptr,
                                           unsigned long long* hw = nullptr) {
    const uint32_t m = __ballot_sync(0xffffffffu, flag);
    if (m == 0u) return;
    unsigned int pos = 0;
    if (lane == 0) pos = atomicAdd(xq.count, (unsigned int)__popc(m));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (!flag) return;
    const unsigned int idx = pos + (unsigned int)__popc(m & lt);
    if (idx < xq.cap)
        xq.e[idx] = entry;
    else
        exact_inline<POLY, VAR, CALLER>(gpc, rb, entry, hc, he, hf, hw);
}

// ---------------------------------------------------------------- FP32 isotropic weight

// FP32 square root of v >= 0: the hardware reciprocal square root and one Newton step (within
// about an ulp of the correctly rounded root); 0 for v = 0.
__device__ __forceinline__ float sqrt_nr(float v) {
    const float y = rsqrtf(v + 1e-30f);
    const float s = v * y;
    return fmaf(fmaf(-s, s, v), 0.5f * y, s);
}

// Half-angle alpha = acos(e / r) of the arc that an edge at distance e cuts from the circle of
// radius r (inv_r = 1 / r), 0 when e >= r.  acos(x) = sqrt(1 - x) P(x), P a degree-7 least-squares
// fit of acos(x) / sqrt(1 - x) on [0, 1] (fit_arc_poly.py; fit error below 3e-8 relative, FP32
// evaluation within 3e-7 absolute); 1 - x is formed as (r - e) / r, whose difference is exact
// when e is near r, so the angle stays accurate up to the tangency band.
__device__ __forceinline__ float arc_half_angle(float e, float r, float inv_r) {
    const float x = fminf(e * inv_r, 1.0f);  // an edge beyond the circle: no arc (P stays finite)
    const float om = fmaxf((r - e) * inv_r, 0.0f);
    float p = -0.0012278304202482104f;
    p = fmaf(p, x, 0.006548574194312096f);
    p = fmaf(p, x, -0.01692071184515953f);
    p = fmaf(p, x, 0.030777458101511f);
    p = fmaf(p, x, -0.05013412609696388f);
    p = fmaf(p, x, 0.08897225558757782f);
    p = fmaf(p, x, -0.2145983725786209f);
    p = fmaf(p, x, 1.570796251296997f);
    return sqrt_nr(om) * p;
}

// Share A of the circle of radius r (inv_r = 1 / r) outside the rectangle, for a centre at
// distances e1 and e2 from its nearer x and y edges (Section 3: the weight is 1 / (1 - A)).
// The radius is at most half of each side, so at most one x-edge and one y-edge cut the circle;
// when the corner lies inside it the two cut arcs overlap and the outside part is
// alpha_1 + alpha_2 + pi / 2 (of 2 pi), else 2 (alpha_1 + alpha_2).
__device__ __forceinline__ float outside_share(float e1, float e2, float r, float inv_r) {
    const float a1 = arc_half_angle(e1, r, inv_r);
    const float a2 = arc_half_angle(e2, r, inv_r);
    return (fmaf(e1, e1, e2 * e2) < r * r) ? (a1 + a2 + 1.57079632679f) * 0.159154943092f
                                           : (a1 + a2) * 0.318309886184f;
}

// r = sqrt(r2) and 1 / r in FP32 from the hardware reciprocal square root with a Newton step
// each (r2 = 0 gives a NaN r, which the callers' range tests send to FP64).
__device__ __forceinline__ void radius_nr(float r2, float& r, float& inv_r) {
    const float y = rsqrtf(r2);
    const float s = r2 * y;
    r = fmaf(fmaf(-s, s, r2), 0.5f * y, s);
    inv_r = y * fmaf(-0.5f * r2 * y, y, 1.5f);
}

// ------------------------------------------------- FP32 polygon weight (pairs of FP32 numbers)
// Values that need more than FP32 precision are carried as unevaluated sums hi + lo of two FP32
// numbers (error-free sums and products; every step stays on the FP32 pipe).

// s + e = a + b exactly (s = a + b rounded).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// p + e = a * b exactly (p = a * b rounded).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Arc half-angle psi = acos(h / r) as a pair, from d = r - h (pair, 0 < d <= r), r (pair) and
// y ~ 1 / rh (within a few ulps; the correction step makes om insensitive to it):
// om = d / r and x = 1 - om to about 2^-46, acos(x) = sqrt(om) P(x) with P a degree-9 fit of
// acos(x) / sqrt(1 - x) on [0, 1] (fit_arc_poly.py, fit error below 1e-9 relative), its
// constant term and last Horner step and the product with sqrt(om) as pairs.  Measured error
// below 1e-8 absolute; the weight's bound takes 3e-8 (kArcErrF32).
constexpr float kArcErrF32 = 3.0e-8f;

__device__ __forceinline__ void arc_half_angle_pair(float dh, float dl, float rh, float rl,
                                                    float y, float& ph, float& pl) {
    const float om0 = dh * y;
    float res = __fmaf_rn(-om0, rh, dh);
    res = __fsub_rn(__fadd_rn(res, dl), om0 * rl);
    const float om1 = res * y;
    const float ys = rsqrtf(om0);
    float s0 = om0 * ys;
    s0 = __fmaf_rn(__fmaf_rn(-s0, s0, om0), 0.5f * ys, s0);
    const float s1 = __fadd_rn(__fmaf_rn(-s0, s0, om0), om1) * (0.5f * ys);
    const float x = __fsub_rn(__fsub_rn(1.0f, om0), om1);
    float p = -0.0004011530545540154f;
    p = __fmaf_rn(p, x, 0.002504516625776887f);
    p = __fmaf_rn(p, x, -0.007419043220579624f);
    p = __fmaf_rn(p, x, 0.014548846520483494f);
    p = __fmaf_rn(p, x, -0.02282850071787834f);
    p = __fmaf_rn(p, x, 0.03330930322408676f);
    p = __fmaf_rn(p, x, -0.050739698112010956f);
    p = __fmaf_rn(p, x, 0.08904469013214111f);
    p = __fmaf_rn(p, x, -0.21460172533988953f);
    float m, me, Ph, Pe;
    two_prod(p, x, m, me);
    two_sum(1.5707963705062866f, m, Ph, Pe);
    const float Pl = __fadd_rn(__fadd_rn(Pe, me), -4.4270890953157505e-08f);
    ph = s0 * Ph;
    pl = __fadd_rn(__fmaf_rn(s0, Ph, -ph), __fmaf_rn(s0, Pl, s1 * Ph));
}

// Share of the circle of radius r = rh + rl around the point c (box frame: c - (x0, y0) =
// (cxh + cxl, cyh + cyl)) that lies inside the polygon, for a centre inside it (Section 3's
// isotropic weight is 1 / inside).  For each edge whose box meets the circle's: f = a - c
// (a the edge's start vertex), the line's signed distance h = f x u and d = r - |h| as pairs
// (u the unit direction); a line with |d| within the band is too close to tangency to call.
// A crossing line meets the circle at u0 -+ t along the edge (u0 = -(f . u),
// t = sqrt(d (r + |h|))); those on the edge, away from its vertices by more than their
// position error, are crossings at polar angle phi_m +- psi (phi_m the normal's direction
// towards the line, psi = acos(|h| / r)), a pair in [0, 2 pi).  Going round the circle from angle
// 0 the inside indicator starts at I0 and steps by +1 at an entering crossing, -1 at a leaving
// one, so the inside measure is 2 pi I0 - sum(delta_c theta_c) in any order of the crossings, and
// I0 = 1 when the crossing of least angle leaves.  Each angle is within
// kArcErrF32 + 2 poly_eh / t (the arc's error and the positions' error eh through dpsi = dh / t)
// of the true one (edges that cannot meet the circle are skipped: those outside its centre's
// bucket list, PairConsts::pb_list, and those whose box misses the circle's); the result is
// refused (false: the order goes to FP64) when the least angle
// lies within its error of 0, the largest within the largest error of 2 pi, or the second least
// within both errors of the least (the choice of I0 would be in doubt), when entering and
// leaving crossings do not balance, or when the errors add up to more than 8.5e-7 of the inside
// share.  No crossing: the whole circle is inside unless it might enclose the polygon
// (2 r >= the polygon's larger bounding-box side: refused).  inv_r ~ 1 / rh (a few ulps).
__device__ __forceinline__ bool poly_share_f32(const PairConsts& pc, float cxh, float cxl,
                                               float cyh, float cyl, float rh, float rl,
                                               float inv_r, float& inside, float& outside) {
    const float kPiH = 3.1415927410125732f, kPiL = -8.742277657347586e-08f;
    const float k2PiH = 6.2831854820251465f, k2PiL = -1.7484555314695172e-07f;
    const float eh = pc.poly_eh;
    const float m = rh * 1e-5f + 1e-6f * (fabsf(cxh) + fabsf(cyh)) + eh;
    const float x0 = cxh - rh - m, x1 = cxh + rh + m, y0 = cyh - rh - m, y1 = cyh + rh + m;
    const float band = 4.0f * eh + rh * 1e-12f;
    float Sh = 0.0f, Sl = 0.0f;              // sum of delta_c theta_c
    float a1h = 4.0e1f, a1l = 0.0f, a1e = 0.0f;  // least angle, its error
    bool a1in = false;                       // ... and whether it enters
    float a2h = 4.0e1f, a2l = 0.0f;          // second least angle
    float zh = -1.0f, zl = 0.0f;             // largest angle
    float esum = 0.0f, emax = 0.0f;
    int bal = 0, na = 0;
    // the edges the circle can meet: its centre's bucket list (every edge when the list
    // overflowed or the radius is beyond the lists' reach)
    const int bi = min(max((int)((cxh - pc.pb_ox) * pc.pb_inv), 0), pc.pb_nx - 1);
    const int bj = min(max((int)((cyh - pc.pb_oy) * pc.pb_inv), 0), pc.pb_ny - 1);
    const uint8_t* L = pc.pb_list + kPolyBucketBytes * (bj * pc.pb_nx + bi);
    const int lc = L[0];
    const bool all = lc > kPolyBucketCap || !(rh <= pc.pb_rmax);
    const int ne = all ? pc.nv : lc;
    for (int i = 0; i < ne; ++i) {
        const int k = all ? i : (int)L[1 + i];
        const float4* E = pc.pe32 + 4 * k;
        const float4 eb = E[3];
        if (eb.x > x1 || eb.y < x0 || eb.z > y1 || eb.w < y0) continue;
        const float4 e0 = E[0], e1 = E[1];
        float fxh, fxe, fyh, fye;
        two_sum(e0.x, -cxh, fxh, fxe);
        two_sum(e0.z, -cyh, fyh, fye);
        const float fxl = __fadd_rn(fxe, __fsub_rn(e0.y, cxl));
        const float fyl = __fadd_rn(fye, __fsub_rn(e0.w, cyl));
        // h = fx uy - fy ux
        float p1, q1, p2, q2, hs, he;
        two_prod(fxh, e1.z, p1, q1);
        two_prod(fyh, e1.x, p2, q2);
        two_sum(p1, -p2, hs, he);
        const float hl0 = __fadd_rn(__fadd_rn(he, __fsub_rn(q1, q2)),
                                    __fsub_rn(__fmaf_rn(fxh, e1.w, fxl * e1.z),
                                              __fmaf_rn(fyh, e1.y, fyl * e1.x)));
        float hh, hl;
        two_sum(hs, hl0, hh, hl);
        const bool neg = hh < 0.0f;
        if (neg) {
            hh = -hh;
            hl = -hl;
        }
        float dh, de, dl;
        two_sum(rh, -hh, dh, de);
        dl = __fadd_rn(de, __fsub_rn(rl, hl));
        two_sum(dh, dl, dh, dl);
        if (dh < -band) continue;   // the line misses the circle
        if (dh <= band) return false;  // nearly tangent
        // t = sqrt(v) and 1 / t from the hardware reciprocal square root (within 2^-21 of
        // 1 / t: the bounds below scale it by 1 + 1e-6)
        const float v = dh * (rh + hh);
        const float yt = rsqrtf(v);
        const float t0 = v * yt;
        const float t = __fmaf_rn(__fmaf_rn(-t0, t0, v), 0.5f * yt, t0);
        const float inv_t = yt * 1.000001f;
        const float u0 = -__fmaf_rn(fxh, e1.x, fyh * e1.z);
        const float4 e2 = E[2];
        const float len = e2.z;
        const float eang = kArcErrF32 + 2.0f * eh * inv_t;
        const float uerr = 2.5e-7f * (fabsf(fxh) + fabsf(fyh)) + 1.5e-7f * t + 6.0e-8f * len +
                           2.0f * eh * (rh * inv_t + 1.0f);
        bool have_psi = false;
        float ph = 0.0f, pl = 0.0f, bh = 0.0f, bl = 0.0f;
        for (int q = -1; q <= 1; q += 2) {
            const float u = fmaf((float)q, t, u0);
            if (fabsf(u) <= uerr || fabsf(u - len) <= uerr) return false;  // at a vertex
            if (u < 0.0f || u >= len) continue;
            if (!have_psi) {
                arc_half_angle_pair(dh, dl, rh, rl, inv_r, ph, pl);
                float be;
                if (neg) {
                    two_sum(e2.x, kPiH, bh, be);
                    bl = __fadd_rn(be, __fadd_rn(e2.y, kPiL));
                } else {
                    bh = e2.x;
                    bl = e2.y;
                }
                have_psi = true;
            }
            // theta = phi_m + q sgn psi, sgn = -1 when h < 0
            const bool plus = (q > 0) != neg;
            float th, te;
            two_sum(bh, plus ? ph : -ph, th, te);
            float tl = __fadd_rn(te, __fadd_rn(bl, plus ? pl : -pl));
            two_sum(th, tl, th, tl);
            // into [0, 2 pi), comparing the whole pair (a hi part equal to 2 pi's may carry
            // a negative low part)
            if (th < 0.0f || (th == 0.0f && tl < 0.0f)) {
                two_sum(th, k2PiH, th, te);
                tl = __fadd_rn(te, __fadd_rn(tl, k2PiL));
                two_sum(th, tl, th, tl);
            } else if (th > k2PiH || (th == k2PiH && tl >= k2PiL)) {
                two_sum(th, -k2PiH, th, te);
                tl = __fadd_rn(te, __fsub_rn(tl, k2PiL));
                two_sum(th, tl, th, tl);
            }
            const bool enter = (q > 0) == (pc.pccw != 0);
            float sh, se;
            two_sum(Sh, enter ? th : -th, sh, se);
            Sl = __fadd_rn(Sl, __fadd_rn(se, enter ? tl : -tl));
            Sh = sh;
            bal += enter ? 1 : -1;
            ++na;
            esum += eang;
            emax = fmaxf(emax, eang);
            if (th < a1h || (th == a1h && tl < a1l)) {
                a2h = a1h;
                a2l = a1l;
                a1h = th;
                a1l = tl;
                a1e = eang;
                a1in = enter;
            } else if (th < a2h || (th == a2h && tl < a2l)) {
                a2h = th;
                a2l = tl;
            }
            if (th > zh || (th == zh && tl > zl)) {
                zh = th;
                zl = tl;
            }
        }
    }
    if (na == 0) {  // the centre is inside and no crossing
        if (!(2.0f * rh * (1.0f + 1e-6f) < pc.poly_span)) return false;
        inside = 1.0f;
        outside = 0.0f;
        return true;
    }
    if (bal != 0) return false;
    // I0's choice: the least angle clear of 0, of the second least and (largest) of 2 pi
    if (!(__fadd_rn(a1h, a1l) > a1e * 1.0001f)) return false;
    if (!(__fadd_rn(__fsub_rn(a2h, a1h), __fsub_rn(a2l, a1l)) > (a1e + emax) * 1.0001f))
        return false;
    if (!(__fadd_rn(__fsub_rn(k2PiH, zh), __fsub_rn(k2PiL, zl)) > emax * 1.0001f)) return false;
    // inside measure 2 pi I0 - S and outside measure 2 pi (1 - I0) + S, each times 1 / (2 pi)
    const float kInvH = 0.15915493667125702f, kInvL = 6.4206382432985265e-09f;
    const bool i0 = !a1in;
    float ih, ie, oh, oe;
    two_sum(i0 ? k2PiH : 0.0f, -Sh, ih, ie);
    const float il = __fadd_rn(ie, __fsub_rn(i0 ? k2PiL : 0.0f, Sl));
    two_sum(i0 ? 0.0f : k2PiH, Sh, oh, oe);
    const float ol = __fadd_rn(oe, __fadd_rn(i0 ? 0.0f : k2PiL, Sl));
    float vh, ve;
    two_prod(ih, kInvH, vh, ve);
    inside = __fadd_rn(vh, __fadd_rn(ve, __fmaf_rn(ih, kInvL, il * kInvH)));
    two_prod(oh, kInvH, vh, ve);
    outside = __fadd_rn(vh, __fadd_rn(ve, __fmaf_rn(oh, kInvL, ol * kInvH)));
    return inside > 0.0f && esum * kInvH <= 8.5e-7f * inside;
}

// Phase C in a polygon study area: the weight of each of `cnt` (<= 32) queued orders.  The
// inside share comes from poly_share_f32 when the job allows it (pc.poly_f32): the pair's
// radius and the centre's box-frame position as pairs of FP32 numbers (the records' hi and
// low parts; y from the centre's cell row cy_u = the unit's row, or the neighbour's), else, or
// when it refuses, from the crossings' directions with FP64 crossing points
// (poly_weight_fast).  FP32-tier weights above 8 (beyond the shared accumulators' bound) are
// added to the realization's global sums (exlo, exhi); what neither tier decides, and FP64
// weights above 8, go to the FP64 queue.  Out of line like the rectangle's version, so
// that the rectangle path does not carry its registers.
__device__ __noinline__ void drain_weights_poly(const PairConsts* pcs, const PairConsts* gpc,
                                                WarpSm* wsp, const float4* __restrict__ Ek,
                                                const float* __restrict__ NXk,
                                                const float* __restrict__ NYk,
                                                const float2* __restrict__ Plok, RealBatch rb,
                                                ExactQueue xq, int off, int cnt, int lane,
                                                unsigned long long* he, uint32_t* hc,
                                                uint32_t real, uint32_t c_begin, int cy_u,
                                                unsigned long long* exlo,
                                                unsigned long long* exhi) {
    const PairConsts& pc = *pcs;
    WarpSm& ws = *wsp;
    (void)Ek;
    bool exact = false;
    uint4 xe = make_uint4(0u, 0u, 0u, 0u);
    if (lane < cnt) {
        const uint2 e = ws.q2[off + lane];
        const uint32_t meta = e.x, j = e.y;
        const int cl = (int)(meta & 31u);
        const uint32_t ci = c_begin + (uint32_t)cl;
        const int dcy = (int)((meta >> 8) & 7u) - pc.g.fs;  // centre i's row - j's row
        const bool other = (meta >> 11) & 1u;
        const bool vhalf = (meta >> 12) & 1u;
        const int bin = (int)(meta >> 13);
        const uint32_t a = other ? j : ci, b = other ? ci : j;  // centre, neighbour
        const float nxj = NXk[j], nyj = NYk[j];
        const float2 lo = Plok[j];
        const float4 ca = ws.cen_a[cl];
        const float4 cb = ws.cen_b[cl];
        float in = 0.0f, out = 0.0f;
        bool done = false;
        if (pc.poly_f32) {
            // offset i - j: hi parts exact (x in the box frame, y with i moved into j's row),
            // low parts rounded once; r^2 and r as pairs
            const float dxh = ca.x + nxj, dxl = cb.x - lo.x;
            const float dyh = fmaf((float)dcy, pc.g.chq, ca.y) + nyj;
            const float dyl = fmaf((float)dcy, pc.g.chl, cb.y - lo.y);
            float p1, e1, p2, e2, s, es;
            two_prod(dxh, dxh, p1, e1);
            two_prod(dyh, dyh, p2, e2);
            two_sum(p1, p2, s, es);
            const float r2l = __fadd_rn(__fadd_rn(es, __fadd_rn(e1, e2)),
                                        __fmaf_rn(2.0f * dxh, dxl,
                                                  __fmaf_rn(2.0f * dyh, dyl,
                                                            dxl * dxl + dyl * dyl)));
            const float ys = rsqrtf(s);
            float rh = s * ys;
            rh = __fmaf_rn(__fmaf_rn(-rh, rh, s), 0.5f * ys, rh);
            const float rl = __fadd_rn(__fmaf_rn(-rh, rh, s), r2l) * (0.5f * ys);
            const float inv_r = ys * __fmaf_rn(-0.5f * s * ys, ys, 1.5f);  // Newton step
            // the centre's box-frame position: x hi + low; y = its row's origin
            // row (chq + chl) plus its offset in the cell
            const int row = other ? cy_u - dcy : cy_u;
            const float cxh = other ? -nxj : ca.x, cxl = other ? lo.x : cb.x;
            const float cyr = other ? -nyj : ca.y, cyrl = other ? lo.y : cb.y;
            float ro, roe, cyh, cye;
            two_prod((float)row, pc.g.chq, ro, roe);
            two_sum(ro, cyr, cyh, cye);
            const float cyl = __fadd_rn(__fadd_rn(cye, roe),
                                        __fmaf_rn((float)row, pc.g.chl, cyrl));
            if (rh > 0.0f && poly_share_f32(pc, cxh, cxl, cyh, cyl, rh, rl, inv_r, in, out)) {
                done = true;
                // weight 1 / (inside v) - 1: outside / inside, or (1 + outside) / inside when
                // the temporal weight is 1/2 (correctly rounded division)
                const float xs = __fdiv_rn(vhalf ? 1.0f + out : out, in);
                if (xs <= 7.0f) {
                    const unsigned long long exc =
                        xs > 0.0f ? __float2ull_rn(xs * 4294967296.0f) : 0ull;
                    if (exc) atomicAdd(&he[bin], exc);
                } else if (xs < 1048576.0f) {
                    // above the shared accumulators' bound: straight to the realization's
                    // global sums (the same fixed point, split into its 32-bit halves)
                    const unsigned long long exc = __float2ull_rn(xs * 4294967296.0f);
                    const int64_t o = (int64_t)real * pc.nbins + bin;
                    atomicAdd(&exlo[o], exc & 0xffffffffull);
                    atomicAdd(&exhi[o], exc >> 32);
                } else {
                    exact = true;
                }
            }
        }
        if (!done) {
            const int64_t base = (int64_t)real * rb.n;
            const double xa = rb.X[base + a], ya = rb.Y[base + a];
            const double dx = __dsub_rn(xa, rb.X[base + b]), dy = __dsub_rn(ya, rb.Y[base + b]);
            const double r64 = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
            int ne;
            const uint8_t* list = poly_edges_of(pc, xa, ya, r64, ne);
            const double in64 = poly_weight_fast<false>(xa, ya, r64, poly_of(pc), pc.pebox,
                                                        pc.pccw, list, ne);
            if (in64 > 0.0) {
                const double w = 1.0 / (in64 * (vhalf ? 0.5 : 1.0));
                if (w > 8.0) {
                    exact = true;
                } else {
                    const unsigned long long exc = excess_fixed64(w);
                    if (exc) atomicAdd(&he[bin], exc);
                }
            } else {
                exact = true;
            }
        }
        if (exact) xe = make_uint4(a, b, real, 1u | ((uint32_t)bin << 2));
    }
    push_exact<true>(gpc, rb, xq, exact, xe, lane, (1u << lane) - 1u, hc, he);
}

// Phase C: isotropic spatial weight for `cnt` (<= 32) entries of queue 2.  Out of line (it
// runs once per 32 deferred orders) with scalar arguments, so that neither its registers nor
// an address-taken copy of the warp state weigh on the filter loop.
template <int CALLER = 0>
__device__ __noinline__ void drain_weights(const PairConsts* pcs, const PairConsts* gpc,
                                           WarpSm* wsp, const float4* __restrict__ Ek,
                                           const float* __restrict__ NXk,
                                           const float* __restrict__ NYk,
                                           const float2* __restrict__ Plok, RealBatch rb,
                                           ExactQueue xq, int off, int cnt, int lane,
                                           unsigned long long* he, uint32_t* hc,
                                           uint32_t real, uint32_t c_begin) {
    const PairConsts& pc = *pcs;
    WarpSm& ws = *wsp;
    bool exact = false;
    uint4 xe = make_uint4(0u, 0u, 0u, 0u);
    if (lane < cnt) {
        const uint2 e = ws.q2[off + lane];
        const uint32_t meta = e.x, j = e.y;
        const int cl = (int)(meta & 31u);
        const float dcy = (float)((int)((meta >> 8) & 7u) - pc.g.fs);
        const bool other = (meta >> 11) & 1u;  // order (j, i): centre j
        const bool vhalf = (meta >> 12) & 1u;
        const int bin = (int)(meta >> 13);
        // the neighbour's hi parts (the filter's arrays, negated: recently read), low parts and
        // edge record (only order (j, i) uses it), issued together
        const float nxj = NXk[j], nyj = NYk[j];
        const float2 lo = Plok[j];
        const float4 pb = Ek[j];
        const float4 ca = ws.cen_a[cl];
        const float4 cb = ws.cen_b[cl];
        // x: box-frame hi parts (exact difference) plus low parts; y: centre i moved into j's
        // cell frame, hi part exact, the low parts' difference and the cell sides' remainder
        // rounded once.  Both are exact negations of the offset taken the other way round, so
        // the distance does not depend on which point of the pair is the centre.
        const float dxa = (ca.x + nxj) + (cb.x - lo.x);
        const float dya = (fmaf(dcy, pc.g.chq, ca.y) + nyj) + fmaf(dcy, pc.g.chl, cb.y - lo.y);
        float ra, inv_r;
        radius_nr(fmaf(dxa, dxa, dya * dya), ra, inv_r);
        const float ex = other ? pb.x : cb.z, ey = other ? pb.y : cb.w;
        const float e1 = fminf(ex, ey), e2 = fmaxf(ex, ey);
        const float band = fmaf(pc.tan_rel, ra, pc.tan_abs);
        if (!(ra >= pc.r_acc_min) || fabsf(ra - e1) <= band || fabsf(ra - e2) <= band) {
            exact = true;  // nearly tangent to an edge, or too short to resolve
            const uint32_t ci = c_begin + (uint32_t)cl;
            xe = make_uint4(other ? j : ci, other ? ci : j, real, 1u | ((uint32_t)bin << 2));
        } else {
            // weight 1 / ((1 - A) v) - 1 in 2^-32 units: A / (1 - A), or (1 + A) / (1 - A)
            // when the temporal weight is 1/2
            const float A = outside_share(e1, e2, ra, inv_r);
            const float xs = __fdividef(vhalf ? 1.0f + A : A, 1.0f - A);
            const unsigned long long exc = xs > 0.0f ? __float2ull_rn(xs * 4294967296.0f) : 0ull;
            if (exc) atomicAdd(&he[bin], exc);
        }
    }
    push_exact<false, kVarPlain, CALLER>(gpc, rb, xq, exact, xe, lane, (1u << lane) - 1u, hc,
                                         he);
}

// Evaluates queue 2 in batches of 32 while it holds that many, and moves the rest (fewer than
// 32) to its front.
template <bool POLY, int CALLER = 0>
__device__ __forceinline__ void flush_weights(WarpSm& ws, const PairConsts& pc,
                                              const PairConsts* gpc, const RealBatch& rb,
                                              const ExactQueue& xq, int lane, WarpCtx& w) {
    int off = 0;
    __syncwarp();
    while (w.q2n - off >= 32) {
        if (POLY)
            drain_weights_poly(&pc, gpc, &ws, w.Ek, w.NX, w.NY, w.Plok, rb, xq, off, 32, lane,
                               w.he, w.hc, w.real, w.c_begin, w.cy, w.exlo, w.exhi);
        else
            drain_weights<CALLER>(&pc, gpc, &ws, w.Ek, w.NX, w.NY, w.Plok, rb, xq, off, 32,
                          lane, w.he, w.hc, w.real, w.c_begin);
        off += 32;
    }
    const int rest = w.q2n - off;
    uint2 v = make_uint2(0u, 0u);
    if (lane < rest) v = ws.q2[off + lane];
    __syncwarp();
    if (lane < rest) ws.q2[lane] = v;
    __syncwarp();
    w.q2n = rest;
}

// FP32 weight W (< 2^32) in the inhomogeneous fixed point (see Fix96): whole part and the
// fraction in units of 2^-64 (exact: the fraction has 24 significant bits).
__device__ __forceinline__ void add_fix96f(float W, Fix96& f) {
    const float wh = floorf(W);
    const unsigned long long m = __float2ull_rn((W - wh) * 18446744073709551616.0f);
    f.whole += (unsigned long long)wh;
    f.lo += m & 0xffffffffull;
    f.hi += m >> 32;
}

// Phase B for `cnt` (<= 64) ring entries starting at index 0: two per lane, loaded together.
// VAR kVarDir: the directional K / translation correction (EDGE and POLY false); kVarInh: the
// inhomogeneous K (POLY false).  Both take every pair's weights here.
template <bool EVEN, bool EDGE, bool POLY, int VAR, int CALLER = 0>
__device__ __forceinline__ void drain_pairs(const PairConsts& pc, const PairConsts* gpc,
                                            WarpSm& ws, const RealBatch& rb,
                                            const ExactQueue& xq, int cnt, int lane,
                                            uint32_t lt, WarpCtx& w) {
    const bool edge = EDGE && !w.deep;  // uniform
    uint4 e[2];
    e[0] = ws.ring[lane];
    e[1] = ws.ring[32 + lane];
    if (32 + lane >= cnt) e[1] = make_uint4(0u, 0u, 0u, 0u);  // stale slot: keep values sane
    float4 pj[2];
    if (edge) {  // neighbour's edge record (dense array: 16 bytes per point)
        pj[0] = w.Ek[lane < cnt ? e[0].w : 0u];
        pj[1] = w.Ek[32 + lane < cnt ? e[1].w : 0u];
    }
    bool rare = false;
    bool full[2], di[2], dj[2], wi[2], wj[2], vi[2], vj[2], aj[2], ai[2];
    int bin[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const bool has = r * 32 + lane < cnt;
        const float d2 = __uint_as_float(e[r].x), u = __uint_as_float(e[r].y);
        const int cl = (int)(e[r].z & 31u);
        bool am = false;
        int a, b;
        if (EVEN) {
            a = bin_even(d2 * rsqrtf(fmaxf(d2, 1e-30f)) * pc.inv_ds, pc.tol_s, pc.top_s, pc.cs, am);
            b = bin_even(u * pc.inv_dt, pc.tol_t, pc.top_t, pc.ct, am);
        } else {
            const PairConsts& pa = *w.pa;  // tables and bands: shared memory
            a = bin_fp32(d2, pc.inv_hs, pa.tab_s, pa.s_lo, pa.s_hi, pc.cs, am);
            b = bin_fp32(u, pc.inv_ht, pa.tab_t, pa.t_lo, pa.t_hi, pc.ct, am);
        }
        bin[r] = a * pc.ct + b;  // always a valid bin, also for lanes without an entry
        // order (i, j) counts when i is a centre and j a neighbour (role flags), (j, i) the
        // other way round
        const uint32_t fj = w.mk == nullptr ? 3u : (has ? (uint32_t)w.mk[e[r].w] : 0u);
        const bool act_i = w.mk == nullptr || (((w.onA >> cl) & 1u) && (fj & 2u));
        const bool act_j = w.mk == nullptr || ((fj & 1u) && ((w.onB >> cl) & 1u));
        ai[r] = act_i;
        aj[r] = act_j;
        const bool counted = has & !am;
        full[r] = has & am;
        if (VAR == kVarPlain)
            atomicAdd(&w.hc[bin[r]], counted ? (uint32_t)act_i + (uint32_t)act_j : 0u);
        di[r] = dj[r] = wi[r] = wj[r] = false;
        if (edge && VAR == kVarPlain) {
            const float te_i = ws.cen_te[cl], rin_i = ws.cen_a[cl].w;
            const float te_j = pj[r].z, rin_j = pj[r].w;
            const bool vhi = u > te_i + pc.g_v, vhj = u > te_j + pc.g_v;
            const bool vai = (u > te_i - pc.g_v) & !vhi, vaj = (u > te_j - pc.g_v) & !vhj;
            const bool ini = d2 <= rin_i, inj = d2 <= rin_j;
            const bool ci = counted & act_i, cj = counted & act_j;
            const uint32_t half = (uint32_t)(ci & vhi & !vai & ini) + (uint32_t)(cj & vhj & !vaj & inj);
            if (half) atomicAdd(&w.hh[bin[r]], half);
            wi[r] = ci & vai;         // temporal weight undecided: FP64 weight of order (i, j)
            wj[r] = cj & vaj;
            di[r] = ci & !vai & !ini;  // spatial weight needed
            dj[r] = cj & !vaj & !inj;

            vi[r] = vhi;
            vj[r] = vhj;
        }
        rare |= full[r] | wi[r] | wj[r] | di[r] | dj[r];
    }
    if (VAR == kVarInh) {
        // h_i h_j times the weights of both orders, in FP32 (a few ulp); the temporal weight
        // and the interior tests as in the rectangle path, the spatial weight inline as in
        // phase C; anything FP32 cannot decide sends the whole pair to FP64.
        bool xf[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            xf[r] = full[r];
            if (!(r * 32 + lane < cnt) || full[r]) continue;
            const uint32_t meta = e[r].z, j = e[r].w;
            const int cl = (int)(meta & 31u);
            const float d2 = __uint_as_float(e[r].x), u = __uint_as_float(e[r].y);
            const float hh = ws.cen_h[cl] * (float)w.H[j];
            float wgt[2] = {1.0f, 1.0f};
            bool und = false;
            if (edge) {
                const float4 ca = ws.cen_a[cl];
                const float4 cb = ws.cen_b[cl];
                const float te[2] = {ws.cen_te[cl], pj[r].z};
                const float rin[2] = {ca.w, pj[r].w};
                const float ex[2] = {cb.z, pj[r].x}, ey[2] = {cb.w, pj[r].y};
                float ra = -1.0f, inv_r = 0.0f;
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    const bool vh = u > te[o] + pc.g_v;
                    und |= (u > te[o] - pc.g_v) & !vh;
                    float wsp = 1.0f;
                    if (!(d2 <= rin[o])) {
                        if (ra < 0.0f) {  // accurate distance from the hi + lo parts
                            const float dcy = (float)((int)((meta >> 8) & 7u) - pc.g.fs);
                            const float2 lo = w.Plok[j];
                            const float dxa = (ca.x + w.NX[j]) + (cb.x - lo.x);
                            const float dya = (fmaf(dcy, pc.g.chq, ca.y) + w.NY[j]) +
                                              fmaf(dcy, pc.g.chl, cb.y - lo.y);
                            radius_nr(fmaf(dxa, dxa, dya * dya), ra, inv_r);
                        }
                        const float e1 = fminf(ex[o], ey[o]), e2 = fmaxf(ex[o], ey[o]);
                        const float band = fmaf(pc.tan_rel, ra, pc.tan_abs);
                        if (!(ra >= pc.r_acc_min) || fabsf(ra - e1) <= band ||
                            fabsf(ra - e2) <= band) {
                            und = true;
                        } else {
                            wsp = __fdividef(1.0f, 1.0f - outside_share(e1, e2, ra, inv_r));
                        }
                    }
                    wgt[o] = (vh ? 2.0f : 1.0f) * wsp;
                }
            }
            if (und) {
                xf[r] = true;
                continue;
            }
            atomicAdd(&w.hc[bin[r]], (uint32_t)ai[r] + (uint32_t)aj[r]);
            Fix96 f;
            if (ai[r]) add_fix96f(wgt[0] * hh, f);
            if (aj[r]) add_fix96f(wgt[1] * hh, f);
            if (f.lo) atomicAdd(&w.he[bin[r]], f.lo);
            if (f.hi) atomicAdd(&w.hf[bin[r]], f.hi);
            if (f.whole) atomicAdd(&w.hw[bin[r]], f.whole);
        }
        if (__any_sync(0xffffffffu, xf[0] | xf[1])) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const uint32_t ci = w.c_begin + (e[r].z & 31u), j = e[r].w;
                push_exact<false, kVarInh>(
                    gpc, rb, xq, xf[r],
                    make_uint4(ci, j, w.real, ((uint32_t)ai[r] << 1) | ((uint32_t)aj[r] << 2)),
                    lane, lt, w.hc, w.he, w.hf, w.hw);
            }
        }
        return;
    }
    if (VAR == kVarDir) {
        // Sector from the accurate offset (exact hi-part difference plus the low parts, as in
        // phase C); a cross product within its guard of a boundary, or an offset within the
        // guard of the axis at angle 0 / pi, leaves the pair to FP64.  Translation weight in
        // FP32 (a few ulp; no cancellation: W - |dx| >= W / 2, D - u >= D / 2).
        bool xf[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            xf[r] = full[r];
            if (!(r * 32 + lane < cnt) || full[r]) continue;
            const uint32_t meta = e[r].z, j = e[r].w;
            const int cl = (int)(meta & 31u);
            const float dcy = (float)((int)((meta >> 8) & 7u) - pc.g.fs);
            const float4 ca = ws.cen_a[cl];
            const float4 cb = ws.cen_b[cl];
            const float2 loj = w.Plok[j];
            float dx = (ca.x + w.NX[j]) + (cb.x - loj.x);
            float dy = (fmaf(dcy, pc.g.chq, ca.y) + w.NY[j]) + fmaf(dcy, pc.g.chl, cb.y - loj.y);
            int k = 0;
            bool und = false;
            if (pc.nsec > 1) {
                und = fabsf(dy) <= pc.sec_gd;
                if (dy < 0.0f) {
                    dx = -dx;
                    dy = -dy;
                }
                for (int m = 0; m < pc.nsec - 1; ++m) {
                    const float cr = fmaf(pc.sec_bxf[m], dy, -(pc.sec_byf[m] * dx));
                    und |= fabsf(cr) <= pc.sec_g;
                    k += cr > 0.0f ? 1 : 0;
                }
            }
            if (und) {
                xf[r] = true;
                continue;
            }
            const int b3 = k * (pc.cs * pc.ct) + bin[r];
            atomicAdd(&w.hc[b3], (uint32_t)ai[r] + (uint32_t)aj[r]);
            if (pc.edge == STK_EDGE_TRANSLATION) {
                const float u = __uint_as_float(e[r].y);
                const float wt = (pc.twf * __frcp_rn(pc.twf - fabsf(dx))) *
                                 (pc.thf * __frcp_rn(pc.thf - fabsf(dy))) *
                                 (pc.tdf * __frcp_rn(pc.tdf - u));
                const float xs = wt - 1.0f;
                const unsigned long long e1 =
                    xs > 0.0f ? __float2ull_rn(xs * 4294967296.0f) : 0ull;
                const unsigned long long exc = (ai[r] ? e1 : 0ull) + (aj[r] ? e1 : 0ull);
                if (exc) atomicAdd(&w.he[b3], exc);
            }
        }
        if (__any_sync(0xffffffffu, xf[0] | xf[1])) {
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const uint32_t ci = w.c_begin + (e[r].z & 31u), j = e[r].w;
                push_exact<false, kVarDir>(
                    gpc, rb, xq, xf[r],
                    make_uint4(ci, j, w.real, ((uint32_t)ai[r] << 1) | ((uint32_t)aj[r] << 2)),
                    lane, lt, w.hc, w.he);
            }
        }
        return;
    }
    if (!__any_sync(0xffffffffu, rare)) return;
    // FP64 entries: rare enough that one vote usually skips them all
    const bool xflag = full[0] | full[1] | wi[0] | wj[0] | wi[1] | wj[1];
    if (__any_sync(0xffffffffu, xflag)) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const uint32_t ci = w.c_begin + (e[r].z & 31u), j = e[r].w;
            if (edge) {
                push_exact<POLY, kVarPlain, CALLER>(gpc, rb, xq, wi[r],
                           make_uint4(ci, j, w.real, 1u | ((uint32_t)bin[r] << 2)), lane, lt,
                           w.hc, w.he);
                push_exact<POLY, kVarPlain, CALLER>(gpc, rb, xq, wj[r],
                           make_uint4(j, ci, w.real, 1u | ((uint32_t)bin[r] << 2)), lane, lt,
                           w.hc, w.he);
            }
            push_exact<POLY, kVarPlain, CALLER>(gpc, rb, xq, full[r],
                       make_uint4(ci, j, w.real, ((uint32_t)ai[r] << 1) | ((uint32_t)aj[r] << 2)),
                       lane, lt, w.hc, w.he);
        }
    }
    if (edge) {
        // spatial weights: up to four orders per lane join queue 2 in one compaction
        const uint32_t b0 = __ballot_sync(0xffffffffu, di[0]);
        const uint32_t b1 = __ballot_sync(0xffffffffu, dj[0]);
        const uint32_t b2 = __ballot_sync(0xffffffffu, di[1]);
        const uint32_t b3 = __ballot_sync(0xffffffffu, dj[1]);
        if ((b0 | b1 | b2 | b3) != 0u) {
            const int o0 = w.q2n, o1 = o0 + __popc(b0), o2 = o1 + __popc(b1),
                      o3 = o2 + __popc(b2);
            const uint32_t m0 = e[0].z | ((uint32_t)bin[0] << 13);
            const uint32_t m1 = e[1].z | ((uint32_t)bin[1] << 13);
            if (di[0]) ws.q2[o0 + __popc(b0 & lt)] = make_uint2(m0 | ((uint32_t)vi[0] << 12), e[0].w);
            if (dj[0])
                ws.q2[o1 + __popc(b1 & lt)] =
                    make_uint2(m0 | (1u << 11) | ((uint32_t)vj[0] << 12), e[0].w);
            if (di[1]) ws.q2[o2 + __popc(b2 & lt)] = make_uint2(m1 | ((uint32_t)vi[1] << 12), e[1].w);
            if (dj[1])
                ws.q2[o3 + __popc(b3 & lt)] =
                    make_uint2(m1 | (1u << 11) | ((uint32_t)vj[1] << 12), e[1].w);
            w.q2n = o3 + __popc(b3);
            if (w.q2n >= 32) flush_weights<POLY, CALLER>(ws, pc, gpc, rb, xq, lane, w);
        }
    }
}

// Drains the warp's queues completely (end of a work unit: the centre data is replaced next).
template <bool EVEN, bool EDGE, bool POLY, int VAR, int CALLER = 0>
__device__ __forceinline__ void drain_all(const PairConsts& pc, const PairConsts* gpc,
                                          WarpSm& ws, const RealBatch& rb,
                                          const ExactQueue& xq, uint32_t& tail, int lane,
                                          uint32_t lt, WarpCtx& w) {
    while (tail > 0) {
        const int cnt = tail < (uint32_t)kDrain ? (int)tail : kDrain;
        __syncwarp();
        drain_pairs<EVEN, EDGE, POLY, VAR, CALLER>(pc, gpc, ws, rb, xq, cnt, lane, lt, w);
        __syncwarp();
        const uint32_t rest = tail - (uint32_t)cnt;
        for (uint32_t i = lane; i < rest; i += 32) ws.ring[i] = ws.ring[cnt + i];
        tail = rest;
    }
    __syncwarp();
    if (w.q2n > 0) {
        if (POLY)
            drain_weights_poly(&pc, gpc, &ws, w.Ek, w.NX, w.NY, w.Plok, rb, xq, 0, w.q2n, lane,
                               w.he, w.hc, w.real, w.c_begin, w.cy, w.exlo, w.exhi);
        else
            drain_weights<CALLER>(&pc, gpc, &ws, w.Ek, w.NX, w.NY, w.Plok, rb, xq, 0,
                          w.q2n, lane, w.he, w.hc, w.real, w.c_begin);
        w.q2n = 0;
    }
    __syncwarp();
}

// One job's realizations [0, m) in a block of the FP32 pair kernel: pc is the job's constants
// (the kernel parameters themselves in the single-job kernel, so that its scalars are
// constant-bank operands; a shared-memory copy in the fused kernel), the shared Smem32's pc
// holds at least the indexed tables and bands before `s2`.  Adds the job's candidate count to
// acc.stats[0].
// BPS: resident blocks per SM the register allocation is made for (2: 128 registers per
// thread; 3: 85, the launch shape the tuner may choose for the plain rectangle kernels).
template <bool EVEN, bool EDGE, bool POLY, int VAR, int BPS = 2>
__global__ void __launch_bounds__(kBlock, BPS)
pair_fp32_kernel(const __grid_constant__ PairConsts pk, const PairConsts* __restrict__ gpc,
                 int m, RealBatch rb,
                 const WorkItem* __restrict__ units, const uint32_t* __restrict__ unit_off,
                 uint32_t* __restrict__ counters, Accum acc, ExactQueue xq, int reps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem32& sm = *reinterpret_cast<Smem32*>(smem_raw);
    const PairConsts& pc = pk;  // scalars: kernel parameters (constant bank)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const int words = (int)(offsetof(PairConsts, s2) / 4);
        const int* src = reinterpret_cast<const int*>(gpc);
        int* dst = reinterpret_cast<int*>(&sm.pc);
        for (int i = tid; i < words; i += kBlock) dst[i] = src[i];
    }
    __syncthreads();
    constexpr int CALLER = 0;
#include "pair_fp32_body.cuh"
}

// Several jobs (point sets, grids, thresholds) in one persistent launch: the blocks take the
// jobs in order, each job's realizations and units as the single-job kernel does; at a job
// switch every block copies the job's whole constants and its descriptor into shared memory
// (block barriers on both sides), so the body reads them from there.  The jobs share the
// kernel class (even thresholds, edge correction; the plain rectangle estimator).  The
// histogram replicas are laid out for the largest job (nbins_max bins) and cleared once:
// every flush clears what it moves, so each job starts on zeros whatever its bin count.
template <bool EVEN, bool EDGE>
__global__ void __launch_bounds__(kBlock, 2)
pair_fp32_fused_kernel(const FusedJob* __restrict__ jobs, int njobs, int reps, int nbins_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem32& sm = *reinterpret_cast<Smem32*>(smem_raw);
    __shared__ FusedJob job;  // the current job's descriptor
    {
        const size_t hist_off = (sizeof(Smem32) + 15) & ~size_t(15);
        uint32_t* hist = reinterpret_cast<uint32_t*>(smem_raw + hist_off);
        const int words = 4 * reps * nbins_max;  // he (u64), hc and hh (u32) per replica
        for (int i = threadIdx.x; i < words; i += kBlock) hist[i] = 0u;
    }
    for (int j = 0; j < njobs; ++j) {
        __syncthreads();  // every warp is done with the previous job's constants
        {
            const int words = (int)(sizeof(PairConsts) / 4);
            const int* src = reinterpret_cast<const int*>(jobs[j].pc);
            int* dst = reinterpret_cast<int*>(&sm.pc);
            for (int i = threadIdx.x; i < words; i += kBlock) dst[i] = src[i];
            const int dwords = (int)(sizeof(FusedJob) / 4);
            const int* dsrc = reinterpret_cast<const int*>(&jobs[j]);
            int* ddst = reinterpret_cast<int*>(&job);
            for (int i = threadIdx.x; i < dwords; i += kBlock) ddst[i] = dsrc[i];
        }
        __syncthreads();
        constexpr bool POLY = false;
        constexpr int VAR = kVarPlain;
        constexpr int CALLER = 1;
        const PairConsts& pc = sm.pc;
        const PairConsts* gpc = job.pc;
        const int m = job.m;
        const RealBatch& rb = job.rb;
        const WorkItem* __restrict__ units = job.units;
        const uint32_t* __restrict__ unit_off = job.unit_off;
        uint32_t* __restrict__ counters = job.counters;
        const Accum& acc = job.acc;
        const ExactQueue& xq = job.xq;
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#include "pair_fp32_body.cuh"
    }
}

// ---------------------------------------------------------------- FP64 plain kernel
//
// The comparison path: the same traversal (each unordered pair once) with every pair in FP64
// and the reference rounding; candidates are compacted per warp and evaluated 32 at a time.

struct WarpSm64 {
    double cx[32], cy[32], ct[32];
    double ch[32];       // inhomogeneous K: h of the centres
    uint2 ring[kRing];   // (lane, neighbour)
};

struct Smem64 {
    PairConsts pc;
    WarpSm64 w[kWarps];
};

// Bins and weights of `cnt` (<= 32) queued pairs, one per lane, with the reference rounding.
template <bool POLY, bool INH, bool DIR>
__device__ __forceinline__ void process64(const PairConsts& pc, const WarpSm64& ws, int cnt,
                                          int lane, const double* X, const double* Y,
                                          const double* T, const double* H, const uint8_t* mk,
                                          uint32_t onA, uint32_t onB,
                                          uint32_t* hc, unsigned long long* he,
                                          unsigned long long* hf, unsigned long long* hw,
                                          unsigned long long* stats) {
    if (lane >= cnt) return;
    const uint2 e = ws.ring[lane];
    const double xi = ws.cx[e.x], yi = ws.cy[e.x], ti = ws.ct[e.x];
    const double xj = X[e.y], yj = Y[e.y], tj = T[e.y];
    const double dx = __dsub_rn(xi, xj);
    const double dy = __dsub_rn(yi, yj);
    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    const double u = fabs(__dsub_rn(ti, tj));
    if (!(d2 <= pc.s2[pc.cs - 1] && u <= pc.tt[pc.ct - 1])) {
        atomicAdd(&stats[2], 1ull);  // cannot happen: the filter used the same arithmetic
        return;
    }
    int ks = (int)(d2 * pc.inv_hs2_64);
    ks = ks < kTab - 1 ? ks : kTab - 1;
    int a = pc.tab_s64[ks];
    while (a < pc.cs - 1 && d2 > pc.s2[a]) ++a;
    int kt = (int)(u * pc.inv_ht_64);
    kt = kt < kTab - 1 ? kt : kTab - 1;
    int b = pc.tab_t64[kt];
    while (b < pc.ct - 1 && u > pc.tt[b]) ++b;
    const uint32_t fj = mk == nullptr ? 3u : (uint32_t)mk[e.y];
    const bool act_i = mk == nullptr || (((onA >> e.x) & 1u) && (fj & 2u));
    const bool act_j = mk == nullptr || ((fj & 1u) && ((onB >> e.x) & 1u));
    if (DIR) {  // directional / translation-corrected K: one weight for both orders
        const int bin = (sector_of(pc, dx, dy) * pc.cs + a) * pc.ct + b;
        const unsigned long long e =
            pc.edge == STK_EDGE_TRANSLATION ? excess_fixed64(translation_weight(pc, dx, dy, u))
                                            : 0ull;
        atomicAdd(&hc[bin], (uint32_t)act_i + (uint32_t)act_j);
        const unsigned long long exc = (act_i ? e : 0ull) + (act_j ? e : 0ull);
        if (exc) atomicAdd(&he[bin], exc);
        return;
    }
    const int bin = a * pc.ct + b;
    if (INH) {
        // Section 7 inhomogeneous variant: each order weighted by h_i h_j / (w v)
        const double hh = __dmul_rn(ws.ch[e.x], H[e.y]);
        double wi = 1.0, wj = 1.0;
        if (pc.edge) {
            const double r = __dsqrt_rn(d2);
            wi = 1.0 / (omega64<POLY>(pc, xi, yi, r) * v64(pc, ti, u));
            wj = 1.0 / (omega64<POLY>(pc, xj, yj, r) * v64(pc, tj, u));
        }
        Fix96 f;
        if (act_i) add_fix96(__dmul_rn(wi, hh), f);
        if (act_j) add_fix96(__dmul_rn(wj, hh), f);
        atomicAdd(&hc[bin], (uint32_t)act_i + (uint32_t)act_j);
        if (f.lo) atomicAdd(&he[bin], f.lo);
        if (f.hi) atomicAdd(&hf[bin], f.hi);
        if (f.whole) atomicAdd(&hw[bin], f.whole);
        return;
    }
    unsigned long long exc = 0;
    if (pc.edge) {
        const double r = __dsqrt_rn(d2);
        if (act_i) exc += excess_fixed64(1.0 / (omega64<POLY>(pc, xi, yi, r) * v64(pc, ti, u)));
        if (act_j) exc += excess_fixed64(1.0 / (omega64<POLY>(pc, xj, yj, r) * v64(pc, tj, u)));
    }
    atomicAdd(&hc[bin], (uint32_t)act_i + (uint32_t)act_j);
    if (exc) atomicAdd(&he[bin], exc);
}

template <bool POLY, bool INH, bool DIR>
__global__ void __launch_bounds__(kBlock, 2)
pair_fp64_kernel(const PairConsts* __restrict__ gpc, int m, RealBatch rb,
                 const WorkItem* __restrict__ units, const uint32_t* __restrict__ unit_off,
                 uint32_t* __restrict__ counters, Accum acc, int reps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem64& sm = *reinterpret_cast<Smem64*>(smem_raw);
    const PairConsts& pc = sm.pc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const int words = (int)(sizeof(PairConsts) / 4);
        const int* src = reinterpret_cast<const int*>(gpc);
        int* dst = reinterpret_cast<int*>(&sm.pc);
        for (int i = tid; i < words; i += kBlock) dst[i] = src[i];
    }
    __syncthreads();
    WarpSm64& ws = sm.w[warp];
    const int nbins = pc.nbins;
    const size_t hist_off = (sizeof(Smem64) + 15) & ~size_t(15);
    // per replica: he [nbins] u64 (excess; inhomogeneous: fraction low halves), then for the
    // inhomogeneous K hf (fraction high halves) and hw (whole parts), then hc [nbins] u32
    unsigned long long* he = reinterpret_cast<unsigned long long*>(smem_raw + hist_off);
    unsigned long long* hf = he + (size_t)reps * nbins;
    unsigned long long* hw = hf + (size_t)reps * nbins;
    uint32_t* hc = reinterpret_cast<uint32_t*>(INH ? hw + (size_t)reps * nbins : hf);
    for (int i = tid; i < reps * nbins; i += kBlock) {
        hc[i] = 0;
        he[i] = 0;
        if (INH) {
            hf[i] = 0;
            hw[i] = 0;
        }
    }
    uint32_t* my_hc = hc + (warp % reps) * nbins;
    unsigned long long* my_he = he + (warp % reps) * nbins;
    unsigned long long* my_hf = hf + (warp % reps) * nbins;
    unsigned long long* my_hw = hw + (warp % reps) * nbins;
    const int64_t n = rb.n;
    const int nx = pc.g.nx, ny = pc.g.ny, nt = pc.g.nt, fs = pc.g.fs, ft = pc.g.ft;
    const int64_t nrows = (int64_t)ny * nt;
    const uint32_t lt = (1u << lane) - 1u;
    const double s2max = pc.s2[pc.cs - 1], tmax = pc.tt[pc.ct - 1];
    unsigned long long n_cand = 0;
    uint64_t since_flush = 0;
    __syncthreads();

    for (int k = 0; k < m; ++k) {
        uint32_t ubeg = unit_off[(int64_t)k * nrows], uend = unit_off[(int64_t)(k + 1) * nrows];
        shard_units(rb, unit_off, nrows, k, &ubeg, &uend);
        const int64_t base = (int64_t)k * n;
        const uint32_t* cs = rb.cell_start + (int64_t)k * (rb.ncells + 1);
        const double* X = rb.X + base;
        const double* Y = rb.Y + base;
        const double* T = rb.T + base;
        const double* H = INH ? rb.H + base : nullptr;
        const uint8_t* mk = (rb.mask != nullptr && (rb.mask_all || k == 0))
                                ? rb.mask + (rb.mask_all ? (int64_t)k * rb.n : 0)
                                : nullptr;
        for (;;) {
            uint32_t u = 0;
            if (lane == 0) u = atomicAdd(&counters[k], 1u);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (ubeg + u >= uend) break;
            const WorkItem wi = units[ubeg + u];
            const int cy = (int)(wi.row % (uint32_t)ny), ct = (int)(wi.row / (uint32_t)ny);
            const bool valid = lane < (int)wi.c_count;
            const uint32_t ci = wi.c_begin + (valid ? lane : 0);
            const double xi = X[ci], yi = Y[ci], ti = T[ci];
            ws.cx[lane] = xi;
            ws.cy[lane] = yi;
            ws.ct[lane] = ti;
            if (INH) ws.ch[lane] = H[ci];
            const int cx = __float_as_int(rb.P[2 * base + ci].w);
            const uint32_t fl = mk == nullptr ? 3u : (uint32_t)mk[ci];
            const uint32_t onA = __ballot_sync(0xffffffffu, valid && (fl & 1u));
            const uint32_t onB = __ballot_sync(0xffffffffu, valid && (fl & 2u));
            const int cxa = __reduce_min_sync(0xffffffffu, valid ? cx : 0x7fffffff);
            const int cxb = __reduce_max_sync(0xffffffffu, valid ? cx : -1);
            const int wb = min(nx - 1, cxb + fs);
            __syncwarp();
            uint32_t tail = 0;
            for (int dt = 0; dt <= ft; ++dt) {
                const int rt = ct + dt;
                if (rt >= nt) break;
                for (int dy = (dt == 0 ? 0 : -fs); dy <= fs; ++dy) {
                    const int ry = cy + dy;
                    if (ry < 0 || ry >= ny) continue;
                    const bool own = (dt == 0) & (dy == 0);
                    const int jlo = own ? (int)ci : -1;
                    const int wa = own ? cxa : max(0, cxa - fs);
                    const int64_t rowkey = ((int64_t)rt * ny + ry) * nx;
                    const uint32_t j0 = cs[rowkey + wa], j1 = cs[rowkey + wb + 1];
                    if (valid) n_cand += j1 - j0;
                    since_flush += 32ull * (j1 - j0);
                    for (uint32_t j = j0; j < j1; ++j) {
                        const double dx = __dsub_rn(xi, X[j]);
                        const double dy2 = __dsub_rn(yi, Y[j]);
                        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy2, dy2));
                        const double uu = fabs(__dsub_rn(ti, T[j]));
                        const bool q = valid && (int)j > jlo && d2 <= s2max && uu <= tmax;
                        const uint32_t mq = __ballot_sync(0xffffffffu, q);
                        if (q) ws.ring[tail + __popc(mq & lt)] = make_uint2((uint32_t)lane, j);
                        tail += __popc(mq);
                        if (tail >= 32u) {
                            __syncwarp();
                            process64<POLY, INH, DIR>(pc, ws, 32, lane, X, Y, T, H, mk, onA, onB,
                                                 my_hc, my_he, my_hf, my_hw, acc.stats);
                            __syncwarp();
                            if ((uint32_t)lane < tail - 32) ws.ring[lane] = ws.ring[32 + lane];
                            __syncwarp();
                            tail -= 32;
                        }
                    }
                }
            }
            __syncwarp();
            if (tail > 0)
                process64<POLY, INH, DIR>(pc, ws, (int)tail, lane, X, Y, T, H, mk, onA, onB, my_hc,
                                     my_he, my_hf, my_hw, acc.stats);
            __syncwarp();
            if (since_flush >= kWarpFlush) {
                if (INH)
                    warp_flush_inh(k, nbins, my_hc, my_he, my_hf, my_hw, acc, lane);
                else
                    warp_flush(k, nbins, my_hc, nullptr, my_he, acc, lane);
                since_flush = 0;
            }
        }
        if (INH)
            flush_hist_inh(k, nbins, reps, hc, he, hf, hw, acc);
        else
            flush_hist(k, nbins, reps, hc, he, acc);
        since_flush = 0;
    }
    for (int o = 16; o > 0; o >>= 1) n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
    if (lane == 0) atomicAdd(&acc.stats[0], n_cand);
}

// ---------------------------------------------------------------- FP64 queue kernel

// Evaluates the pairs the FP32 kernel queued, 32 per warp, and adds them to the global
// accumulators (integer atomics, so the order does not matter).
template <bool POLY, int VAR>
__global__ void __launch_bounds__(256)
exact_kernel(const PairConsts* __restrict__ gpc, RealBatch rb, Accum acc, ExactQueue xq) {
    const unsigned int pushed = *xq.count;
    const unsigned int total = min(pushed, xq.cap);
    const PairConsts& pc = *gpc;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&acc.stats[1], (unsigned long long)pushed);
    for (unsigned int i = blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += gridDim.x * blockDim.x) {
        const uint4 q = xq.e[i];
        int bin;
        uint32_t counts;
        unsigned long long exc;
        Fix96 f;
        if (!exact_eval<POLY, VAR>(pc, rb, q, bin, counts, exc, &f)) continue;
        const int64_t o = (int64_t)q.z * pc.nbins + bin;
        if (counts) atomicAdd(&acc.cnt[o], (unsigned long long)counts);
        if (exc & 0xffffffffull) atomicAdd(&acc.exc_lo[o], exc & 0xffffffffull);
        if (exc >> 32) atomicAdd(&acc.exc_hi[o], exc >> 32);
        if (VAR == kVarInh) add_fix96_global(acc, o, f.whole, f.lo, f.hi);
    }
}

// ---------------------------------------------------------------- finalize / envelope

// One block per realization: integer histogram -> cumulative grids (exact, in 128-bit fixed
// point) -> S, K (Eq. 2 normalisation) and L (Eq. 4).
__global__ void finalize_kernel(int cs, int ct, const double* __restrict__ s,
                                const double* __restrict__ tt, double coef,
                                const int64_t* __restrict__ self_pairs, Accum acc,
                                double* __restrict__ K, double* __restrict__ L,
                                double* __restrict__ S, int64_t* __restrict__ C, double lfac) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int nb = cs * ct;
    unsigned long long* cc = reinterpret_cast<unsigned long long*>(fsm);
    unsigned __int128* ee = reinterpret_cast<unsigned __int128*>(cc + ((nb + 1) & ~1));
    const int k = blockIdx.x;
    const int64_t o = (int64_t)k * nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        cc[i] = acc.cnt[o + i];
        ee[i] = ((unsigned __int128)acc.exc_hi[o + i] << 32) + (unsigned __int128)acc.exc_lo[o + i];
        if (acc.whole) ee[i] += (unsigned __int128)acc.whole[o + i] << 64;
    }
    __syncthreads();
    if (threadIdx.x == 0) cc[0] -= (unsigned long long)self_pairs[k];  // (i, i) lands in bin (0, 0)
    __syncthreads();
    for (int a = threadIdx.x; a < cs; a += blockDim.x) {  // prefix along t
        for (int b = 1; b < ct; ++b) {
            cc[a * ct + b] += cc[a * ct + b - 1];
            ee[a * ct + b] += ee[a * ct + b - 1];
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < ct; b += blockDim.x) {  // prefix along s
        for (int a = 1; a < cs; ++a) {
            cc[a * ct + b] += cc[(a - 1) * ct + b];
            ee[a * ct + b] += ee[(a - 1) * ct + b];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const int a = i / ct, b = i - (i / ct) * ct;
        const unsigned __int128 e = ee[i];
        double sv;
        if (acc.whole) {  // inhomogeneous K: the weights themselves, in units of 2^-64
            sv = (double)(unsigned long long)(e >> 64) +
                 (double)(unsigned long long)e * (1.0 / 18446744073709551616.0);
        } else {
            const double ed = (double)(unsigned long long)(e >> 64) * 18446744073709551616.0 +
                              (double)(unsigned long long)e;
            sv = (double)cc[i] + ed * (1.0 / 4294967296.0);
        }
        const double kv = coef * sv;
        if (K) K[o + i] = kv;
        if (L) L[o + i] = sqrt(lfac * kv / (2.0 * 3.141592653589793 * tt[b])) - s[a];
        if (S) S[o + i] = sv;
        if (C) C[o + i] = (int64_t)cc[i];
    }
}

__global__ void envelope_kernel(int m, int nbins, int cs, int ct, const double* __restrict__ K,
                                const double* __restrict__ s, const double* __restrict__ tt,
                                double* __restrict__ K_lo, double* __restrict__ K_hi,
                                double* __restrict__ L_lo, double* __restrict__ L_hi,
                                double lfac) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbins) return;
    double lo = K[i], hi = K[i];
    for (int k = 1; k < m; ++k) {
        const double v = K[(int64_t)k * nbins + i];
        lo = fmin(lo, v);
        hi = fmax(hi, v);
    }
    const int a = (i / ct) % cs, b = i - (i / ct) * ct;
    const double den = 2.0 * 3.141592653589793 * tt[b] / lfac;
    K_lo[i] = lo;
    K_hi[i] = hi;
    L_lo[i] = sqrt(lo / den) - s[a];
    L_hi[i] = sqrt(hi / den) - s[a];
}

size_t hist_bytes(int nbins, int reps) { return (size_t)reps * nbins * 16; }

size_t smem_with_reps(size_t base, int nbins, int* reps, size_t budget) {
    const size_t b = (base + 15) & ~size_t(15);
    int r = 8;
    while (r > 1 && b + hist_bytes(nbins, r) > budget) --r;
    *reps = r;
    return b + hist_bytes(nbins, r);
}

}  // namespace

size_t pair_fp32_poly_extra(int nbins, int reps) { return hist_bytes(nbins, reps); }

size_t pair_fp32_smem(int nbins, int* reps, bool inh) {
    if (inh) {  // three u64 sums and a u32 count per bin and replica
        const size_t b = (sizeof(Smem32) + 15) & ~size_t(15);
        int r = 8;
        while (r > 1 && b + (size_t)r * nbins * 32 > 56 * 1024) --r;
        *reps = r;
        return b + (size_t)r * nbins * 32;
    }
    return smem_with_reps(sizeof(Smem32), nbins, reps, 56 * 1024);
}
size_t pair_fp64_smem(int nbins, int* reps, bool inh) {
    if (inh) {  // three u64 sums and a u32 count per bin and replica
        const size_t b = (sizeof(Smem64) + 15) & ~size_t(15);
        int r = 8;
        while (r > 1 && b + (size_t)r * nbins * 32 > 72 * 1024) --r;
        *reps = r;
        return b + (size_t)r * nbins * 32;
    }
    return smem_with_reps(sizeof(Smem64), nbins, reps, 72 * 1024);
}

// Largest dynamic shared memory a pair kernel can ask for (any threshold grid).
size_t smem_cap(size_t base) {
    const size_t one = ((base + 15) & ~size_t(15)) + hist_bytes(kMaxThr * kMaxThr, 1);
    return std::max<size_t>(72 * 1024, one);
}

// The attributes are process-wide and jobs on other threads may launch at any time, so they
// are set to one fixed cap that covers every grid, never lowered.
cudaError_t pair_kernels_configure(size_t smem32, size_t smem64) {
    smem32 = std::max(smem32, smem_cap(sizeof(Smem32)));
    smem64 = std::max(smem64, smem_cap(sizeof(Smem64)));
    cudaError_t e = cudaFuncSetAttribute(finalize_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kMaxThr * kMaxThr * 24 + 16));
    if (e != cudaSuccess) return e;
    const void* k32[16] = {(const void*)pair_fp32_kernel<false, false, false, kVarPlain>,
                          (const void*)pair_fp32_kernel<false, true, false, kVarPlain>,
                          (const void*)pair_fp32_kernel<true, false, false, kVarPlain>,
                          (const void*)pair_fp32_kernel<true, true, false, kVarPlain>,
                          (const void*)pair_fp32_kernel<false, true, true, kVarPlain>,
                          (const void*)pair_fp32_kernel<true, true, true, kVarPlain>,
                          (const void*)pair_fp32_kernel<false, false, false, kVarDir>,
                          (const void*)pair_fp32_kernel<true, false, false, kVarDir>,
                          (const void*)pair_fp32_kernel<false, false, false, kVarPlain, 3>,
                          (const void*)pair_fp32_kernel<false, true, false, kVarPlain, 3>,
                          (const void*)pair_fp32_kernel<true, false, false, kVarPlain, 3>,
                          (const void*)pair_fp32_kernel<true, true, false, kVarPlain, 3>,
                          (const void*)pair_fp32_fused_kernel<false, false>,
                          (const void*)pair_fp32_fused_kernel<false, true>,
                          (const void*)pair_fp32_fused_kernel<true, false>,
                          (const void*)pair_fp32_fused_kernel<true, true>};
    for (const void* f : k32) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32);
        if (e != cudaSuccess) return e;
    }
    // inhomogeneous K: 32 bytes per bin and replica
    const size_t smem32_inh = std::max<size_t>(
        smem32, ((sizeof(Smem32) + 15) & ~size_t(15)) + (size_t)kMaxThr * kMaxThr * 32);
    // polygon study areas: two histogram sets (pair_fp32_poly_extra), within the same cap
    for (const void* f : {(const void*)pair_fp32_kernel<false, true, true, kVarPlain>,
                          (const void*)pair_fp32_kernel<true, true, true, kVarPlain>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem32_inh);
        if (e != cudaSuccess) return e;
    }
    const void* k32i[4] = {(const void*)pair_fp32_kernel<false, false, false, kVarInh>,
                           (const void*)pair_fp32_kernel<false, true, false, kVarInh>,
                           (const void*)pair_fp32_kernel<true, false, false, kVarInh>,
                           (const void*)pair_fp32_kernel<true, true, false, kVarInh>};
    for (const void* f : k32i) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem32_inh);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(pair_fp64_kernel<true, false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(pair_fp64_kernel<false, false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(pair_fp64_kernel<false, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
    if (e != cudaSuccess) return e;
    const size_t smem_inh = std::max<size_t>(
        72 * 1024, ((sizeof(Smem64) + 15) & ~size_t(15)) + (size_t)kMaxThr * kMaxThr * 32);
    return cudaFuncSetAttribute(pair_fp64_kernel<false, true, false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_inh);
}

int pair_fp32_blocks_per_sm(size_t smem, int bps) {
    int b = 0;
    const cudaError_t e =
        bps == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                       &b, pair_fp32_kernel<true, true, false, kVarPlain, 3>, kBlock, smem)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                       &b, pair_fp32_kernel<true, true, false, kVarPlain>, kBlock, smem);
    if (e != cudaSuccess) return 1;
    return b > 0 ? b : 1;
}

int pair_fp32_fused_blocks_per_sm(size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pair_fp32_fused_kernel<true, true>,
                                                      kBlock, smem) != cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

cudaError_t launch_pair_fp32_fused(bool even, bool edge, size_t smem, int reps, int nbins_max,
                                   int grid, const FusedJob* d_jobs, int njobs, cudaStream_t st) {
    if (njobs < 1 || reps < 1 || nbins_max < 1) return cudaErrorInvalidValue;
    if (even && edge)
        pair_fp32_fused_kernel<true, true><<<grid, kBlock, smem, st>>>(d_jobs, njobs, reps,
                                                                      nbins_max);
    else if (even)
        pair_fp32_fused_kernel<true, false><<<grid, kBlock, smem, st>>>(d_jobs, njobs, reps,
                                                                       nbins_max);
    else if (edge)
        pair_fp32_fused_kernel<false, true><<<grid, kBlock, smem, st>>>(d_jobs, njobs, reps,
                                                                       nbins_max);
    else
        pair_fp32_fused_kernel<false, false><<<grid, kBlock, smem, st>>>(d_jobs, njobs, reps,
                                                                        nbins_max);
    return cudaGetLastError();
}

bool pair_fp32_shape_tunable(const PairConsts& hpc, bool inh) {
    const bool dir = hpc.nsec > 1 || hpc.edge == STK_EDGE_TRANSLATION;
    return !(hpc.nv > 0) && !dir && !inh;
}

int pair_fp64_blocks_per_sm(size_t smem, bool inh) {
    int b = 0;
    const cudaError_t e =
        inh ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &b, pair_fp64_kernel<false, true, false>, kBlock, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &b, pair_fp64_kernel<false, false, false>, kBlock, smem);
    if (e != cudaSuccess) return 1;
    return b > 0 ? b : 1;
}

cudaError_t launch_pair_fp32(const PairConsts& hpc, const PairConsts* d_pc, bool even, bool edge,
                             size_t smem, int reps,
                             int grid, int m, RealBatch rb, const WorkItem* units,
                             const uint32_t* unit_off, uint32_t* counters, Accum acc,
                             ExactQueue xq, cudaStream_t st, int bps) {
    if (hpc.tile_units < 1) return cudaErrorInvalidValue;
    const bool poly = edge && hpc.nv > 0;
    // directional K / translation correction and inhomogeneous K: their own instantiations
    const bool dir = hpc.nsec > 1 || hpc.edge == STK_EDGE_TRANSLATION;
    const bool inh = rb.H != nullptr;
#define STK_PAIR32V(E, D, P, V)                                                              \
    pair_fp32_kernel<E, D, P, V><<<grid, kBlock, smem, st>>>(hpc, d_pc, m, rb, units,        \
                                                             unit_off, counters, acc, xq, reps)
#define STK_PAIR32(E, D, P) STK_PAIR32V(E, D, P, kVarPlain)
#define STK_PAIR32S(E, D)                                                                     \
    if (bps == 3)                                                                             \
        pair_fp32_kernel<E, D, false, kVarPlain, 3><<<grid, kBlock, smem, st>>>(               \
            hpc, d_pc, m, rb, units, unit_off, counters, acc, xq, reps);                      \
    else                                                                                      \
        STK_PAIR32(E, D, false)
    if ((dir && (poly || inh)) || (inh && (poly || acc.whole == nullptr)))
        return cudaErrorInvalidValue;
    if (inh && even && edge)
        STK_PAIR32V(true, true, false, kVarInh);
    else if (inh && even)
        STK_PAIR32V(true, false, false, kVarInh);
    else if (inh && edge)
        STK_PAIR32V(false, true, false, kVarInh);
    else if (inh)
        STK_PAIR32V(false, false, false, kVarInh);
    else if (dir && even)
        STK_PAIR32V(true, false, false, kVarDir);
    else if (dir)
        STK_PAIR32V(false, false, false, kVarDir);
    else if (poly && even)
        STK_PAIR32(true, true, true);
    else if (poly)
        STK_PAIR32(false, true, true);
    else if (even && edge)
        STK_PAIR32S(true, true);
    else if (even)
        STK_PAIR32S(true, false);
    else if (edge)
        STK_PAIR32S(false, true);
    else
        STK_PAIR32S(false, false);
#undef STK_PAIR32S
#undef STK_PAIR32
#undef STK_PAIR32V
    return cudaGetLastError();
}

cudaError_t launch_exact(const PairConsts* d_pc, int grid, RealBatch rb, Accum acc,
                         ExactQueue xq, cudaStream_t st, bool poly, bool dir) {
    const bool inh = rb.H != nullptr;
    if ((dir && (poly || inh)) || (inh && (poly || acc.whole == nullptr)))
        return cudaErrorInvalidValue;
    if (inh)
        exact_kernel<false, kVarInh><<<grid, 256, 0, st>>>(d_pc, rb, acc, xq);
    else if (dir)
        exact_kernel<false, kVarDir><<<grid, 256, 0, st>>>(d_pc, rb, acc, xq);
    else if (poly)
        exact_kernel<true, kVarPlain><<<grid, 256, 0, st>>>(d_pc, rb, acc, xq);
    else
        exact_kernel<false, kVarPlain><<<grid, 256, 0, st>>>(d_pc, rb, acc, xq);
    return cudaGetLastError();
}

cudaError_t launch_pair_fp64(const PairConsts* d_pc, size_t smem, int reps, int grid, int m,
                             RealBatch rb, const WorkItem* units, const uint32_t* unit_off,
                             uint32_t* counters, Accum acc, cudaStream_t st, bool poly,
                             bool inh, bool dir) {
    if (inh && (poly || dir || rb.H == nullptr || acc.whole == nullptr))
        return cudaErrorInvalidValue;
    if (dir && poly) return cudaErrorInvalidValue;
#define STK_PAIR64(P, I, D)                                                                     \
    pair_fp64_kernel<P, I, D><<<grid, kBlock, smem, st>>>(d_pc, m, rb, units, unit_off, counters, \
                                                          acc, reps)
    if (inh)
        STK_PAIR64(false, true, false);
    else if (dir)
        STK_PAIR64(false, false, true);
    else if (poly)
        STK_PAIR64(true, false, false);
    else
        STK_PAIR64(false, false, false);
#undef STK_PAIR64
    return cudaGetLastError();
}

cudaError_t launch_finalize(int m, int cs, int ct, const double* s, const double* tt,
                            double coef, const int64_t* self_pairs, Accum acc, double* K,
                            double* L, double* S, int64_t* C, cudaStream_t st, double lfac) {
    const int nb = cs * ct;
    const size_t smem = (size_t)((nb + 1) & ~1) * 8 + (size_t)nb * 16;
    finalize_kernel<<<m, 128, smem, st>>>(cs, ct, s, tt, coef, self_pairs, acc, K, L, S, C,
                                          lfac);
    return cudaGetLastError();
}

cudaError_t launch_envelope(int m, int nbins, int cs, int ct, const double* K, const double* s,
                            const double* tt, double* K_lo, double* K_hi, double* L_lo,
                            double* L_hi, cudaStream_t st, double lfac) {
    envelope_kernel<<<(nbins + 127) / 128, 128, 0, st>>>(m, nbins, cs, ct, K, s, tt, K_lo, K_hi,
                                                         L_lo, L_hi, lfac);
    return cudaGetLastError();
}

}  // namespace stk
