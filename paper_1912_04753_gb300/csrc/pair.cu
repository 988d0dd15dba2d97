// Fused pair kernels: the hot loop of the space-time K estimator (Section 3, Eq. 2 and 3).
//
// Replaces the paper's per-point cylinder range query on an R-tree (Section 4.2) and its
// 2-tier weight cache (Section 4.3): each block takes work items (up to 256 centres of one
// grid cell of one realization), stages the 27-cell neighbourhood through shared memory in
// chunks, evaluates every candidate pair once, and adds qualifying pairs into a block-private
// (s_bin, t_bin) histogram.  Each pair contributes to exactly one bin: the first spatial
// threshold s_a with d <= s_a and the first temporal threshold t_b with u <= t_b, so the
// cumulative grid over (a, b) reproduces the indicator sum of Eq. 2 at every threshold pair.
//
// Two precisions:
//   * pair_fp32: candidate filter, binning and weights in FP32 on cell-relative coordinates.
//     Every decision that FP32 cannot make with a proven error bound (a squared distance or a
//     time lag inside the guard band of a threshold, a temporal weight near its switch, a
//     circle nearly tangent to an edge) is recomputed in FP64 with the reference arithmetic,
//     so counts are exact.  Weights enter as fixed-point (w - 1) * 2^32, so sums are
//     order-independent integers.
//   * pair_fp64: the same tiling with every pair in FP64 (the plain comparison path).
//
// This is CUDA-core work (no dense contraction), bound by instruction issue.
#include "stk_internal.h"

#include <math.h>

namespace stk {
namespace {

constexpr int kWarps = kBlock / 32;
constexpr uint64_t kFlushLimit = 1ull << 28;  // candidates per histogram flush (no overflow)

struct Segs {
    int start[9];   // first sorted index of the run of up to three x-cells
    int b1[9];      // first index of the centre column's x-cell in this row
    int b2[9];      // one past its last index
    int pref[10];   // prefix of run lengths (position of the run in the staged sequence)
    int dy[9], dt[9];
};

__device__ __forceinline__ void make_segments(const Grid& g, uint32_t cell,
                                              const uint32_t* __restrict__ cs, Segs& sg) {
    // thread 0 builds all nine runs (dy, dt in -1..1)
    const int cx = (int)(cell % (uint32_t)g.nx);
    const int cy = (int)((cell / (uint32_t)g.nx) % (uint32_t)g.ny);
    const int ct = (int)(cell / ((uint32_t)g.nx * (uint32_t)g.ny));
    int acc = 0;
    for (int s = 0; s < 9; ++s) {
        const int dy = s / 3 - 1, dt = s % 3 - 1;
        const int ry = cy + dy, rt = ct + dt;
        sg.dy[s] = dy;
        sg.dt[s] = dt;
        sg.pref[s] = acc;
        if (ry < 0 || ry >= g.ny || rt < 0 || rt >= g.nt) {
            sg.start[s] = 0;
            sg.b1[s] = 0;
            sg.b2[s] = 0;
            continue;
        }
        const int row = (rt * g.ny + ry) * g.nx;
        const int lo = row + (cx > 0 ? cx - 1 : 0);
        const int hi = row + (cx + 1 < g.nx ? cx + 1 : cx);
        const int st = (int)cs[lo];
        const int en = (int)cs[hi + 1];
        sg.start[s] = st;
        sg.b1[s] = (int)cs[row + cx];
        sg.b2[s] = (int)cs[row + cx + 1];
        acc += en - st;
    }
    sg.pref[9] = acc;
}

// ---------------------------------------------------------------- exact FP64 pair (reference)

// Section 3 isotropic weight for a rectangle when the radius is at most half of each side:
// at most one x-edge and one y-edge cut the circle.  An edge at distance e < r removes an arc
// of half-angle acos(e/r) around its normal; when the corner lies inside the circle the two
// arcs overlap and the outside part is alpha_x + alpha_y + pi/2 (out of 2 pi).
__device__ __forceinline__ double omega64(const PairConsts& pc, double xi, double yi,
                                          double r) {
    if (r == 0.0) return 1.0;
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

// Exact pair evaluation with the reference rounding (every operation rounded separately).
// Returns false when the pair does not qualify.
__device__ __noinline__ bool pair_exact(const PairConsts& pc, double xi, double yi, double ti,
                                        double xj, double yj, double tj, int& a, int& b,
                                        unsigned long long& exc) {
    const double dx = __dsub_rn(xi, xj);
    const double dy = __dsub_rn(yi, yj);
    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (d2 > pc.s2[pc.cs - 1]) return false;
    const double u = fabs(__dsub_rn(ti, tj));
    if (u > pc.tt[pc.ct - 1]) return false;
    a = 0;
    while (d2 > pc.s2[a]) ++a;
    b = 0;
    while (u > pc.tt[b]) ++b;
    exc = 0;
    if (pc.edge) {
        const double om = omega64(pc, xi, yi, __dsqrt_rn(d2));
        const double w = 1.0 / (om * v64(pc, ti, u));
        exc = excess_fixed64(w);
    }
    return true;
}

// ---------------------------------------------------------------- histogram flush

__device__ __forceinline__ void flush_hist(int real, int nbins, int reps, uint32_t* hc,
                                           unsigned long long* he, const Accum& acc) {
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += kBlock) {
        uint32_t c = 0;
        unsigned long long e = 0;
        for (int r = 0; r < reps; ++r) {
            c += hc[r * nbins + b];
            e += he[r * nbins + b];
            hc[r * nbins + b] = 0;
            he[r * nbins + b] = 0;
        }
        const int64_t o = (int64_t)real * nbins + b;
        if (c) atomicAdd(&acc.cnt[o], (unsigned long long)c);
        if (e) {
            atomicAdd(&acc.exc_lo[o], e & 0xffffffffull);
            if (e >> 32) atomicAdd(&acc.exc_hi[o], e >> 32);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- FP32 guarded kernel

struct Smem32 {
    PairConsts pc;
    Segs sg;
    float4 stage[kStage32];      // x_hi, y_hi, t_hi (centre-cell frame), sorted index bits
    float2 stage_lo[kStage32];   // x_lo, y_lo (centre-cell frame)
    float4 cen_a[kCentreMax];    // x_hi, y_hi, t_hi, interior fast-path bound on d2_hi
    float4 cen_b[kCentreMax];    // x_lo, y_lo, e_x, e_y
    float cen_te[kCentreMax];    // distance to the nearer end of the study period
    uint8_t cen_on[kCentreMax];
    uint32_t item;
    // histograms follow (dynamic size)
};

__device__ __forceinline__ int bin_fp32(float v2_or_v, float key, float inv_h,
                                        const uint8_t* tab, const float* lo, const float* hi,
                                        int nthr, bool& amb) {
    int k = (int)(key * inv_h);
    k = k < kTab - 1 ? k : kTab - 1;
    const uint32_t e = tab[k];
    int a = (int)(e & 0x7fu);
    if (e & 0x80u) {
        while (a < nthr - 1 && v2_or_v > hi[a]) ++a;
        if (v2_or_v >= lo[a]) amb = true;
    }
    return a;
}

__global__ void __launch_bounds__(kBlock, 3)
pair_fp32_kernel(const PairConsts* __restrict__ gpc, RealBatch rb,
                 const WorkItem* __restrict__ items, const uint32_t* __restrict__ n_items_p,
                 uint32_t* __restrict__ counter, Accum acc, int reps) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem32& sm = *reinterpret_cast<Smem32*>(smem_raw);
    const PairConsts& pc = sm.pc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {
        const int words = (int)(sizeof(PairConsts) / 4);
        const int* src = reinterpret_cast<const int*>(gpc);
        int* dst = reinterpret_cast<int*>(&sm.pc);
        for (int i = tid; i < words; i += kBlock) dst[i] = src[i];
    }
    __syncthreads();
    const int nbins = pc.nbins;
    const size_t hist_off = (sizeof(Smem32) + 15) & ~size_t(15);
    unsigned long long* he = reinterpret_cast<unsigned long long*>(smem_raw + hist_off);
    uint32_t* hc = reinterpret_cast<uint32_t*>(he + (size_t)reps * nbins);
    for (int i = tid; i < reps * nbins; i += kBlock) {
        hc[i] = 0;
        he[i] = 0;
    }
    uint32_t* my_hc = hc + (warp % reps) * nbins;
    unsigned long long* my_he = he + (warp % reps) * nbins;

    const uint32_t n_items = *n_items_p;
    const int64_t n = rb.n;
    int cur_real = -1;
    uint64_t since_flush = 0;
    unsigned long long n_cand = 0, n_exact = 0;
    __syncthreads();

    for (;;) {
        if (tid == 0) sm.item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t it = sm.item;
        if (it >= n_items) break;
        const WorkItem w = items[it];
        if ((int)w.real != cur_real) {
            if (cur_real >= 0) flush_hist(cur_real, nbins, reps, hc, he, acc);
            cur_real = (int)w.real;
            since_flush = 0;
        }
        const int64_t base = (int64_t)w.real * n;
        const uint32_t* cs = rb.cell_start + (int64_t)w.real * (rb.ncells + 1);
        const int C = (int)w.c_count;
        if (tid < C) {
            const int64_t ci = base + w.c_begin + tid;
            const float4 p = rb.P[ci];
            const float2 lo = rb.Plo[ci];
            const double xi = rb.X[ci], yi = rb.Y[ci], ti = rb.T[ci];
            const float ex = (float)fmin(xi - pc.g.x0, pc.g.x1 - xi);
            const float ey = (float)fmin(yi - pc.g.y0, pc.g.y1 - yi);
            const float te = (float)fmin(ti - pc.g.t0, pc.g.t1 - ti);
            const float em = fminf(ex, ey);
            // interior: r_true < e_min * (1 - tan_rel) - tan_abs, so omega = 1 exactly
            float rin = em * (1.0f - pc.tan_rel) - pc.tan_abs - pc.fast_abs -
                        em * 4.76837158e-7f;
            rin = fmaxf(rin, 0.0f);
            sm.cen_a[tid] = make_float4(p.x, p.y, p.z, rin * rin * 0.99999f);
            sm.cen_b[tid] = make_float4(lo.x, lo.y, ex, ey);
            sm.cen_te[tid] = te;
            sm.cen_on[tid] =
                (rb.mask != nullptr && w.real == 0) ? rb.mask[w.c_begin + tid] : (uint8_t)1;
        }
        if (tid == 0) make_segments(pc.g, w.cell, cs, sm.sg);
        __syncthreads();
        const int M = sm.sg.pref[9];
        for (int cb = 0; cb < M; cb += kStage32) {
            const int mlen = min(kStage32, M - cb);
            if (since_flush + (uint64_t)C * (uint64_t)mlen > kFlushLimit) {
                flush_hist(cur_real, nbins, reps, hc, he, acc);
                since_flush = 0;
            }
            since_flush += (uint64_t)C * (uint64_t)mlen;
            // stage the chunk, moving each point into the centre cell's frame
            for (int e = tid; e < mlen; e += kBlock) {
                const int gp = cb + e;
                int s = 0;
                while (s < 8 && gp >= sm.sg.pref[s + 1]) ++s;
                const int idx = sm.sg.start[s] + (gp - sm.sg.pref[s]);
                float4 p = rb.P[base + idx];
                float2 lo = rb.Plo[base + idx];
                const float sx = (float)(-1 + (idx >= sm.sg.b1[s]) + (idx >= sm.sg.b2[s]));
                const float sy = (float)sm.sg.dy[s], st = (float)sm.sg.dt[s];
                p.x += sx * pc.g.cwq;
                p.y += sy * pc.g.chq;
                p.z += st * pc.g.cdq;
                lo.x += sx * pc.g.cwl;
                lo.y += sy * pc.g.chl;
                sm.stage[e] = p;
                sm.stage_lo[e] = lo;
            }
            __syncthreads();
            // warp units: 32 consecutive centres x one slice of the staged chunk
            const int G = (C + 31) >> 5;
            int S = (2 * kWarps + G - 1) / G;
            const int smax = mlen / 64 > 1 ? mlen / 64 : 1;
            S = S < smax ? S : smax;
            const int units = G * S;
            for (int un = warp; un < units; un += kWarps) {
                const int g = un % G, sl = un / G;
                const int c = g * 32 + lane;
                const bool on = c < C && sm.cen_on[c];
                const int cc = c < C ? c : 0;
                const float4 ca = sm.cen_a[cc];
                const float4 cbv = sm.cen_b[cc];
                const float te = sm.cen_te[cc];
                const int j0 = (int)(((int64_t)mlen * sl) / S);
                const int j1 = (int)(((int64_t)mlen * (sl + 1)) / S);
                if (on) n_cand += (unsigned long long)(j1 - j0);
                for (int j = j0; j < j1; ++j) {
                    const float4 p = sm.stage[j];
                    const float dx = ca.x - p.x;
                    const float dy = ca.y - p.y;
                    const float d2 = fmaf(dx, dx, dy * dy);
                    const float u = fabsf(ca.z - p.z);
                    if (!(on && d2 <= pc.s2_cut && u <= pc.u_cut)) continue;
                    bool amb = false;
                    const float r = sqrtf(d2);
                    int a = bin_fp32(d2, r, pc.inv_hs, pc.tab_s, pc.s_lo, pc.s_hi, pc.cs, amb);
                    int b = bin_fp32(u, u, pc.inv_ht, pc.tab_t, pc.t_lo, pc.t_hi, pc.ct, amb);
                    unsigned long long exc = 0;
                    if (pc.edge && !amb) {
                        bool vhalf = false;
                        if (u > te - pc.g_v) {
                            if (u > te + pc.g_v)
                                vhalf = true;
                            else
                                amb = true;
                        }
                        float A = 0.0f;
                        if (!amb && d2 > ca.w) {
                            const float2 lo = sm.stage_lo[j];
                            const float dxa = dx + (cbv.x - lo.x);
                            const float dya = dy + (cbv.y - lo.y);
                            const float ra = sqrtf(fmaf(dxa, dxa, dya * dya));
                            const float ex = cbv.z, ey = cbv.w;
                            const float band = fmaf(pc.tan_rel, ra, pc.tan_abs);
                            if (ra < pc.r_acc_min || fabsf(ra - ex) <= band ||
                                fabsf(ra - ey) <= band) {
                                amb = true;
                            } else {
                                float ax = 0.0f, ay = 0.0f;
                                if (ex < ra) ax = atan2f(sqrtf((ra - ex) * (ra + ex)), ex);
                                if (ey < ra) ay = atan2f(sqrtf((ra - ey) * (ra + ey)), ey);
                                if (fmaf(ex, ex, ey * ey) < ra * ra)
                                    A = (ax + ay + 1.57079632679f) * 0.159154943092f;
                                else
                                    A = (ax + ay) * 0.318309886184f;
                            }
                        }
                        if (!amb) {
                            const float xs = vhalf ? (1.0f + A) / (1.0f - A) : A / (1.0f - A);
                            if (xs > 0.0f) exc = __float2ull_rn(xs * 4294967296.0f);
                        }
                    }
                    if (amb) {
                        ++n_exact;
                        const int64_t ci = base + w.c_begin + c;
                        const int64_t cj = base + __float_as_int(p.w);
                        if (!pair_exact(pc, rb.X[ci], rb.Y[ci], rb.T[ci], rb.X[cj], rb.Y[cj],
                                        rb.T[cj], a, b, exc))
                            continue;
                    }
                    const int bin = a * pc.ct + b;
                    atomicAdd(&my_hc[bin], 1u);
                    if (exc) atomicAdd(&my_he[bin], exc);
                }
            }
            __syncthreads();
        }
    }
    if (cur_real >= 0) flush_hist(cur_real, nbins, reps, hc, he, acc);
    // block totals of the statistics
    for (int o = 16; o > 0; o >>= 1) {
        n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
        n_exact += __shfl_xor_sync(0xffffffffu, n_exact, o);
    }
    if (lane == 0) {
        atomicAdd(&acc.stats[0], n_cand);
        atomicAdd(&acc.stats[1], n_exact);
    }
}

// ---------------------------------------------------------------- FP64 plain kernel

struct Smem64 {
    PairConsts pc;
    Segs sg;
    double sx[kStage64], sy[kStage64], st[kStage64];
    double cx[kCentreMax], cy[kCentreMax], ct[kCentreMax];
    uint8_t cen_on[kCentreMax];
    uint32_t item;
};

__global__ void __launch_bounds__(kBlock, 2)
pair_fp64_kernel(const PairConsts* __restrict__ gpc, RealBatch rb,
                 const WorkItem* __restrict__ items, const uint32_t* __restrict__ n_items_p,
                 uint32_t* __restrict__ counter, Accum acc, int reps) {
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
    const int nbins = pc.nbins;
    const size_t hist_off = (sizeof(Smem64) + 15) & ~size_t(15);
    unsigned long long* he = reinterpret_cast<unsigned long long*>(smem_raw + hist_off);
    uint32_t* hc = reinterpret_cast<uint32_t*>(he + (size_t)reps * nbins);
    for (int i = tid; i < reps * nbins; i += kBlock) {
        hc[i] = 0;
        he[i] = 0;
    }
    uint32_t* my_hc = hc + (warp % reps) * nbins;
    unsigned long long* my_he = he + (warp % reps) * nbins;
    const uint32_t n_items = *n_items_p;
    const int64_t n = rb.n;
    int cur_real = -1;
    uint64_t since_flush = 0;
    unsigned long long n_cand = 0;
    const double s2max = pc.s2[pc.cs - 1], tmax = pc.tt[pc.ct - 1];
    __syncthreads();

    for (;;) {
        if (tid == 0) sm.item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t it = sm.item;
        if (it >= n_items) break;
        const WorkItem w = items[it];
        if ((int)w.real != cur_real) {
            if (cur_real >= 0) flush_hist(cur_real, nbins, reps, hc, he, acc);
            cur_real = (int)w.real;
            since_flush = 0;
        }
        const int64_t base = (int64_t)w.real * n;
        const uint32_t* cs = rb.cell_start + (int64_t)w.real * (rb.ncells + 1);
        const int C = (int)w.c_count;
        if (tid < C) {
            const int64_t ci = base + w.c_begin + tid;
            sm.cx[tid] = rb.X[ci];
            sm.cy[tid] = rb.Y[ci];
            sm.ct[tid] = rb.T[ci];
            sm.cen_on[tid] =
                (rb.mask != nullptr && w.real == 0) ? rb.mask[w.c_begin + tid] : (uint8_t)1;
        }
        if (tid == 0) make_segments(pc.g, w.cell, cs, sm.sg);
        __syncthreads();
        const int M = sm.sg.pref[9];
        for (int cb = 0; cb < M; cb += kStage64) {
            const int mlen = min(kStage64, M - cb);
            if (since_flush + (uint64_t)C * (uint64_t)mlen > kFlushLimit) {
                flush_hist(cur_real, nbins, reps, hc, he, acc);
                since_flush = 0;
            }
            since_flush += (uint64_t)C * (uint64_t)mlen;
            for (int e = tid; e < mlen; e += kBlock) {
                const int gp = cb + e;
                int s = 0;
                while (s < 8 && gp >= sm.sg.pref[s + 1]) ++s;
                const int64_t idx = base + sm.sg.start[s] + (gp - sm.sg.pref[s]);
                sm.sx[e] = rb.X[idx];
                sm.sy[e] = rb.Y[idx];
                sm.st[e] = rb.T[idx];
            }
            __syncthreads();
            const int G = (C + 31) >> 5;
            int S = (2 * kWarps + G - 1) / G;
            const int smax = mlen / 64 > 1 ? mlen / 64 : 1;
            S = S < smax ? S : smax;
            const int units = G * S;
            for (int un = warp; un < units; un += kWarps) {
                const int g = un % G, sl = un / G;
                const int c = g * 32 + lane;
                const bool on = c < C && sm.cen_on[c];
                const int cc = c < C ? c : 0;
                const double xi = sm.cx[cc], yi = sm.cy[cc], ti = sm.ct[cc];
                const int j0 = (int)(((int64_t)mlen * sl) / S);
                const int j1 = (int)(((int64_t)mlen * (sl + 1)) / S);
                if (on) n_cand += (unsigned long long)(j1 - j0);
                for (int j = j0; j < j1; ++j) {
                    const double dx = __dsub_rn(xi, sm.sx[j]);
                    const double dy = __dsub_rn(yi, sm.sy[j]);
                    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                    const double u = fabs(__dsub_rn(ti, sm.st[j]));
                    if (!(on && d2 <= s2max && u <= tmax)) continue;
                    int ks = (int)(d2 * pc.inv_hs2_64);
                    ks = ks < kTab - 1 ? ks : kTab - 1;
                    int a = pc.tab_s64[ks];
                    while (d2 > pc.s2[a]) ++a;
                    int kt = (int)(u * pc.inv_ht_64);
                    kt = kt < kTab - 1 ? kt : kTab - 1;
                    int b = pc.tab_t64[kt];
                    while (u > pc.tt[b]) ++b;
                    unsigned long long exc = 0;
                    if (pc.edge) {
                        const double om = omega64(pc, xi, yi, __dsqrt_rn(d2));
                        exc = excess_fixed64(1.0 / (om * v64(pc, ti, u)));
                    }
                    const int bin = a * pc.ct + b;
                    atomicAdd(&my_hc[bin], 1u);
                    if (exc) atomicAdd(&my_he[bin], exc);
                }
            }
            __syncthreads();
        }
    }
    if (cur_real >= 0) flush_hist(cur_real, nbins, reps, hc, he, acc);
    for (int o = 16; o > 0; o >>= 1) n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
    if (lane == 0) atomicAdd(&acc.stats[0], n_cand);
}

// ---------------------------------------------------------------- finalize / envelope

// One block per realization: integer histogram -> cumulative grids (exact, in 128-bit fixed
// point) -> S, K (Eq. 2 normalisation) and L (Eq. 4).
__global__ void finalize_kernel(int cs, int ct, const double* __restrict__ s,
                                const double* __restrict__ tt, double coef,
                                const int64_t* __restrict__ self_pairs, Accum acc,
                                double* __restrict__ K, double* __restrict__ L,
                                double* __restrict__ S, int64_t* __restrict__ C) {
    extern __shared__ __align__(16) unsigned char fsm[];
    const int nb = cs * ct;
    unsigned long long* cc = reinterpret_cast<unsigned long long*>(fsm);
    unsigned __int128* ee = reinterpret_cast<unsigned __int128*>(cc + ((nb + 1) & ~1));
    const int k = blockIdx.x;
    const int64_t o = (int64_t)k * nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        cc[i] = acc.cnt[o + i];
        ee[i] = ((unsigned __int128)acc.exc_hi[o + i] << 32) + (unsigned __int128)acc.exc_lo[o + i];
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
        const double ed = (double)(unsigned long long)(e >> 64) * 18446744073709551616.0 +
                          (double)(unsigned long long)e;
        const double sv = (double)cc[i] + ed * (1.0 / 4294967296.0);
        const double kv = coef * sv;
        if (K) K[o + i] = kv;
        if (L) L[o + i] = sqrt(kv / (2.0 * 3.141592653589793 * tt[b])) - s[a];
        if (S) S[o + i] = sv;
        if (C) C[o + i] = (int64_t)cc[i];
    }
}

__global__ void envelope_kernel(int m, int nbins, int ct, const double* __restrict__ K,
                                const double* __restrict__ s, const double* __restrict__ tt,
                                double* __restrict__ K_lo, double* __restrict__ K_hi,
                                double* __restrict__ L_lo, double* __restrict__ L_hi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbins) return;
    double lo = K[i], hi = K[i];
    for (int k = 1; k < m; ++k) {
        const double v = K[(int64_t)k * nbins + i];
        lo = fmin(lo, v);
        hi = fmax(hi, v);
    }
    const int a = i / ct, b = i - (i / ct) * ct;
    const double den = 2.0 * 3.141592653589793 * tt[b];
    K_lo[i] = lo;
    K_hi[i] = hi;
    L_lo[i] = sqrt(lo / den) - s[a];
    L_hi[i] = sqrt(hi / den) - s[a];
}

size_t hist_bytes(int nbins, int reps) { return (size_t)reps * nbins * 12; }

size_t smem_with_reps(size_t base, int nbins, int* reps, size_t budget) {
    const size_t b = (base + 15) & ~size_t(15);
    int r = 8;
    while (r > 1 && b + hist_bytes(nbins, r) > budget) --r;
    *reps = r;
    return b + hist_bytes(nbins, r);
}

}  // namespace

size_t pair_fp32_smem(int nbins, int* reps) {
    return smem_with_reps(sizeof(Smem32), nbins, reps, 72 * 1024);
}
size_t pair_fp64_smem(int nbins, int* reps) {
    return smem_with_reps(sizeof(Smem64), nbins, reps, 100 * 1024);
}

cudaError_t pair_kernels_configure(size_t smem32, size_t smem64) {
    cudaError_t e = cudaFuncSetAttribute(finalize_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kMaxThr * kMaxThr * 24 + 16));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(pair_fp32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem32);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(pair_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem64);
}

int pair_fp32_blocks_per_sm(size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pair_fp32_kernel, kBlock, smem) !=
        cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

int pair_fp64_blocks_per_sm(size_t smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pair_fp64_kernel, kBlock, smem) !=
        cudaSuccess)
        return 1;
    return b > 0 ? b : 1;
}

cudaError_t launch_pair_fp32(const PairConsts* d_pc, size_t smem, int reps, int grid,
                             RealBatch rb, const WorkItem* items, const uint32_t* n_items,
                             uint32_t* counter, Accum acc, cudaStream_t st) {
    pair_fp32_kernel<<<grid, kBlock, smem, st>>>(d_pc, rb, items, n_items, counter, acc, reps);
    return cudaGetLastError();
}

cudaError_t launch_pair_fp64(const PairConsts* d_pc, size_t smem, int reps, int grid,
                             RealBatch rb, const WorkItem* items, const uint32_t* n_items,
                             uint32_t* counter, Accum acc, cudaStream_t st) {
    pair_fp64_kernel<<<grid, kBlock, smem, st>>>(d_pc, rb, items, n_items, counter, acc, reps);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int m, int cs, int ct, const double* s, const double* tt,
                            double coef, const int64_t* self_pairs, Accum acc, double* K,
                            double* L, double* S, int64_t* C, cudaStream_t st) {
    const int nb = cs * ct;
    const size_t smem = (size_t)((nb + 1) & ~1) * 8 + (size_t)nb * 16;
    finalize_kernel<<<m, 128, smem, st>>>(cs, ct, s, tt, coef, self_pairs, acc, K, L, S, C);
    return cudaGetLastError();
}

cudaError_t launch_envelope(int m, int nbins, int ct, const double* K, const double* s,
                            const double* tt, double* K_lo, double* K_hi, double* L_lo,
                            double* L_hi, cudaStream_t st) {
    envelope_kernel<<<(nbins + 127) / 128, 128, 0, st>>>(m, nbins, ct, K, s, tt, K_lo, K_hi,
                                                         L_lo, L_hi);
    return cudaGetLastError();
}

}  // namespace stk
