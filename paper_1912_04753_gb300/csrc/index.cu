// Grid index build: CSR point generation, cell keys, counting sort by cell, work list.
//
// Replaces the paper's R-tree / STR bulk loading (Section 4.2) and KDB-tree partitioning
// (Section 4.4) with a uniform spatio-temporal grid whose cells are at least as large as the
// largest thresholds, so the spatio-temporal cylinder around any point (Section 4.2) lies in
// the 27 cells around the point's own cell.  Every kernel here is bound by HBM bandwidth.
#include "stk_internal.h"

#include <math.h>

#include "poly.cuh"

namespace stk {
namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds, each multiplying words 0 and
// 2 by the round constants and folding the high product halves into words 1 and 3 with the
// key; the key advances by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Uniform double in [0,1) from 27 + 26 random bits (exact in FP64).
__device__ __forceinline__ double u01(uint32_t w0, uint32_t w1) {
    return ((double)(w0 >> 5) * 67108864.0 + (double)(w1 >> 6)) * (1.0 / 9007199254740992.0);
}

// lo + (hi - lo) * u with each operation rounded separately, clamped into the closed box.
__device__ __forceinline__ double csr_coord(uint64_t seed, uint32_t sim, int64_t i,
                                            uint32_t stream, double lo, double hi) {
    const uint4 w = philox4x32_10(
        make_uint4((uint32_t)i, sim, stream, (uint32_t)((uint64_t)i >> 32)),
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const double u = u01(w.x, w.y);
    const double span = __dsub_rn(hi, lo);
    const double v = __dadd_rn(lo, __dmul_rn(span, u));
    return v > hi ? hi : v;
}

__device__ __forceinline__ int cell_of(double v, double v0, double inv, int nc) {
    const double f = floor(__dmul_rn(__dsub_rn(v, v0), inv));
    int c = (int)fmax(0.0, fmin(f, (double)(nc - 1)));
    return c;
}

struct GridDev {
    int nx, ny, nt;
    double x0, y0, t0, inv_cw, inv_ch, inv_cd;
};

__host__ GridDev grid_dev(const Grid& g) {
    GridDev d;
    d.nx = g.nx;
    d.ny = g.ny;
    d.nt = g.nt;
    d.x0 = g.x0;
    d.y0 = g.y0;
    d.t0 = g.t0;
    d.inv_cw = 1.0 / g.cw;
    d.inv_ch = 1.0 / g.ch;
    d.inv_cd = 1.0 / g.cd;
    return d;
}

__device__ __forceinline__ uint32_t key_of(const GridDev& g, double x, double y, double t) {
    const int cx = cell_of(x, g.x0, g.inv_cw, g.nx);
    const int cy = cell_of(y, g.y0, g.inv_ch, g.ny);
    const int ct = cell_of(t, g.t0, g.inv_cd, g.nt);
    return (uint32_t)((ct * g.ny + cy) * g.nx + cx);
}

__global__ void keys_observed_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                     const double* __restrict__ t, int64_t n, GridDev g,
                                     double x1, double y1, double t1, uint32_t* __restrict__ key,
                                     uint32_t* __restrict__ rank, uint32_t* __restrict__ cnt,
                                     int* __restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double xi = x[i], yi = y[i], ti = t[i];
        // inside the closed box (also rejects NaN); infinities fail the range test
        const bool ok = (xi >= g.x0) && (xi <= x1) && (yi >= g.y0) && (yi <= y1) &&
                        (ti >= g.t0) && (ti <= t1);
        if (!ok) {
            atomicOr(bad, 1);
            key[i] = 0;
            rank[i] = atomicAdd(&cnt[0], 1u);
            continue;
        }
        const uint32_t k = key_of(g, xi, yi, ti);
        key[i] = k;
        rank[i] = atomicAdd(&cnt[k], 1u);
    }
}

__global__ void validate_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                const double* __restrict__ t, int64_t n, double x0, double x1,
                                double y0, double y1, double t0, double t1,
                                int* __restrict__ bad) {
    int local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double xi = x[i], yi = y[i], ti = t[i];
        local |= !((xi >= x0) && (xi <= x1) && (yi >= y0) && (yi <= y1) && (ti >= t0) &&
                   (ti <= t1));
    }
    if (__any_sync(0xffffffffu, local) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

constexpr int kPolyAttempts = 4096;  // CSR draws per point in a polygon (area >= box / 64)

__global__ void gen_csr_kernel(int64_t n, int m, const uint64_t* __restrict__ seeds,
                               const uint32_t* __restrict__ sims, GridDev g,
                               double x1, double y1, double t1, int64_t ncells,
                               double* __restrict__ x, double* __restrict__ y,
                               double* __restrict__ t, uint32_t* __restrict__ key,
                               uint32_t* __restrict__ rank, uint32_t* __restrict__ cnt,
                               Polygon poly, unsigned long long* __restrict__ err) {
    const int64_t total = n * (int64_t)m;
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(gi / n);
        const int64_t i = gi - (int64_t)k * n;
        const uint32_t sim = sims[k];
        const uint64_t seed = seeds[k];
        double xi, yi;
        if (poly.nv == 0) {
            xi = csr_coord(seed, sim, i, 0u, g.x0, x1);
            yi = csr_coord(seed, sim, i, 1u, g.y0, y1);
        } else {
            // uniform in the polygon: the first attempt inside, x from words 0-1 and y from
            // words 2-3 of Philox block (i, sim, 32 + attempt, i >> 32) in the bounding box
            const uint2 kk2 = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
            const double sx = __dsub_rn(x1, g.x0), sy = __dsub_rn(y1, g.y0);
            bool found = false;
            xi = g.x0;
            yi = g.y0;
            for (int a = 0; a < kPolyAttempts && !found; ++a) {
                const uint4 w = philox4x32_10(
                    make_uint4((uint32_t)i, sim, 32u + (uint32_t)a, (uint32_t)((uint64_t)i >> 32)),
                    kk2);
                double px = __dadd_rn(g.x0, __dmul_rn(sx, u01(w.x, w.y)));
                double py = __dadd_rn(g.y0, __dmul_rn(sy, u01(w.z, w.w)));
                px = px > x1 ? x1 : px;
                py = py > y1 ? y1 : py;
                if (poly.band ? poly_contains_banded(px, py, poly)
                              : poly_contains(px, py, poly.vx, poly.vy, poly.nv)) {
                    xi = px;
                    yi = py;
                    found = true;
                }
            }
            if (!found && err) atomicAdd(err, 1ull);  // never expected: area >= box / 64
        }
        const double ti = csr_coord(seed, sim, i, 2u, g.t0, t1);
        x[gi] = xi;
        y[gi] = yi;
        t[gi] = ti;
        const uint32_t kk = key_of(g, xi, yi, ti);
        key[gi] = kk;
        rank[gi] = atomicAdd(&cnt[(int64_t)k * ncells + kk], 1u);
    }
}

// ---------------------------------------------------------------------------- intensity
// Inhomogeneous K (Section 7 future work): the relative intensity rho is piecewise constant on
// nix x niy x nit equal cells of the box.  Cell of v along one axis:
// floor(((v - lo) / (hi - lo)) * nc), each operation rounded separately, clamped to the axis.
__device__ __forceinline__ int intensity_axis(double v, double lo, double hi, int nc) {
    const double f = floor(__dmul_rn(__ddiv_rn(__dsub_rn(v, lo), __dsub_rn(hi, lo)), (double)nc));
    return (int)fmax(0.0, fmin(f, (double)(nc - 1)));
}

struct IntensityBox {
    double x0, x1, y0, y1, t0, t1;
};

__global__ void intensity_lookup_kernel(const double* __restrict__ x,
                                        const double* __restrict__ y,
                                        const double* __restrict__ t, int64_t count,
                                        IntensityBox b, Intensity in, double* __restrict__ h,
                                        unsigned long long* __restrict__ zero) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int ix = intensity_axis(x[i], b.x0, b.x1, in.nix);
        const int iy = intensity_axis(y[i], b.y0, b.y1, in.niy);
        const int it = intensity_axis(t[i], b.t0, b.t1, in.nit);
        const double v = in.hcell[((int64_t)it * in.niy + iy) * in.nix + ix];
        h[i] = v;
        if (v == 0.0) atomicAdd(zero, 1ull);
    }
}

// Point i of a realization: cell c = the first whose running sum of rho exceeds u * total
// (u from Philox block (i, sim, 40, i >> 32); the last cell with rho > 0 when rounding leaves
// none), then lo + (hi - lo) * ((cell index + u_axis) / cells on the axis), u_axis the uniform
// of the CSR coordinate stream of that axis.  One cell gives exactly the CSR realization.
__global__ void gen_inhom_kernel(int64_t n, int m, const uint64_t* __restrict__ seeds,
                                 const uint32_t* __restrict__ sims, GridDev g, double x1,
                                 double y1, double t1, int64_t ncells, Intensity in,
                                 double* __restrict__ x, double* __restrict__ y,
                                 double* __restrict__ t, double* __restrict__ h,
                                 uint32_t* __restrict__ key, uint32_t* __restrict__ rank,
                                 uint32_t* __restrict__ cnt) {
    const int64_t total = n * (int64_t)m;
    const int cells = in.nix * in.niy * in.nit;
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(gi / n);
        const int64_t i = gi - (int64_t)k * n;
        const uint32_t sim = sims[k];
        const uint64_t seed = seeds[k];
        const uint2 kk2 = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
        const uint4 w = philox4x32_10(
            make_uint4((uint32_t)i, sim, 40u, (uint32_t)((uint64_t)i >> 32)), kk2);
        const double target = __dmul_rn(u01(w.x, w.y), in.total);
        int lo = 0, hi = cells;  // first c with cum[c] > target
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (in.cum[mid] > target)
                hi = mid;
            else
                lo = mid + 1;
        }
        const int c = lo < cells ? lo : in.last_pos;
        const int ix = c % in.nix, iy = (c / in.nix) % in.niy, it = c / (in.nix * in.niy);
        const double b0[3] = {g.x0, g.y0, g.t0}, b1[3] = {x1, y1, t1};
        const int idx[3] = {ix, iy, it}, nc[3] = {in.nix, in.niy, in.nit};
        double v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const uint4 wa = philox4x32_10(
                make_uint4((uint32_t)i, sim, (uint32_t)a, (uint32_t)((uint64_t)i >> 32)), kk2);
            const double q = __ddiv_rn(__dadd_rn((double)idx[a], u01(wa.x, wa.y)), (double)nc[a]);
            const double c1 = __dadd_rn(b0[a], __dmul_rn(__dsub_rn(b1[a], b0[a]), q));
            v[a] = c1 > b1[a] ? b1[a] : c1;
        }
        x[gi] = v[0];
        y[gi] = v[1];
        t[gi] = v[2];
        h[gi] = in.hcell[c];
        const uint32_t kk = key_of(g, v[0], v[1], v[2]);
        key[gi] = kk;
        rank[gi] = atomicAdd(&cnt[(int64_t)k * ncells + kk], 1u);
    }
}

// ---------------------------------------------------------------------------- resampling
// Bootstrapping (Section 3): point i of a realization is observed point floor(u n), u the
// 53-bit uniform of Philox block (i, sim, 4, i >> 32), a product that rounds up to n taken
// as n - 1.
__device__ __forceinline__ int64_t bootstrap_src(uint64_t seed, uint32_t sim, int64_t i,
                                                 int64_t n) {
    const uint4 w = philox4x32_10(
        make_uint4((uint32_t)i, sim, 4u, (uint32_t)((uint64_t)i >> 32)),
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    int64_t src = (int64_t)__dmul_rn(u01(w.x, w.y), (double)n);
    return src < n ? src : n - 1;
}

// Random permutation (Section 3): a balanced 4-round Feistel network on b-bit values whose
// round r mixes the right half into the left with the low half-width bits of word 0 of
// Philox block (right, sim, 16 + r, 0) (Luby-Rackoff), restricted to [0, n) by cycle walking
// (Black and Rogaway, 2002).
__device__ __forceinline__ uint64_t feistel(uint64_t v, int b, uint64_t seed, uint32_t sim) {
    const int half = b >> 1;
    const uint64_t mask = (1ull << half) - 1ull;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    uint64_t left = v >> half, right = v & mask;
#pragma unroll
    for (uint32_t r = 0; r < 4; ++r) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)right, sim, 16u + r, 0u), key);
        const uint64_t nr = left ^ ((uint64_t)w.x & mask);
        left = right;
        right = nr;
    }
    return (left << half) | right;
}

constexpr int kWalkLimit = 1 << 16;  // cycle-walk steps (the expected number is below 4)

__global__ void gen_resample_kernel(int method, int64_t n, int m, int bits,
                                    const uint64_t* __restrict__ seeds,
                                    const uint32_t* __restrict__ sims, GridDev g,
                                    int64_t ncells, const double* __restrict__ x0,
                                    const double* __restrict__ y0,
                                    const double* __restrict__ t0, double* __restrict__ x,
                                    double* __restrict__ y, double* __restrict__ t,
                                    uint32_t* __restrict__ key, uint32_t* __restrict__ rank,
                                    uint32_t* __restrict__ cnt,
                                    unsigned long long* __restrict__ err) {
    const int64_t total = n * (int64_t)m;
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(gi / n);
        const int64_t i = gi - (int64_t)k * n;
        const uint32_t sim = sims[k];
        const uint64_t seed = seeds[k];
        double xi, yi, ti;
        if (method == STK_SIM_BOOTSTRAP) {
            const int64_t src = bootstrap_src(seed, sim, i, n);
            xi = x0[src];
            yi = y0[src];
            ti = t0[src];
        } else {
            uint64_t v = feistel((uint64_t)i, bits, seed, sim);
            int steps = 0;
            while (v >= (uint64_t)n && ++steps < kWalkLimit) v = feistel(v, bits, seed, sim);
            if (v >= (uint64_t)n) {  // never expected; keep the index valid and report it
                atomicAdd(err, 1ull);
                v = (uint64_t)i;
            }
            xi = x0[i];
            yi = y0[i];
            ti = t0[v];
        }
        x[gi] = xi;
        y[gi] = yi;
        t[gi] = ti;
        const uint32_t kk = key_of(g, xi, yi, ti);
        key[gi] = kk;
        rank[gi] = atomicAdd(&cnt[(int64_t)k * ncells + kk], 1u);
    }
}

// ---------------------------------------------------------------------------- scan
// Exclusive scan of uint32 in tiles of kThreads*kItems, with the tile sums scanned
// recursively.  tmp holds the tile sums of every level.
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t nb = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += nb;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < kThreads / 32 ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t nb = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += nb;
        }
        if (lane < kThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t before = (wid > 0 ? warp_sums[wid - 1] : 0u) + inc - v;
    if (total) *total = warp_sums[kThreads / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void scan_tiles_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                  int64_t count, uint32_t* __restrict__ tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    uint32_t v[kItems];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        v[k] = (base + k < count) ? in[base + k] : 0u;
        sum += v[k];
    }
    uint32_t total;
    uint32_t run = block_excl_scan(sum, &total);
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < count) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = total;
}

__global__ void scan_add_kernel(uint32_t* __restrict__ out, int64_t count,
                                const uint32_t* __restrict__ tile_offsets) {
    const uint32_t add = tile_offsets[blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int k = threadIdx.x; k < kTile; k += kThreads) {
        if (base + k < count) out[base + k] += add;
    }
}

// ---------------------------------------------------------------------------- scatter

struct ScatterGrid {
    int nx, ny;
    double x0, y0, t0, x1, y1, t1, cw, ch, cd;
    double inv_qx, inv_qy, inv_qt;
    double qx, qy, qt;
    double qX, inv_qX;  // the filter's box-frame x quantum
    int64_t nF;         // floats per realization and axis of the filter arrays
    float tan_rel, tan_abs, fast_abs;
    Polygon poly;
    int mask_all;  // role flags for every realization (indexed by the point's index in it)
};

// The counting sort's scatter in two passes.  Points arrive in random order, so writing each
// per-point array at the point's sorted position is a store of 4-16 bytes into a random DRAM
// sector for each of nine arrays, most of them partial sectors that the memory system merges
// by read-modify-write.  Instead pass 1 moves each point as one 32-byte record (FP64
// coordinates, cell key, index within its realization: one whole sector) to its sorted
// position in a staging array, and pass 2 reads the records in sorted order and writes every
// per-point array with coalesced stores.

// Pass 1: inputs of slots slot0 .. slot0 + m - 1; the record of the point that goes to sorted
// position pos lands at S[pos - slot0 * n] (two double2: (x, y) and (t, key | src << 32)).
__global__ void stage_kernel(int m, int64_t n, int64_t ncells, const double* __restrict__ x,
                             const double* __restrict__ y, const double* __restrict__ t,
                             const uint32_t* __restrict__ key, const uint32_t* __restrict__ rank,
                             const uint32_t* __restrict__ start, int slot0,
                             double2* __restrict__ S) {
    const int64_t total = n * (int64_t)m;
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int kr = (int)(gi / n);
        const int k = slot0 + kr;
        const uint32_t kk = key[gi];
        const int64_t q = (int64_t)start[(int64_t)k * ncells + kk] + rank[gi] - (int64_t)slot0 * n;
        const uint32_t src = (uint32_t)(gi - (int64_t)kr * n);
        const unsigned long long tag = (unsigned long long)kk | ((unsigned long long)src << 32);
        S[2 * q] = make_double2(x[gi], y[gi]);
        S[2 * q + 1] = make_double2(t[gi], __longlong_as_double((long long)tag));
    }
}

// Pass 2: sorted position pos = slot0 * n + q of realization (slot) k = pos / n.
// P holds two float4 per point, the coordinate record (x_hi, y_hi, t_hi, cell x) in the
// first half of the realization's [2n] and the edge record (e_x, e_y, e_t, rin2) in the
// second: distances to the nearer x edge, y edge and end of the period, and a bound on d2
// below which the circle around the point stays clear of every edge (interior: weight 1).
// Plo holds (x - x0 - X_hi, y_lo): x's remainder below the filter's box-frame hi part
// X_hi, and y's below its cell-frame hi part.  The role flags and h of a point come from its
// input slot (index src within the realization).
__global__ void records_kernel(int m, int64_t n, ScatterGrid g, const double2* __restrict__ S,
                               const uint8_t* __restrict__ mask_in, double* __restrict__ X,
                               double* __restrict__ Y, double* __restrict__ T,
                               float4* __restrict__ P, float2* __restrict__ Plo,
                               uint8_t* __restrict__ mask_out,
                               const double* __restrict__ h_in, double* __restrict__ H,
                               float* __restrict__ F, int slot0) {
    const int64_t total = n * (int64_t)m;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int kr = (int)(q / n);
        const int k = slot0 + kr;
        const int64_t pos = (int64_t)slot0 * n + q;
        const double2 r0 = S[2 * q], r1 = S[2 * q + 1];
        const double xi = r0.x, yi = r0.y, ti = r1.x;
        const unsigned long long tag = (unsigned long long)__double_as_longlong(r1.y);
        const uint32_t kk = (uint32_t)tag, src = (uint32_t)(tag >> 32);
        X[pos] = xi;
        Y[pos] = yi;
        T[pos] = ti;
        const int cx = (int)(kk % (uint32_t)g.nx);
        const int cy = (int)((kk / (uint32_t)g.nx) % (uint32_t)g.ny);
        const int ct = (int)(kk / ((uint32_t)g.nx * (uint32_t)g.ny));
        // offsets from the cell origin; hi = offset rounded to the quantum (exact in FP32),
        // lo = the exact FP64 remainder rounded to FP32
        const double ox = __dsub_rn(xi, __dadd_rn(g.x0, __dmul_rn((double)cx, g.cw)));
        const double oy = __dsub_rn(yi, __dadd_rn(g.y0, __dmul_rn((double)cy, g.ch)));
        const double ot = __dsub_rn(ti, __dadd_rn(g.t0, __dmul_rn((double)ct, g.cd)));
        const double hx = rint(ox * g.inv_qx) * g.qx;
        const double hy = rint(oy * g.inv_qy) * g.qy;
        const double ht = rint(ot * g.inv_qt) * g.qt;
        // realization k's records: [k][2n] float4, the coordinate records first, then the
        // edge records
        const int64_t local = pos - (int64_t)k * n;
        float4* Pr = P + 2 * (int64_t)k * n;
        Pr[local] = make_float4((float)hx, (float)hy, (float)ht, __int_as_float(cx));
        // the filter's arrays: -x_hi relative to x0 (exact multiple of qX below 2^24 qX),
        // -y_hi, -t_hi as above; x's low part is taken relative to x0 too
        const double oX = __dsub_rn(xi, g.x0);
        const double hX = rint(oX * g.inv_qX) * g.qX;
        {
            float* f = F + (int64_t)k * 3 * g.nF + local;
            f[0] = -(float)hX;
            f[g.nF] = -(float)hy;
            f[2 * g.nF] = -(float)ht;
        }
        float ex = (float)fmin(__dsub_rn(xi, g.x0), __dsub_rn(g.x1, xi));
        float ey = (float)fmin(__dsub_rn(yi, g.y0), __dsub_rn(g.y1, yi));
        const float te = (float)fmin(__dsub_rn(ti, g.t0), __dsub_rn(g.t1, ti));
        // interior: r_true < e_min * (1 - tan_rel) - tan_abs, so omega = 1 exactly; in a
        // polygon e_min is the distance to its boundary (its weights are all taken in FP64)
        float em = fminf(ex, ey);
        if (g.poly.nv > 0) {
            em = (float)poly_boundary_distance(xi, yi, g.poly.vx, g.poly.vy, g.poly.nv);
            ex = ey = 3.0e38f;
        }
        float rin = em * (1.0f - g.tan_rel) - g.tan_abs - g.fast_abs - em * 4.76837158e-7f;
        rin = fmaxf(rin, 0.0f);
        Pr[n + local] = make_float4(ex, ey, te, rin * rin * 0.99999f);
        Plo[pos] = make_float2((float)(oX - hX), (float)(oy - hy));
        if (mask_out && (g.mask_all || k == 0)) mask_out[pos] = mask_in[src];
        if (H) H[pos] = h_in[(int64_t)kr * n + src];
    }
}

__global__ void cell_starts_kernel(int m, int64_t n, int64_t ncells,
                                   const uint32_t* __restrict__ start,
                                   uint32_t* __restrict__ cell_start) {
    const int64_t total = (ncells + 1) * (int64_t)m;
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(gi / (ncells + 1));
        const int64_t c = gi - (int64_t)k * (ncells + 1);
        cell_start[gi] = (c == ncells) ? (uint32_t)n
                                       : (uint32_t)((int64_t)start[(int64_t)k * ncells + c] -
                                                    (int64_t)k * n);
    }
}

// Work units: each (realization, grid row) is cut into groups of kUnit consecutive centres.
__global__ void work_counts_kernel(int m, int64_t nrows, int nx, const uint32_t* __restrict__ cs,
                                   int64_t ncells, uint32_t* __restrict__ counts) {
    const int64_t total = nrows * (int64_t)m;
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi <= total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        if (gi == total) {
            counts[gi] = 0u;  // slot that the exclusive scan turns into the total
            continue;
        }
        const int k = (int)(gi / nrows);
        const int64_t r = gi - (int64_t)k * nrows;
        const uint32_t* s = cs + (int64_t)k * (ncells + 1);
        const uint32_t cnt = s[(r + 1) * nx] - s[r * nx];
        counts[gi] = (cnt + kUnit - 1) / kUnit;
    }
}

__global__ void work_fill_kernel(int m, int64_t nrows, int nx, const uint32_t* __restrict__ cs,
                                 int64_t ncells, const uint32_t* __restrict__ off,
                                 WorkItem* __restrict__ units) {
    const int64_t total = nrows * (int64_t)m;
    for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(gi / nrows);
        const int64_t r = gi - (int64_t)k * nrows;
        const uint32_t* s = cs + (int64_t)k * (ncells + 1);
        const uint32_t b = s[r * nx], cnt = s[(r + 1) * nx] - b;
        const uint32_t o = off[gi];
        for (uint32_t g = 0; g * kUnit < cnt; ++g) {
            WorkItem w;
            w.real = (uint32_t)k;
            w.row = (uint32_t)r;
            w.c_begin = b + g * kUnit;
            w.c_count = min((uint32_t)kUnit, cnt - g * kUnit);
            units[o + g] = w;
        }
    }
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

cudaError_t launch_keys_observed(const double* x, const double* y, const double* t, int64_t n,
                                 const Grid& g, uint32_t* key, uint32_t* rank,
                                 uint32_t* cell_count, int* bad_flag, cudaStream_t st) {
    keys_observed_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(
        x, y, t, n, grid_dev(g), g.x1, g.y1, g.t1, key, rank, cell_count, bad_flag);
    return cudaGetLastError();
}

cudaError_t launch_validate(const double* x, const double* y, const double* t, int64_t n,
                            const double box[6], int* bad_flag, cudaStream_t st) {
    validate_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(x, y, t, n, box[0], box[1],
                                                                 box[2], box[3], box[4], box[5],
                                                                 bad_flag);
    return cudaGetLastError();
}

cudaError_t launch_gen_csr(int64_t n, int m, const uint64_t* seeds, const uint32_t* sims,
                           const Grid& g, double* x, double* y, double* t, uint32_t* key,
                           uint32_t* rank, uint32_t* cell_count, cudaStream_t st, Polygon poly,
                           unsigned long long* err) {
    gen_csr_kernel<<<grid_for(n * (int64_t)m, kThreads), kThreads, 0, st>>>(
        n, m, seeds, sims, grid_dev(g), g.x1, g.y1, g.t1, g.ncells, x, y, t, key, rank,
        cell_count, poly, err);
    return cudaGetLastError();
}

__global__ void poly_validate_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                     int64_t n, Polygon poly, int* __restrict__ bad) {
    int local = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        local |= !poly_contains(x[i], y[i], poly.vx, poly.vy, poly.nv);
    if (__any_sync(0xffffffffu, local) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

cudaError_t launch_poly_validate(const double* x, const double* y, int64_t n, Polygon poly,
                                 int* bad, cudaStream_t st) {
    poly_validate_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(x, y, n, poly, bad);
    return cudaGetLastError();
}

// One thread per bucket: the edges whose closest point lies within `reach` of the bucket's
// centre, in edge order (FP64).  A circle of radius r around a point of the bucket meets only
// edges within r + half the bucket's diagonal of that centre, so with reach above the largest
// pair radius plus half the diagonal the list holds every edge the bucket's circles can cross.
__global__ void poly_bucket_kernel(Polygon poly, double x0, double y0, double ox, double oy,
                                   double bs, int nx, int ny, double reach,
                                   uint8_t* __restrict__ list) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nx * ny) return;
    const double cx = x0 + ox + ((b % nx) + 0.5) * bs, cy = y0 + oy + ((b / nx) + 0.5) * bs;
    uint8_t* L = list + (size_t)b * kPolyBucketBytes;
    int cnt = 0;
    for (int k = 0; k < poly.nv; ++k) {
        const int k1 = k + 1 < poly.nv ? k + 1 : 0;
        const double ax = poly.vx[k] - cx, ay = poly.vy[k] - cy;
        const double dx = poly.vx[k1] - poly.vx[k], dy = poly.vy[k1] - poly.vy[k];
        const double len2 = dx * dx + dy * dy;
        const double s = len2 > 0.0 ? fmin(1.0, fmax(0.0, -(ax * dx + ay * dy) / len2)) : 0.0;
        const double ex = ax + s * dx, ey = ay + s * dy;
        if (ex * ex + ey * ey <= reach * reach) {
            if (cnt == kPolyBucketCap) {
                cnt = 255;
                break;
            }
            L[1 + cnt++] = (uint8_t)k;
        }
    }
    L[0] = (uint8_t)cnt;
}

cudaError_t launch_poly_buckets(Polygon poly, double x0, double y0, double ox, double oy,
                                double bs, int nx, int ny, double reach, uint8_t* list,
                                cudaStream_t st) {
    poly_bucket_kernel<<<(nx * ny + 127) / 128, 128, 0, st>>>(poly, x0, y0, ox, oy, bs, nx, ny,
                                                              reach, list);
    return cudaGetLastError();
}

int feistel_bits(int64_t n) {
    int b = 2;
    while (((int64_t)1 << b) < n) b += 2;
    return b;
}

cudaError_t launch_gen_resample(int method, int64_t n, int m, const uint64_t* seeds,
                                const uint32_t* sims, const Grid& g, const double* x0,
                                const double* y0, const double* t0, double* x, double* y,
                                double* t, uint32_t* key, uint32_t* rank, uint32_t* cell_count,
                                unsigned long long* err, cudaStream_t st) {
    gen_resample_kernel<<<grid_for(n * (int64_t)m, kThreads), kThreads, 0, st>>>(
        method, n, m, feistel_bits(n), seeds, sims, grid_dev(g), g.ncells, x0, y0, t0, x, y, t,
        key, rank, cell_count, err);
    return cudaGetLastError();
}

int64_t scan_tmp_words(int64_t count) {
    int64_t words = 0;
    while (count > kTile) {
        const int64_t tiles = (count + kTile - 1) / kTile;
        words += 2 * tiles;  // tile sums and their scanned offsets
        count = tiles;
    }
    return words + 1;
}

cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t count,
                                  uint32_t* tmp, int64_t tmp_words, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int64_t tiles = (count + kTile - 1) / kTile;
    if (tiles == 1) {
        scan_tiles_kernel<<<1, kThreads, 0, st>>>(in, out, count, nullptr);
        return cudaGetLastError();
    }
    if (tmp_words < 2 * tiles) return cudaErrorInvalidValue;
    uint32_t* sums = tmp;
    uint32_t* offs = tmp + tiles;
    scan_tiles_kernel<<<(unsigned)tiles, kThreads, 0, st>>>(in, out, count, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_exclusive_scan(sums, offs, tiles, tmp + 2 * tiles, tmp_words - 2 * tiles, st);
    if (e != cudaSuccess) return e;
    scan_add_kernel<<<(unsigned)tiles, kThreads, 0, st>>>(out, count, offs);
    return cudaGetLastError();
}

cudaError_t launch_scatter(int m, int64_t n, const Grid& g, const double* x, const double* y,
                           const double* t, const uint32_t* key, const uint32_t* rank,
                           const uint32_t* start_global, const uint8_t* mask_in, double* X,
                           double* Y, double* T, float4* P, float2* Plo, uint8_t* mask_out,
                           float tan_rel, float tan_abs, float fast_abs, float* F, int64_t nF,
                           double2* stage, cudaStream_t st, Polygon poly, bool mask_all,
                           const double* h_in, double* H, int slot0) {
    if (stage == nullptr) return cudaErrorInvalidValue;
    ScatterGrid s;
    s.qX = g.qX;
    s.inv_qX = 1.0 / (double)g.qX;
    s.nF = nF;
    s.poly = poly;
    s.mask_all = mask_all ? 1 : 0;
    s.x1 = g.x1;
    s.y1 = g.y1;
    s.t1 = g.t1;
    s.tan_rel = tan_rel;
    s.tan_abs = tan_abs;
    s.fast_abs = fast_abs;
    s.nx = g.nx;
    s.ny = g.ny;
    s.x0 = g.x0;
    s.y0 = g.y0;
    s.t0 = g.t0;
    s.cw = g.cw;
    s.ch = g.ch;
    s.cd = g.cd;
    s.qx = g.qx;
    s.qy = g.qy;
    s.qt = g.qt;
    s.inv_qx = 1.0 / (double)g.qx;
    s.inv_qy = 1.0 / (double)g.qy;
    s.inv_qt = 1.0 / (double)g.qt;
    stage_kernel<<<grid_for(n * (int64_t)m, kThreads), kThreads, 0, st>>>(
        m, n, g.ncells, x, y, t, key, rank, start_global, slot0, stage);
    records_kernel<<<grid_for(n * (int64_t)m, kThreads), kThreads, 0, st>>>(
        m, n, s, stage, mask_in, X, Y, T, P, Plo, mask_in ? mask_out : nullptr, h_in,
        h_in ? H : nullptr, F, slot0);
    return cudaGetLastError();
}

cudaError_t launch_intensity_lookup(const double* x, const double* y, const double* t,
                                    int64_t count, const double box[6], Intensity in, double* h,
                                    unsigned long long* zero, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    IntensityBox b;
    b.x0 = box[0];
    b.x1 = box[1];
    b.y0 = box[2];
    b.y1 = box[3];
    b.t0 = box[4];
    b.t1 = box[5];
    intensity_lookup_kernel<<<grid_for(count, kThreads), kThreads, 0, st>>>(x, y, t, count, b,
                                                                            in, h, zero);
    return cudaGetLastError();
}

cudaError_t launch_gen_inhom(int64_t n, int m, const uint64_t* seeds, const uint32_t* sims,
                             const Grid& g, Intensity in, double* x, double* y, double* t,
                             double* h, uint32_t* key, uint32_t* rank, uint32_t* cell_count,
                             cudaStream_t st) {
    gen_inhom_kernel<<<grid_for(n * (int64_t)m, kThreads), kThreads, 0, st>>>(
        n, m, seeds, sims, grid_dev(g), g.x1, g.y1, g.t1, g.ncells, in, x, y, t, h, key, rank,
        cell_count);
    return cudaGetLastError();
}

cudaError_t launch_cell_starts(int m, int64_t n, int64_t ncells, const uint32_t* start_global,
                               uint32_t* cell_start, cudaStream_t st) {
    cell_starts_kernel<<<grid_for((ncells + 1) * m, kThreads), kThreads, 0, st>>>(
        m, n, ncells, start_global, cell_start);
    return cudaGetLastError();
}

cudaError_t launch_work_counts(int m, const Grid& g, const uint32_t* cell_start,
                               uint32_t* counts, cudaStream_t st) {
    const int64_t nrows = (int64_t)g.ny * g.nt;
    work_counts_kernel<<<grid_for(nrows * m + 1, kThreads), kThreads, 0, st>>>(
        m, nrows, g.nx, cell_start, g.ncells, counts);
    return cudaGetLastError();
}

cudaError_t launch_work_fill(int m, const Grid& g, const uint32_t* cell_start,
                             const uint32_t* unit_off, WorkItem* units, cudaStream_t st) {
    const int64_t nrows = (int64_t)g.ny * g.nt;
    work_fill_kernel<<<grid_for(nrows * m, kThreads), kThreads, 0, st>>>(
        m, nrows, g.nx, cell_start, g.ncells, unit_off, units);
    return cudaGetLastError();
}

}  // namespace stk
