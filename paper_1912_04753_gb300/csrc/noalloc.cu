// stk_k_noalloc: observed K of one pattern without allocating any memory.
//
// Some callers cannot allocate device memory at the point where they need K: code that runs
// inside a caching allocator's reserved pool, inside a region where the host must not call
// cudaMalloc / cudaFree (they synchronise the device and would stall or break pipelined
// work), or inside an embedding that hands out only the buffers it owns.  This entry point
// takes the caller's device inputs and outputs and keeps every intermediate buffer in one
// statically sized device array that belongs to this library.
//
// Properties (also stated in include/stk.h):
//   - the array holds kScratchBytes on every GPU that loads the library, until the process
//     exits; the largest accepted pattern has kMaxPoints points and kMaxCells grid cells;
//   - the first call on a device looks up the array's device address (once per device);
//     make that first call before any stream capture;
//   - all calls share the array: concurrent calls, from several threads or on streams that
//     overlap on the GPU, race and must be serialised by the caller;
//   - no cudaMalloc, cudaFree or allocating library routine is called.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "stk.h"
#include "stk_internal.h"

using namespace stk;

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int64_t kMaxPoints = 262144;
constexpr int64_t kMaxCells = int64_t(1) << 20;
constexpr unsigned int kExactCap = 1u << 16;         // FP64 queue entries (overflow is exact)

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_dev[kMaxDevices];  // device address of g_scratch, per device
std::mutex g_scratch_mu;

int nofail(int code, const char* msg) {
    stk_note_error(code, msg);
    return code;
}

int nofail_cuda(cudaError_t e, const char* what) {
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof buf, "stk_k_noalloc: %s: %s", what, cudaGetErrorString(e));
    return nofail(STK_ECUDA, buf);
}

#define NK(expr, what)                                          \
    do {                                                        \
        cudaError_t e_ = (expr);                                \
        if (e_ != cudaSuccess) return nofail_cuda(e_, what);    \
    } while (0)

// The host-side name g_scratch is not a device address; look the address up once per device,
// with that device current.
int scratch_address(void** out) {
    int dev = 0;
    NK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return nofail(STK_ENODEV, "stk_k_noalloc: device index too large");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        NK(cudaGetSymbolAddress(&p, g_scratch), "cudaGetSymbolAddress");
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return STK_OK;
}

// Bump allocator over the static array (256-byte aligned slices).
struct Carve {
    unsigned char* base;
    size_t used;
    template <class T>
    T* take(size_t count) {
        const size_t off = (used + 255) & ~size_t(255);
        used = off + sizeof(T) * count;
        return reinterpret_cast<T*>(base + off);
    }
};

}  // namespace

extern "C" int stk_k_noalloc(const double* d_x, const double* d_y, const double* d_t, int64_t n,
                             const stk_box* box, const double* s, int cs, const double* tt,
                             int ct, int edge_mode, double* d_K, double* d_L, double* d_S,
                             int64_t* d_C, void* stream) {
    if (!d_x || !d_y || !d_t || !box || !s || !tt || !d_K || !d_L || !d_S || !d_C)
        return nofail(STK_EINVAL, "stk_k_noalloc: NULL argument");
    if (n < 2) return nofail(STK_EINVAL, "stk_k_noalloc: need n >= 2 points");
    if (n > kMaxPoints) {
        char buf[160];
        snprintf(buf, sizeof buf, "stk_k_noalloc: n = %lld exceeds the fixed scratch limit of %lld points",
                 (long long)n, (long long)kMaxPoints);
        return nofail(STK_EINVAL, buf);
    }
    if (edge_mode != STK_EDGE_NONE && edge_mode != STK_EDGE_ISOTROPIC)
        return nofail(STK_EINVAL, "stk_k_noalloc: unknown edge_mode");
    const double b6[6] = {box->x0, box->x1, box->y0, box->y1, box->t0, box->t1};
    if (!(box->x0 < box->x1 && box->y0 < box->y1 && box->t0 < box->t1))
        return nofail(STK_EINVAL, "stk_k_noalloc: box must satisfy x0<x1, y0<y1, t0<t1");
    char err[256];
    if (validate_thresholds(b6, s, cs, tt, ct, err, sizeof err)) return nofail(STK_EINVAL, err);
    Grid g;
    if (build_grid(b6, s[cs - 1], tt[ct - 1], n, 0, &g, err, sizeof err)) return nofail(STK_EINVAL, err);
    if (g.ncells > kMaxCells)
        return nofail(STK_EINVAL, "stk_k_noalloc: threshold grid too fine for the fixed scratch");
    PairConsts pc;
    build_pair_consts(g, n, s, cs, tt, ct, edge_mode, &pc);
    {  // failure-detection test hook, as in the handle's jobs (see PairConsts::never_publish)
        const char* np = getenv("STK_TEST_NEVER_PUBLISH");
        pc.never_publish = (np && atoi(np) != 0) ? 1 : 0;
    }
    const int nbins = cs * ct;
    const int64_t ncells = g.ncells, nrows = (int64_t)g.ny * g.nt;
    const int64_t units_max = nrows + n / kUnit + 1;

    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    Carve cv{reinterpret_cast<unsigned char*>(scratch), 0};
    PairConsts* d_pc = cv.take<PairConsts>(1);
    double* d_thr = cv.take<double>(2 * kMaxThr);
    uint32_t* key = cv.take<uint32_t>(n);
    uint32_t* rank = cv.take<uint32_t>(n);
    uint32_t* counts = cv.take<uint32_t>(ncells);
    uint32_t* start = cv.take<uint32_t>(ncells);
    const int64_t tmp_words = std::max(scan_tmp_words(ncells), scan_tmp_words(nrows + 1));
    uint32_t* scan_tmp = cv.take<uint32_t>(tmp_words);
    double* X = cv.take<double>(n);
    double* Y = cv.take<double>(n);
    double* T = cv.take<double>(n);
    float4* P = cv.take<float4>(2 * (n + 8));
    float2* Plo = cv.take<float2>(n);
    float* F = cv.take<float>(3 * filter_stride(n));
    double2* stage = cv.take<double2>(2 * n);
    uint32_t* cell_start = cv.take<uint32_t>(ncells + 1);
    uint32_t* ucount = cv.take<uint32_t>(nrows + 1);
    uint32_t* uoff = cv.take<uint32_t>(nrows + 1);
    WorkItem* units = cv.take<WorkItem>(units_max);
    uint32_t* counter = cv.take<uint32_t>(4);
    unsigned long long* acc_cnt = cv.take<unsigned long long>(nbins);
    unsigned long long* acc_lo = cv.take<unsigned long long>(nbins);
    unsigned long long* acc_hi = cv.take<unsigned long long>(nbins);
    unsigned long long* stats = cv.take<unsigned long long>(8);
    int64_t* selfp = cv.take<int64_t>(1);
    uint4* xq_e = cv.take<uint4>(kExactCap);
    unsigned int* xq_count = cv.take<unsigned int>(4);
    if (cv.used > kScratchBytes)
        return nofail(STK_EINVAL, "stk_k_noalloc: pattern and grid do not fit the fixed scratch");

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double thr[2 * kMaxThr] = {0};
    for (int a = 0; a < cs; ++a) thr[a] = s[a];
    for (int b = 0; b < ct; ++b) thr[kMaxThr + b] = tt[b];
    // pageable host sources: each copy has read its source when the call returns
    NK(cudaMemcpyAsync(d_pc, &pc, sizeof pc, cudaMemcpyHostToDevice, st), "constants");
    NK(cudaMemcpyAsync(d_thr, thr, sizeof thr, cudaMemcpyHostToDevice, st), "thresholds");
    // the array keeps the previous call's contents: clear everything that accumulates
    NK(cudaMemsetAsync(counts, 0, 4 * (size_t)ncells, st), "clear");
    NK(cudaMemsetAsync(counter, 0, 16, st), "clear");
    NK(cudaMemsetAsync(acc_cnt, 0, 8 * (size_t)nbins, st), "clear");
    NK(cudaMemsetAsync(acc_lo, 0, 8 * (size_t)nbins, st), "clear");
    NK(cudaMemsetAsync(acc_hi, 0, 8 * (size_t)nbins, st), "clear");
    NK(cudaMemsetAsync(stats, 0, 64, st), "clear");
    NK(cudaMemsetAsync(selfp, 0, 8, st), "clear");
    NK(cudaMemsetAsync(xq_count, 0, 16, st), "clear");

    NK(launch_keys_observed(d_x, d_y, d_t, n, g, key, rank, counts,
                            reinterpret_cast<int*>(stats + 3), st), "cell keys");
    NK(launch_exclusive_scan(counts, start, ncells, scan_tmp, tmp_words, st), "cell scan");
    NK(launch_scatter(1, n, g, d_x, d_y, d_t, key, rank, start, nullptr, X, Y, T, P, Plo, nullptr,
                      pc.tan_rel, pc.tan_abs, pc.fast_abs, F, filter_stride(n), stage, st),
       "scatter");
    NK(launch_cell_starts(1, n, ncells, start, cell_start, st), "cell starts");
    NK(launch_work_counts(1, g, cell_start, ucount, st), "work counts");
    NK(launch_exclusive_scan(ucount, uoff, nrows + 1, scan_tmp, tmp_words, st), "work scan");
    NK(launch_work_fill(1, g, cell_start, uoff, units, st), "work fill");
    int reps = 1, reps64 = 1;
    const size_t smem = pair_fp32_smem(nbins, &reps);
    NK(pair_kernels_configure(smem, pair_fp64_smem(nbins, &reps64)), "kernel configuration");
    int dev = 0, sms = 0;
    NK(cudaGetDevice(&dev), "cudaGetDevice");
    NK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device query");
    RealBatch rb;
    rb.P = P;
    rb.Plo = Plo;
    rb.F = F;
    rb.nF = filter_stride(n);
    rb.X = X;
    rb.Y = Y;
    rb.T = T;
    rb.cell_start = cell_start;
    rb.mask = nullptr;
    rb.n = n;
    rb.ncells = ncells;
    Accum acc;
    acc.cnt = acc_cnt;
    acc.exc_lo = acc_lo;
    acc.exc_hi = acc_hi;
    acc.stats = stats;
    ExactQueue xq;
    xq.e = xq_e;
    xq.count = xq_count;
    xq.cap = kExactCap;
    const int grid = pair_fp32_blocks_per_sm(smem) * sms;
    NK(launch_pair_fp32(pc, d_pc, pc.even_s && pc.even_t, edge_mode != 0, smem, reps, grid, 1, rb,
                        units, uoff, counter, acc, xq, st),
       "pair kernel");
    NK(launch_exact(d_pc, 4 * sms, rb, acc, xq, st), "FP64 queue");
    const double area = (box->x1 - box->x0) * (box->y1 - box->y0);
    const double nn = (double)n;
    const double coef = area * (box->t1 - box->t0) / (nn * (nn - 1.0));
    NK(launch_finalize(1, cs, ct, d_thr, d_thr + kMaxThr, coef, selfp, acc, d_K, d_L, d_S, d_C, st),
       "finalize");
    unsigned long long h_stats[8];
    NK(cudaMemcpyAsync(h_stats, stats, sizeof h_stats, cudaMemcpyDeviceToHost, st), "status");
    NK(cudaStreamSynchronize(st), "synchronise");
    if (h_stats[3]) return nofail(STK_EDOMAIN, "stk_k_noalloc: a point lies outside the study box");
    if (h_stats[2]) return nofail(STK_ECUDA, "stk_k_noalloc: internal consistency check failed");
    if (h_stats[4])
        return nofail(STK_ETIMEOUT,
                      "stk_k_noalloc: bounded waits for work in the pair kernel ran out; the "
                      "outputs are incomplete");
    return STK_OK;
}
