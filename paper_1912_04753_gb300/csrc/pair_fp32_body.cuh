// Body of the FP32 pair kernels (pair.cu): one job's realizations [0, m) in a block.  It is
// included inside pair_fp32_kernel and pair_fp32_fused_kernel, which define the names it uses:
// the template parameters EVEN, EDGE, POLY, VAR and CALLER (see exact_inline); the job's constants `pc` (the kernel
// parameters themselves in the single-job kernel, so that its scalars are constant-bank
// operands; a shared-memory copy in the fused kernel) and their device copy `gpc`; m, rb,
// units, unit_off, counters, acc, xq, reps; the dynamic shared memory `smem_raw` viewed as
// `sm` (Smem32, whose pc holds at least the indexed tables and bands before `s2`); tid, lane,
// warp.  Compiled as part of each kernel rather than called, the single-job kernel keeps the
// code and register allocation of a kernel written out in full (a shared device function
// taking these by reference measured 2% slower there).  Adds the job's candidate count to
// acc.stats[0].
{
    WarpSm& ws = sm.w[warp];
    const int nbins = pc.nbins;
    const size_t hist_off = (sizeof(Smem32) + 15) & ~size_t(15);
    // per replica: he [nbins] u64, then for the inhomogeneous K hf and hw [nbins] u64, then hc
    // [nbins] u32 and (otherwise) hh [nbins] u32
    unsigned long long* he = reinterpret_cast<unsigned long long*>(smem_raw + hist_off);
    unsigned long long* hf = he + (size_t)reps * nbins;
    unsigned long long* hw = hf + (size_t)reps * nbins;
    uint32_t* hc = reinterpret_cast<uint32_t*>(VAR == kVarInh ? hw + (size_t)reps * nbins : hf);
    uint32_t* hh = hc + (size_t)reps * nbins;
    for (int i = tid; i < reps * nbins; i += kBlock) {
        hc[i] = 0;
        he[i] = 0;
        if (VAR == kVarInh) {
            hf[i] = 0;
            hw[i] = 0;
        } else {
            hh[i] = 0;
        }
    }
    // In a polygon study area the cost of a work unit varies so much (units along the outline
    // weigh many times the others) that a block barrier at the end of each realization left its
    // warps waiting for the slowest: there, realizations of either parity have their own
    // histogram set (a second set follows the first) and cursor, the last warp done with a
    // realization flushes its set, claims the block's first tile of the realization two on and
    // marks the slot ready for it, and a warp waits only for its next realization's slot.
    const size_t set_bytes = (size_t)reps * nbins * 16;
    if (POLY) {
        uint32_t* s1 = reinterpret_cast<uint32_t*>(smem_raw + hist_off + set_bytes);
        for (size_t i = tid; i < set_bytes / 4; i += kBlock) s1[i] = 0u;
        if (tid == 0) {
            sm.pcur[0] = (unsigned long long)atomicAdd(&counters[0], 1u) << 32;
            sm.pcur[1] = m > 1 ? (unsigned long long)atomicAdd(&counters[1], 1u) << 32 : 0ull;
            sm.pdone[0] = sm.pdone[1] = 0;
            sm.pready[0] = 0;
            sm.pready[1] = 1;
        }
    }
    WarpCtx w;
    w.hc = hc + (warp % reps) * nbins;
    w.hh = hh + (warp % reps) * nbins;
    w.he = he + (warp % reps) * nbins;
    w.hf = hf + (warp % reps) * nbins;
    w.hw = hw + (warp % reps) * nbins;
    w.H = nullptr;
    w.Plok = nullptr;
    w.q2n = 0;
    w.deep = false;
    w.pa = &sm.pc;
    if (POLY) {
        w.exlo = acc.exc_lo;
        w.exhi = acc.exc_hi;
    }
    const int64_t n = rb.n;
    const int nx = pc.g.nx, ny = pc.g.ny, nt = pc.g.nt, fs = pc.g.fs, ft = pc.g.ft;
    const int64_t nrows = (int64_t)ny * nt;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t tile = pc.tile_units;  // >= 1 (host)
    unsigned long long n_cand = 0;
    uint64_t since_flush = 0;  // candidates this warp added since it last flushed (uniform)
    __syncthreads();

    for (int k = 0; k < m; ++k) {
        uint32_t ubeg = unit_off[(int64_t)k * nrows], uend = unit_off[(int64_t)(k + 1) * nrows];
        shard_units(rb, unit_off, nrows, k, &ubeg, &uend);
        const uint32_t ntiles = (uend - ubeg + tile - 1) / tile;
        const int64_t base = (int64_t)k * n;
        const uint32_t* cs = rb.cell_start + (int64_t)k * (rb.ncells + 1);
        const float4* Pk = rb.P + 2 * base;
        w.Pk = Pk;
        w.Ek = Pk + n;
        w.NX = rb.F + (int64_t)k * 3 * rb.nF;
        w.NY = w.NX + rb.nF;
        w.real = (uint32_t)k;
        w.Plok = rb.Plo + base;
        if (VAR == kVarInh) w.H = rb.H + base;
        w.mk = (rb.mask != nullptr && (rb.mask_all || k == 0))
                   ? rb.mask + (rb.mask_all ? base : 0)
                   : nullptr;
        if (POLY) {
            // wait (bounded) until this realization's slot is flushed and its cursor claimed
            const int slot = k & 1;
            if (lane == 0) {
                int spin = 0;
                while (*reinterpret_cast<volatile int*>(&sm.pready[slot]) != k) {
                    if (++spin > kSpinLimit) {
                        atomicAdd(&acc.stats[4], 1ull);  // never expected: the flusher runs
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __syncwarp();
            __threadfence_block();
            const size_t so = slot ? set_bytes : 0;
            unsigned long long* hes = reinterpret_cast<unsigned long long*>(
                smem_raw + hist_off + so);
            uint32_t* hcs = reinterpret_cast<uint32_t*>(hes + (size_t)reps * nbins);
            w.he = hes + (warp % reps) * nbins;
            w.hc = hcs + (warp % reps) * nbins;
            w.hh = hcs + (size_t)reps * nbins + (warp % reps) * nbins;
            since_flush = 0;
        } else {
            if (tid == 0) sm.cursor = (unsigned long long)atomicAdd(&counters[k], 1u) << 32;
            __syncthreads();
        }
        unsigned long long* cursor = POLY ? &sm.pcur[k & 1] : &sm.cursor;
        for (;;) {
            const uint32_t ui = next_unit(cursor, &counters[k], ubeg, uend, tile, ntiles,
                                          lane, acc.stats, pc.never_publish != 0);
            if (ui == kNoUnit) break;
            const WorkItem wi = units[ui];
            w.c_begin = wi.c_begin;
            const int cy = (int)(wi.row % (uint32_t)ny), ct = (int)(wi.row / (uint32_t)ny);
            if (POLY) w.cy = cy;
            // centres: one per lane
            const bool valid = lane < (int)wi.c_count;
            const uint32_t myi = wi.c_begin + (valid ? lane : 0);
            const float4 p = Pk[myi];
            const float4 pe = w.Ek[myi];
            const float2 plo = rb.Plo[base + myi];
            const int cx = __float_as_int(p.w);
            // x: the box-frame hi part (with plo.x its remainder); y, t: the cell frame
            ws.cen_a[lane] = make_float4(-w.NX[myi], p.y, p.z, pe.w);
            ws.cen_b[lane] = make_float4(plo.x, plo.y, pe.x, pe.y);
            ws.cen_te[lane] = pe.z;
            if (VAR == kVarInh) ws.cen_h[lane] = (float)w.H[myi];
            const uint32_t fl = w.mk == nullptr ? 3u : (uint32_t)w.mk[myi];
            w.onA = __ballot_sync(0xffffffffu, valid && (fl & 1u));
            w.onB = __ballot_sync(0xffffffffu, valid && (fl & 2u));
            const float cut2 = valid ? pc.s2_cut : -1.0f;  // idle lanes never qualify
            const float ucut = pc.u_cut;
            const int cxa = __reduce_min_sync(0xffffffffu, valid ? cx : 0x7fffffff);
            const int cxb = __reduce_max_sync(0xffffffffu, valid ? cx : -1);
            const int wb = min(nx - 1, cxb + fs);
            // units whose whole neighbourhood is deep inside the box skip the weight logic
            w.deep = EDGE && max(0, cxa - fs) >= pc.deep_x[0] && wb <= pc.deep_x[1] &&
                     cy - fs >= pc.deep_y[0] && cy + fs <= pc.deep_y[1] &&
                     ct >= pc.deep_t[0] && ct + ft <= pc.deep_t[1];
            // the filter's copy of the coordinates (negated hi parts; x relative to the box)
            const float* NXk = rb.F + (int64_t)k * 3 * rb.nF;
            const float* NYk = NXk + rb.nF;
            const float* NTk = NYk + rb.nF;
            const float xcb = -NXk[myi];  // the centre's x in the box frame
            const float2 xc2 = make_float2(xcb, xcb);
            __syncwarp();
            uint32_t tail = 0;
            // rows from the centres' own row onward in key order (t major, y minor); the cells
            // wa .. wb of a row are one contiguous run of points in one coordinate frame (x
            // relative to the box, y and t relative to the row's cell origin), scanned four
            // points at a time
            for (int dt = 0; dt <= ft; ++dt) {
                const int rt = ct + dt;
                if (rt >= nt) break;
                const float tc = fmaf((float)(-dt), pc.g.cdq, p.z);
                const float2 tc2 = make_float2(tc, tc);
                for (int dy = (dt == 0 ? 0 : -fs); dy <= fs; ++dy) {
                    const int ry = cy + dy;
                    if (ry < 0 || ry >= ny) continue;
                    const bool own = (dt == 0) & (dy == 0);
                    // in the own row only neighbours after the centre (sorted index > myi),
                    // all of them after the unit's first centre
                    const int wa = own ? cxa : max(0, cxa - fs);
                    const int64_t rowkey = ((int64_t)rt * ny + ry) * nx;
                    const uint32_t J1 = cs[rowkey + wb + 1];
                    const uint32_t jstart = own ? wi.c_begin + 1u : cs[rowkey + wa];
                    if (jstart >= J1) continue;
                    // first index this lane may pair with; from jfull on no lane's bound binds
                    const uint32_t jmin = own ? myi + 1u : jstart;
                    const uint32_t jfull = own ? wi.c_begin + (uint32_t)kUnit : jstart;
                    const float yc = fmaf((float)(-dy), pc.g.chq, p.y);
                    const float2 yc2 = make_float2(yc, yc);
                    const uint32_t meta = (uint32_t)lane | ((uint32_t)(fs - dy) << 8);
                    if (valid && J1 > jmin) n_cand += J1 - jmin;
                    since_flush += 32ull * (J1 - jstart);
                    for (uint32_t j = jstart & ~3u; j < J1; j += 4) {
                        // four consecutive neighbours per step, one float4 per axis
                        const float4 qx = *reinterpret_cast<const float4*>(NXk + j);
                        const float4 qy = *reinterpret_cast<const float4*>(NYk + j);
                        const float4 qt = *reinterpret_cast<const float4*>(NTk + j);
                        const float2 dxa = __fadd2_rn(xc2, make_float2(qx.x, qx.y));
                        const float2 dxb = __fadd2_rn(xc2, make_float2(qx.z, qx.w));
                        const float2 dya = __fadd2_rn(yc2, make_float2(qy.x, qy.y));
                        const float2 dyb = __fadd2_rn(yc2, make_float2(qy.z, qy.w));
                        const float2 dta = __fadd2_rn(tc2, make_float2(qt.x, qt.y));
                        const float2 dtb = __fadd2_rn(tc2, make_float2(qt.z, qt.w));
                        const float2 d2a = __ffma2_rn(dxa, dxa, __fmul2_rn(dya, dya));
                        const float2 d2b = __ffma2_rn(dxb, dxb, __fmul2_rn(dyb, dyb));
                        bool k0 = (d2a.x <= cut2) & (fabsf(dta.x) <= ucut);
                        bool k1 = (d2a.y <= cut2) & (fabsf(dta.y) <= ucut);
                        bool k2 = (d2b.x <= cut2) & (fabsf(dtb.x) <= ucut);
                        bool k3 = (d2b.y <= cut2) & (fabsf(dtb.y) <= ucut);
                        if (j < jfull || j + 4u > J1) {  // the ends of the run
                            k0 &= (j >= jmin) & (j < J1);
                            k1 &= (j + 1u >= jmin) & (j + 1u < J1);
                            k2 &= (j + 2u >= jmin) & (j + 2u < J1);
                            k3 &= (j + 3u >= jmin) & (j + 3u < J1);
                        }
                        const uint32_t m0 = __ballot_sync(0xffffffffu, k0);
                        const uint32_t m1 = __ballot_sync(0xffffffffu, k1);
                        const uint32_t m2 = __ballot_sync(0xffffffffu, k2);
                        const uint32_t m3 = __ballot_sync(0xffffffffu, k3);
                        const uint32_t t1 = tail + (uint32_t)__popc(m0);
                        const uint32_t t2 = t1 + (uint32_t)__popc(m1);
                        const uint32_t t3 = t2 + (uint32_t)__popc(m2);
                        if (k0)
                            ws.ring[tail + __popc(m0 & lt)] =
                                make_uint4(__float_as_uint(d2a.x), __float_as_uint(fabsf(dta.x)),
                                           meta, j);
                        if (k1)
                            ws.ring[t1 + __popc(m1 & lt)] =
                                make_uint4(__float_as_uint(d2a.y), __float_as_uint(fabsf(dta.y)),
                                           meta, j + 1);
                        if (k2)
                            ws.ring[t2 + __popc(m2 & lt)] =
                                make_uint4(__float_as_uint(d2b.x), __float_as_uint(fabsf(dtb.x)),
                                           meta, j + 2);
                        if (k3)
                            ws.ring[t3 + __popc(m3 & lt)] =
                                make_uint4(__float_as_uint(d2b.y), __float_as_uint(fabsf(dtb.y)),
                                           meta, j + 3);
                        tail = t3 + (uint32_t)__popc(m3);
                        while (tail >= (uint32_t)kDrain) {
                            __syncwarp();
                            drain_pairs<EVEN, EDGE, POLY, VAR, CALLER>(pc, gpc, ws, rb, xq,
                                                                       kDrain, lane, lt, w);
                            __syncwarp();
                            const uint32_t rest = tail - kDrain;
                            uint4 v[4];
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                if ((uint32_t)(lane + 32 * c) < rest)
                                    v[c] = ws.ring[kDrain + lane + 32 * c];
                            __syncwarp();
#pragma unroll
                            for (int c = 0; c < 4; ++c)
                                if ((uint32_t)(lane + 32 * c) < rest) ws.ring[lane + 32 * c] = v[c];
                            __syncwarp();
                            tail = rest;
                        }
                    }
                }
            }
            drain_all<EVEN, EDGE, POLY, VAR, CALLER>(pc, gpc, ws, rb, xq, tail, lane, lt, w);
            if (since_flush >= kWarpFlush) {
                if (VAR == kVarInh)
                    warp_flush_inh(k, nbins, w.hc, w.he, w.hf, w.hw, acc, lane);
                else
                    warp_flush(k, nbins, w.hc, w.hh, w.he, acc, lane);
                since_flush = 0;
            }
        }
        if (POLY) {
            // done with realization k; the last warp of the block flushes the slot's set
            const int slot = k & 1;
            __threadfence_block();
            int last = 0;
            if (lane == 0) last = atomicAdd(&sm.pdone[slot], 1) == kWarps - 1;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence_block();
                const size_t so = slot ? set_bytes : 0;
                unsigned long long* hes = reinterpret_cast<unsigned long long*>(
                    smem_raw + hist_off + so);
                uint32_t* hcs = reinterpret_cast<uint32_t*>(hes + (size_t)reps * nbins);
                for (int r = 0; r < reps; ++r)
                    warp_flush(k, nbins, hcs + r * nbins, hcs + (size_t)(reps + r) * nbins,
                               hes + r * nbins, acc, lane);
                __syncwarp();
                if (lane == 0) {
                    sm.pdone[slot] = 0;
                    if (k + 2 < m)
                        sm.pcur[slot] = (unsigned long long)atomicAdd(&counters[k + 2], 1u) << 32;
                    __threadfence_block();
                    *reinterpret_cast<volatile int*>(&sm.pready[slot]) = k + 2;
                }
                __syncwarp();
            }
        } else {
            __syncthreads();
            // every warp of the block is done with realization k: add its histograms
            if (VAR == kVarInh)
                flush_hist_inh(k, nbins, reps, hc, he, hf, hw, acc);
            else
                flush_hist(k, nbins, reps, hc, he, acc, hh);
            since_flush = 0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
    if (lane == 0) atomicAdd(&acc.stats[0], n_cand);
}
