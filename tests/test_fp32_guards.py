"""The FP32 directional path decides a pair's sector in FP32 only outside a guard band and
leaves the rest to FP64.  This test emulates, with numpy FP32 arithmetic, the device's point
representation (x: the offset from the box's x0 rounded to the quantum qX = 2^-24 P_W, P_W the
power of two >= the box width; y: the offset from the cell origin rounded to q = 2^-22 P, P the
power of two >= the cell side; FP32 low parts) and its sector test, on offsets placed
adversarially close to the sector boundaries and to the axis at angle 0 / pi, at projected-size
coordinates, and checks that whenever the FP32 test clears its guards the sector equals the
one the reference FP64 arithmetic gives.  It also checks that the guards leave almost every
random pair to FP32."""
import math

import numpy as np
import pytest

f32 = np.float32


def _pow2_at_least(v):
    return 2.0 ** math.ceil(math.log2(v))


def _rep(v, lo, side, nc):
    """Cell index, FP32 hi part and FP32 low part of coordinates v (as the scatter kernel)."""
    c = np.clip(np.floor((v - lo) * (1.0 / side)), 0, nc - 1)
    o = v - (lo + c * side)
    q = _pow2_at_least(side) * 2.0 ** -22
    hi = np.rint(o * (1.0 / q)) * q
    return c, hi.astype(f32), (o - hi).astype(f32), q


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def _sectors(n_sec, dx, dy, bx, by):
    flip = ~((dy > 0) | ((dy == 0) & (dx > 0)))
    dx = np.where(flip, -dx, dx)
    dy = np.where(flip, -dy, dy)
    return dx, dy


@pytest.mark.parametrize("n_sec,x0", [(8, 5.0e5), (6, 0.0), (3, 3.3e6)])
def test_sector_guard_is_sound(n_sec, x0):
    rng = np.random.default_rng(n_sec)
    s_max, fs = 1000.0, 2
    W = H = 49_999.37  # a cell side that is not a multiple of the quantum
    y0 = x0 + 1234.5
    nx = ny = int(W // (s_max / fs))
    cw = W / nx
    N = 400_000
    m = rng.integers(0, n_sec, N)  # boundary index (0: the axis at angle 0 / pi)
    eps = np.exp(rng.uniform(math.log(1e-13), math.log(1e-3), N)) * rng.choice([-1, 1], N)
    eps[:2000] = 0.0
    ang = m * math.pi / n_sec + eps + np.where(rng.random(N) < 0.5, 0.0, math.pi)
    r = rng.uniform(0.0, s_max, N)
    r[2000:2100] = 0.0
    xi = x0 + s_max + rng.uniform(0, W - 2 * s_max, N)
    yi = y0 + s_max + rng.uniform(0, H - 2 * s_max, N)
    xj = xi - r * np.cos(ang)
    yj = yi - r * np.sin(ang)
    # reference: FP64 offset, upper half plane, count of boundaries with cross >= 0
    bx64 = np.array([math.cos(k * math.pi / n_sec) for k in range(1, n_sec)])
    by64 = np.array([math.sin(k * math.pi / n_sec) for k in range(1, n_sec)])
    dx64, dy64 = _sectors(n_sec, xi - xj, yi - yj, bx64, by64)
    k64 = ((bx64[None, :] * dy64[:, None] - by64[None, :] * dx64[:, None]) >= 0).sum(axis=1)
    k64 = np.where((xi - xj == 0) & (yi - yj == 0), 0, k64)
    # device: FP32 accurate offset from hi + lo parts, FP32 boundaries, guards
    # x relative to the box (the filter's hi part, quantum qX = 2^-24 P_W, and its remainder);
    # y relative to the point's cell, the centre moved into the neighbour's cell frame
    qX = _pow2_at_least(W) * 2.0 ** -24
    oxi, oxj = xi - x0, xj - x0
    hxi = (np.rint(oxi / qX) * qX).astype(f32)
    hxj = (np.rint(oxj / qX) * qX).astype(f32)
    lxi = (oxi - hxi.astype(np.float64)).astype(f32)
    lxj = (oxj - hxj.astype(np.float64)).astype(f32)
    cyi, hyi, lyi, qy = _rep(yi, y0, cw, ny)
    cyj, hyj, lyj, _ = _rep(yj, y0, cw, ny)
    cwq = f32(np.rint(cw / qy) * qy)
    cwl = f32(cw - np.rint(cw / qy) * qy)
    dcy = (cyi - cyj).astype(f32)
    cwq_v, cwl_v = np.full(N, cwq, f32), np.full(N, cwl, f32)
    dx = ((hxi - hxj).astype(f32) + (lxi - lxj).astype(f32)).astype(f32)
    dy = ((_fma32(dcy, cwq_v, hyi) - hyj).astype(f32) +
          _fma32(dcy, cwl_v, (lyi - lyj).astype(f32))).astype(f32)
    q = max(qX, qy)
    big = max(abs(x0), abs(x0 + W), abs(y0), abs(y0 + H))
    sec_g = f32(1.0e-6 * s_max + 1.0e-6 * q + 4.0e-16 * big + 1e-30)
    sec_gd = f32(1.0e-6 * q + 4.0e-16 * big + 1e-30)
    und = np.abs(dy) <= sec_gd
    dxf, dyf = _sectors(n_sec, dx, dy, None, None)
    k32 = np.zeros(N, int)
    for bxm, bym in zip(bx64.astype(f32), by64.astype(f32)):
        t = (bym * dxf).astype(f32)
        cr = (bxm.astype(np.float64) * dyf.astype(np.float64) - t.astype(np.float64)).astype(f32)
        und |= np.abs(cr) <= sec_g
        k32 += (cr > 0).astype(int)
    decided = ~und
    assert decided.sum() > 0.1 * N  # many decisions close to a boundary are exercised
    bad = np.flatnonzero(decided & (k32 != k64))
    assert bad.size == 0, (bad[:5], k32[bad[:5]], k64[bad[:5]], eps[bad[:5]])
    # on random (non-adversarial) offsets the guards send very few pairs to FP64
    a2 = rng.uniform(0, 2 * math.pi, 50_000)
    r2 = rng.uniform(1.0, s_max, 50_000)
    c2 = np.abs(np.stack([np.cos(k * math.pi / n_sec) * r2 * np.sin(a2) -
                          np.sin(k * math.pi / n_sec) * r2 * np.cos(a2)
                          for k in range(1, n_sec)]))
    frac = np.mean((c2 <= sec_g).any(axis=0) | (np.abs(r2 * np.sin(a2)) <= sec_gd))
    assert frac < 1e-3


@pytest.mark.parametrize("x0,W,fs", [(5.0e5, 49_999.37, 2), (0.0, 50_000.0, 2),
                                     (3.3e6, 123_456.7, 3), (-7.5e4, 8_000.0, 1)])
def test_filter_distance_within_guard(x0, W, fs):
    """The pair filter's squared distance (x relative to the box, quantum qX = 2^-24 P_W, P_W
    the power of two >= the box width; y relative to the neighbour's cell, the centre moved
    into it; FP32 adds and a fused multiply-add, as the kernel) stays within half the guard
    band G of the reference FP64 squared distance, so every bin FP32 decides outside the band
    is the reference bin.  G restates the band of the job set-up: with eps_x = qX and
    eps_y = 2 q_y (plus 2^-50 of the coordinates), sp = s (1 + 1e-6) + eps_x + eps_y,
    G = 2 (2 sp (eps_x + eps_y) + eps_x^2 + eps_y^2 + 2^-22 sp^2) + 2^-48 sp^2."""
    rng = np.random.default_rng(int(W) % 1000 + fs)
    H = W * 0.8
    y0 = x0 - 4321.0
    s_max = min(W, H) / 20
    ny = int(H // (s_max / fs))
    ch = H / ny
    N = 300_000
    r = s_max * np.sqrt(rng.uniform(0, 1.0, N))
    near = rng.random(N) < 0.5  # half of the pairs a hair from a threshold
    thr = s_max * rng.integers(1, 26, N) / 25
    r = np.where(near, thr + rng.uniform(-1e-3, 1e-3, N), r)
    ang = rng.uniform(0, 2 * math.pi, N)
    xi = x0 + rng.uniform(0, W, N)
    yi = y0 + s_max + rng.uniform(0, H - 2 * s_max, N)
    xj = np.clip(xi - r * np.cos(ang), x0, x0 + W)
    yj = yi - r * np.sin(ang)
    dx, dy = xi - xj, yi - yj
    d2_ref = dx * dx + dy * dy
    # filter representation
    qX = _pow2_at_least(W) * 2.0 ** -24
    hxi = (np.rint((xi - x0) / qX) * qX).astype(f32)
    hxj = (np.rint((xj - x0) / qX) * qX).astype(f32)
    cyi, hyi, _, qy = _rep(yi, y0, ch, ny)
    cyj, hyj, _, _ = _rep(yj, y0, ch, ny)
    chq = f32(np.rint(ch / qy) * qy)
    dcell = (cyi - cyj).astype(f32)
    keep = np.abs(dcell) <= fs
    yc = _fma32(-(-dcell), chq, hyi)  # centre moved into the neighbour's row frame
    dxf = (hxi + (-hxj)).astype(f32)
    dyf = (yc + (-hyj)).astype(f32)
    d2f = _fma32(dxf, dxf, (dyf * dyf).astype(f32))
    ex = qX + 2.0 ** -50 * (abs(x0) + abs(x0 + W))
    ey = 2 * qy + 2.0 ** -50 * (abs(y0) + abs(y0 + H))
    s = np.sqrt(np.maximum(d2_ref, 0))
    sp = s * (1 + 1e-6) + ex + ey
    G = 2 * (2 * sp * (ex + ey) + ex * ex + ey * ey + 2.0 ** -22 * sp * sp) + 2.0 ** -48 * sp * sp
    err = np.abs(d2f.astype(np.float64) - d2_ref)[keep]
    assert keep.sum() > N // 2
    assert (err <= 0.5 * G[keep]).all(), (err / G[keep]).max()
    # the x hi parts are exact FP32 multiples of qX over the whole box
    assert np.array_equal(hxi.astype(np.float64), np.rint((xi - x0) / qX) * qX)


def test_accurate_offset_is_antisymmetric():
    """The accurate offset of a pair (x: box-frame hi difference plus low difference; y: the
    other point moved into the neighbour's cell frame, the low parts' difference and the cell
    side's remainder rounded once) is the exact negation of the offset taken the other way
    round, so a weight does not depend on which point of the pair the traversal makes the
    centre (the counting sort does not fix the order of points inside a cell)."""
    rng = np.random.default_rng(4)
    N = 200_000
    qX, qy = 2.0 ** -8, 2.0 ** -12
    hxi, hxj = (rng.integers(0, 2**23, N) * qX).astype(f32), (rng.integers(0, 2**23, N) * qX).astype(f32)
    lxi, lxj = (rng.uniform(-qX / 2, qX / 2, N)).astype(f32), (rng.uniform(-qX / 2, qX / 2, N)).astype(f32)
    # close pairs across cell boundaries (the hi part of the offset is small), where the low
    # parts decide the last bits
    dcy = rng.integers(-3, 4, N).astype(f32)
    chq = np.full(N, f32(2.0 ** 21 * qy / 4))
    hyi = (rng.integers(0, 2**19, N) * qy).astype(f32)
    hyj = (hyi.astype(np.float64) + dcy.astype(np.float64) * chq + rng.integers(-64, 65, N) * qy
           ).astype(f32)
    lyi, lyj = (rng.uniform(-qy / 2, qy / 2, N)).astype(f32), (rng.uniform(-qy / 2, qy / 2, N)).astype(f32)
    chl = rng.uniform(-qy / 2, qy / 2, N).astype(f32)  # the cell side's remainder

    def off(hxa, lxa, hya, lya, hxb, lxb, hyb, lyb, dc, fused=True):
        dx = ((hxa + (-hxb)).astype(f32) + (lxa - lxb).astype(f32)).astype(f32)
        lo = (_fma32(dc, chl, (lya - lyb).astype(f32)) if fused else
              (_fma32(dc, chl, lya) - lyb).astype(f32))
        dy = ((_fma32(dc, chq, hya) + (-hyb)).astype(f32) + lo).astype(f32)
        return dx, dy

    dx1, dy1 = off(hxi, lxi, hyi, lyi, hxj, lxj, hyj, lyj, dcy)
    dx2, dy2 = off(hxj, lxj, hyj, lyj, hxi, lxi, hyi, lyi, -dcy)
    assert np.array_equal(dx1, -dx2) and np.array_equal(dy1, -dy2)
    # rounding the low part in two steps (each point's remainder moved separately) is not
    # antisymmetric: the reason for the single rounding
    _, e1 = off(hxi, lxi, hyi, lyi, hxj, lxj, hyj, lyj, dcy, fused=False)
    _, e2 = off(hxj, lxj, hyj, lyj, hxi, lxi, hyi, lyi, -dcy, fused=False)
    assert not np.array_equal(e1, -e2)
