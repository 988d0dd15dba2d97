"""The FP32-guarded isotropic weight in a polygon study area (pair.cu, poly_share_f32 and
arc_half_angle_pair), emulated on the host with numpy FP32 arithmetic in the kernel's order:
pairs hi + lo of FP32 numbers for the centre's box-frame position (built from the records' hi
and low parts and a row origin, as the kernel builds it), the radius, the line distance h and
r - |h|, the arc half-angle psi = acos(|h| / r) and the crossing angles; the inside share as
2 pi I0 - sum(delta_c theta_c) over the crossings in any order; and the guards (tangency,
vertices, the choice of I0, the error bound).  Whenever the guards let a circle through, its
inside share must match the oracle's (Section 3: proportion of the circumference inside the
polygon, FP64) to the bound the kernel claims; and the guards must let nearly every circle near
the boundary through, spiky outlines with many crossings included."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_04753_gb300", "csrc")
f32 = np.float32
TWO_PI = 6.283185307179586
ARC_ERR = 3.0e-8  # kArcErrF32


def _fma(a, b, c):
    """fmaf: the product of two FP32 numbers is exact in FP64; one rounding to FP32 after the
    sum (a double rounding that can differ from the hardware's by an ulp in rare ties)."""
    return f32(float(a) * float(b) + float(c))


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def _two_prod(a, b):
    p = f32(a * b)
    return p, f32(float(a) * float(b) - float(p))  # exact: the FP64 product is exact


def _split(v):
    h = f32(v)
    return h, f32(v - float(h))


def _coefficients():
    sys.path.insert(0, CSRC)
    import fit_arc_poly

    c = fit_arc_poly.fit(9)
    c0h, c0l = _split(float(c[0]))
    return c.astype(f32), c0h, c0l


def _rsqrt(v):
    return f32(1.0 / math.sqrt(float(v)))


def _inv(v):
    """1 / v as the kernel forms it from the reciprocal square root of v^2 and a Newton step
    (the hardware's approximation taken as correctly rounded here)."""
    s = f32(v * v)
    ys = _rsqrt(s)
    return f32(ys * _fma(f32(f32(f32(-0.5) * s) * ys), ys, f32(1.5)))


def arc_pair(dh, dl, rh, rl, coef, y=None):
    """Emulation of arc_half_angle_pair: psi = acos(1 - d / r) as (hi, lo); y ~ 1 / rh."""
    c, c0h, c0l = coef
    y = _inv(rh) if y is None else y
    om0 = f32(dh * y)
    res = _fma(-om0, rh, dh)
    res = f32(f32(res + dl) - f32(om0 * rl))
    om1 = f32(res * y)
    ys = _rsqrt(om0)
    s0 = f32(om0 * ys)
    s0 = _fma(_fma(-s0, s0, om0), f32(f32(0.5) * ys), s0)
    s1 = f32(f32(_fma(-s0, s0, om0) + om1) * f32(f32(0.5) * ys))
    x = f32(f32(f32(1.0) - om0) - om1)
    p = c[9]
    for k in range(8, 0, -1):
        p = _fma(p, x, c[k])
    m, me = _two_prod(p, x)
    Ph, Pe = _two_sum(c0h, m)
    Pl = f32(f32(Pe + me) + c0l)
    ph = f32(s0 * Ph)
    pl = f32(_fma(s0, Ph, -ph) + _fma(s0, Pl, f32(s1 * Ph)))
    return ph, pl


class Frame:
    """The records' representation of a box and grid (index.cu, records_kernel): x relative to
    the box in a hi part on the quantum qX plus a low part, y relative to its cell row's origin
    (hi part on the quantum q_y, low part), rows of height ch = chq + chl."""

    def __init__(self, box, ny):
        self.x0, self.x1, self.y0, self.y1 = box
        W, H = self.x1 - self.x0, self.y1 - self.y0
        self.ny = ny
        self.ch = H / ny
        p2 = lambda v: 2.0 ** math.ceil(math.log2(v))  # noqa: E731
        self.qX = f32(math.ldexp(p2(W), -24))
        self.qy = f32(math.ldexp(p2(self.ch), -22))
        chq = round(self.ch / float(self.qy)) * float(self.qy)
        self.chq = f32(chq)
        self.chl = f32(self.ch - chq)
        acc_x = math.ldexp(float(self.qX), -24) + math.ldexp(abs(self.x0) + abs(self.x1), -50)
        acc_y = math.ldexp(float(self.qy), -22) + math.ldexp(abs(self.y0) + abs(self.y1), -50)
        ext = W + H
        self.acc = acc_x + acc_y
        # the host's poly_eh (stk.cu, run_job)
        self.eh = f32(2.0 * (2.0 * (acc_x + acc_y) + math.ldexp(ny * float(self.qy), -23) +
                             math.ldexp(ext, -43)) * 1.001)

    def centre(self, x, y):
        """(cxh, cxl, cyh, cyl) as the kernel forms them from the records."""
        oX = x - self.x0
        hX = f32(round(oX / float(self.qX)) * float(self.qX))
        lox = f32(oX - float(hX))
        row = min(self.ny - 1, max(0, int((y - self.y0) / self.ch)))
        origin = self.y0 + row * self.ch
        oy = y - origin
        hy = f32(round(oy / float(self.qy)) * float(self.qy))
        loy = f32(oy - float(hy))
        ro, roe = _two_prod(f32(row), self.chq)
        cyh, cye = _two_sum(ro, hy)
        cyl = f32(f32(cye + roe) + _fma(f32(row), self.chl, loy))
        return hX, lox, cyh, cyl


def tables(vx, vy, frame):
    """The host's per-edge table (stk.cu, stk_set_polygon) and the polygon's span."""
    nv = len(vx)
    out = []
    for k in range(nv):
        k1 = (k + 1) % nv
        ax, ay = vx[k] - frame.x0, vy[k] - frame.y0
        bx, by = vx[k1] - frame.x0, vy[k1] - frame.y0
        dx, dy = vx[k1] - vx[k], vy[k1] - vy[k]
        ln = math.sqrt(dx * dx + dy * dy)
        e = dict(a=_split(ax) + _split(ay), u=(f32(0),) * 4, phi=(f32(0), f32(0)), len=f32(0))
        if ln > 0:
            ux, uy = dx / ln, dy / ln
            phi = math.atan2(-ux, uy)
            if phi < 0:
                phi += TWO_PI
            e.update(u=_split(ux) + _split(uy), phi=_split(phi), len=f32(ln))
        box = []
        for lo, hi in ((min(ax, bx), max(ax, bx)), (min(ay, by), max(ay, by))):
            lf, hf = f32(lo), f32(hi)
            if float(lf) > lo:
                lf = np.nextafter(lf, f32(-np.inf))
            if float(hf) < hi:
                hf = np.nextafter(hf, f32(np.inf))
            box += [lf, hf]
        e["box"] = box
        out.append(e)
    span = f32(max(vx.max() - vx.min(), vy.max() - vy.min()) * (1.0 - 1e-6))
    return out, span


class Buckets:
    """The bucket lists (stk.cu, run_job; index.cu, poly_bucket_kernel): a grid over the
    polygon's bounding box (box frame) with side max(r_max / 2, larger side / 63.5), each bucket
    listing the edges within r_max + half its diagonal (plus margins) of its centre; 255 when
    more than 47 (then every edge is scanned)."""

    def __init__(self, vx, vy, frame, r_max):
        bb = (vx.min() - frame.x0, vx.max() - frame.x0, vy.min() - frame.y0, vy.max() - frame.y0)
        r_max = r_max * (1.0 + 1e-6)
        bw, bh = bb[1] - bb[0], bb[3] - bb[2]
        bs = max(0.5 * r_max, max(bw, bh) / 63.5)
        self.nx = max(1, min(64, math.ceil(bw / bs)))
        self.ny = max(1, min(64, math.ceil(bh / bs)))
        reach = r_max + 0.5 * math.sqrt(2.0) * bs * 1.001 + 1e-5 * (abs(bb[0]) + abs(bb[2]) +
                                                                   bw + bh)
        self.ox, self.oy, self.inv = f32(bb[0]), f32(bb[2]), f32(1.0 / bs)
        self.rmax = f32(r_max * (1.0 - 1e-6))
        nv = len(vx)
        self.lists = []
        for b in range(self.nx * self.ny):
            cx = frame.x0 + bb[0] + (b % self.nx + 0.5) * bs
            cy = frame.y0 + bb[2] + (b // self.nx + 0.5) * bs
            lst = []
            for k in range(nv):
                k1 = (k + 1) % nv
                ax, ay = vx[k] - cx, vy[k] - cy
                dx, dy = vx[k1] - vx[k], vy[k1] - vy[k]
                len2 = dx * dx + dy * dy
                t = min(1.0, max(0.0, -(ax * dx + ay * dy) / len2)) if len2 > 0 else 0.0
                ex, ey = ax + t * dx, ay + t * dy
                if ex * ex + ey * ey <= reach * reach:
                    lst.append(k)
            self.lists.append(lst if len(lst) <= 47 else None)

    def edges(self, cxh, cyh, rh, nv):
        bi = min(max(int(f32(f32(cxh - self.ox) * self.inv)), 0), self.nx - 1)
        bj = min(max(int(f32(f32(cyh - self.oy) * self.inv)), 0), self.ny - 1)
        lst = self.lists[bj * self.nx + bi]
        if lst is None or not rh <= self.rmax:
            return range(nv)
        return lst


def _sqrt_nr(v):
    y = _rsqrt(float(v) + 1e-30)
    s = f32(v * y)
    return _fma(_fma(-s, s, v), f32(f32(0.5) * y), s)


def share_f32(c, rh, rl, edges, span, ccw, eh, coef, buckets=None):
    """Emulation of poly_share_f32: (inside, outside, error bound) or None where it refuses
    (the edges of the centre's bucket list when `buckets` is given, else all)."""
    cxh, cxl, cyh, cyl = c
    inv_r = _inv(rh)
    k2h, k2l = f32(6.2831854820251465), f32(-1.7484555314695172e-07)
    kph, kpl = f32(3.1415927410125732), f32(-8.742277657347586e-08)
    m = f32(f32(f32(rh * f32(1e-5)) + f32(f32(1e-6) * f32(abs(cxh) + abs(cyh)))) + eh)
    x0, x1 = f32(f32(cxh - rh) - m), f32(f32(cxh + rh) + m)
    y0, y1 = f32(f32(cyh - rh) - m), f32(f32(cyh + rh) + m)
    band = f32(f32(f32(4.0) * eh) + f32(rh * f32(1e-12)))
    Sh = Sl = f32(0)
    a1, a1e, a1in, a2, z = (f32(40), f32(0)), f32(0), False, (f32(40), f32(0)), (f32(-1), f32(0))
    esum = emax = f32(0)
    bal = na = 0
    scan = range(len(edges)) if buckets is None else buckets.edges(cxh, cyh, rh, len(edges))
    for k in scan:
        e = edges[k]
        bx0, bx1, by0, by1 = e["box"]
        if bx0 > x1 or bx1 < x0 or by0 > y1 or by1 < y0:
            continue
        axh, axl, ayh, ayl = e["a"]
        uxh, uxl, uyh, uyl = e["u"]
        fxh, fxe = _two_sum(axh, -cxh)
        fyh, fye = _two_sum(ayh, -cyh)
        fxl = f32(fxe + f32(axl - cxl))
        fyl = f32(fye + f32(ayl - cyl))
        p1, q1 = _two_prod(fxh, uyh)
        p2, q2 = _two_prod(fyh, uxh)
        hs, he = _two_sum(p1, -p2)
        hl0 = f32(f32(he + f32(q1 - q2)) +
                  f32(_fma(fxh, uyl, f32(fxl * uyh)) - _fma(fyh, uxl, f32(fyl * uxh))))
        hh, hl = _two_sum(hs, hl0)
        neg = hh < 0
        if neg:
            hh, hl = -hh, -hl
        dh, de = _two_sum(rh, -hh)
        dl = f32(de + f32(rl - hl))
        dh, dl = _two_sum(dh, dl)
        if dh < -band:
            continue
        if dh <= band:
            return None
        v = f32(dh * f32(rh + hh))
        yt = _rsqrt(v)
        t0 = f32(v * yt)
        t = _fma(_fma(-t0, t0, v), f32(f32(0.5) * yt), t0)
        inv_t = f32(yt * f32(1.000001))
        u0 = -_fma(fxh, uxh, f32(fyh * uyh))
        ln = e["len"]
        eang = f32(f32(ARC_ERR) + f32(f32(f32(2.0) * eh) * inv_t))
        uerr = f32(f32(f32(f32(2.5e-7) * f32(abs(fxh) + abs(fyh))) + f32(f32(1.5e-7) * t)) +
                   f32(f32(f32(6.0e-8) * ln) +
                       f32(f32(f32(2.0) * eh) * f32(f32(rh * inv_t) + f32(1)))))
        psi = None
        for q in (-1, 1):
            u = _fma(f32(q), t, u0)
            if abs(u) <= uerr or abs(f32(u - ln)) <= uerr:
                return None
            if u < 0 or u >= ln:
                continue
            if psi is None:
                psi = arc_pair(dh, dl, rh, rl, coef, inv_r)
                ph0, pl0 = e["phi"]
                if neg:
                    bh, be = _two_sum(ph0, kph)
                    bl = f32(be + f32(pl0 + kpl))
                else:
                    bh, bl = ph0, pl0
            ph, pl = psi
            plus = (q > 0) != neg
            th, te = _two_sum(bh, ph if plus else -ph)
            tl = f32(te + f32(bl + (pl if plus else -pl)))
            th, tl = _two_sum(th, tl)
            if th < 0 or (th == 0 and tl < 0):  # the whole pair against 0 and 2 pi
                th, te = _two_sum(th, k2h)
                tl = f32(te + f32(tl + k2l))
                th, tl = _two_sum(th, tl)
            elif th > k2h or (th == k2h and tl >= k2l):
                th, te = _two_sum(th, -k2h)
                tl = f32(te + f32(tl - k2l))
                th, tl = _two_sum(th, tl)
            enter = (q > 0) == ccw
            sh, se = _two_sum(Sh, th if enter else -th)
            Sl = f32(Sl + f32(se + (tl if enter else -tl)))
            Sh = sh
            bal += 1 if enter else -1
            na += 1
            esum = f32(esum + eang)
            emax = max(emax, eang)
            if (th, tl) < a1:
                a2, a1, a1e, a1in = a1, (th, tl), eang, enter
            elif (th, tl) < a2:
                a2 = (th, tl)
            if (th, tl) > z:
                z = (th, tl)
    if na == 0:
        if not f32(f32(f32(2.0) * rh) * f32(1.0 + 1e-6)) < span:
            return None
        return f32(1), f32(0), 0.0
    if bal != 0:
        return None
    if not f32(a1[0] + a1[1]) > f32(a1e * f32(1.0001)):
        return None
    if not f32(f32(a2[0] - a1[0]) + f32(a2[1] - a1[1])) > f32(f32(a1e + emax) * f32(1.0001)):
        return None
    if not f32(f32(k2h - z[0]) + f32(k2l - z[1])) > f32(emax * f32(1.0001)):
        return None
    kih, kil = f32(0.15915493667125702), f32(6.4206382432985265e-09)
    i0 = not a1in
    ih, ie = _two_sum(k2h if i0 else f32(0), -Sh)
    il = f32(ie + f32((k2l if i0 else f32(0)) - Sl))
    oh, oe = _two_sum(f32(0) if i0 else k2h, Sh)
    ol = f32(oe + f32((f32(0) if i0 else k2l) + Sl))
    vh, ve = _two_prod(ih, kih)
    inside = f32(vh + f32(ve + _fma(ih, kil, f32(il * kih))))
    vh, ve = _two_prod(oh, kih)
    outside = f32(vh + f32(ve + _fma(oh, kil, f32(ol * kih))))
    bound = float(f32(esum * kih))
    if not (inside > 0 and f32(esum * kih) <= f32(f32(8.5e-7) * inside)):
        return None
    return inside, outside, bound


def _polygons():
    from paper_1912_04753_gb300 import workloads as wl

    star = wl.star_polygon(85, 5000.0, 3400.0, 5000.0, 5000.0, 1)
    smooth = wl.smooth_polygon(85, 3800.0, 5000.0, 5000.0, 3)
    rng = np.random.default_rng(3)
    ang = np.sort(rng.uniform(0, 2 * np.pi, 24))
    rad = rng.uniform(600.0, 1000.0, 24)
    poly24 = (1200.0 + rad * np.cos(ang), 1100.0 + rad * np.sin(ang))
    # a clockwise outline at projected coordinates
    vx, vy = wl.star_polygon(40, 2500.0, 1800.0, 5.0e5 + 3000.0, 3.3e6 + 3000.0, 5)
    projected = (vx[::-1].copy(), vy[::-1].copy())
    return {
        "star85": (star, 1000.0, (0.0, 10000.0, 0.0, 10000.0), 20),
        "smooth85": (smooth, 1000.0, (0.0, 10000.0, 0.0, 10000.0), 20),
        "poly24": (poly24, 300.0, (0.0, 2500.0, 0.0, 2500.0), 16),
        "projected40": (projected, 900.0, (5.0e5, 5.06e5, 3.3e6, 3.306e6), 12),
    }


def _setup(name):
    (vx, vy), r_max, box, ny = _polygons()[name]
    vx, vy = np.asarray(vx, np.float64), np.asarray(vy, np.float64)
    frame = Frame(box, ny)
    edges, span = tables(vx, vy, frame)
    ccw = float(np.sum(vx * np.roll(vy, -1) - np.roll(vx, -1) * vy)) > 0
    return vx, vy, r_max, frame, edges, span, ccw


def _radius(r, frame, rng):
    """The kernel's radius pair: within acc + 2^-45 r of the true one (records' parts, pair
    arithmetic)."""
    rk = r * (1.0 + rng.uniform(-1, 1) * 2.0 ** -45) + rng.uniform(-1, 1) * frame.acc
    return _split(rk)


def _circles(orc, vx, vy, r_max, count, seed):
    """Centres inside the polygon, a third of them within a few metres of an edge, radii from
    1 m to r_max with a share near the boundary."""
    rng = np.random.default_rng(seed)
    x0, x1, y0, y1 = vx.min(), vx.max(), vy.min(), vy.max()
    out = []
    nv = len(vx)
    while len(out) < count:
        if rng.uniform() < 0.35:
            k = int(rng.integers(0, nv))
            k1 = (k + 1) % nv
            s = rng.uniform()
            px = vx[k] + s * (vx[k1] - vx[k])
            py = vy[k] + s * (vy[k1] - vy[k])
            ang = rng.uniform(0, 2 * np.pi)
            d = 10.0 ** rng.uniform(-3, 1)
            px, py = px + d * math.cos(ang), py + d * math.sin(ang)
        else:
            px, py = rng.uniform(x0, x1), rng.uniform(y0, y1)
        if not orc.point_in_polygon(px, py, vx, vy):
            continue
        r = 10.0 ** rng.uniform(0.0, math.log10(r_max))
        out.append((px, py, r))
    return out


@pytest.mark.parametrize("name", ["star85", "smooth85", "poly24", "projected40"])
def test_fp32_polygon_share_within_its_bound(orc, name):
    vx, vy, r_max, frame, edges, span, ccw = _setup(name)
    coef = _coefficients()
    rng = np.random.default_rng(11)
    decided = cut = crossed = 0
    worst = 0.0
    buckets = Buckets(vx, vy, frame, r_max)
    for px, py, r in _circles(orc, vx, vy, r_max, 1500, 7):
        want = orc.polygon_weight(px, py, r, vx, vy)
        rh, rl = _radius(r, frame, rng)
        got = share_f32(frame.centre(px, py), rh, rl, edges, span, ccw, frame.eh, coef,
                        buckets)
        if got is None:
            cut += 1
            continue
        decided += 1
        ins, out, bound = got
        crossed += bound > 0
        rel = abs(float(ins) - want) / want
        worst = max(worst, rel)
        # the claimed bound (8.5e-7 of the share, before its rounding to FP32) and the result
        assert rel <= bound / want + 2.0 ** -24 + 1e-15, (name, px, py, r, float(ins), want)
        assert rel <= 8.5e-7 + 2.0 ** -24, (name, px, py, r, float(ins), want, rel)
        assert abs(float(ins) + float(out) - 1.0) <= 2.4e-7
    # nearly every circle is decided, many crossings included
    assert decided >= 0.97 * (decided + cut), (decided, cut)
    assert crossed > 200 and worst > 0


@pytest.mark.parametrize("name", ["star85", "projected40"])
def test_bucket_lists_hold_every_edge_a_circle_meets(orc, name):
    """For circles of radius up to the lists' reach around points of the polygon, every edge
    that comes within r of the centre (FP64 point-segment distance) is in the list the kernel
    picks for it; and the lists are far shorter than the edge count."""
    vx, vy, r_max, frame, edges, span, ccw = _setup(name)
    buckets = Buckets(vx, vy, frame, r_max)
    nv = len(vx)
    rng = np.random.default_rng(23)
    listed = []
    for px, py, _ in _circles(orc, vx, vy, r_max, 800, 29):
        c = frame.centre(px, py)
        r = float(buckets.rmax) * rng.uniform(0.5, 1.0)
        scan = set(buckets.edges(c[0], c[2], f32(r), nv))
        listed.append(len(scan))
        for k in range(nv):
            k1 = (k + 1) % nv
            ax, ay = vx[k] - px, vy[k] - py
            dx, dy = vx[k1] - vx[k], vy[k1] - vy[k]
            t = min(1.0, max(0.0, -(ax * dx + ay * dy) / (dx * dx + dy * dy)))
            if math.hypot(ax + t * dx, ay + t * dy) <= r:
                assert k in scan, (name, px, py, r, k)
    assert np.mean(listed) < 0.5 * nv, np.mean(listed)


def test_arc_pair_error_bound():
    """arc_half_angle_pair against FP64 acos, from pairs r and d = r - h, up to the tangency
    band: within 1e-8 (the kernel's bound takes 3e-8)."""
    coef = _coefficients()
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(20000):
        r = 10.0 ** rng.uniform(-1, 3.5)
        mode = rng.uniform()
        if mode < 0.3:
            h = r * rng.uniform(0, 1)
        elif mode < 0.6:
            h = r * (1 - 10.0 ** rng.uniform(-7, 0))
        else:
            h = r * 10.0 ** rng.uniform(-8, 0)
        rh, rl = _split(r)
        hh, hl = _split(h)
        dh, de = _two_sum(rh, -hh)
        dl = f32(de + f32(rl - hl))
        dh, dl = _two_sum(dh, dl)
        if float(dh) + float(dl) <= r * 2.0 ** -36:
            continue
        rr, d = float(rh) + float(rl), float(dh) + float(dl)
        want = 2.0 * math.asin(math.sqrt(d / rr / 2.0))  # acos(1 - d / r), accurate for small d
        ph, pl = arc_pair(dh, dl, rh, rl, coef)
        worst = max(worst, abs(float(ph) + float(pl) - want))
    assert worst < 1.0e-8, worst


def _square():
    vx = np.array([0.0, 1000.0, 1000.0, 0.0])
    vy = np.array([0.0, 0.0, 800.0, 800.0])
    frame = Frame((0.0, 1000.0, 0.0, 800.0), 8)
    edges, span = tables(vx, vy, frame)
    return vx, vy, frame, edges, span


def test_fp32_polygon_share_refuses_what_it_cannot_decide(orc):
    """Circles tangent to an edge, through a vertex, with a crossing at polar angle 0 (the
    choice of I0 in doubt), and a circle that might enclose the polygon go to FP64."""
    coef = _coefficients()
    vx, vy, frame, edges, span = _square()

    def share(x, y, r, ed=edges, sp=span, fr=frame, ccw=True):
        return share_f32(fr.centre(x, y), *_split(r), ed, sp, ccw, fr.eh, coef)

    assert share(500.0, 250.0, 250.0) is None  # tangent to the bottom edge
    assert share(300.0, 400.0, 500.0) is None  # through the corner (0, 0)
    # an ordinary circle cut by one edge is decided, and matches the closed form
    got = share(500.0, 100.0, 200.0)
    want = 1.0 - math.acos(100.0 / 200.0) / math.pi
    assert got is not None and abs(float(got[0]) - want) / want <= 1e-6
    # a crossing at polar angle 0: the edge (840, 250) - (940, 350) passes through
    # (890, 300) = centre (500, 300) + (390, 0)
    px = np.array([100.0, 700.0, 840.0, 940.0, 100.0])
    py = np.array([100.0, 100.0, 250.0, 350.0, 700.0])
    fr = Frame((0.0, 1000.0, 0.0, 1000.0), 8)
    ed, sp = tables(px, py, fr)
    assert orc.point_in_polygon(500.0, 300.0, px, py)
    assert share(500.0, 300.0, 390.0, ed, sp, fr) is None
    for ang in (1e-9, -1e-9, 2e-8, -2e-8):  # within the angle's error either way
        assert share(500.0, 300.0 - 390.0 * ang, 390.0, ed, sp, fr) is None
    # well clear of angle 0 the same outline is decided and matches the oracle
    got = share(500.0, 330.0, 390.0, ed, sp, fr)
    want = orc.polygon_weight(500.0, 330.0, 390.0, px, py)
    assert got is not None and abs(float(got[0]) - want) / want <= 1e-6
    # no crossing, yet the disc could enclose the polygon (2 r above its larger side)
    tx = np.array([0.0, 100.0, 50.0])
    ty = np.array([0.0, 0.0, 80.0])
    fr = Frame((0.0, 1000.0, 0.0, 1000.0), 8)
    ed, sp = tables(tx, ty, fr)
    assert share(50.0, 30.0, 300.0, ed, sp, fr) is None
    assert share(50.0, 30.0, 10.0, ed, sp, fr)[0] == 1.0  # small circle, wholly inside


def test_many_crossings_are_decided(orc):
    """A comb whose ten teeth a wide circle crosses twice each (20 crossings) is decided: the
    crossings are summed without a sort or a cap, and the result matches the oracle in both
    orientations of the outline."""
    coef = _coefficients()
    xs, ys = [0.0], [0.0]
    for k in range(10):
        xs += [k * 100.0 + 20.0, k * 100.0 + 50.0, k * 100.0 + 80.0, k * 100.0 + 100.0]
        ys += [600.0, 600.0, 0.0, 0.0]
    xs += [1000.0, 0.0]
    ys += [-300.0, -300.0]
    vx, vy = np.array(xs), np.array(ys)
    frame = Frame((0.0, 1000.0, -300.0, 600.0), 8)
    area2 = float(np.sum(vx * np.roll(vy, -1) - np.roll(vx, -1) * vy))
    want = orc.polygon_weight(500.0, -100.0, 450.0, vx, vy)
    for ox, oy, ccw in ((vx, vy, area2 > 0), (vx[::-1].copy(), vy[::-1].copy(), area2 < 0)):
        edges, span = tables(ox, oy, frame)
        got = share_f32(frame.centre(500.0, -100.0), *_split(450.0), edges, span, ccw,
                        frame.eh, coef)
        assert got is not None
        assert abs(float(got[0]) - want) / want <= 1e-6


def test_planted_mistake_fails_the_oracle(orc):
    """With the orientation flipped (entering and leaving crossings swapped) the shares of
    circles that cross the boundary no longer match the oracle: the comparison above is
    sensitive to the crossings' classification."""
    coef = _coefficients()
    vx, vy, r_max, frame, edges, span, ccw = _setup("poly24")
    bad = 0
    for px, py, r in _circles(orc, vx, vy, r_max, 300, 19):
        got = share_f32(frame.centre(px, py), *_split(r), edges, span, not ccw, frame.eh, coef)
        if got is None or got[2] == 0:
            continue
        want = orc.polygon_weight(px, py, r, vx, vy)
        bad += abs(float(got[0]) - want) / want > 1e-3
    assert bad > 20
