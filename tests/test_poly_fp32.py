"""The FP32-guarded isotropic weight in a polygon study area (pair.cu, poly_share_f32),
emulated on the host with numpy FP32 arithmetic in the kernel's order: per edge the line's
distance h and the centre's projection from FP64, the half chord t and the arc half-angle
psi = acos(h / r) (the fitted polynomial of fit_arc_poly.py) in FP32, the crossings' angles
phi_m -+ psi in FP64, and the guards (tangency, vertices, order, alternation, the error bound).
Whenever the guards let a circle through, its inside share must match the oracle's (Section 3:
proportion of the circumference inside the polygon, FP64) to the bound the kernel claims; and
the guards must let most circles near the boundary through."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_04753_gb300", "csrc")
f32 = np.float32
TWO_PI = 6.283185307179586


def _coefficients():
    sys.path.insert(0, CSRC)
    import fit_arc_poly

    return fit_arc_poly.fit().astype(f32)


def _sqrt_nr(v):
    y = f32(1.0 / math.sqrt(float(v) + 1e-30))
    s = f32(v * y)
    corr = f32(float(v) - float(s) * float(s))
    return f32(float(corr) * float(f32(f32(0.5) * y)) + float(s))


def _arc(e, r, inv_r, c):
    x = min(f32(e * inv_r), f32(1.0))
    om = max(f32(f32(r - e) * inv_r), f32(0.0))
    p = c[7]
    for k in range(6, -1, -1):
        p = f32(float(p) * float(x) + float(c[k]))
    return f32(_sqrt_nr(om) * p)


def _edges(vx, vy):
    """Host tables of the kernel: FP32 boxes rounded outwards and FP64 edge directions."""
    nv = len(vx)
    out = []
    for k in range(nv):
        k1 = (k + 1) % nv
        dx, dy = vx[k1] - vx[k], vy[k1] - vy[k]
        ln = math.sqrt(dx * dx + dy * dy)
        box = []
        for lo, hi in ((min(vx[k], vx[k1]), max(vx[k], vx[k1])),
                       (min(vy[k], vy[k1]), max(vy[k], vy[k1]))):
            lf, hf = f32(lo), f32(hi)
            if float(lf) > lo:
                lf = np.nextafter(lf, f32(-np.inf))
            if float(hf) < hi:
                hf = np.nextafter(hf, f32(np.inf))
            box += [lf, hf]
        if ln > 0:
            ux, uy = dx / ln, dy / ln
            out.append((box, vx[k], vy[k], ux, uy, ln, math.atan2(-ux, uy)))
        else:
            out.append((box, vx[k], vy[k], 0.0, 0.0, 0.0, 0.0))
    return out


def share_f32(cx, cy, r, edges, ccw, c):
    """Emulation of poly_share_f32: (inside, outside) or None where FP64 decides."""
    r = f32(r)
    inv_r = f32(f32(1.0) / r)
    cxf, cyf = f32(cx), f32(cy)
    m = f32(f32(f32(r * f32(1e-4)) + f32(f32(1e-6) * f32(abs(cxf) + abs(cyf)))) + f32(1e-30))
    x0, x1 = f32(f32(cxf - r) - m), f32(f32(cxf + r) + m)
    y0, y1 = f32(f32(cyf - r) - m), f32(f32(cyf + r) + m)
    band = f32(math.ldexp(float(r), -19))
    cmag = f32(abs(cxf) + abs(cyf))
    cross = []
    for box, ax, ay, ux, uy, ln, phi0 in edges:
        if box[0] > x1 or box[1] < x0 or box[2] > y1 or box[3] < y0:
            continue
        # FP32 pre-test of the line's distance (fmaf: one rounding of the exact a * b + c)
        axf, ayf, uxf, uyf = f32(ax), f32(ay), f32(ux), f32(uy)
        prod = f32(f32(ayf - cyf) * uxf)
        h32 = abs(f32(float(f32(axf - cxf)) * float(uyf) - float(prod)))
        lim = f32(f32(r + band) + f32(f32(2.4e-7) * f32(f32(f32(abs(axf) + abs(ayf)) + cmag) + h32)))
        if h32 > lim:
            continue
        if not ln > 0:
            continue
        fx, fy = ax - cx, ay - cy
        hd = fx * uy - fy * ux
        h = abs(f32(hd))
        if h >= f32(r + band):
            continue
        if h > f32(r - band):
            return None
        t = _sqrt_nr(f32(f32(r - h) * f32(r + h)))
        psi = _arc(h, r, inv_r, c)
        u0 = f32(-(fx * ux + fy * uy))
        lnf = f32(ln)
        rt = f32(r / t)
        err = f32(f32(4.2e-7) + f32(f32(3.0e-7) * rt))
        uerr = f32(f32(f32(1.2e-7) * f32(f32(abs(u0) + lnf) + t)) +
                   f32(f32(f32(3.0e-7) * r) * rt) + f32(f32(1.5e-7) * t))
        phi = phi0 + (math.pi if hd < 0 else 0.0)
        sgn = -1.0 if hd < 0 else 1.0
        for q in (-1, 1):
            u = f32(float(q) * float(t) + float(u0))
            if abs(u) <= uerr or abs(f32(u - lnf)) <= uerr:
                return None
            if u < 0 or u >= lnf:
                continue
            if len(cross) == 8:
                return None
            a = q * sgn * float(psi) + phi
            a = a + TWO_PI if a < 0 else (a - TWO_PI if a >= TWO_PI else a)
            cross.append((a, err, (q > 0) == ccw))
    if not cross:
        return f32(1.0), f32(0.0)
    if len(cross) % 2:
        return None
    cross.sort(key=lambda v: v[0])
    n = len(cross)
    inside, bound = 0.0, f32(0.0)
    for k in range(n):
        k1 = (k + 1) % n
        gap = cross[k1][0] - cross[k][0] if k + 1 < n else cross[0][0] + TWO_PI - cross[k][0]
        if not gap > float(f32(cross[k][1] + cross[k1][1])):
            return None
        if cross[k][2] == cross[k1][2]:
            return None
        if cross[k][2]:
            inside += gap
        bound = f32(bound + cross[k][1])
    ins = f32(inside * 0.15915494309189535)
    out = f32((TWO_PI - inside) * 0.15915494309189535)
    if not f32(bound * f32(0.15915494309189535)) <= f32(f32(8.5e-7) * ins):
        return None
    return ins, out


def _polygons():
    from paper_1912_04753_gb300 import workloads as wl

    star = wl.star_polygon(85, 5000.0, 3400.0, 5000.0, 5000.0, 1)
    rng = np.random.default_rng(3)
    ang = np.sort(rng.uniform(0, 2 * np.pi, 24))
    rad = rng.uniform(600.0, 1000.0, 24)
    poly24 = (1200.0 + rad * np.cos(ang), 1100.0 + rad * np.sin(ang))
    # a clockwise outline at projected coordinates
    vx, vy = wl.star_polygon(40, 2500.0, 1800.0, 5.0e5 + 3000.0, 3.3e6 + 3000.0, 5)
    projected = (vx[::-1].copy(), vy[::-1].copy())
    return {"star85": (star, 1000.0), "poly24": (poly24, 300.0), "projected40": (projected, 900.0)}


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


@pytest.mark.parametrize("name", ["star85", "poly24", "projected40"])
def test_fp32_polygon_share_within_its_bound(orc, name):
    c = _coefficients()
    (vx, vy), r_max = _polygons()[name]
    vx, vy = np.asarray(vx, np.float64), np.asarray(vy, np.float64)
    area2 = float(np.sum(vx * np.roll(vy, -1) - np.roll(vx, -1) * vy))
    ccw = area2 > 0
    edges = _edges(vx, vy)
    rng = np.random.default_rng(11)
    decided = cut = 0
    worst = 0.0
    circles = _circles(orc, vx, vy, r_max, 2500, 7)
    for px, py, r in circles:
        want = orc.polygon_weight(px, py, r, vx, vy)
        # the kernel's radius is the reference one within 2^-22 r (accurate offset, Newton root)
        rk = float(f32(r * (1.0 + rng.uniform(-1, 1) * 2.0 ** -22)))
        got = share_f32(px, py, rk, edges, ccw, c)
        if got is None:
            cut += 1
            continue
        decided += 1
        ins, out = got
        # the share of the true radius r: the kernel's radius differs by up to 2^-22 r, whose
        # effect on the share is inside the bound as well (it is part of h / r's rounding)
        rel = abs(float(ins) - want) / want
        worst = max(worst, rel)
        assert rel <= 1e-6, (name, px, py, r, float(ins), want, rel)
        assert abs(float(ins) + float(out) - 1.0) <= 2e-7
    assert decided >= 0.8 * len(circles), (decided, cut)
    assert worst > 0  # exercised


def test_fp32_polygon_share_refuses_what_it_cannot_decide(orc):
    """Circles tangent to an edge, through a vertex, and many crossings go to FP64."""
    c = _coefficients()
    vx = np.array([0.0, 1000.0, 1000.0, 0.0])
    vy = np.array([0.0, 0.0, 800.0, 800.0])
    edges = _edges(vx, vy)
    # tangent to the bottom edge (distance 250 from it)
    assert share_f32(500.0, 250.0, 250.0, edges, True, c) is None
    # through the corner (0, 0): centre at (300, 400), r = 500
    assert share_f32(300.0, 400.0, 500.0, edges, True, c) is None
    # an ordinary circle cut by one edge is decided, and matches the closed form
    got = share_f32(500.0, 100.0, 200.0, edges, True, c)
    assert got is not None
    want = 1.0 - math.acos(100.0 / 200.0) / math.pi
    assert abs(float(got[0]) - want) / want <= 1e-6
    # a comb whose ten teeth a wide circle crosses twice each: more than 8 crossings
    xs, ys = [0.0], [0.0]
    for k in range(10):
        xs += [k * 100.0 + 20.0, k * 100.0 + 50.0, k * 100.0 + 80.0, k * 100.0 + 100.0]
        ys += [600.0, 600.0, 0.0, 0.0]
    xs += [1000.0, 0.0]
    ys += [-300.0, -300.0]
    ex = _edges(np.array(xs), np.array(ys))
    area2 = sum(xs[k] * ys[(k + 1) % len(xs)] - xs[(k + 1) % len(xs)] * ys[k]
                for k in range(len(xs)))
    assert share_f32(500.0, -100.0, 450.0, ex, area2 > 0, c) is None


def share_f64(cx, cy, r, edges, ccw):
    """Emulation of poly_share_f64 (the FP64 middle tier): the inside share, or None."""
    band = 1e-12 * r
    cross = []
    for box, ax, ay, ux, uy, ln, phi0 in edges:
        if (box[0] > cx + r * 1.0001 + 1 or box[1] < cx - r * 1.0001 - 1 or
                box[2] > cy + r * 1.0001 + 1 or box[3] < cy - r * 1.0001 - 1):
            continue
        if not ln > 0:
            continue
        fx, fy = ax - cx, ay - cy
        hd = fx * uy - fy * ux
        h = abs(hd)
        if h >= r + band:
            continue
        if h > r - band:
            return None
        t = math.sqrt((r - h) * (r + h))
        psi = math.acos(h / r)
        u0 = -(fx * ux + fy * uy)
        uerr = 1e-12 * (abs(u0) + ln + r)
        phi = phi0 + (math.pi if hd < 0 else 0.0)
        sgn = -1.0 if hd < 0 else 1.0
        for q in (-1, 1):
            u = u0 + q * t
            if abs(u) <= uerr or abs(u - ln) <= uerr:
                return None
            if u < 0 or u >= ln:
                continue
            if len(cross) == 16:
                return None
            a = (phi + q * sgn * psi) % TWO_PI
            cross.append((a, (q > 0) == ccw))
    if not cross:
        return 1.0
    if len(cross) % 2:
        return None
    cross.sort(key=lambda v: v[0])
    n, inside = len(cross), 0.0
    for k in range(n):
        k1 = (k + 1) % n
        if cross[k][1] == cross[k1][1]:
            return None
        if cross[k][1]:
            inside += cross[k1][0] - cross[k][0] if k + 1 < n else cross[0][0] + TWO_PI - cross[k][0]
    return inside / TWO_PI


@pytest.mark.parametrize("name", ["star85", "poly24", "projected40"])
def test_fp64_tier_matches_the_oracle(orc, name):
    """The FP64 middle tier decides nearly every circle (the FP32 tier's refusals included)
    and equals the oracle's share (a different FP64 construction) to rounding: both carry
    the FP64 rounding of the coordinates relative to the radius (below 1e-9 here)."""
    (vx, vy), r_max = _polygons()[name]
    vx, vy = np.asarray(vx, np.float64), np.asarray(vy, np.float64)
    ccw = float(np.sum(vx * np.roll(vy, -1) - np.roll(vx, -1) * vy)) > 0
    edges = _edges(vx, vy)
    circles = _circles(orc, vx, vy, r_max, 2500, 13)
    refused = 0
    for px, py, r in circles:
        got = share_f64(px, py, r, edges, ccw)
        if got is None:
            refused += 1
            continue
        want = orc.polygon_weight(px, py, r, vx, vy)
        assert abs(got - want) <= 1e-9 * want, (px, py, r, got, want)
    assert refused <= 0.005 * len(circles), refused
