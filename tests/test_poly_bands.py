"""The y-band edge lists of a polygon (stk.cu, build_poly_bands; poly.cuh,
poly_contains_banded), emulated on the host in FP64 with the device's operations: the closed
point-in-polygon test restricted to the edges of the point's band must decide exactly as the
oracle's test over every edge (Section 3's CSR in a polygon keeps the draws that lie inside, and
the device's draws are compared with the oracle's bit for bit).  Points drawn at random, on the
outline, at the heights of vertices and on the band boundaries themselves."""
import math

import numpy as np
import pytest

BANDS = 32  # kPolyBands


def build_bands(vx, vy):
    """build_poly_bands: per band the edges whose closed y-range meets it, widened by eps."""
    nv = len(vx)
    lo, hi = float(np.min(vy)), float(np.max(vy))
    bh = (hi - lo) / BANDS
    eps = 1e-9 * (hi - lo) + 1e-12 * (abs(lo) + abs(hi))
    bands = []
    for b in range(BANDS):
        blo, bhi = lo + b * bh - eps, lo + (b + 1) * bh + eps
        bands.append([k for k in range(nv)
                      if min(vy[k], vy[(k + 1) % nv]) <= bhi and
                      max(vy[k], vy[(k + 1) % nv]) >= blo])
    return bands, lo, hi, BANDS / (hi - lo)


def _on_segment(px, py, ax, ay, bx, by):
    cross = (bx - ax) * (py - ay) - (by - ay) * (px - ax)  # each operation rounded (FP64)
    if cross != 0.0:
        return False
    return min(ax, bx) <= px <= max(ax, bx) and min(ay, by) <= py <= max(ay, by)


def contains_banded(px, py, vx, vy, bands, lo, hi, inv):
    """poly_contains_banded."""
    if not (lo <= py <= hi):
        return False
    b = min(max(int((py - lo) * inv), 0), BANDS - 1)
    nv = len(vx)
    inside = False
    for k in bands[b]:
        k1 = (k + 1) % nv
        ax, ay, bx, by = vx[k], vy[k], vx[k1], vy[k1]
        if _on_segment(px, py, ax, ay, bx, by):
            return True
        if (ay > py) != (by > py):
            xc = ax + ((py - ay) * (bx - ax)) / (by - ay)
            if px < xc:
                inside = not inside
    return inside


def _outlines():
    from paper_1912_04753_gb300 import workloads as wl

    star = wl.star_polygon(85, 5000.0, 3400.0, 5000.0, 5000.0, 1)
    smooth = wl.smooth_polygon(85, 3800.0, 5000.0, 5000.0, 3)
    # an axis-aligned staircase: horizontal edges at band boundaries and repeated heights
    xs, ys = [0.0], [0.0]
    for k in range(12):
        xs += [100.0 * (k + 1), 100.0 * (k + 1)]
        ys += [50.0 * k, 50.0 * (k + 1)]
    xs += [0.0]
    ys += [600.0]
    proj = wl.star_polygon(40, 2500.0, 1800.0, 5.0e5 + 3000.0, 3.3e6 + 3000.0, 5)
    return {"star85": star, "smooth85": smooth, "staircase": (np.array(xs), np.array(ys)),
            "projected40": proj}


@pytest.mark.parametrize("name", ["star85", "smooth85", "staircase", "projected40"])
def test_banded_test_decides_as_the_oracle(orc, name):
    vx, vy = (np.asarray(v, np.float64) for v in _outlines()[name])
    bands, lo, hi, inv = build_bands(vx, vy)
    nv = len(vx)
    rng = np.random.default_rng(31)
    x0, x1 = vx.min() - 10.0, vx.max() + 10.0
    pts = [(rng.uniform(x0, x1), rng.uniform(lo - 10.0, hi + 10.0)) for _ in range(1500)]
    for k in range(nv):  # on the outline: vertices, points along edges, vertex heights
        k1 = (k + 1) % nv
        pts.append((vx[k], vy[k]))
        s = rng.uniform()
        pts.append((vx[k] + s * (vx[k1] - vx[k]), vy[k] + s * (vy[k1] - vy[k])))
        pts.append((rng.uniform(x0, x1), vy[k]))
    bh = (hi - lo) / BANDS
    for b in range(BANDS + 1):  # band boundaries and their neighbours in FP64
        y = lo + b * bh
        for yy in (y, math.nextafter(y, -math.inf), math.nextafter(y, math.inf)):
            pts.append((rng.uniform(x0, x1), yy))
    assert max(len(b) for b in bands) < nv or name == "staircase"
    for px, py in pts:
        want = orc.point_in_polygon(px, py, vx, vy)
        got = contains_banded(px, py, vx, vy, bands, lo, hi, inv)
        assert got == want, (name, px, py, got, want)


def test_bands_are_short_on_the_benchmark_outlines():
    """The star's and the smooth outline's bands hold a fraction of the edges (what makes the
    banded test cheaper), and every edge is in at least one band."""
    for name in ("star85", "smooth85"):
        vx, vy = (np.asarray(v, np.float64) for v in _outlines()[name])
        bands, *_ = build_bands(vx, vy)
        assert np.mean([len(b) for b in bands]) < 0.4 * len(vx)
        assert set().union(*map(set, bands)) == set(range(len(vx)))
