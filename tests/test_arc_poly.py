"""The FP32 isotropic weight of the pair kernel's weight phase, emulated on the host with numpy
FP32 arithmetic: the arc half-angle acos(e / r) from the polynomial of fit_arc_poly.py with
1 - x formed as (r - e) / r, the overlapping arcs at a corner, and 1 / (1 - A).  Outside the
tangency band (|r - e| <= 1e-3 r, which the kernel sends to FP64) it must match the oracle's
weight (Section 3: share of the circumference inside the rectangle, computed there as a union
of arcs) to well within the FP32-guarded tolerance; and the coefficients written in pair.cu
must be the fit's."""
import math
import os
import re
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_04753_gb300", "csrc")
f32 = np.float32


def _coefficients_in_kernel():
    src = open(os.path.join(CSRC, "pair.cu")).read()
    body = src[src.index("float arc_half_angle("):]
    body = body[:body.index("return sqrt_nr")]
    vals = [float(v) for v in re.findall(r"p = [^;]*?(-?\d+\.\d+(?:e-?\d+)?)f\)?;", body)]
    return vals[::-1]  # Horner runs from c7 down to c0


def test_kernel_coefficients_are_the_fit():
    sys.path.insert(0, CSRC)
    import fit_arc_poly

    c = fit_arc_poly.fit().astype(f32)
    got = np.array(_coefficients_in_kernel(), dtype=f32)
    assert got.shape == c.shape
    assert np.array_equal(got, c)


def test_pair_coefficients_are_the_fit():
    """arc_half_angle_pair (the polygon weight): c9 .. c1 in its Horner steps and c0 as a pair
    hi + lo are the degree-9 fit's."""
    sys.path.insert(0, CSRC)
    import fit_arc_poly

    src = open(os.path.join(CSRC, "pair.cu")).read()
    body = src[src.index("void arc_half_angle_pair("):]
    body = body[:body.index("ph = s0 * Ph;")]
    horner = [float(v) for v in re.findall(r"p = [^;]*?(-?\d+\.\d+(?:e-?\d+)?)f\)?;", body)]
    c0 = [float(v) for v in
          re.findall(r"two_sum\((-?\d+\.\d+(?:e-?\d+)?)f, m", body)]
    c0l = [float(v) for v in re.findall(r"Pe, me\), (-?\d+\.\d+(?:e-?\d+)?)f\)", body)]
    c = fit_arc_poly.fit(fit_arc_poly.PAIR_DEGREE)
    want = c.astype(f32)
    assert np.array_equal(np.array(horner[::-1], f32), want[1:])
    hi = f32(c[0])
    assert c0 == [float(hi)] and c0l == [float(f32(c[0] - float(hi)))]


def _sqrt_nr(v):
    y = (1.0 / np.sqrt(v.astype(np.float64) + 1e-30)).astype(f32)
    s = (v * y).astype(f32)
    corr = (v.astype(np.float64) - s.astype(np.float64) * s).astype(f32)
    return (corr.astype(np.float64) * (f32(0.5) * y) + s).astype(f32)


def _arc(e, r, inv_r, c):
    x = np.minimum((e * inv_r).astype(f32), f32(1))
    om = np.maximum(((r - e).astype(f32) * inv_r).astype(f32), f32(0))
    p = np.full_like(x, c[7])
    for k in range(6, -1, -1):
        p = (p.astype(np.float64) * x + c[k]).astype(f32)
    return (_sqrt_nr(om) * p).astype(f32)


def _weight32(e1, e2, r, c):
    inv_r = (f32(1) / r).astype(f32)
    a1, a2 = _arc(e1, r, inv_r, c), _arc(e2, r, inv_r, c)
    corner = (e1.astype(np.float64) * e1 + (e2 * e2).astype(f32)).astype(f32) < (r * r).astype(f32)
    A = np.where(corner, ((a1 + a2 + f32(1.57079632679)) * f32(0.159154943092)).astype(f32),
                 ((a1 + a2) * f32(0.318309886184)).astype(f32))
    return (f32(1) / (f32(1) - A)).astype(f32)


@pytest.mark.parametrize("seed", [0, 1])
def test_fp32_weight_matches_oracle_outside_the_tangency_band(orc, seed):
    sys.path.insert(0, CSRC)
    import fit_arc_poly

    c = fit_arc_poly.fit().astype(f32)
    rng = np.random.default_rng(seed)
    W = H = 10_000.0
    box = (0.0, W, 0.0, H, 0.0, 1.0)
    n = 6000
    r = rng.uniform(1.0, 0.5 * W, n)
    # centres near an edge, near a corner, and anywhere
    kind = rng.integers(0, 3, n)
    xi = np.where(kind == 0, rng.uniform(0, 1.2, n) * r, rng.uniform(0, W, n))
    yi = np.where(kind == 1, rng.uniform(0, 1.2, n) * r, rng.uniform(0, H, n))
    xi = np.where(kind == 2, rng.uniform(0, 1.5, n) * r, xi)
    yi = np.where(kind == 2, rng.uniform(0, 1.5, n) * r, yi)
    # dyadic geometry (multiples of 2^-6 below 2^14): e and r are exact in FP32, so what is
    # measured is the arc formula and its FP32 evaluation, not the rounding of the inputs
    xi, yi, r = (np.clip(np.round(v * 64) / 64, 1 / 64, W - 1 / 64) for v in (xi, yi, r))
    ex = np.minimum(xi, W - xi)
    ey = np.minimum(yi, H - yi)
    e1, e2 = np.minimum(ex, ey), np.maximum(ex, ey)
    out_band = (np.abs(r - e1) > 1e-3 * r) & (np.abs(r - e2) > 1e-3 * r)
    w32 = _weight32(e1.astype(f32), e2.astype(f32), r.astype(f32), c).astype(np.float64)
    checked = 0
    for k in np.nonzero(out_band)[0]:
        w_ref = 1.0 / orc.spatial_weight(float(xi[k]), float(yi[k]), float(r[k]), box)
        rel = abs(w32[k] - w_ref) / w_ref
        # exact inputs: half the FP32-guarded tolerance of 1e-6 (the kernel's e and r carry
        # their own rounding besides, which the tangency band keeps below the other half)
        assert rel <= 5e-7, (k, xi[k], yi[k], r[k], w32[k], w_ref)
        checked += 1
    assert checked > 4000
    # the interior and the corner are exercised
    assert (w32 == 1.0).any() and (w32 > 2.0).any()


def test_arc_polynomial_error_bound():
    sys.path.insert(0, CSRC)
    import fit_arc_poly

    c = fit_arc_poly.fit()
    x = np.linspace(0.0, 1.0, 100001)
    rel = np.abs(np.polyval(c[::-1], x) * np.sqrt(1 - x) - np.arccos(x)) / np.maximum(
        np.arccos(x), 1e-300)
    assert rel[:-1].max() < 3e-8
    r = np.float32(1000.0)
    e = (r * np.linspace(0, 0.999, 20001)).astype(f32)
    a = _arc(e, np.full_like(e, r), np.full_like(e, f32(1) / r), c.astype(f32))
    assert np.abs(a - np.arccos(e.astype(np.float64) / np.float64(r))).max() < 4e-7
    assert math.isclose(float(_arc(np.array([r], f32), np.array([r], f32),
                                   np.array([f32(1) / r], f32), c.astype(f32))[0]), 0.0,
                        abs_tol=1e-6)


def test_far_edges_of_tiny_circles_add_no_arc():
    """An edge far beyond a tiny circle (e / r up to 1e9) cuts no arc: the angle is exactly 0,
    not a NaN from the polynomial at a huge argument."""
    sys.path.insert(0, CSRC)
    import fit_arc_poly

    c = fit_arc_poly.fit().astype(f32)
    r = np.array([1e-6, 1e-3, 0.5, 2.0], f32)
    e = np.array([2500.0, 2500.0, 1e4, 2.0], f32)
    a = _arc(e, r, (f32(1) / r).astype(f32), c)
    assert np.array_equal(a, np.zeros(4, f32))
    w = _weight32(np.zeros(4, f32), e, r, c)
    assert np.all(np.abs(w.astype(np.float64) - 2.0) < 1e-6)  # one edge through the centre
