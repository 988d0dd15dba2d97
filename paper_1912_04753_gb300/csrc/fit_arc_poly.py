"""Coefficients of the FP32 arc polynomial of the pair kernel (pair.cu, arc_half_angle).

An edge at distance e from a centre cuts from the circle of radius r > e an arc of half-angle
alpha = acos(e / r) (Section 3's isotropic weight removes such arcs).  With x = e / r,

    acos(x) = sqrt(1 - x) * f(x),    f(x) = acos(x) / sqrt(1 - x),

and f is analytic on [0, 1] (f(1) = sqrt(2)), so a short polynomial fits it closely; the
square-root factor carries the singular part, and the kernel forms 1 - x as (r - e) / r so that
it stays accurate up to tangency.  This script fits P ~ f by least squares in the relative error
on Chebyshev nodes of [0, 1] (monomial basis) and prints the coefficients: degree 7 for the
rectangle's arcs (arc_half_angle, c0 .. c7 rounded to FP32) and degree 9 for the polygon weight
(arc_half_angle_pair, c1 .. c9 rounded to FP32 and c0 as a pair hi + lo of FP32 numbers).
tests/test_arc_poly.py checks the coefficients written in pair.cu against this fit and the
evaluations against acos.

    python paper_1912_04753_gb300/csrc/fit_arc_poly.py
"""
import numpy as np

DEGREE = 7
NODES = 4000


def fit(degree=DEGREE, nodes=NODES):
    k = np.arange(nodes)
    x = 0.5 - 0.5 * np.cos(np.pi * (k + 0.5) / nodes)  # Chebyshev nodes of [0, 1]
    f = np.arccos(x) / np.sqrt(1.0 - x)
    V = np.vander(x, degree + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V / f[:, None], np.ones_like(f), rcond=None)
    return c


PAIR_DEGREE = 9


if __name__ == "__main__":
    for i, v in enumerate(fit().astype(np.float32)):
        print(f"c{i} = {float(v)!r}f")
    c = fit(PAIR_DEGREE)
    hi = np.float32(c[0])
    print(f"pair: c0 = {float(hi)!r}f + {float(np.float32(c[0] - float(hi)))!r}f")
    for i, v in enumerate(c.astype(np.float32)[1:], start=1):
        print(f"pair: c{i} = {float(v)!r}f")
