"""The pins have the power to see plausible mistakes: each mistake below is planted in a copy
of the oracle's C source (on the CPU), the copy is compiled, and the pin files run against it
in a subprocess must fail.  Mistakes: n^2 normalisation, no temporal weight, an open temporal
interval, a strict threshold test, a dropped dy term, an unsigned time lag lost, the weight
not inverted, arcs summed without their union, a wrong Philox constant, the inhomogeneous
weight with one intensity twice, the intensity not scaled to n, a simulated coordinate scaled
by the wrong axis's cell count, the translation correction with dx in place of dy, the
sector test with its operands transposed, a signed polygon area, an open polygon boundary, a
ray test inclusive at both ends, an arc judged at its start instead of its midpoint, the
cross-K denominator of the same-label case used for two labels, the intensity grid's x cell
count used along y, the grid-accelerated histogram skipping the cells on one side, grids not
cumulated over time, L without the factor 2 of the cylinder's height, a bootstrap that never
draws the last point, a permutation that maps out-of-range Feistel values to the identity
instead of walking the cycle, and CSR points that never reach the last tenth of each axis."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "stk_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_inhom.py", "tests/test_oracle_dir.py",
        "tests/test_oracle_grid.py", "tests/test_oracle_properties.py"]

MUTANTS = {
    "n2_normalisation": ("nn * (nn - 1.0)", "nn * nn"),
    "no_temporal_weight": ("return (ti - u >= t0 && ti + u <= t1) ? 1.0 : 0.5;", "return 1.0;"),
    "open_temporal_interval": ("ti - u >= t0 && ti + u <= t1", "ti - u > t0 && ti + u < t1"),
    "strict_threshold": ("if (d2 > s2max) continue;", "if (d2 >= s2max) continue;"),
    "dropped_dy": ("const double d2 = dx * dx + dy * dy;", "const double d2 = dx * dx;"),
    "signed_lag": ("fabs(t[i] - t[j])", "(t[i] - t[j])"),
    "weight_not_inverted": ("w = 1.0 / (om * v);", "w = om * v;"),
    "no_arc_union": ("if (arcs[k].lo <= cur_hi) {", "if (0) {"),
    "philox_constant": ("0xD2511F53u", "0xD2511F57u"),
    "inhom_one_intensity": ("lam[i] * lam[j]", "lam[i] * lam[i]"),
    "inhom_not_scaled": ("lam_cell[c] = (double)n * rho[c] / mass;",
                         "lam_cell[c] = rho[c] / mass;"),
    "inhom_cell_axis": ("(((double)idx[a] + u) / (double)cnt[a])",
                        "(((double)idx[a] + u) / (double)cnt[0])"),
    "translation_index": ("((w - fabs(dx)) * (h - fabs(dy)))", "((w - fabs(dx)) * (h - fabs(dx)))"),
    "sector_transposed": ("const double cr = bx * dy - by * dx;",
                          "const double cr = bx * dx - by * dy;"),
    "polygon_area_signed": ("return fabs(a) * 0.5;", "return a * 0.5;"),
    "polygon_boundary_open": ("if (on_segment(px, py, ax, ay, bx, by)) return 1;", ""),
    "polygon_ray_inclusive": ("if ((ay > py) != (by > py)) {", "if ((ay >= py) != (by > py)) {"),
    "polygon_arc_start_not_mid": ("const double mid = 0.5 * (a0 + a1);",
                                  "const double mid = a0;"),
    "cross_denominator": ("(a != b) ? fa * fb", "(a != b) ? fa * (fb - 1.0)"),
    "intensity_lookup_axis": ("axis_cell(y, box[2], box[3], niy)",
                              "axis_cell(y, box[2], box[3], nix)"),
    "grid_neighbours_one_side": ("for (int dxx = -1; dxx <= 1; ++dxx)",
                                 "for (int dxx = -1; dxx <= 0; ++dxx)"),
    "no_cumulation_over_time": ("for (int b2 = 0; b2 <= b; ++b2)",
                                "for (int b2 = b; b2 <= b; ++b2)"),
    "l_without_factor_2": ("sqrt(kv / (2.0 * ORACLE_PI * tt[b])) - s[a]",
                           "sqrt(kv / (ORACLE_PI * tt[b])) - s[a]"),
    "bootstrap_never_last": ("int64_t src = (int64_t)(u * (double)n);",
                             "int64_t src = (int64_t)(u * (double)(n - 1));"),
    "permutation_no_cycle_walk": ("while (v >= (uint64_t)n) v = oracle_feistel(v, b, seed, sim);",
                                  "if (v >= (uint64_t)n) v = (uint64_t)i;"),
    "csr_short_of_the_box": ("const double span = hi - lo;", "const double span = 0.9 * (hi - lo);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, f"mutation {name} no longer applies"
    mut = tmp_path / "stk_oracle.c"
    mut.write_text(src.replace(old, new))
    (tmp_path / "stk_oracle.h").write_text(open(SRC[:-1] + "h").read())
    lib = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-pthread", "-o", str(lib), str(mut), "-lm"])
    env = dict(os.environ, STK_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"no pin caught {name}:\n{r.stdout[-2000:]}"
