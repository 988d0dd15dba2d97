"""Seeded synthetic point patterns that stand in for the paper's datasets.

The paper evaluates on the Hubei enterprise-registration POI set and on random points inside
an 85-vertex US outline (Section 6.1, Appendix Table A); neither is available here, so these
generators produce patterns of the same shape: complete spatio-temporal randomness (CSR),
Thomas cluster processes, and POI-like mixtures of lognormal-sized clusters over a uniform
background with timestamps at one-second granularity.

This module holds input generation only: no part of the estimator's arithmetic.  It is shared
by the tests (CUDA path and oracle alike), the benchmark and the smoke check.  Generation uses
numpy's PCG64 with the stated seed, so every workload is reproducible.
"""
from __future__ import annotations

import math

from dataclasses import dataclass, field

import numpy as np

DAY = 86400.0


@dataclass
class Workload:
    """A point pattern plus the analysis parameters that go with it."""

    name: str
    x: np.ndarray
    y: np.ndarray
    t: np.ndarray
    box: tuple  # (x0, x1, y0, y1, t0, t1)
    s: np.ndarray  # spatial thresholds, strictly increasing
    tt: np.ndarray  # temporal thresholds, strictly increasing
    n_sims: int
    sim_seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def even_thresholds(vmax: float, count: int) -> np.ndarray:
    """Thresholds vmax*a/count for a = 1..count (zero excluded: L divides by t)."""
    return np.array([vmax * a / count for a in range(1, count + 1)], dtype=np.float64)


def csr(n: int, box, seed: int):
    """n points uniform in the spatio-temporal box (binomial CSR)."""
    rng = np.random.default_rng(seed)
    x0, x1, y0, y1, t0, t1 = box
    x = rng.uniform(x0, x1, n)
    y = rng.uniform(y0, y1, n)
    t = rng.uniform(t0, t1, n)
    return x, y, t


def _redraw_inside(rng, centres, sigma, lo, hi):
    """Gaussian offspring around `centres`; any offspring outside [lo, hi] is redrawn."""
    out = centres + rng.normal(0.0, sigma, centres.shape[0])
    bad = (out < lo) | (out > hi)
    while bad.any():
        out[bad] = centres[bad] + rng.normal(0.0, sigma, int(bad.sum()))
        bad = (out < lo) | (out > hi)
    return out


def thomas(n: int, box, n_parents: int, sigma_s: float, sigma_t: float, rng,
           lognormal_sigma: float | None = None):
    """Thomas process with exactly n offspring.

    Parents are uniform in the box.  Offspring are assigned to parents multinomially, with
    equal probabilities or, if `lognormal_sigma` is given, with lognormal(0, sigma) relative
    cluster sizes.  Offsets are isotropic Gaussian in space and Gaussian in time; offspring
    that leave the box are redrawn around the same parent.
    """
    x0, x1, y0, y1, t0, t1 = box
    px = rng.uniform(x0, x1, n_parents)
    py = rng.uniform(y0, y1, n_parents)
    pt = rng.uniform(t0, t1, n_parents)
    if lognormal_sigma is None:
        p = np.full(n_parents, 1.0 / n_parents)
    else:
        w = rng.lognormal(0.0, lognormal_sigma, n_parents)
        p = w / w.sum()
    counts = rng.multinomial(n, p)
    parent = np.repeat(np.arange(n_parents), counts)
    x = _redraw_inside(rng, px[parent], sigma_s, x0, x1)
    y = _redraw_inside(rng, py[parent], sigma_s, y0, y1)
    t = _redraw_inside(rng, pt[parent], sigma_t, t0, t1)
    return x, y, t


def config_csr_small(seed: int = 0, n: int = 2000) -> Workload:
    """CSR n=2,000 in 1000 m x 1000 m x 365 d; 10 x 10 thresholds to 100 m / 30 d; 19 sims."""
    box = (0.0, 1000.0, 0.0, 1000.0, 0.0, 365.0)
    x, y, t = csr(n, box, seed)
    return Workload("csr_n2000", x, y, t, box, even_thresholds(100.0, 10),
                    even_thresholds(30.0, 10), 19, seed, {"time_unit": "day"})


def config_thomas(seed: int = 0, n: int = 200_000) -> Workload:
    """Thomas n=200,000 in 10 km x 10 km x 730 d; parents Poisson(400), sigma 150 m / 10 d.

    20 x 20 thresholds to 1 km / 60 d; 99 CSR simulations.
    """
    rng = np.random.default_rng(seed)
    box = (0.0, 10_000.0, 0.0, 10_000.0, 0.0, 730.0)
    n_par = max(1, int(rng.poisson(400)))
    x, y, t = thomas(n, box, n_par, 150.0, 10.0, rng)
    return Workload("thomas_n200k", x, y, t, box, even_thresholds(1000.0, 20),
                    even_thresholds(60.0, 20), 99, seed,
                    {"time_unit": "day", "parents": n_par})


def poi_mixture(n: int, box, n_parents: int, rng, cluster_frac: float = 0.7,
                sigma_s: float = 150.0, sigma_t_s: float = 10 * DAY):
    """POI-shaped mixture: lognormal-sized Thomas clusters plus a uniform background,
    timestamps floored to whole seconds (time unit = s)."""
    x0, x1, y0, y1, t0, t1 = box
    nc = int(round(cluster_frac * n))
    cx, cy, ctt = thomas(nc, box, n_parents, sigma_s, sigma_t_s, rng, lognormal_sigma=1.0)
    nb = n - nc
    bx = rng.uniform(x0, x1, nb)
    by = rng.uniform(y0, y1, nb)
    bt = rng.uniform(t0, t1, nb)
    x = np.concatenate([cx, bx])
    y = np.concatenate([cy, by])
    t = np.floor(np.concatenate([ctt, bt]))
    perm = rng.permutation(n)
    return x[perm], y[perm], t[perm]


def config_poi(seed: int = 0, n: int = 2_000_000) -> Workload:
    """POI mixture n=2,000,000 in 50 km x 50 km x 1095 d (time in s), 2,000 parents.

    25 x 25 thresholds: s_a = 80 a m, t_b = 311,040 b s (3.6 b days); 99 CSR simulations.
    """
    rng = np.random.default_rng(seed)
    box = (0.0, 50_000.0, 0.0, 50_000.0, 0.0, 1095 * DAY)
    n_par = max(1, int(round(2000 * n / 2_000_000)))
    x, y, t = poi_mixture(n, box, n_par, rng)
    return Workload("poi_n2M", x, y, t, box, even_thresholds(2000.0, 25),
                    np.array([311_040.0 * b for b in range(1, 26)]), 99, seed,
                    {"time_unit": "s", "parents": n_par, "lognormal_sigma": 1.0,
                     "cluster_frac": 0.7})


def config_large(seed: int = 0, n: int = 10_000_000) -> Workload:
    """Same POI generator at 5x density: n=10,000,000, 10,000 parents.

    20 x 20 thresholds to 1 km / 30 d (t in s); 199 CSR simulations.
    """
    rng = np.random.default_rng(seed)
    box = (0.0, 50_000.0, 0.0, 50_000.0, 0.0, 1095 * DAY)
    n_par = max(1, int(round(10_000 * n / 10_000_000)))
    x, y, t = poi_mixture(n, box, n_par, rng)
    return Workload("poi_n10M", x, y, t, box, even_thresholds(1000.0, 20),
                    np.array([129_600.0 * b for b in range(1, 21)]), 199, seed,
                    {"time_unit": "s", "parents": n_par, "lognormal_sigma": 1.0,
                     "cluster_frac": 0.7})


def serving_stream(count: int, seed: int = 0, n_datasets: int = 12, presets: int = 2,
                   n_lo: int = 1000, n_hi: int = 1_000_000, max_sims: int = 199,
                   rate_hz: float = 50.0, neighbours: float = 300.0):
    """Synthetic request stream for the serving loop (Poisson arrivals of K / envelope jobs).

    A pool of `n_datasets` point sets stays registered with the server (the analyst's layers):
    n log-uniform in [n_lo, n_hi], drawn from the CSR, Thomas or POI-mixture generator, at a
    fixed density of one point per 500 m^2 over 365 days.  Each dataset carries `presets`
    threshold grids (5-50 thresholds per axis, evenly spaced) whose largest spatial threshold
    gives about `neighbours` CSR neighbours per point at a 60-day window, capped at a quarter
    of the side.  Each request picks a dataset, one of its grids, 0..max_sims simulations and
    its own simulation seed; arrivals are exponential with mean 1/rate_hz.

    Returns (datasets, requests): datasets is a list of Workload (n_sims 0), requests a list of
    dicts {arrival_s, dataset, s, tt, n_sims, seed}.
    """
    rng = np.random.default_rng(seed)
    datasets, grids = [], []
    for d in range(n_datasets):
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        kind = d % 3
        side = float((500.0 * n) ** 0.5)
        box = (0.0, side, 0.0, side, 0.0, 365.0)
        sub = int(rng.integers(0, 2**31))
        r = np.random.default_rng(sub)
        if kind == 0:
            x, y, t = csr(n, box, sub)
        elif kind == 1:
            x, y, t = thomas(n, box, max(1, n // 500), 150.0, 10.0, r)
        else:
            x, y, t = poi_mixture(n, box, max(1, n // 1000), r, sigma_s=150.0, sigma_t_s=10.0)
        s_max = min(0.25 * side, float((neighbours * 500.0 * 365.0 / (60.0 * math.pi)) ** 0.5))
        mine = []
        for _ in range(presets):
            cs = int(rng.integers(5, 51))
            ct = int(rng.integers(5, 51))
            mine.append((even_thresholds(s_max, cs), even_thresholds(30.0, ct)))
        grids.append(mine)
        datasets.append(Workload(f"layer{d}", x, y, t, box, mine[0][0], mine[0][1], 0, 0,
                                 {"kind": ("csr", "thomas", "poi_mixture")[kind]}))
    requests = []
    clock = 0.0
    for _ in range(count):
        clock += float(rng.exponential(1.0 / rate_hz))
        d = int(rng.integers(0, n_datasets))
        s_, tt_ = grids[d][int(rng.integers(0, presets))]
        requests.append({"arrival_s": clock, "dataset": d, "s": s_, "tt": tt_,
                         "n_sims": int(rng.integers(0, max_sims + 1)),
                         "seed": int(rng.integers(0, 2**63))})
    return datasets, requests


def star_polygon(nv: int, r_out: float, r_in: float, cx: float, cy: float, seed: int):
    """A simple star-shaped polygon of nv vertices (alternating outer / inner radius with
    jitter, sorted angles): a stand-in for an irregular administrative outline."""
    rng = np.random.default_rng(seed)
    th = np.sort(rng.uniform(0.0, 2.0 * math.pi, nv))
    rad = np.where(np.arange(nv) % 2 == 0, r_out, r_in) * rng.uniform(0.85, 1.0, nv)
    return cx + rad * np.cos(th), cy + rad * np.sin(th)


def smooth_polygon(nv: int, r_mean: float, cx: float, cy: float, seed: int):
    """A simple polygon of nv vertices whose radius varies slowly with the angle (a few low
    harmonics of 5-15% and 1% jitter): a stand-in for an administrative outline without
    spikes."""
    rng = np.random.default_rng(seed)
    ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, nv))
    ph = rng.uniform(0.0, 2.0 * np.pi, 3)
    rad = r_mean * (1.0 + 0.15 * np.sin(2.0 * ang + ph[0]) + 0.08 * np.sin(3.0 * ang + ph[1]) +
                    0.05 * np.sin(5.0 * ang + ph[2]) + 0.01 * rng.uniform(-1.0, 1.0, nv))
    return cx + rad * np.cos(ang), cy + rad * np.sin(ang)


def inside_polygon(px, py, vx, vy):
    """Vectorised even-odd test (input generation only; boundary cases are immaterial)."""
    inside = np.zeros(np.shape(px), bool)
    n = len(vx)
    for k in range(n):
        ax, ay, bx, by = vx[k], vy[k], vx[(k + 1) % n], vy[(k + 1) % n]
        straddle = (ay > py) != (by > py)
        with np.errstate(divide="ignore", invalid="ignore"):
            xc = ax + (py - ay) * (bx - ax) / (by - ay)
        inside ^= straddle & (px < xc)
    return inside


def config_polygon(seed: int = 0, n: int = 200_000) -> Workload:
    """The Thomas configuration (10 km x 10 km x 730 d, sigma 150 m / 10 d) inside an
    85-vertex star polygon (the paper's experiments use an 85-vertex outline): n points drawn
    from the Thomas process and kept when inside; 20 x 20 thresholds to 1 km / 60 d; 99 CSR
    simulations in the polygon.  meta["polygon"] holds (vx, vy)."""
    rng = np.random.default_rng(seed)
    box = (0.0, 10_000.0, 0.0, 10_000.0, 0.0, 730.0)
    vx, vy = star_polygon(85, 5000.0, 3400.0, 5000.0, 5000.0, seed + 1)
    xs, ys, ts = [], [], []
    have = 0
    while have < n:
        x, y, t = thomas(n, box, 400, 150.0, 10.0, rng)
        keep = inside_polygon(x, y, vx, vy)
        xs.append(x[keep]), ys.append(y[keep]), ts.append(t[keep])
        have += int(keep.sum())
    x, y, t = (np.concatenate(a)[:n] for a in (xs, ys, ts))
    return Workload("thomas_polygon85_n200k", x, y, t, box, even_thresholds(1000.0, 20),
                    even_thresholds(60.0, 20), 99, seed,
                    {"time_unit": "day", "polygon": (vx, vy)})


def config_polygon_smooth(seed: int = 0, n: int = 200_000) -> Workload:
    """As config_polygon, inside an 85-vertex outline without spikes (smooth_polygon, mean
    radius 3800 m)."""
    rng = np.random.default_rng(seed)
    box = (0.0, 10_000.0, 0.0, 10_000.0, 0.0, 730.0)
    vx, vy = smooth_polygon(85, 3800.0, 5000.0, 5000.0, seed + 2)
    xs, ys, ts = [], [], []
    have = 0
    while have < n:
        x, y, t = thomas(n, box, 400, 150.0, 10.0, rng)
        keep = inside_polygon(x, y, vx, vy)
        xs.append(x[keep]), ys.append(y[keep]), ts.append(t[keep])
        have += int(keep.sum())
    x, y, t = (np.concatenate(a)[:n] for a in (xs, ys, ts))
    return Workload("thomas_smooth85_n200k", x, y, t, box, even_thresholds(1000.0, 20),
                    even_thresholds(60.0, 20), 99, seed,
                    {"time_unit": "day", "polygon": (vx, vy)})


def histogram_intensity(x, y, t, box, shape, floor: float = 0.05) -> np.ndarray:
    """A relative intensity for the inhomogeneous K: the point counts on `shape` = (nit, niy,
    nix) equal cells of the box plus `floor` times the mean count, so that every cell is
    positive (a stand-in for a smoothed estimate of the first-order intensity)."""
    nit, niy, nix = shape
    x0, x1, y0, y1, t0, t1 = box
    ix = np.clip(((np.asarray(x) - x0) / (x1 - x0) * nix).astype(np.int64), 0, nix - 1)
    iy = np.clip(((np.asarray(y) - y0) / (y1 - y0) * niy).astype(np.int64), 0, niy - 1)
    it = np.clip(((np.asarray(t) - t0) / (t1 - t0) * nit).astype(np.int64), 0, nit - 1)
    counts = np.bincount((it * niy + iy) * nix + ix, minlength=nit * niy * nix).astype(float)
    return (counts + floor * counts.mean()).reshape(nit, niy, nix)


def config_inhom(seed: int = 0, n: int = 200_000) -> Workload:
    """The Thomas configuration with a relative intensity for the inhomogeneous K: point
    counts on 10 x 10 x 8 cells (1 km x 1 km x 91.25 d) plus 5 % of the mean count;
    meta["rho"] holds it ([nit][niy][nix]).  99 intensity-weighted simulations."""
    w = config_thomas(seed, n)
    rho = histogram_intensity(w.x, w.y, w.t, w.box, (8, 10, 10))
    return Workload("thomas_inhom_n200k", w.x, w.y, w.t, w.box, w.s, w.tt, w.n_sims,
                    w.sim_seed, dict(w.meta, rho=rho))


CONFIGS = {
    "csr_n2000": config_csr_small,
    "thomas_n200k": config_thomas,
    "poi_n2M": config_poi,
    "poi_n10M": config_large,
    "thomas_polygon85_n200k": config_polygon,
    "thomas_smooth85_n200k": config_polygon_smooth,
    "thomas_inhom_n200k": config_inhom,
}
