"""Oracle for the edge-corrected space-time Ripley's K estimator (test infrastructure).

A plain, single-threaded FP64 CPU restatement of the paper's Section 3 (Eq. 2-4 and the
simulation envelopes: Monte Carlo CSR, bootstrapping, random permutation), compiled from ``stk_oracle.c`` with gcc and loaded through
ctypes.  Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference legs may import it; the CUDA library never calls it and shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "stk_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
             "-fno-fast-math", "-pthread", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        # STK_ORACLE_LIB: a deliberately broken copy, for the tests that check that the pins
        # catch planted mistakes
        lib = ctypes.CDLL(os.environ.get("STK_ORACLE_LIB") or build())
        d, i64, i32, u64, u32 = (ctypes.c_double, ctypes.c_int64, ctypes.c_int,
                                 ctypes.c_uint64, ctypes.c_uint32)
        P = ctypes.c_void_p
        lib.oracle_philox4x32_10.argtypes = [P, P, P]
        lib.oracle_philox4x32_10.restype = None
        lib.oracle_u01.argtypes = [u32, u32]
        lib.oracle_u01.restype = d
        lib.oracle_csr_points.argtypes = [i64, P, u64, u32, P, P, P]
        lib.oracle_csr_points.restype = None
        lib.oracle_spatial_weight.argtypes = [d, d, d, P]
        lib.oracle_spatial_weight.restype = d
        lib.oracle_temporal_weight.argtypes = [d, d, d, d]
        lib.oracle_temporal_weight.restype = d
        lib.oracle_pair_hist.argtypes = [i64, P, P, P, P, P, i32, P, i32, i32, P, P, P]
        lib.oracle_pair_hist.restype = i64
        lib.oracle_finalize.argtypes = [i64, P, P, i32, P, i32, i32, P, P, P, P, P, P]
        lib.oracle_finalize.restype = None
        lib.oracle_k.argtypes = [i64, P, P, P, P, P, i32, P, i32, i32, i32, P, P, P, P]
        lib.oracle_k.restype = i64
        lib.oracle_envelope.argtypes = [i64, P, P, i32, P, i32, i32, i32, i32, u64, P, P, P,
                                        P, P]
        lib.oracle_envelope.restype = ctypes.c_int
        lib.oracle_bootstrap_index.argtypes = [i64, u64, u32, i64]
        lib.oracle_bootstrap_index.restype = i64
        lib.oracle_bootstrap_points.argtypes = [P, P, P, i64, u64, u32, P, P, P]
        lib.oracle_bootstrap_points.restype = None
        lib.oracle_feistel_bits.argtypes = [i64]
        lib.oracle_feistel_bits.restype = ctypes.c_int
        lib.oracle_feistel.argtypes = [u64, ctypes.c_int, u64, u32]
        lib.oracle_feistel.restype = u64
        lib.oracle_permutation_index.argtypes = [i64, u64, u32, i64]
        lib.oracle_permutation_index.restype = i64
        lib.oracle_permutation_points.argtypes = [P, P, P, i64, u64, u32, P, P, P]
        lib.oracle_permutation_points.restype = None
        lib.oracle_finalize_area.argtypes = [i64, d, d, P, i32, P, i32, i32, P, P, P, P, P, P]
        lib.oracle_finalize_area.restype = None
        lib.oracle_polygon_area.argtypes = [P, P, i32]
        lib.oracle_polygon_area.restype = d
        lib.oracle_point_in_polygon.argtypes = [d, d, P, P, i32]
        lib.oracle_point_in_polygon.restype = i32
        lib.oracle_polygon_weight.argtypes = [d, d, d, P, P, i32]
        lib.oracle_polygon_weight.restype = d
        lib.oracle_pair_hist_polygon.argtypes = [i64, P, P, P, P, P, P, i32, P, i32, P, i32,
                                                 i32, P, P]
        lib.oracle_pair_hist_polygon.restype = i64
        lib.oracle_csr_polygon_points.argtypes = [i64, P, P, P, i32, u64, u32, i32, P, P, P]
        lib.oracle_csr_polygon_points.restype = i32
        lib.oracle_k_cross.argtypes = [i64, P, P, P, P, i32, i32, P, P, i32, P, i32, i32, i32,
                                       P, P, P, P]
        lib.oracle_k_cross.restype = i64
        lib.oracle_intensity_cell.argtypes = [P, i32, i32, i32, d, d, d]
        lib.oracle_intensity_cell.restype = i32
        lib.oracle_intensity_lambda.argtypes = [P, i32, i32, i32, P, i64, P]
        lib.oracle_intensity_lambda.restype = None
        lib.oracle_inhom_points.argtypes = [i64, P, P, i32, i32, i32, u64, u32, P, P, P, P]
        lib.oracle_inhom_points.restype = None
        lib.oracle_pair_hist_inhom.argtypes = [i64, P, P, P, P, P, P, i32, P, i32, i32, P, P,
                                               P]
        lib.oracle_pair_hist_inhom.restype = i64
        lib.oracle_finalize_inhom.argtypes = [i64, P, P, i32, P, i32, i32, P, P, P, P, P, P]
        lib.oracle_finalize_inhom.restype = None
        lib.oracle_translation_weight.argtypes = [d, d, d, P]
        lib.oracle_translation_weight.restype = d
        lib.oracle_sector.argtypes = [d, d, i32]
        lib.oracle_sector.restype = i32
        lib.oracle_pair_hist_dir.argtypes = [i64, P, P, P, P, P, i32, P, i32, i32, i32, P, P,
                                             P]
        lib.oracle_pair_hist_dir.restype = i64
        lib.oracle_pair_hist_grid.argtypes = [i64, P, P, P, P, P, i32, P, i32, i32, P, i32, P, P]
        lib.oracle_pair_hist_grid.restype = i64
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _box(box):
    b = _f64(box)
    assert b.shape == (6,)
    return b


def philox4x32_10(ctr, key):
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(w0: int, w1: int) -> float:
    return _load().oracle_u01(w0, w1)


def csr_points(n: int, box, seed: int, sim: int):
    """Realization `sim` of the Monte Carlo CSR simulation (Section 3)."""
    x = np.empty(n, np.float64)
    y = np.empty(n, np.float64)
    t = np.empty(n, np.float64)
    b = _box(box)
    _load().oracle_csr_points(n, _ptr(b), seed, sim, _ptr(x), _ptr(y), _ptr(t))
    return x, y, t


def spatial_weight(xi: float, yi: float, r: float, box) -> float:
    b = _box(box)
    return _load().oracle_spatial_weight(xi, yi, r, _ptr(b))


def temporal_weight(ti: float, u: float, t0: float, t1: float) -> float:
    return _load().oracle_temporal_weight(ti, u, t0, t1)


def pair_hist(x, y, t, box, s, tt, edge_mode=1, centre_mask=None):
    """Non-cumulative (count, weighted sum) histograms over ordered pairs (Eq. 2, 3)."""
    x, y, t, s, tt = map(_f64, (x, y, t, s, tt))
    b = _box(box)
    cs, ct = len(s), len(tt)
    cnt = np.zeros(cs * ct, np.int64)
    wsum = np.zeros(cs * ct, np.float64)
    m = None if centre_mask is None else np.ascontiguousarray(centre_mask, dtype=np.uint8)
    q = _load().oracle_pair_hist(len(x), _ptr(x), _ptr(y), _ptr(t), _ptr(b), _ptr(s), cs,
                                 _ptr(tt), ct, edge_mode, _ptr(m), _ptr(cnt), _ptr(wsum))
    return cnt.reshape(cs, ct), wsum.reshape(cs, ct), int(q)


def pair_hist_grid(x, y, t, box, s, tt, edge_mode=1, centre_mask=None, threads=None):
    """pair_hist over the same pairs with a grid and threads (for whole grids at large n)."""
    x, y, t, s, tt = map(_f64, (x, y, t, s, tt))
    b = _box(box)
    cs, ct = len(s), len(tt)
    cnt = np.zeros(cs * ct, np.int64)
    wsum = np.zeros(cs * ct, np.float64)
    m = None if centre_mask is None else np.ascontiguousarray(centre_mask, dtype=np.uint8)
    nt = threads or (os.cpu_count() or 1)
    q = _load().oracle_pair_hist_grid(len(x), _ptr(x), _ptr(y), _ptr(t), _ptr(b), _ptr(s), cs,
                                      _ptr(tt), ct, edge_mode, _ptr(m), nt, _ptr(cnt),
                                      _ptr(wsum))
    return cnt.reshape(cs, ct), wsum.reshape(cs, ct), int(q)


def finalize(n, box, s, tt, cnt, wsum, norm=0):
    """Cumulative C, S and K (Eq. 2), L (Eq. 4) from a non-cumulative histogram."""
    s, tt = _f64(s), _f64(tt)
    b = _box(box)
    cs, ct = len(s), len(tt)
    cnt = np.ascontiguousarray(cnt, dtype=np.int64).reshape(-1)
    wsum = _f64(wsum).reshape(-1)
    C = np.zeros(cs * ct, np.int64)
    S, K, L = (np.zeros(cs * ct, np.float64) for _ in range(3))
    _load().oracle_finalize(n, _ptr(b), _ptr(s), cs, _ptr(tt), ct, norm, _ptr(cnt), _ptr(wsum),
                            _ptr(C), _ptr(S), _ptr(K), _ptr(L))
    sh = (cs, ct)
    return C.reshape(sh), S.reshape(sh), K.reshape(sh), L.reshape(sh)


def k_function(x, y, t, box, s, tt, edge_mode=1, norm=0):
    """Full estimator: returns dict with cumulative C, S, K, L and the qualifying count."""
    x, y, t, s, tt = map(_f64, (x, y, t, s, tt))
    b = _box(box)
    cs, ct = len(s), len(tt)
    C = np.zeros(cs * ct, np.int64)
    S, K, L = (np.zeros(cs * ct, np.float64) for _ in range(3))
    q = _load().oracle_k(len(x), _ptr(x), _ptr(y), _ptr(t), _ptr(b), _ptr(s), cs, _ptr(tt), ct,
                         edge_mode, norm, _ptr(C), _ptr(S), _ptr(K), _ptr(L))
    sh = (cs, ct)
    return {"C": C.reshape(sh), "S": S.reshape(sh), "K": K.reshape(sh), "L": L.reshape(sh),
            "pairs": int(q)}


def envelope(n, box, s, tt, n_sims, seed, edge_mode=1, norm=0, keep_all=False):
    """Monte Carlo CSR envelope (Section 3): min / max of K over the simulations."""
    s, tt = _f64(s), _f64(tt)
    b = _box(box)
    cs, ct = len(s), len(tt)
    K_lo, K_hi, L_lo, L_hi = (np.zeros(cs * ct, np.float64) for _ in range(4))
    K_all = np.zeros(n_sims * cs * ct, np.float64) if keep_all else None
    rc = _load().oracle_envelope(n, _ptr(b), _ptr(s), cs, _ptr(tt), ct, edge_mode, norm,
                                 n_sims, seed, _ptr(K_lo), _ptr(K_hi), _ptr(L_lo), _ptr(L_hi),
                                 _ptr(K_all))
    if rc != 0:
        raise ValueError("oracle_envelope: invalid arguments")
    sh = (cs, ct)
    out = {"K_lo": K_lo.reshape(sh), "K_hi": K_hi.reshape(sh), "L_lo": L_lo.reshape(sh),
           "L_hi": L_hi.reshape(sh)}
    if keep_all:
        out["K_all"] = K_all.reshape(n_sims, cs, ct)
    return out


SIM_CSR, SIM_PERMUTATION, SIM_BOOTSTRAP = 0, 1, 2


def bootstrap_index(n: int, seed: int, sim: int, i: int) -> int:
    return int(_load().oracle_bootstrap_index(n, seed, sim, i))


def bootstrap_points(x, y, t, seed: int, sim: int):
    """Realization `sim` of the bootstrapping simulation (Section 3): n draws with
    replacement from the observed points."""
    x, y, t = _f64(x), _f64(y), _f64(t)
    n = len(x)
    ox, oy, ot = (np.empty(n, np.float64) for _ in range(3))
    _load().oracle_bootstrap_points(_ptr(x), _ptr(y), _ptr(t), n, seed, sim, _ptr(ox),
                                    _ptr(oy), _ptr(ot))
    return ox, oy, ot


def feistel_bits(n: int) -> int:
    return int(_load().oracle_feistel_bits(n))


def feistel(v: int, b: int, seed: int, sim: int) -> int:
    return int(_load().oracle_feistel(v, b, seed, sim))


def permutation_index(n: int, seed: int, sim: int, i: int) -> int:
    return int(_load().oracle_permutation_index(n, seed, sim, i))


def permutation_points(x, y, t, seed: int, sim: int):
    """Realization `sim` of the random-permutation simulation (Section 3): the observed
    points with their timestamps exchanged by a pseudo-random bijection."""
    x, y, t = _f64(x), _f64(y), _f64(t)
    n = len(x)
    ox, oy, ot = (np.empty(n, np.float64) for _ in range(3))
    _load().oracle_permutation_points(_ptr(x), _ptr(y), _ptr(t), n, seed, sim, _ptr(ox),
                                      _ptr(oy), _ptr(ot))
    return ox, oy, ot


def polygon_area(vx, vy) -> float:
    vx, vy = _f64(vx), _f64(vy)
    return _load().oracle_polygon_area(_ptr(vx), _ptr(vy), len(vx))


def point_in_polygon(px: float, py: float, vx, vy) -> bool:
    vx, vy = _f64(vx), _f64(vy)
    return bool(_load().oracle_point_in_polygon(px, py, _ptr(vx), _ptr(vy), len(vx)))


def polygon_weight(xi: float, yi: float, r: float, vx, vy) -> float:
    """Proportion of the circle's circumference inside the polygon (isotropic weight)."""
    vx, vy = _f64(vx), _f64(vy)
    return _load().oracle_polygon_weight(xi, yi, r, _ptr(vx), _ptr(vy), len(vx))


def k_function_polygon(x, y, t, box, vx, vy, s, tt, edge_mode=1, norm=0):
    """The estimator over a polygon study area (A = polygon area, period box[4..5])."""
    x, y, t, s, tt, vx, vy = map(_f64, (x, y, t, s, tt, vx, vy))
    b = _box(box)
    cs, ct = len(s), len(tt)
    cnt = np.zeros(cs * ct, np.int64)
    wsum = np.zeros(cs * ct, np.float64)
    lib = _load()
    q = lib.oracle_pair_hist_polygon(len(x), _ptr(x), _ptr(y), _ptr(t), _ptr(b), _ptr(vx),
                                     _ptr(vy), len(vx), _ptr(s), cs, _ptr(tt), ct, edge_mode,
                                     _ptr(cnt), _ptr(wsum))
    C = np.zeros(cs * ct, np.int64)
    S, K, L = (np.zeros(cs * ct, np.float64) for _ in range(3))
    lib.oracle_finalize_area(len(x), polygon_area(vx, vy), b[5] - b[4], _ptr(s), cs, _ptr(tt),
                             ct, norm, _ptr(cnt), _ptr(wsum), _ptr(C), _ptr(S), _ptr(K),
                             _ptr(L))
    sh = (cs, ct)
    return {"C": C.reshape(sh), "S": S.reshape(sh), "K": K.reshape(sh), "L": L.reshape(sh),
            "pairs": int(q)}


def csr_polygon_points(n: int, box, vx, vy, seed: int, sim: int, max_attempts: int = 4096):
    """Realization `sim` of CSR in a polygon (rejection from the bounding rectangle)."""
    vx, vy = _f64(vx), _f64(vy)
    b = _box(box)
    x, y, t = (np.empty(n, np.float64) for _ in range(3))
    rc = _load().oracle_csr_polygon_points(n, _ptr(b), _ptr(vx), _ptr(vy), len(vx), seed, sim,
                                           max_attempts, _ptr(x), _ptr(y), _ptr(t))
    if rc != 0:
        raise ValueError("a point found no position inside the polygon")
    return x, y, t


def _rho(rho):
    r = _f64(rho)
    assert r.ndim == 3, "rho is indexed [t][y][x]"
    return np.ascontiguousarray(r), r.shape[2], r.shape[1], r.shape[0]


def intensity_cell(box, rho_shape, x: float, y: float, t: float) -> int:
    """Cell of the intensity grid (shape [nit, niy, nix]) holding the point (x, y, t)."""
    nit, niy, nix = rho_shape
    return int(_load().oracle_intensity_cell(_ptr(_box(box)), nix, niy, nit, x, y, t))


def intensity_lambda(rho, box, n: int):
    """Intensity per cell: rho scaled to integrate to n over the box."""
    r, nix, niy, nit = _rho(rho)
    lam = np.empty(r.size, np.float64)
    _load().oracle_intensity_lambda(_ptr(r), nix, niy, nit, _ptr(_box(box)), n, _ptr(lam))
    return lam


def intensity_at(x, y, t, box, rho):
    """Intensity at each point: lambda of the cell that holds it."""
    lam = intensity_lambda(rho, box, len(x))
    cells = np.array([intensity_cell(box, np.shape(rho), float(a), float(b), float(c))
                      for a, b, c in zip(x, y, t)], dtype=np.int64)
    return lam[cells] if len(cells) else np.zeros(0)


def inhom_points(n: int, box, rho, seed: int, sim: int):
    """Realization `sim` of n points drawn with density proportional to rho, and the cell of
    each point."""
    r, nix, niy, nit = _rho(rho)
    x, y, t = (np.empty(n, np.float64) for _ in range(3))
    cell = np.empty(n, np.int32)
    _load().oracle_inhom_points(n, _ptr(_box(box)), _ptr(r), nix, niy, nit, seed, sim, _ptr(x),
                                _ptr(y), _ptr(t), _ptr(cell))
    return x, y, t, cell


def k_function_inhom(x, y, t, box, s, tt, lam, edge_mode=1, norm=0, centre_mask=None):
    """Inhomogeneous estimator with the intensity lam[i] at each point (see stk_oracle.c)."""
    x, y, t, s, tt, lam = map(_f64, (x, y, t, s, tt, lam))
    b = _box(box)
    cs, ct = len(s), len(tt)
    cnt = np.zeros(cs * ct, np.int64)
    wsum = np.zeros(cs * ct, np.float64)
    m = None if centre_mask is None else np.ascontiguousarray(centre_mask, dtype=np.uint8)
    lib = _load()
    q = lib.oracle_pair_hist_inhom(len(x), _ptr(x), _ptr(y), _ptr(t), _ptr(lam), _ptr(b),
                                   _ptr(s), cs, _ptr(tt), ct, edge_mode, _ptr(m), _ptr(cnt),
                                   _ptr(wsum))
    C = np.zeros(cs * ct, np.int64)
    S, K, L = (np.zeros(cs * ct, np.float64) for _ in range(3))
    lib.oracle_finalize_inhom(len(x), _ptr(b), _ptr(s), cs, _ptr(tt), ct, norm, _ptr(cnt),
                              _ptr(wsum), _ptr(C), _ptr(S), _ptr(K), _ptr(L))
    sh = (cs, ct)
    return {"C": C.reshape(sh), "S": S.reshape(sh), "K": K.reshape(sh), "L": L.reshape(sh),
            "pairs": int(q)}


def translation_weight(dx: float, dy: float, u: float, box) -> float:
    """Translation edge correction of a pair at offset (dx, dy) and time lag u."""
    return _load().oracle_translation_weight(dx, dy, u, _ptr(_box(box)))


def sector(dx: float, dy: float, n_sec: int) -> int:
    """Axial-direction sector of the offset (dx, dy) among n_sec equal sectors of [0, pi)."""
    return int(_load().oracle_sector(dx, dy, n_sec))


def k_function_dir(x, y, t, box, s, tt, n_sec, edge_mode=2, norm=0, centre_mask=None):
    """Directional (sector) K, translation-corrected with edge_mode 2 (see stk_oracle.c):
    cumulative C, S, K and L per sector, arrays [n_sec, cs, ct].  L of a sector is
    sqrt(n_sec K / (2 pi t)) - s, zero in expectation under CSR like Eq. 4."""
    x, y, t, s, tt = map(_f64, (x, y, t, s, tt))
    b = _box(box)
    cs, ct = len(s), len(tt)
    cnt = np.zeros(n_sec * cs * ct, np.int64)
    wsum = np.zeros(n_sec * cs * ct, np.float64)
    m = None if centre_mask is None else np.ascontiguousarray(centre_mask, dtype=np.uint8)
    q = _load().oracle_pair_hist_dir(len(x), _ptr(x), _ptr(y), _ptr(t), _ptr(b), _ptr(s), cs,
                                     _ptr(tt), ct, n_sec, edge_mode, _ptr(m), _ptr(cnt),
                                     _ptr(wsum))
    out = {k: [] for k in ("C", "S", "K", "L")}
    nb = cs * ct
    for k in range(n_sec):
        C, S_, K, _ = finalize(len(x), box, s, tt, cnt[k * nb:(k + 1) * nb],
                               wsum[k * nb:(k + 1) * nb], norm=norm)
        out["C"].append(C)
        out["S"].append(S_)
        out["K"].append(K)
        out["L"].append(np.sqrt(n_sec * K / (2.0 * np.pi * tt[None, :])) - s[:, None])
    res = {k: np.stack(v) for k, v in out.items()}
    res["pairs"] = int(q)
    return res


def simulation_points(method: int, x, y, t, box, seed: int, sim: int, polygon=None):
    """Realization `sim` of the given simulation method (Section 3)."""
    if method == SIM_CSR and polygon is not None:
        return csr_polygon_points(len(x), box, polygon[0], polygon[1], seed, sim)
    if method == SIM_CSR:
        return csr_points(len(x), box, seed, sim)
    if method == SIM_PERMUTATION:
        return permutation_points(x, y, t, seed, sim)
    if method == SIM_BOOTSTRAP:
        return bootstrap_points(x, y, t, seed, sim)
    raise ValueError(f"unknown simulation method {method}")


def envelope_of(method: int, x, y, t, box, s, tt, n_sims, seed, edge_mode=1, norm=0,
                polygon=None, rho=None, n_sec=0):
    """Envelope (Section 3) over n_sims realizations of any simulation method (optionally in
    a polygon study area, or of the inhomogeneous K with relative intensity rho, whose CSR
    realizations are then drawn with density proportional to rho): the element-wise min /
    max of K (and L of those), plus every realization's K."""
    Ks = []
    for k in range(n_sims):
        if n_sec > 0:
            px, py, pt = simulation_points(method, x, y, t, box, seed, k)
            Ks.append(k_function_dir(px, py, pt, box, s, tt, n_sec, edge_mode=edge_mode,
                                     norm=norm)["K"])
            continue
        if rho is not None:
            if method == SIM_CSR:
                px, py, pt, cell = inhom_points(len(x), box, rho, seed, k)
                lam = intensity_lambda(rho, box, len(x))[cell]
            else:
                px, py, pt = simulation_points(method, x, y, t, box, seed, k)
                lam = intensity_at(px, py, pt, box, rho)
            r = k_function_inhom(px, py, pt, box, s, tt, lam, edge_mode=edge_mode, norm=norm)
            Ks.append(r["K"])
            continue
        px, py, pt = simulation_points(method, x, y, t, box, seed, k, polygon)
        if polygon is None:
            r = k_function(px, py, pt, box, s, tt, edge_mode=edge_mode, norm=norm)
        else:
            r = k_function_polygon(px, py, pt, box, polygon[0], polygon[1], s, tt,
                                   edge_mode=edge_mode, norm=norm)
        Ks.append(r["K"])
    Ks = np.stack(Ks)
    s, tt = _f64(s), _f64(tt)
    lo, hi = Ks.min(axis=0), Ks.max(axis=0)
    den = 2.0 * np.pi * tt[None, :] / max(1, n_sec)
    return {"K_lo": lo, "K_hi": hi, "L_lo": np.sqrt(lo / den) - s[:, None],
            "L_hi": np.sqrt(hi / den) - s[:, None], "K_all": Ks}


def k_cross(x, y, t, labels, a, b, box, s, tt, edge_mode=1, norm=0):
    """Bivariate (cross) K between centres labelled a and neighbours labelled b."""
    x, y, t, s, tt = map(_f64, (x, y, t, s, tt))
    lab = np.ascontiguousarray(labels, dtype=np.uint8)
    bx = _box(box)
    cs, ct = len(s), len(tt)
    C = np.zeros(cs * ct, np.int64)
    S, K, L = (np.zeros(cs * ct, np.float64) for _ in range(3))
    q = _load().oracle_k_cross(len(x), _ptr(x), _ptr(y), _ptr(t), _ptr(lab), a, b, _ptr(bx),
                               _ptr(s), cs, _ptr(tt), ct, edge_mode, norm, _ptr(C), _ptr(S),
                               _ptr(K), _ptr(L))
    sh = (cs, ct)
    return {"C": C.reshape(sh), "S": S.reshape(sh), "K": K.reshape(sh), "L": L.reshape(sh),
            "pairs": int(q)}

