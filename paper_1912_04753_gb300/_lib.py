"""ctypes binding of libstk.so: the C ABI declared in include/stk.h, same names.

Argument marshalling only: every step of the computation runs in the CUDA library.  There is
no fallback: if libstk.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libstk.so")

STK_OK, STK_EINVAL, STK_EDOMAIN, STK_ENOMEM, STK_ECUDA, STK_ETIMEOUT, STK_EBUSY, STK_ENODEV = range(8)
STK_EDGE_NONE, STK_EDGE_ISOTROPIC, STK_EDGE_TRANSLATION = 0, 1, 2
STK_PREC_FP64, STK_PREC_FP32_GUARDED = 0, 1
STK_NORM_N_NM1, STK_NORM_N2 = 0, 1
STK_EXEC_BATCHED, STK_EXEC_PLAIN = 0, 1
STK_SIM_CSR, STK_SIM_PERMUTATION, STK_SIM_BOOTSTRAP = 0, 1, 2
STK_MAX_THRESHOLDS = 64

_P = ctypes.c_void_p


class StkError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[stk status {code}] {msg}")
        self.code = code


class stk_box(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("x0", "x1", "y0", "y1", "t0", "t1")]


class stk_request(ctypes.Structure):
    _fields_ = [("s", _P), ("cs", ctypes.c_int), ("tt", _P), ("ct", ctypes.c_int),
                ("edge_mode", ctypes.c_int), ("prec", ctypes.c_int), ("norm", ctypes.c_int),
                ("n_sims", ctypes.c_int), ("seed", ctypes.c_uint64), ("exec", ctypes.c_int),
                ("centre_mask", _P), ("sim_method", ctypes.c_int), ("first_sim", ctypes.c_uint32),
                ("labels", _P), ("cross_a", ctypes.c_int), ("cross_b", ctypes.c_int),
                ("n_sectors", ctypes.c_int), ("shard_count", ctypes.c_int),
                ("shard_index", ctypes.c_int)]


class stk_result(ctypes.Structure):
    _fields_ = [(k, _P) for k in ("K", "L", "raw_sum", "pair_count", "K_lo", "K_hi", "L_lo",
                                  "L_hi", "K_sims", "count_sims")]


class stk_stats(ctypes.Structure):
    _fields_ = [("qualifying_pairs", ctypes.c_int64), ("candidate_pairs", ctypes.c_int64),
                ("fp64_recomputed", ctypes.c_int64), ("work_items", ctypes.c_int64),
                ("realizations", ctypes.c_int32), ("waves", ctypes.c_int32),
                ("ms_total", ctypes.c_double), ("ms_pair", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("internal_errors", ctypes.c_int64),
                ("grid_refinement", ctypes.c_int32), ("graph_replays", ctypes.c_int32),
                ("grid_refinement_t", ctypes.c_int32), ("obs_index_reused", ctypes.c_int32),
                ("tile_units", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]


class stk_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("slots", ctypes.c_int),
                ("mem_budget_bytes", ctypes.c_int64), ("max_batch_sims", ctypes.c_int),
                ("max_queue", ctypes.c_int), ("no_merge", ctypes.c_int), ("fuse", ctypes.c_int)]


class stk_job(ctypes.Structure):
    _fields_ = [("dataset", ctypes.c_uint64), ("s", _P), ("cs", ctypes.c_int), ("tt", _P),
                ("ct", ctypes.c_int), ("edge_mode", ctypes.c_int), ("prec", ctypes.c_int),
                ("norm", ctypes.c_int), ("n_sims", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("want_sims", ctypes.c_int), ("sim_method", ctypes.c_int),
                ("n_sectors", ctypes.c_int)]


class stk_serve_stats(ctypes.Structure):
    _fields_ = ([(k, ctypes.c_int64) for k in (
        "submitted", "completed", "failed", "queued", "running", "max_queue_depth", "batches",
        "merged_jobs", "simulations", "qualifying_pairs")] +
        [(k, ctypes.c_double) for k in (
            "p50_ms", "p99_ms", "max_ms", "mean_ms", "wall_s", "jobs_per_s", "sims_per_s")] +
        [(k, ctypes.c_int64) for k in ("resident_bytes", "peak_bytes", "budget_bytes",
                                        "kernel_launches", "fused_jobs")])


_lib = None


def load(build_if_missing: bool = False):
    """Load libstk.so (raises OSError if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        if build_if_missing:
            from . import build as _b

            _b.build()
        else:
            raise OSError(f"libstk.so not built ({LIB_PATH}); run paper_1912_04753_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    i32, i64, u64, u32 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
    PP = ctypes.POINTER(_P)
    sig = {
        "stk_create": ([_P, _P, _P, i64, ctypes.POINTER(stk_box), PP], i32),
        "stk_create_device": ([_P, _P, _P, i64, ctypes.POINTER(stk_box), _P, PP], i32),
        "stk_set_stream": ([_P, _P], i32),
        "stk_k": ([_P, _P, i32, _P, i32, i32, i32, i32, _P, _P, _P, _P], i32),
        "stk_envelope": ([_P, _P, i32, _P, i32, i32, i32, i32, i32, u64, _P, _P, _P, _P], i32),
        "stk_run": ([_P, ctypes.POINTER(stk_request), ctypes.POINTER(stk_result)], i32),
        "stk_run_fused": ([ctypes.POINTER(_P), ctypes.POINTER(stk_request),
                           ctypes.POINTER(stk_result), i32, ctypes.POINTER(i32)], i32),
        "stk_last_stats": ([_P, ctypes.POINTER(stk_stats)], i32),
        "stk_last_accumulators": ([_P, i32, i32, _P], i32),
        "stk_merge_grids": ([_P, ctypes.POINTER(stk_request), _P, i32, _P, _P, _P, _P], i32),
        "stk_envelope_merge": ([_P, i32, i32, i32, i32, _P, _P, _P, _P, _P, _P], i32),
        "stk_sim_points": ([ctypes.POINTER(stk_box), i64, u64, u32, _P, _P, _P], i32),
        "stk_sim_resample": ([_P, _P, _P, i64, i32, u64, u32, _P, _P, _P], i32),
        "stk_sim_points_polygon": ([ctypes.POINTER(stk_box), _P, _P, i32, i64, u64, u32, _P, _P,
                                    _P], i32),
        "stk_set_polygon": ([_P, _P, _P, i32], i32),
        "stk_set_intensity": ([_P, _P, i32, i32, i32], i32),
        "stk_sim_points_inhom": ([ctypes.POINTER(stk_box), _P, i32, i32, i32, i64, u64, u32,
                                  _P, _P, _P], i32),
        "stk_k_noalloc": ([_P, _P, _P, i64, ctypes.POINTER(stk_box), _P, i32, _P, i32, i32, _P,
                           _P, _P, _P, _P], i32),
        "stk_server_create": ([ctypes.POINTER(stk_server_config), PP], i32),
        "stk_server_register": ([_P, _P, _P, _P, i64, ctypes.POINTER(stk_box),
                                 ctypes.POINTER(u64)], i32),
        "stk_server_unregister": ([_P, u64], i32),
        "stk_server_set_polygon": ([_P, u64, _P, _P, i32], i32),
        "stk_server_set_intensity": ([_P, u64, _P, i32, i32, i32], i32),
        "stk_submit": ([_P, ctypes.POINTER(stk_job), ctypes.POINTER(u64)], i32),
        "stk_poll": ([_P, u64, ctypes.POINTER(stk_result), i32, ctypes.POINTER(ctypes.c_double)],
                     i32),
        "stk_server_stats": ([_P, ctypes.POINTER(stk_serve_stats)], i32),
        "stk_server_reset_stats": ([_P], i32),
        "stk_server_destroy": ([_P], None),
        "stk_destroy": ([_P], None),
        "stk_last_error": ([], ctypes.c_char_p),
        "stk_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int):
    if rc != STK_OK:
        raise StkError(rc, load().stk_last_error().decode())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _box(box) -> stk_box:
    return stk_box(*[float(v) for v in box])


def stk_version() -> str:
    return load().stk_version().decode()


def stk_last_error() -> str:
    return load().stk_last_error().decode()


def stk_create(x, y, t, box):
    """Copy n host points into a new handle (returns an opaque handle)."""
    x, y, t = _f64(x), _f64(y), _f64(t)
    if not (x.shape == y.shape == t.shape and x.ndim == 1):
        raise ValueError("x, y, t must be 1-D arrays of equal length")
    h = _P()
    b = _box(box)
    _check(load().stk_create(_ptr(x), _ptr(y), _ptr(t), x.shape[0], ctypes.byref(b),
                             ctypes.byref(h)))
    return h


def stk_create_device(x, y, t, box, stream=None):
    """Create a handle from device-resident FP64 torch tensors (copied on the device)."""
    for v in (x, y, t):
        if not (v.is_cuda and v.dtype.is_floating_point and v.element_size() == 8
                and v.is_contiguous()):
            raise ValueError("device inputs must be contiguous float64 CUDA tensors")
    h = _P()
    b = _box(box)
    st = None if stream is None else _P(stream.cuda_stream)
    _check(load().stk_create_device(_P(x.data_ptr()), _P(y.data_ptr()), _P(t.data_ptr()),
                                    x.numel(), ctypes.byref(b), st, ctypes.byref(h)))
    return h


def stk_set_stream(h, stream=None):
    st = None if stream is None else _P(stream.cuda_stream)
    _check(load().stk_set_stream(h, st))


def stk_destroy(h):
    if h:
        load().stk_destroy(h)


def stk_k(h, s, tt, edge_mode=STK_EDGE_ISOTROPIC, prec=STK_PREC_FP32_GUARDED,
          norm=STK_NORM_N_NM1):
    """Observed K, L, raw weighted sum and pair count grids ([cs, ct], cumulative)."""
    s, tt = _f64(s), _f64(tt)
    cs, ct = s.shape[0], tt.shape[0]
    K, L, S = (np.zeros(cs * ct) for _ in range(3))
    C = np.zeros(cs * ct, np.int64)
    _check(load().stk_k(h, _ptr(s), cs, _ptr(tt), ct, edge_mode, prec, norm, _ptr(K), _ptr(L),
                        _ptr(S), _ptr(C)))
    sh = (cs, ct)
    return {"K": K.reshape(sh), "L": L.reshape(sh), "S": S.reshape(sh), "C": C.reshape(sh)}


def stk_envelope(h, s, tt, n_sims, seed, edge_mode=STK_EDGE_ISOTROPIC,
                 prec=STK_PREC_FP32_GUARDED, norm=STK_NORM_N_NM1):
    s, tt = _f64(s), _f64(tt)
    cs, ct = s.shape[0], tt.shape[0]
    out = [np.zeros(cs * ct) for _ in range(4)]
    _check(load().stk_envelope(h, _ptr(s), cs, _ptr(tt), ct, edge_mode, prec, norm, n_sims,
                               seed, *[_ptr(o) for o in out]))
    sh = (cs, ct)
    return {k: v.reshape(sh) for k, v in zip(("K_lo", "K_hi", "L_lo", "L_hi"), out)}


def _request(s, tt, n_sims=0, seed=0, edge_mode=STK_EDGE_ISOTROPIC,
             prec=STK_PREC_FP32_GUARDED, norm=STK_NORM_N_NM1, exec_mode=STK_EXEC_BATCHED,
             centre_mask=None, sim_method=STK_SIM_CSR, first_sim=0, labels=None, cross=(0, 0),
             n_sectors=0, shard=(0, 0)):
    """(stk_request, arrays it points to): the arrays must outlive the call."""
    mask = None if centre_mask is None else np.ascontiguousarray(centre_mask, dtype=np.uint8)
    lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.uint8)
    q = stk_request(_ptr(s), s.shape[0], _ptr(tt), tt.shape[0], edge_mode, prec, norm, n_sims,
                    seed, exec_mode, _ptr(mask), sim_method, first_sim, _ptr(lab),
                    int(cross[0]), int(cross[1]), int(n_sectors), int(shard[0]), int(shard[1]))
    return q, (s, tt, mask, lab)


def stk_run(h, s, tt, n_sims=0, seed=0, edge_mode=STK_EDGE_ISOTROPIC,
            prec=STK_PREC_FP32_GUARDED, norm=STK_NORM_N_NM1, exec_mode=STK_EXEC_BATCHED,
            centre_mask=None, want_sims=False, sim_method=STK_SIM_CSR, first_sim=0,
            labels=None, cross=(0, 0), n_sectors=0, shard=(0, 0)):
    """A whole job: observed grids plus the n_sims CSR envelope (and optionally every sim).
    With n_sectors > 1 (directional K) every grid is [n_sectors, cs, ct].  shard = (count,
    index) evaluates only that shard of the observed pattern's pairs (see stk_request)."""
    q, keep, o, r, shape = _job(s, tt, n_sims, seed, edge_mode, prec, norm, exec_mode,
                                centre_mask, want_sims, sim_method, first_sim, labels, cross,
                                n_sectors, shard)
    _check(load().stk_run(h, ctypes.byref(q), ctypes.byref(r)))
    return _shaped(o, shape)


def _job(s, tt, n_sims=0, seed=0, edge_mode=STK_EDGE_ISOTROPIC, prec=STK_PREC_FP32_GUARDED,
         norm=STK_NORM_N_NM1, exec_mode=STK_EXEC_BATCHED, centre_mask=None, want_sims=False,
         sim_method=STK_SIM_CSR, first_sim=0, labels=None, cross=(0, 0), n_sectors=0,
         shard=(0, 0)):
    """Request and result structures of one job, with the arrays they point to."""
    s, tt = _f64(s), _f64(tt)
    cs, ct = s.shape[0], tt.shape[0]
    grid = (n_sectors, cs, ct) if n_sectors > 1 else (cs, ct)
    nb = int(np.prod(grid))
    q, keep = _request(s, tt, n_sims, seed, edge_mode, prec, norm, exec_mode, centre_mask,
                       sim_method, first_sim, labels, cross, n_sectors, shard)
    o = {"K": np.zeros(nb), "L": np.zeros(nb), "S": np.zeros(nb), "C": np.zeros(nb, np.int64)}
    if n_sims > 0:
        for k in ("K_lo", "K_hi", "L_lo", "L_hi"):
            o[k] = np.zeros(nb)
        if want_sims:
            o["K_sims"] = np.zeros(n_sims * nb)
            o["C_sims"] = np.zeros(n_sims * nb, np.int64)
    r = stk_result(_ptr(o["K"]), _ptr(o["L"]), _ptr(o["S"]), _ptr(o["C"]), _ptr(o.get("K_lo")),
                   _ptr(o.get("K_hi")), _ptr(o.get("L_lo")), _ptr(o.get("L_hi")),
                   _ptr(o.get("K_sims")), _ptr(o.get("C_sims")))
    return q, keep, o, r, (n_sims, grid)


def _shaped(o, shape):
    n_sims, grid = shape
    return {k: v.reshape((n_sims,) + grid) if k in ("K_sims", "C_sims") else v.reshape(grid)
            for k, v in o.items()}


def stk_run_fused(handles, jobs):
    """Several jobs, job i on handles[i] (distinct point sets) with the keywords of stk_run in
    the dict jobs[i] (s and tt included), their pair kernels in one persistent launch (see
    stk_run_fused in stk.h).  Returns (list of result dicts as stk_run's, pair launches)."""
    if len(handles) != len(jobs) or not handles:
        raise ValueError("one job per handle, at least one")
    built = [_job(**j) for j in jobs]
    nj = len(built)
    hs = (_P * nj)(*handles)
    qs = (stk_request * nj)(*[b[0] for b in built])
    rs = (stk_result * nj)(*[b[3] for b in built])
    launches = ctypes.c_int32(0)
    _check(load().stk_run_fused(hs, qs, rs, nj, ctypes.byref(launches)))
    return [_shaped(b[2], b[4]) for b in built], int(launches.value)


def stk_last_accumulators(h, row0=0, rows=1, n_sectors=0, cs=None, ct=None):
    """Raw integer accumulators of realizations row0 .. row0 + rows - 1 of the last job on h
    (row 0 = observed when the job had one): uint64 [rows, 4, nbins] (count, excess low half,
    excess high half, whole part; per bin, not cumulative).  cs, ct: the job's grid."""
    nb = int(cs) * int(ct) * (n_sectors if n_sectors > 1 else 1)
    out = np.zeros((rows, 4, nb), np.uint64)
    _check(load().stk_last_accumulators(h, row0, rows, _ptr(out)))
    return out


def stk_merge_grids(h, acc, s, tt, **kw):
    """Cumulative K, L, S, C grids from merged accumulators acc [rows, 4, nbins] (uint64),
    normalised as a request with the keywords of stk_run would be on h.  Returns the dict of
    grids, each [rows, (n_sectors,) cs, ct]."""
    s, tt = _f64(s), _f64(tt)
    acc = np.ascontiguousarray(acc, dtype=np.uint64)
    if acc.ndim != 3 or acc.shape[1] != 4:
        raise ValueError("acc must be [rows, 4, nbins]")
    rows, nbins = acc.shape[0], acc.shape[2]
    nsec = kw.get("n_sectors", 0)
    grid = (nsec, s.shape[0], tt.shape[0]) if nsec > 1 else (s.shape[0], tt.shape[0])
    if int(np.prod(grid)) != nbins:
        raise ValueError("acc's bin count does not match the thresholds and sectors")
    kw.pop("want_sims", None)
    q, keep = _request(s, tt, **kw)
    o = {"K": np.zeros(rows * nbins), "L": np.zeros(rows * nbins), "S": np.zeros(rows * nbins),
         "C": np.zeros(rows * nbins, np.int64)}
    _check(load().stk_merge_grids(h, ctypes.byref(q), _ptr(acc), rows, _ptr(o["K"]),
                                  _ptr(o["L"]), _ptr(o["S"]), _ptr(o["C"])))
    return {k: v.reshape((rows,) + grid) for k, v in o.items()}


def stk_envelope_merge(K_rows, s, tt, n_sectors=0):
    """Element-wise min / max over the rows of K_rows [rows, (n_sectors,) cs, ct] and L of
    those (computed by the library on the current device): dict K_lo, K_hi, L_lo, L_hi."""
    s, tt = _f64(s), _f64(tt)
    K = np.ascontiguousarray(K_rows, dtype=np.float64)
    cs, ct = s.shape[0], tt.shape[0]
    grid = (n_sectors, cs, ct) if n_sectors > 1 else (cs, ct)
    nb = int(np.prod(grid))
    if K.size % nb or K.size == 0:
        raise ValueError("K_rows must hold whole grids of the thresholds' shape")
    rows = K.size // nb
    out = [np.zeros(nb) for _ in range(4)]
    _check(load().stk_envelope_merge(_ptr(K), rows, cs, ct, int(n_sectors), _ptr(s), _ptr(tt),
                                     *[_ptr(o) for o in out]))
    return {k: v.reshape(grid) for k, v in zip(("K_lo", "K_hi", "L_lo", "L_hi"), out)}


def stk_last_stats(h) -> dict:
    st = stk_stats()
    _check(load().stk_last_stats(h, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in stk_stats._fields_}


def stk_sim_points(box, n, seed, sim):
    """Realization `sim` of the device CSR generator, copied back to host arrays."""
    x, y, t = (np.zeros(n) for _ in range(3))
    b = _box(box)
    _check(load().stk_sim_points(ctypes.byref(b), n, seed, sim, _ptr(x), _ptr(y), _ptr(t)))
    return x, y, t


def stk_set_polygon(h, vx=None, vy=None):
    """Make the polygon (vx, vy) the study area of later jobs on h (None: back to the box)."""
    if vx is None:
        _check(load().stk_set_polygon(h, None, None, 0))
        return
    vx, vy = _f64(vx), _f64(vy)
    _check(load().stk_set_polygon(h, _ptr(vx), _ptr(vy), vx.shape[0]))


def _rho3(rho):
    r = np.ascontiguousarray(rho, dtype=np.float64)
    if r.ndim != 3:
        raise ValueError("rho must be a 3-D array indexed [t][y][x]")
    return r


def stk_set_intensity(h, rho=None):
    """Relative intensity rho[nit, niy, nix] over the box for the inhomogeneous K of later jobs
    on h (None: back to the homogeneous estimator)."""
    if rho is None:
        _check(load().stk_set_intensity(h, None, 0, 0, 0))
        return
    r = _rho3(rho)
    _check(load().stk_set_intensity(h, _ptr(r), r.shape[2], r.shape[1], r.shape[0]))


def stk_sim_points_inhom(box, rho, n, seed, sim):
    """Realization `sim` of the intensity-weighted simulation (device generator), copied back
    to the host."""
    r = _rho3(rho)
    x, y, t = (np.zeros(n) for _ in range(3))
    b = _box(box)
    _check(load().stk_sim_points_inhom(ctypes.byref(b), _ptr(r), r.shape[2], r.shape[1],
                                       r.shape[0], n, seed, sim, _ptr(x), _ptr(y), _ptr(t)))
    return x, y, t


def stk_sim_points_polygon(box, vx, vy, n, seed, sim):
    """Realization `sim` of CSR in the polygon (device generator), copied back to the host."""
    vx, vy = _f64(vx), _f64(vy)
    x, y, t = (np.zeros(n) for _ in range(3))
    b = _box(box)
    _check(load().stk_sim_points_polygon(ctypes.byref(b), _ptr(vx), _ptr(vy), vx.shape[0], n,
                                         seed, sim, _ptr(x), _ptr(y), _ptr(t)))
    return x, y, t


def stk_sim_resample(x, y, t, method, seed, sim):
    """Realization `sim` of the device permutation / bootstrap generator (Section 3) of the
    host points x, y, t, copied back to host arrays."""
    x, y, t = _f64(x), _f64(y), _f64(t)
    n = x.shape[0]
    ox, oy, ot = (np.zeros(n) for _ in range(3))
    _check(load().stk_sim_resample(_ptr(x), _ptr(y), _ptr(t), n, method, seed, sim, _ptr(ox),
                                   _ptr(oy), _ptr(ot)))
    return ox, oy, ot


def _check_noalloc_tensors(x, y, t, K, L, S, C, cells, current=None):
    """The device buffers stk_k_noalloc reads and writes, checked before the call: a wrong
    dtype, size or device would otherwise turn into out-of-bounds device accesses.  `current`:
    the current CUDA device index (looked up when None)."""
    import torch

    named = (("x", x, torch.float64), ("y", y, torch.float64), ("t", t, torch.float64),
             ("K", K, torch.float64), ("L", L, torch.float64), ("S", S, torch.float64),
             ("C", C, torch.int64))
    for name, v, _ in named:
        if not getattr(v, "is_cuda", False):
            raise ValueError(f"{name} must be a CUDA tensor")
    if current is None:
        current = torch.cuda.current_device()
    for name, v, dt in named:
        if v.device.index != current:
            raise ValueError(f"{name} must live on the current CUDA device (cuda:{current})")
        if v.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {v.dtype}")
        if not v.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if not (x.numel() == y.numel() == t.numel()):
        raise ValueError("x, y and t must have the same number of points")
    for name, v in (("K", K), ("L", L), ("S", S), ("C", C)):
        if v.numel() < cells:
            raise ValueError(f"{name} must hold at least cs * ct = {cells} values")


def stk_k_noalloc(x, y, t, box, s, tt, K, L, S, C, edge_mode=STK_EDGE_ISOTROPIC, stream=None):
    """K of one pattern with no allocation inside the library.  x, y, t and the outputs K, L,
    S (float64) and C (int64), each [cs, ct], are caller-owned contiguous CUDA tensors on the
    current device (checked here; ValueError otherwise)."""
    s, tt = _f64(s), _f64(tt)
    _check_noalloc_tensors(x, y, t, K, L, S, C, s.shape[0] * tt.shape[0])
    b = _box(box)
    st = None if stream is None else _P(stream.cuda_stream)
    _check(load().stk_k_noalloc(_P(x.data_ptr()), _P(y.data_ptr()), _P(t.data_ptr()), x.numel(),
                                ctypes.byref(b), _ptr(s), s.shape[0], _ptr(tt), tt.shape[0],
                                edge_mode, _P(K.data_ptr()), _P(L.data_ptr()), _P(S.data_ptr()),
                                _P(C.data_ptr()), st))


def stk_server_create(device=0, slots=0, mem_budget_bytes=0, max_batch_sims=0, max_queue=0,
                      no_merge=False, fuse=False):
    """Start a serving loop on `device` (returns an opaque server)."""
    cfg = stk_server_config(device, slots, int(mem_budget_bytes), max_batch_sims, max_queue,
                            1 if no_merge else 0, 1 if fuse else 0)
    sv = _P()
    _check(load().stk_server_create(ctypes.byref(cfg), ctypes.byref(sv)))
    return sv


def stk_server_register(sv, x, y, t, box) -> int:
    """Make a point set resident on the server's device; returns its dataset id."""
    x, y, t = _f64(x), _f64(y), _f64(t)
    if not (x.shape == y.shape == t.shape and x.ndim == 1):
        raise ValueError("x, y, t must be 1-D arrays of equal length")
    b = _box(box)
    d = ctypes.c_uint64()
    _check(load().stk_server_register(sv, _ptr(x), _ptr(y), _ptr(t), x.shape[0],
                                      ctypes.byref(b), ctypes.byref(d)))
    return d.value


def stk_server_unregister(sv, dataset: int):
    _check(load().stk_server_unregister(sv, dataset))


def stk_submit(sv, dataset, s, tt, n_sims=0, seed=0, edge_mode=STK_EDGE_ISOTROPIC,
               prec=STK_PREC_FP32_GUARDED, norm=STK_NORM_N_NM1, want_sims=False,
               sim_method=STK_SIM_CSR, n_sectors=0) -> int:
    """Queue a K / envelope job on a registered point set; returns its ticket."""
    s, tt = _f64(s), _f64(tt)
    j = stk_job(dataset, _ptr(s), s.shape[0], _ptr(tt), tt.shape[0], edge_mode, prec, norm,
                n_sims, seed, 1 if want_sims else 0, sim_method, n_sectors)
    tk = ctypes.c_uint64()
    _check(load().stk_submit(sv, ctypes.byref(j), ctypes.byref(tk)))
    return tk.value


def stk_poll(sv, ticket, cs, ct, n_sims=0, want_sims=False, wait_ms=-1, n_sectors=0):
    """Wait for a job.  Returns (grids, latency_ms), or None while it is still running after
    wait_ms; raises StkError if the job failed."""
    grid = (n_sectors, cs, ct) if n_sectors > 1 else (cs, ct)
    nb = int(np.prod(grid))
    o = {"K": np.zeros(nb), "L": np.zeros(nb), "S": np.zeros(nb), "C": np.zeros(nb, np.int64)}
    if n_sims > 0:
        for k in ("K_lo", "K_hi", "L_lo", "L_hi"):
            o[k] = np.zeros(nb)
        if want_sims:
            o["K_sims"] = np.zeros(n_sims * nb)
            o["C_sims"] = np.zeros(n_sims * nb, np.int64)
    r = stk_result(_ptr(o["K"]), _ptr(o["L"]), _ptr(o["S"]), _ptr(o["C"]), _ptr(o.get("K_lo")),
                   _ptr(o.get("K_hi")), _ptr(o.get("L_lo")), _ptr(o.get("L_hi")),
                   _ptr(o.get("K_sims")), _ptr(o.get("C_sims")))
    lat = ctypes.c_double()
    rc = load().stk_poll(sv, ticket, ctypes.byref(r), wait_ms, ctypes.byref(lat))
    if rc == STK_ETIMEOUT:
        return None
    _check(rc)
    out = {}
    for k, v in o.items():
        out[k] = v.reshape((n_sims,) + grid) if k in ("K_sims", "C_sims") else v.reshape(grid)
    return out, lat.value


def stk_server_stats(sv) -> dict:
    st = stk_serve_stats()
    _check(load().stk_server_stats(sv, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in stk_serve_stats._fields_}


def stk_server_reset_stats(sv):
    _check(load().stk_server_reset_stats(sv))


def stk_server_destroy(sv):
    if sv:
        load().stk_server_destroy(sv)


class Server:
    """Owning wrapper of a serving loop; remembers each ticket's grid shape for poll()."""

    def __init__(self, **cfg):
        self.sv = stk_server_create(**cfg)
        self._shape = {}

    def register(self, x, y, t, box) -> int:
        return stk_server_register(self.sv, x, y, t, box)

    def unregister(self, dataset):
        stk_server_unregister(self.sv, dataset)

    def set_polygon(self, dataset, vx=None, vy=None):
        """Polygon study area of a registered point set (None: back to its box)."""
        if vx is None:
            _check(load().stk_server_set_polygon(self.sv, dataset, None, None, 0))
            return
        vx, vy = _f64(vx), _f64(vy)
        _check(load().stk_server_set_polygon(self.sv, dataset, _ptr(vx), _ptr(vy), vx.shape[0]))

    def set_intensity(self, dataset, rho=None):
        """Relative intensity rho[nit, niy, nix] of a registered point set (None: none)."""
        if rho is None:
            _check(load().stk_server_set_intensity(self.sv, dataset, None, 0, 0, 0))
            return
        r = _rho3(rho)
        _check(load().stk_server_set_intensity(self.sv, dataset, _ptr(r), r.shape[2],
                                               r.shape[1], r.shape[0]))

    def submit(self, dataset, s, tt, n_sims=0, seed=0, want_sims=False, **kw) -> int:
        tk = stk_submit(self.sv, dataset, s, tt, n_sims=n_sims, seed=seed, want_sims=want_sims,
                        **kw)
        self._shape[tk] = (len(s), len(tt), n_sims, want_sims, kw.get("n_sectors", 0))
        return tk

    def poll(self, ticket, wait_ms=-1):
        cs, ct, n_sims, want, nsec = self._shape[ticket]
        r = stk_poll(self.sv, ticket, cs, ct, n_sims, want, wait_ms, nsec)
        if r is not None:
            del self._shape[ticket]
        return r

    def stats(self):
        return stk_server_stats(self.sv)

    def reset_stats(self):
        stk_server_reset_stats(self.sv)

    def close(self):
        if self.sv:
            stk_server_destroy(self.sv)
            self.sv = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pattern:
    """Owning wrapper of a handle: ``with Pattern(x, y, t, box) as p: p.k(s, tt)``."""

    def __init__(self, x, y, t, box):
        self.box = tuple(float(v) for v in box)
        self.n = len(x)
        self.h = stk_create(x, y, t, box)

    def k(self, s, tt, **kw):
        return stk_k(self.h, s, tt, **kw)

    def envelope(self, s, tt, n_sims, seed, **kw):
        return stk_envelope(self.h, s, tt, n_sims, seed, **kw)

    def run(self, s, tt, **kw):
        return stk_run(self.h, s, tt, **kw)

    def stats(self):
        return stk_last_stats(self.h)

    def set_polygon(self, vx=None, vy=None):
        stk_set_polygon(self.h, vx, vy)

    def set_intensity(self, rho=None):
        """Inhomogeneous K from now on, with relative intensity rho[nit, niy, nix]."""
        stk_set_intensity(self.h, rho)

    def close(self):
        if self.h:
            stk_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
