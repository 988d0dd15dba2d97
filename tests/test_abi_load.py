"""CPU-side checks of the boundary: the library builds, loads without a GPU and exports every
entry point that include/stk.h declares; argument errors are reported without device work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1912_04753_gb300 import build as b

    b.build()
    import paper_1912_04753_gb300 as stk

    return stk.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(stk_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "stk_create" in names and "stk_run" in names
    for nm in names:
        assert hasattr(lib, nm), f"{nm} declared in include/ but not exported"


def test_version_and_error_string(lib):
    import paper_1912_04753_gb300 as stk

    assert "sm_103a" in stk.stk_version()
    assert isinstance(stk.stk_last_error(), str)


def test_argument_errors_need_no_device(lib):
    import paper_1912_04753_gb300 as stk

    box = (0, 10, 0, 10, 0, 10)
    x = np.array([1.0, 2.0, 3.0])
    with pytest.raises(stk.StkError) as e:
        stk.stk_create(x[:1], x[:1], x[:1], box)  # n < 2
    assert e.value.code == 1
    with pytest.raises(stk.StkError) as e:
        stk.stk_create(x, x, x, (0, 10, 5, 1, 0, 10))  # y0 > y1
    assert e.value.code == 1
    with pytest.raises(stk.StkError) as e:
        stk.stk_create(x, np.array([1.0, 11.0, 2.0]), x, box)  # outside the box
    assert e.value.code == 2
    with pytest.raises(stk.StkError) as e:
        stk.stk_create(x, np.array([1.0, np.nan, 2.0]), x, box)  # not finite
    assert e.value.code == 2


def test_python_binding_has_no_fallback(monkeypatch, tmp_path):
    import paper_1912_04753_gb300._lib as L

    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(OSError):
        L.load()


def test_server_argument_errors(lib):
    import torch

    import paper_1912_04753_gb300 as stk

    with pytest.raises(stk.StkError) as e:
        stk.stk_server_create(slots=100)
    assert e.value.code == stk.STK_EINVAL
    with pytest.raises(stk.StkError) as e:
        stk.stk_server_create(mem_budget_bytes=-1)
    assert e.value.code == stk.STK_EINVAL
    if not torch.cuda.is_available():
        with pytest.raises(stk.StkError) as e:
            stk.stk_server_create()
        assert e.value.code == 7  # STK_ENODEV


def test_intensity_argument_errors_need_no_device(lib):
    """The relative intensity is checked on the host before any device call."""
    import paper_1912_04753_gb300 as stk

    box = (0, 10, 0, 10, 0, 10)
    good = np.ones((2, 2, 2))
    for bad in (good * -1.0, np.full((2, 2, 2), np.nan), np.zeros((2, 2, 2))):
        with pytest.raises(stk.StkError) as e:
            stk.stk_sim_points_inhom(box, bad, 10, 1, 0)
        assert e.value.code == 1
    wide = np.ones((1, 1, 4))
    wide[0, 0, 0] = 1e-6  # 2^14 below the mean
    with pytest.raises(stk.StkError) as e:
        stk.stk_sim_points_inhom(box, wide, 10, 1, 0)
    assert e.value.code == 1 and "2^14" in str(e.value)
    with pytest.raises(ValueError):
        stk.stk_sim_points_inhom(box, np.ones((2, 2)), 10, 1, 0)
    with pytest.raises(stk.StkError) as e:
        stk.stk_set_intensity(None, good)
    assert e.value.code == 1


def test_null_handles_and_servers_are_rejected(lib):
    """Every entry point that takes a handle or a server checks it on the host first."""
    import ctypes

    import paper_1912_04753_gb300 as stk

    L = stk.load()
    v = np.array([0.0, 1.0, 0.0])
    P = ctypes.c_void_p
    assert L.stk_set_polygon(None, v.ctypes.data_as(P), v.ctypes.data_as(P), 3) == 1
    assert L.stk_set_intensity(None, None, 0, 0, 0) == 1
    assert L.stk_server_set_polygon(None, 1, v.ctypes.data_as(P), v.ctypes.data_as(P), 3) == 1
    assert L.stk_server_set_intensity(None, 1, None, 0, 0, 0) == 1
    assert L.stk_server_unregister(None, 1) == 1
    assert L.stk_run(None, None, None) == 1
    assert "NULL" in stk.stk_last_error()
    # fused jobs: NULL arrays and a job count outside 1 .. STK_MAX_FUSED_JOBS
    assert L.stk_run_fused(None, None, None, 1, None) == 1
    hs = (P * 1)(None)
    qs = (stk._lib.stk_request * 1)()
    rs = (stk._lib.stk_result * 1)()
    assert L.stk_run_fused(hs, qs, rs, 0, None) == 1
    assert L.stk_run_fused(hs, qs, rs, 257, None) == 1
    assert L.stk_run_fused(hs, qs, rs, 1, None) == 1  # a NULL handle
    assert "NULL" in stk.stk_last_error()


def test_merge_entry_points_reject_bad_arguments_without_a_device(lib):
    """stk_last_accumulators, stk_merge_grids and stk_envelope_merge check their arguments
    before touching a device."""
    import paper_1912_04753_gb300 as stk
    from paper_1912_04753_gb300 import _lib as L

    P = ctypes.c_void_p
    buf = (ctypes.c_uint64 * 16)()
    assert lib.stk_last_accumulators(None, 0, 1, ctypes.cast(buf, P)) == stk.STK_EINVAL
    s = np.array([1.0, 2.0])
    q, keep = L._request(s, s)
    assert lib.stk_merge_grids(None, ctypes.byref(q), ctypes.cast(buf, P), 1, None, None, None,
                               None) == stk.STK_EINVAL
    K = np.zeros(4)
    sp = s.ctypes.data_as(P)
    # NULL input, no rows, a grid beyond 64 thresholds, sectors x grid beyond 4096 bins,
    # a non-positive temporal threshold
    bad = [(None, 1, 2, 2, 0, sp, sp), (K.ctypes.data_as(P), 0, 2, 2, 0, sp, sp),
           (K.ctypes.data_as(P), 1, 65, 2, 0, sp, sp), (K.ctypes.data_as(P), 1, 64, 64, 2, sp, sp),
           (K.ctypes.data_as(P), 1, 2, 2, 0, sp, np.array([0.0, 1.0]).ctypes.data_as(P))]
    for a in bad:
        assert lib.stk_envelope_merge(*a, None, None, None, None) == stk.STK_EINVAL
