"""The allocation-free entry point (stk_k_noalloc) against the regular one (stk_k) and the
oracle.

Some callers cannot allocate device memory where they need K (inside a caching allocator's
reserved pool, in a region where cudaMalloc / cudaFree would synchronise the device, in an
embedding that owns every buffer); stk_k_noalloc keeps its intermediate buffers in a fixed
array inside the library and writes into the caller's device buffers.  Two calls in a row, on
different patterns, must each match stk_k on the same input and the FP64 oracle (counts exact,
K / L / raw sums within the FP32-guarded tolerance), which also shows that the shared array is
cleared between calls; warm calls must leave the device's free memory unchanged.  This file is
collected last so that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) / np.where(b == 0, 1.0, np.abs(b))


def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1912_04753_gb300 import build as b

    b.build()
    import paper_1912_04753_gb300 as stk

    stk.load()
    return stk


def _buffers(w, dev):
    import torch

    cs, ct = len(w.s), len(w.tt)
    x, y, t = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (w.x, w.y, w.t))
    K, L, S = (torch.full((cs, ct), -1.0, dtype=torch.float64, device=dev) for _ in range(3))
    C = torch.full((cs, ct), -1, dtype=torch.int64, device=dev)
    return x, y, t, K, L, S, C


def _check(w, got, want, tol):
    K, L, S, C = (v.cpu().numpy() for v in got)
    np.testing.assert_array_equal(C, want["C"])
    assert _rel(K, want["K"]).max() <= tol
    assert _rel(S, want["S"]).max() <= tol
    s_col = np.asarray(w.s)[:, None]
    assert _rel(L + s_col, want["L"] + s_col).max() <= tol


def test_no_alloc_matches_regular_entry_point_and_oracle_twice():
    import torch

    import oracle
    from paper_1912_04753_gb300 import workloads as wl

    stk = _lib()
    oracle.build()
    cases = [wl.config_csr_small(seed=21, n=3000), wl.config_thomas(seed=4, n=20_000)]
    dev = torch.device("cuda", 0)
    for w in cases:
        x, y, t, K, L, S, C = _buffers(w, dev)
        stk.stk_k_noalloc(x, y, t, w.box, w.s, w.tt, K, L, S, C)
        torch.cuda.synchronize()
        with stk.Pattern(w.x, w.y, w.t, w.box) as p:
            want = p.k(w.s, w.tt, prec=stk.STK_PREC_FP32_GUARDED)
        _check(w, (K, L, S, C), want, TOL)
        ref = oracle.k_function(w.x, w.y, w.t, w.box, w.s, w.tt)
        _check(w, (K, L, S, C), ref, TOL)


def test_warm_calls_allocate_no_device_memory():
    """After a warm-up call, repeated calls (on the default and on an explicit stream) leave
    the device's free memory exactly unchanged; no stk handle is alive meanwhile."""
    import torch

    from paper_1912_04753_gb300 import workloads as wl

    stk = _lib()
    dev = torch.device("cuda", 0)
    w = wl.config_thomas(seed=6, n=15_000)
    bufs = _buffers(w, dev)
    stream = torch.cuda.Stream()
    stk.stk_k_noalloc(*bufs[:3], w.box, w.s, w.tt, *bufs[3:])
    stk.stk_k_noalloc(*bufs[:3], w.box, w.s, w.tt, *bufs[3:], stream=stream)
    torch.cuda.synchronize()
    first = [b.clone() for b in bufs[3:]]
    free0, _ = torch.cuda.mem_get_info()
    for k in range(4):
        stk.stk_k_noalloc(*bufs[:3], w.box, w.s, w.tt, *bufs[3:],
                          stream=stream if k % 2 else None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    for a, b in zip(first, bufs[3:]):
        assert torch.equal(a, b)


def test_no_alloc_bounded_wait_reports_timeout_then_recovers(monkeypatch):
    """With the failure-detection hook set, a warp that should publish the next tile of work
    publishes none; the other warps' bounded waits run out, the kernel returns and the call
    reports STK_ETIMEOUT.  The next normal call on the shared array is exact again."""
    import torch

    from paper_1912_04753_gb300 import workloads as wl

    stk = _lib()
    dev = torch.device("cuda", 0)
    w = wl.config_thomas(seed=7, n=40_000)
    bufs = _buffers(w, dev)
    monkeypatch.setenv("STK_TEST_NEVER_PUBLISH", "1")
    with pytest.raises(stk.StkError) as e:
        stk.stk_k_noalloc(*bufs[:3], w.box, w.s, w.tt, *bufs[3:])
    assert e.value.code == stk.STK_ETIMEOUT
    monkeypatch.delenv("STK_TEST_NEVER_PUBLISH")
    stk.stk_k_noalloc(*bufs[:3], w.box, w.s, w.tt, *bufs[3:])
    torch.cuda.synchronize()
    with stk.Pattern(w.x, w.y, w.t, w.box) as p:
        want = p.k(w.s, w.tt, prec=stk.STK_PREC_FP32_GUARDED)
    _check(w, bufs[3:], want, TOL)


def test_no_alloc_rejects_oversized_patterns():
    import torch

    stk = _lib()
    n = 262_145  # one more than the fixed limit
    x = torch.full((n,), 1.0, dtype=torch.float64, device="cuda")
    K = L = S = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    C = torch.zeros((1, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(stk.StkError) as e:
        stk.stk_k_noalloc(x, x, x, (0, 10, 0, 10, 0, 10), [1.0], [1.0], K, L, S, C)
    assert e.value.code == 1 and "limit" in str(e.value)
