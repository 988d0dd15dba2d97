"""The allocation-free entry point (stk_k_noalloc) against the regular one (stk_k).

Some callers cannot allocate device memory where they need K; stk_k_noalloc keeps its
intermediate buffers in a fixed array inside the library and writes into the caller's device
buffers.  Two calls in a row, on different patterns, must each match stk_k on the same input
(counts exact, K / L / raw sums within the FP32-guarded tolerance), which also shows that the
shared array is cleared between calls.  This file is collected last so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-6


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) / np.where(b == 0, 1.0, np.abs(b))


def test_no_alloc_matches_regular_entry_point_twice():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1912_04753_gb300 import build as b

    b.build()
    import paper_1912_04753_gb300 as stk
    from paper_1912_04753_gb300 import workloads as wl

    cases = [wl.config_csr_small(seed=21, n=3000), wl.config_thomas(seed=4, n=20_000)]
    dev = torch.device("cuda", 0)
    for w in cases:
        cs, ct = len(w.s), len(w.tt)
        x, y, t = (torch.tensor(a, dtype=torch.float64, device=dev) for a in (w.x, w.y, w.t))
        K, L, S = (torch.full((cs, ct), -1.0, dtype=torch.float64, device=dev) for _ in range(3))
        C = torch.full((cs, ct), -1, dtype=torch.int64, device=dev)
        stk.stk_k_noalloc(x, y, t, w.box, w.s, w.tt, K, L, S, C)
        torch.cuda.synchronize()
        with stk.Pattern(w.x, w.y, w.t, w.box) as p:
            want = p.k(w.s, w.tt, prec=stk.STK_PREC_FP32_GUARDED)
        np.testing.assert_array_equal(C.cpu().numpy(), want["C"])
        assert _rel(K.cpu().numpy(), want["K"]).max() <= TOL
        assert _rel(S.cpu().numpy(), want["S"]).max() <= TOL
        s_col = np.asarray(w.s)[:, None]
        assert _rel(L.cpu().numpy() + s_col, want["L"] + s_col).max() <= TOL


def test_no_alloc_rejects_oversized_patterns():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_1912_04753_gb300 as stk

    n = 262_145  # one more than the fixed limit
    x = torch.full((n,), 1.0, dtype=torch.float64, device="cuda")
    K = L = S = torch.zeros((1, 1), dtype=torch.float64, device="cuda")
    C = torch.zeros((1, 1), dtype=torch.int64, device="cuda")
    with pytest.raises(stk.StkError) as e:
        stk.stk_k_noalloc(x, x, x, (0, 10, 0, 10, 0, 10), [1.0], [1.0], K, L, S, C)
    assert e.value.code == 1 and "limit" in str(e.value)
