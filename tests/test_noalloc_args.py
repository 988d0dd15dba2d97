"""Argument checks of the stk_k_noalloc binding, on the host: every buffer it hands to the
library must be a contiguous CUDA tensor of the right dtype on the current device, x, y, t of
equal length and the outputs at least cs * ct long, or the call raises ValueError before any
device work (a wrong buffer would otherwise be read or written out of bounds on the GPU)."""
import os
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1912_04753_gb300 import _lib  # noqa: E402


class FakeCuda:
    """Stands in for a CUDA tensor (no GPU here): the attributes the check reads."""

    def __init__(self, n, dtype=torch.float64, dev=0, contiguous=True, cuda=True):
        self.n, self.dtype, self.is_cuda, self._c = n, dtype, cuda, contiguous
        self.device = torch.device("cuda", dev)

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self._c


def _args(**over):
    a = dict(x=FakeCuda(10), y=FakeCuda(10), t=FakeCuda(10), K=FakeCuda(6), L=FakeCuda(6),
             S=FakeCuda(6), C=FakeCuda(6, torch.int64))
    a.update(over)
    return a


def test_valid_buffers_pass():
    _lib._check_noalloc_tensors(**_args(), cells=6, current=0)


@pytest.mark.parametrize("over,msg", [
    (dict(x=FakeCuda(10, cuda=False)), "CUDA tensor"),
    (dict(K=FakeCuda(6, dev=1)), "current CUDA device"),
    (dict(t=FakeCuda(10, torch.float32)), "torch.float64"),
    (dict(C=FakeCuda(6, torch.float64)), "torch.int64"),
    (dict(L=FakeCuda(6, torch.int64)), "torch.float64"),
    (dict(y=FakeCuda(10, contiguous=False)), "contiguous"),
    (dict(y=FakeCuda(9)), "same number of points"),
    (dict(S=FakeCuda(5)), "cs * ct"),
    (dict(C=FakeCuda(5, torch.int64)), "cs * ct"),
])
def test_each_mismatch_is_rejected(over, msg):
    with pytest.raises(ValueError, match=msg.replace("*", r"\*")):
        _lib._check_noalloc_tensors(**_args(**over), cells=6, current=0)


def test_cpu_tensors_are_rejected_before_the_library():
    x = torch.zeros(10, dtype=torch.float64)
    out = torch.zeros(4, dtype=torch.float64)
    c = torch.zeros(4, dtype=torch.int64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        _lib.stk_k_noalloc(x, x, x, (0, 1, 0, 1, 0, 1), [0.1, 0.2], [0.1, 0.2], out, out, out, c)
