"""The allocation-free entry point writes into device buffers the caller owns; the binding refuses a
buffer of the wrong kind, type or size before anything is launched (no GPU needed for these)."""
import pytest
import torch

from paper_2406_03762_gb300 import cortex
from paper_2406_03762_gb300 import workloads as W

SPEC = W.NetSpec(800, 200, 80, 20)


class _FakeCuda:
    """Stands in for a CUDA tensor of a given size and dtype (never dereferenced: refused first)."""
    is_cuda = True

    def __init__(self, n, dtype):
        self._n, self.dtype = n, dtype
        self.device = None

    def numel(self):
        return self._n

    def is_contiguous(self):
        return True

    def data_ptr(self):
        raise AssertionError("the library must not be called with a refused buffer")


def _bufs(nnz, row=None, tgt=None, dly=None, w=None):
    return (row or _FakeCuda(SPEC.n + 1, torch.int32), tgt or _FakeCuda(nnz, torch.int32),
            dly or _FakeCuda(nnz, torch.int32), w or _FakeCuda(nnz, torch.float32))


@pytest.mark.parametrize("which,bad", [
    (0, _FakeCuda(SPEC.n, torch.int32)),             # row_ptr one short
    (1, _FakeCuda(10, torch.int32)),                 # tgt too short
    (2, _FakeCuda(250 * 100, torch.int64)),          # delay of the wrong type
    (3, _FakeCuda(250 * 100, torch.float64)),        # weight of the wrong type
    (1, torch.zeros(250 * 100, dtype=torch.int32)),  # a CPU tensor
])
def test_noalloc_refuses_bad_buffers_before_any_launch(which, bad):
    nnz = 250 * SPEC.k
    bufs = list(_bufs(nnz))
    bufs[which] = bad
    with pytest.raises(cortex.CortexError) as e:
        cortex.subgraph_noalloc(SPEC, 1, 0, 250, *bufs)
    assert e.value.code == cortex.ERR_ARG
