"""The entry point's smoke run (one small FP64 and FP32 solve against the
oracle through the C ABI) passes on the GPU."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.smoke()
