"""The package's smoke check (one small forward + backward on cuda:0 against
the oracle) passes."""
import pytest
import torch

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def test_smoke():
    import __graft_entry__
    __graft_entry__.smoke()
