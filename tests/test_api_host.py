"""Host-side argument checks of the Python binding (no GPU): Gaussian arrays
must be float32 with the documented layout before their pointers cross the
C ABI, and tensors must be contiguous CUDA tensors."""
import pytest
import torch

from paper_2312_10070_gb300 import api


def params(n=5, **over):
    t = dict(mean=torch.zeros(n, 3), log_scale=torch.zeros(n, 3), quat=torch.zeros(n, 4),
             opacity_logit=torch.zeros(n), rgb=torch.zeros(n, 3))
    t.update(over)
    return api.GaussianParams(*[t[k] for k in api.GaussianParams.NAMES])


def test_documented_layout_passes_the_check():
    assert params().check().n == 5
    assert params(0).check().n == 0


@pytest.mark.parametrize("name,bad", [
    ("mean", torch.zeros(5, 3, dtype=torch.float64)),
    ("quat", torch.zeros(5, 3)),
    ("opacity_logit", torch.zeros(5, 1)),
    ("rgb", torch.zeros(4, 3)),
    ("log_scale", torch.zeros(5, 3, dtype=torch.float16)),
])
def test_wrong_dtype_or_shape_is_rejected_before_the_abi(name, bad):
    g = params(**{name: bad})
    with pytest.raises(ValueError, match=name):
        g.check()
    with pytest.raises(ValueError, match=name):
        g.c()


def test_host_tensors_are_rejected():
    with pytest.raises(ValueError, match="CUDA"):
        params().c()
