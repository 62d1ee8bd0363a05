"""Host-side code of the Python package, on the CPU: argument checks of the
binding (Gaussian arrays must be float32 with the documented layout before
their pointers cross the C ABI; tensors must be contiguous CUDA tensors),
the evaluation helpers (pose errors against scipy, twist sampling ranges),
and that the product path holds no host copy of the SE(3) retraction (the
pose update runs on the device, gsr_pose_retract / gsr_render_forward_xi)."""
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


def test_no_host_pose_retraction_in_the_product_path():
    import inspect
    from paper_2312_10070_gb300 import autograd, warmstart
    assert not hasattr(api, "pose_exp_left")
    for mod in (api, autograd, warmstart):
        src = inspect.getsource(mod)
        assert "pose_exp_left" not in src and ".cpu()" not in inspect.getsource(autograd)


def test_pose_error_and_twist_sampling():
    """warmstart.pose_error against scipy rotations; random_twist stays in
    its ball and angle range."""
    import numpy as np
    from scipy.spatial.transform import Rotation
    from paper_2312_10070_gb300 import warmstart as W
    rng = np.random.default_rng(5)
    for _ in range(10):
        q, qg = rng.standard_normal(4), rng.standard_normal(4)
        t, tg = rng.standard_normal(3), rng.standard_normal(3)
        R = Rotation.from_quat(np.roll(q / np.linalg.norm(q), -1)).as_matrix()
        Rg = Rotation.from_quat(np.roll(qg / np.linalg.norm(qg), -1)).as_matrix()
        d, ang = W.pose_error(q, t, qg, tg)
        assert abs(d - np.linalg.norm(-R.T @ t + Rg.T @ tg)) < 1e-12
        assert abs(ang - np.degrees(Rotation.from_matrix(R @ Rg.T).magnitude())) < 1e-9
    for _ in range(200):
        xi = W.random_twist(rng, 0.05, 3.0)
        assert np.linalg.norm(xi[:3]) <= 0.05 + 1e-15 and np.linalg.norm(xi[3:]) <= np.deg2rad(3.0) + 1e-15


def test_no_cpu_fallback_without_a_gpu():
    """Without a CUDA device the rasterizer refuses to run instead of falling
    back to host code (this container has none; on a GPU machine it is skipped)."""
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        api.Context()
    from paper_2312_10070_gb300 import warmstart as W
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        W.WarmStartNet(max_batch=4)


def test_missing_library_raises(monkeypatch, tmp_path):
    """A missing libgsr.so raises on load (when not rebuilt) rather than
    degrading to anything else."""
    from paper_2312_10070_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libgsr.so"))
    with pytest.raises(ImportError):
        _lib.load(build_if_missing=False)
