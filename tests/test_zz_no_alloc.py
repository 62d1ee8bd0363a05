"""The allocation-free tracking loss (gsr_loss_track_noalloc) against the
context-based entry point (gsr_loss_track).

Callers that cannot call cudaMalloc (a fixed memory pool, a real-time loop)
use the allocation-free variant; it must give the same loss, median and
gradients.  Two calls in a row check that the shared static scratch carries
nothing from one call into the next.  This file is collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_10070_gb300 import _lib, api

pytestmark = pytest.mark.gpu


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def frame(H, W, seed, invalid):
    rng = np.random.default_rng(seed)
    rgb = rng.random((3, H, W)).astype(np.float32)
    rgb_t = np.clip(rgb + rng.normal(0, 0.1, rgb.shape), 0, 1).astype(np.float32)
    d = rng.uniform(1, 4, (H, W)).astype(np.float32)
    d_t = (d * (1 + rng.normal(0, 0.02, d.shape))).astype(np.float32)
    d_t[rng.random((H, W)) < invalid] = 0
    d[3, 3] = d_t[3, 3] + 25.0
    a = rng.random((H, W)).astype(np.float32)
    return [cu(x) for x in (rgb, d, a, rgb_t, d_t)]


def noalloc(lib, H, W, rgb, d, a, rgb_t, d_t):
    d_rgb, d_d = torch.full_like(rgb, np.nan), torch.full_like(d, np.nan)
    loss, med = torch.full((1,), np.nan, device="cuda"), torch.full((1,), np.nan, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = lib.gsr_loss_track_noalloc(W, H, p(rgb), p(d), p(a), p(rgb_t), p(d_t), 0.5, 50.0, 3.0, p(d_rgb), p(d_d),
                                    p(loss), p(med), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, _lib.STATUS.get(st, st)
    torch.cuda.synchronize()
    return loss, med, d_rgb, d_d


def test_noalloc_track_loss_matches_context_entry_point():
    lib = _lib.load()
    ctx = api.Context()
    # calls in a row with different inputs and sizes: the largest image the
    # static scratch holds (1280 x 720 = GSR_NOALLOC_MAX_PIXELS), a smaller one
    # that must not see the first call's leftovers, then a mid-sized one
    assert 720 * 1280 == _lib.NOALLOC_MAX_PIXELS
    for (H, W, seed, invalid) in ((720, 1280, 3, 0.1), (120, 160, 2, 0.3), (680, 1200, 1, 0.05)):
        inp = frame(H, W, seed, invalid)
        loss, med, g_rgb, g_d = noalloc(lib, H, W, *inp)
        ref_loss, ref_med, ref_rgb, ref_d = api.loss_track(ctx, *inp)
        torch.cuda.synchronize()
        assert float(med) == float(ref_med)
        assert abs(float(loss) - float(ref_loss)) <= 1e-5 * abs(float(ref_loss)) + 1e-6
        np.testing.assert_allclose(g_rgb.cpu().numpy(), ref_rgb.cpu().numpy(), rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(g_d.cpu().numpy(), ref_d.cpu().numpy(), rtol=1e-5, atol=1e-6)
    ctx.close()


def test_noalloc_rejects_images_beyond_its_scratch():
    lib = _lib.load()
    H, W = 721, 1280  # one row more than the 1280 x 720 maximum
    x = torch.zeros((3, H, W), device="cuda")
    y = torch.zeros((H, W), device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = lib.gsr_loss_track_noalloc(W, H, p(x), p(y), p(y), p(x), p(y), 0.5, 50.0, 3.0, p(x), p(y), None, None,
                                    None)
    assert st == -4  # GSR_ERR_CAPACITY, nothing launched
    assert lib.gsr_loss_track_noalloc(0, 10, p(x), p(y), p(y), p(x), p(y), 0.5, 50.0, 3.0, p(x), p(y), None, None,
                                      None) == -1


def test_noalloc_nonfinite_loss_shows_in_the_loss_value():
    """The call does not synchronise, so a NaN input is not reported as a
    status; it shows in the loss it writes (documented in gsr.h)."""
    lib = _lib.load()
    H, W = 64, 96
    rgb, d, a, rgb_t, d_t = frame(H, W, 4, 0.1)
    rgb_t[1, 5, 7] = float("nan")
    loss, med, _, _ = noalloc(lib, H, W, rgb, d, a, rgb_t, d_t)
    assert not np.isfinite(float(loss))
    # the next call on clean inputs is unaffected
    rgb_t[1, 5, 7] = 0.5
    loss, med, _, _ = noalloc(lib, H, W, rgb, d, a, rgb_t, d_t)
    assert np.isfinite(float(loss))
