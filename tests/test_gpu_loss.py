"""GPU parity of the fused losses and the optimiser steps against the FP64
oracle, on identical float32 inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2312_10070_gb300 import api, synth as S
from tests.gpu_common import grad_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context()
    yield c
    c.close()


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def images(H, W, seed, invalid=0.1):
    rng = np.random.default_rng(seed)
    rgb = rng.random((3, H, W)).astype(np.float32)
    rgb_t = np.clip(rgb + rng.normal(0, 0.1, rgb.shape), 0, 1).astype(np.float32)
    d = rng.uniform(1, 4, (H, W)).astype(np.float32)
    d_t = (d * (1 + rng.normal(0, 0.02, d.shape))).astype(np.float32)
    d_t[rng.random((H, W)) < invalid] = 0
    a = rng.random((H, W)).astype(np.float32)
    return rgb, d, a, rgb_t, d_t


@pytest.mark.parametrize("H,W", [(120, 160), (37, 50), (680, 1200)])
def test_loss_map_matches_oracle(ctx, H, W):
    rgb, d, _, rgb_t, d_t = images(H, W, 1)
    loss, g_rgb, g_d = api.loss_map(ctx, cu(rgb), cu(d), cu(rgb_t), cu(d_t), 0.2, 1.0, 1.0, 1.0)
    ref = O.loss_map(rgb, d, rgb_t, d_t, 0.2, 1.0, 1.0)
    assert abs(float(loss) - ref["loss"]) <= 1e-5 * abs(ref["loss"]) + 1e-7
    g = g_rgb.cpu().numpy()
    assert np.abs(g - ref["d_rgb"]).max() <= 1e-3 * np.abs(ref["d_rgb"]).max()
    np.testing.assert_allclose(g_d.cpu().numpy(), ref["d_depth"], rtol=1e-5, atol=1e-12)


def test_loss_map_scale_and_weights(ctx):
    rgb, d, _, rgb_t, d_t = images(64, 48, 2)
    loss, g_rgb, g_d = api.loss_map(ctx, cu(rgb), cu(d), cu(rgb_t), cu(d_t), 0.3, 0.7, 2.0, 0.25)
    ref = O.loss_map(rgb, d, rgb_t, d_t, 0.3, 0.7, 2.0)
    assert abs(float(loss) - 0.25 * ref["loss"]) <= 1e-5 * abs(ref["loss"])
    assert np.abs(g_rgb.cpu().numpy() - 0.25 * ref["d_rgb"]).max() <= 1e-3 * 0.25 * np.abs(ref["d_rgb"]).max()


@pytest.mark.parametrize("H,W,invalid", [(120, 160, 0.1), (37, 50, 0.5), (680, 1200, 0.05), (16, 16, 1.0)])
def test_loss_track_matches_oracle(ctx, H, W, invalid):
    rgb, d, a, rgb_t, d_t = images(H, W, 3, invalid)
    d[5 % H, 5 % W] = d_t[5 % H, 5 % W] + 30.0  # an outlier
    loss, med, g_rgb, g_d = api.loss_track(ctx, cu(rgb), cu(d), cu(a), cu(rgb_t), cu(d_t))
    ref = O.loss_track(rgb, d, a, rgb_t, d_t)
    # the median is one of the float32 residuals: exact
    e = np.abs(d.astype(np.float32) - d_t.astype(np.float32))
    assert float(med) == np.float32(ref["median"]) or (ref["median"] == 0 and float(med) == 0)
    assert abs(float(loss) - ref["loss"]) <= 1e-5 * abs(ref["loss"]) + 1e-6
    np.testing.assert_allclose(g_rgb.cpu().numpy(), ref["d_rgb"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(g_d.cpu().numpy(), ref["d_depth"], rtol=1e-5, atol=1e-6)
    del e


def test_adam_and_lreg_match_oracle(ctx):
    sc = S.random_scene(3000, 5)
    g = api.GaussianParams.from_numpy(sc)
    st = api.AdamMoments(g)
    cfg = api.AdamConfig(w_reg=0.7)
    rng = np.random.default_rng(4)
    ref_p = {k: sc[k].astype(np.float64).copy() for k in api.GaussianParams.NAMES}
    ref_m = {k: np.zeros_like(v) for k, v in ref_p.items()}
    ref_v = {k: np.zeros_like(v) for k, v in ref_p.items()}
    lrs = dict(mean=cfg.lr_mean, log_scale=cfg.lr_log_scale, quat=cfg.lr_quat, opacity_logit=cfg.lr_opacity,
               rgb=cfg.lr_rgb)
    for step in range(1, 4):
        grads = {k: rng.standard_normal(v.shape).astype(np.float32) for k, v in ref_p.items()}
        gr = api.GaussianParams(*[cu(grads[k]) for k in api.GaussianParams.NAMES])
        lreg_dev = torch.zeros(1, device="cuda")
        api.adam_step(ctx, g, gr, st, cfg, lreg_dev)
        L, gl = O.lreg(ref_p["log_scale"], 0.7)
        for k in ref_p:
            gk = grads[k].astype(np.float64) + (gl.reshape(ref_p[k].shape) if k == "log_scale" else 0)
            O.adam(ref_p[k], np.ascontiguousarray(gk), ref_m[k], ref_v[k], step, lrs[k], 0.9, 0.999, 1e-15)
        assert abs(float(lreg_dev) - 0.7 * L) <= 1e-4 * 0.7 * L
    for k in api.GaussianParams.NAMES:
        np.testing.assert_allclose(getattr(g, k).cpu().numpy(), ref_p[k], rtol=1e-5, atol=1e-6)
    assert int(st.step) == 3


@pytest.mark.parametrize("alpha_pow,k_median", [(0.0, 1e30), (3.0, 1e30), (0.0, 50.0), (3.0, 50.0), (1.0, 5.0)])
def test_loss_track_ablation_variants_match_oracle(ctx, alpha_pow, k_median):
    """The tracking-loss variants of the mask ablation (the alpha mask off:
    exponent 0; the inlier mask off: an infinite factor) and an off-default
    pair, each against the oracle with the same parameters."""
    rgb, d, a, rgb_t, d_t = images(120, 160, 4, 0.1)
    d[7, 9] = d_t[7, 9] + 30.0
    d[50, 60] = d_t[50, 60] * 0.3
    loss, med, g_rgb, g_d = api.loss_track(ctx, cu(rgb), cu(d), cu(a), cu(rgb_t), cu(d_t), 0.5, k_median, alpha_pow)
    ref = O.loss_track(rgb, d, a, rgb_t, d_t, 0.5, k_median, alpha_pow)
    assert float(med) == np.float32(ref["median"])
    assert abs(float(loss) - ref["loss"]) <= 1e-5 * abs(ref["loss"]) + 1e-6
    np.testing.assert_allclose(g_rgb.cpu().numpy(), ref["d_rgb"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(g_d.cpu().numpy(), ref["d_depth"], rtol=1e-5, atol=1e-6)
