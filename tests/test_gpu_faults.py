"""Failure detection without a GPU fault (no trap, no hang, no bad address):
device-side conditions are latched in the context's status word, returned by
the next synchronising call, and the context stays usable afterwards.

- capacity: a fixed-capacity context with room for 64 tile instances renders
  a scene with thousands; the emission kernel bounds every write by the
  capacity, the sort and the ranges read at most that many, the overflow is
  latched and gsr_frame_stats_get returns GSR_ERR_CAPACITY once.
- non-finite: a NaN in the mapping target makes the loss NaN; gsr_map_step
  returns GSR_ERR_NONFINITE, and a step on clean inputs afterwards succeeds.
- timeout: the radix sort's bounded look-back wait, run on a word nothing
  publishes, gives up after a few thousand polls; GSR_ERR_TIMEOUT is returned
  and the same context then renders bit-identically to a fresh one.
- allocation failure: a scratch hint of 2^40 Gaussians asks cudaMalloc for
  4 TiB, which it refuses without allocating; gsr_create returns GSR_ERR_OOM,
  frees what it had allocated, and a new context works.
"""
import numpy as np
import pytest
import torch

from paper_2312_10070_gb300 import _lib, api, synth as S

pytestmark = pytest.mark.gpu


def unit_scene():
    spec = S.camera_unit()
    return (api.GaussianParams.from_numpy(S.random_scene(5000, seed=1)), api.camera_from_spec(spec),
            api.make_pose(*S.IDENTITY_POSE))


def test_capacity_overflow_is_latched_and_reported():
    g, cam, pose = unit_scene()
    ctx = api.Context(fixed_capacity=True, max_instances=64)
    out = api.render_forward(ctx, g, cam, pose)
    with pytest.raises(_lib.GsrError) as e:
        api.frame_stats(ctx)
    assert e.value.status == -4, e.value
    st = api.frame_stats(ctx)  # reported once, then cleared
    assert st["capacity_instances"] == 64 and st["n_instances"] > 64
    torch.cuda.synchronize()
    for k in ("rgb", "depth", "alpha", "final_T"):
        assert bool(torch.isfinite(out[k]).all()), k
    # a grow-on-demand context renders the same scene in full
    ref_ctx = api.Context()
    ref = api.render_forward(ref_ctx, g, cam, pose)
    assert api.frame_stats(ref_ctx)["n_instances"] == st["n_instances"]
    assert float(ref["alpha"].max()) > 0.5
    ctx.close()
    ref_ctx.close()


def test_non_finite_loss_is_latched_and_reported():
    sc = S.random_scene(5000, seed=1)
    _, cam, pose = unit_scene()
    ctx = api.Context()
    tgt = api.render_forward(ctx, api.GaussianParams.from_numpy(sc), cam, pose)
    rgb_t, depth_t = tgt["rgb"].clone(), tgt["depth"].clone()
    bad = rgb_t.clone()
    bad[1, 60, 80] = float("nan")
    cfg = api.MapConfig(use_graph=False)
    g = api.GaussianParams.from_numpy(S.noisy_copy(sc, seed=3))
    with pytest.raises(_lib.GsrError) as e:
        api.map_step(ctx, g, api.AdamMoments(g), cam, [(pose, bad, depth_t)], cfg=cfg)
    assert e.value.status == -6, e.value
    # fresh parameters and a clean target: the step succeeds on the same context
    g2 = api.GaussianParams.from_numpy(S.noisy_copy(sc, seed=3))
    st = api.map_step(ctx, g2, api.AdamMoments(g2), cam, [(pose, rgb_t, depth_t)], cfg=cfg)
    assert np.isfinite(st["loss_last"]) and st["loss_last"] > 0
    ctx.close()


def test_bounded_wait_expires_with_timeout_status():
    g, cam, pose = unit_scene()
    ctx = api.Context()
    with pytest.raises(_lib.GsrError) as e:
        api.check_wait_timeout(ctx, polls=4096)
    assert e.value.status == -5 and "bounded device wait" in str(e.value), e.value
    with pytest.raises(_lib.GsrError) as e:
        _lib.check(ctx.lib.gsr_check_wait_timeout(ctx.handle, 0, None), ctx.handle)
    assert e.value.status == -1
    # the context is usable afterwards: its render equals a fresh context's
    out = api.render_forward(ctx, g, cam, pose)
    assert api.frame_stats(ctx)["n_visible"] > 0
    ref_ctx = api.Context()
    ref = api.render_forward(ref_ctx, g, cam, pose)
    for k in ("rgb", "depth", "alpha", "final_T", "last_idx"):
        assert torch.equal(out[k], ref[k]), k
    ctx.close()
    ref_ctx.close()


def test_allocation_failure_is_reported_and_cleaned_up():
    with pytest.raises(_lib.GsrError) as e:
        api.Context(max_gaussians=1 << 40)
    assert e.value.status == -3, e.value
    g, cam, pose = unit_scene()
    ctx = api.Context()
    out = api.render_forward(ctx, g, cam, pose)
    assert api.frame_stats(ctx)["n_visible"] > 0
    assert float(out["alpha"].max()) > 0.5
    ctx.close()
