"""GPU parity of sub-map seeding (gsr_seed_keyframe) against the FP64 oracle
(oracle/seed.py).

Frames are the oracle's renders of synthetic rooms (inputs to both sides);
the existing sub-map is a seeded subset of the room's Gaussians.  Bars:
- candidate pixels: identical sets, except pixels whose FP64 squared gradient
  lies within 1e-5 (relative) of the selection cut (FP32 may order them
  differently);
- kept flags: identical, except candidates whose squared distance to the
  sub-map lies within 5e-3 rho^2 of rho^2 (the FP32 back-projection moves a
  point by up to a few micrometres);
- new Gaussians (matched by pixel): means within 2e-5 m, colours exact,
  rotation and opacity exact, log-scales within 2e-3, except points whose
  nearest neighbour could be an ambiguous candidate.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import seed as SD
from paper_2312_10070_gb300 import synth as S

pytestmark = pytest.mark.gpu


def frame(scene, q, t, spec):
    cam = O.Camera(spec.width, spec.height, spec.fx, spec.fy, spec.cx, spec.cy)
    r = O.render(O.Scene.from_dict(scene), q, t, cam)
    return (r["rgb"].astype(np.float32), r["depth"].astype(np.float32), r["alpha"].astype(np.float32))


def run_gpu(spec, q, t, rgb, depth, alpha, existing, cfg):
    from paper_2312_10070_gb300 import api
    ctx = api.Context()
    P = spec.width * spec.height
    sub = api.SubMap(len(existing) + P)
    g = api.GaussianParams.from_numpy(dict(mean=existing, log_scale=np.zeros_like(existing),
                                           quat=np.tile([1, 0, 0, 0], (len(existing), 1)).astype(np.float32),
                                           opacity_logit=np.zeros(len(existing), np.float32),
                                           rgb=np.zeros_like(existing)))
    sub.append(g)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda() if a is not None else None
    st = api.seed_keyframe(ctx, sub, api.camera_from_spec(spec), api.make_pose(q, t), T(rgb), T(depth), T(alpha), cfg)
    pix, keep, d2 = api.seed_candidates(ctx, P)
    new = {k: v[len(existing):].cpu().numpy() for k, v in zip(api.GaussianParams.NAMES, sub.params().tensors())}
    return st, pix.cpu().numpy(), keep.cpu().numpy().astype(bool), d2.cpu().numpy(), new


def compare(spec, rgb, depth, alpha, existing, cfg, out, st, pix, keep, d2, new, first):
    rho2 = cfg.rho ** 2
    # candidates
    amb_pix = set()
    if first and cfg.m_c > 0:
        g2 = SD.gradient2(rgb.astype(np.float64)).ravel()
        valid = depth.ravel() > 0
        cut = np.sort(g2[valid])[::-1][min(cfg.m_c, valid.sum()) - 1]
        amb_pix = set(np.nonzero(valid & (np.abs(g2 - cut) <= 1e-5 * cut + 1e-12))[0].tolist())
    diff = set(pix.tolist()) ^ set(out["pix"].tolist())
    assert diff <= amb_pix, sorted(diff - amb_pix)[:10]
    # kept flags on the common candidates
    o_idx = {p: i for i, p in enumerate(out["pix"].tolist())}
    common = [(i, o_idx[p]) for i, p in enumerate(pix.tolist()) if p in o_idx]
    gi = np.array([a for a, _ in common])
    oi = np.array([b for _, b in common])
    od2 = out["d2_existing"][oi]
    amb = np.abs(od2 - rho2) <= 5e-3 * rho2
    bad = (keep[gi] != out["keep"][oi]) & ~amb
    assert not bad.any(), (np.nonzero(bad)[0][:10], od2[bad][:5])
    near = od2 < 0.99 * rho2
    np.testing.assert_allclose(d2[gi][near], od2[near], rtol=2e-3, atol=1e-9)
    n_amb = int(amb.sum()) + len(diff)
    assert abs(st["n_added"] - int(out["keep"].sum())) <= n_amb
    # new Gaussians matched by pixel
    g_new_pix = pix[keep]
    o_new_pix = out["pix"][out["keep"]]
    og = out["gaussians"]
    o_map = {p: k for k, p in enumerate(o_new_pix.tolist())}
    pairs = [(k, o_map[p]) for k, p in enumerate(g_new_pix.tolist()) if p in o_map]
    assert len(pairs) >= len(o_new_pix) - n_amb
    gk = np.array([a for a, _ in pairs])
    ok = np.array([b for _, b in pairs])
    np.testing.assert_allclose(new["mean"][gk], og["mean"][ok], atol=2e-5)
    np.testing.assert_array_equal(new["rgb"][gk], og["rgb"][ok].astype(np.float32))
    np.testing.assert_array_equal(new["quat"][gk], np.tile([1, 0, 0, 0], (len(gk), 1)))
    np.testing.assert_array_equal(new["opacity_logit"][gk], 0)
    # scales: skip points whose nearest neighbour may be an ambiguous candidate
    amb_pts = out["points"][oi[amb]] if amb.any() else np.zeros((0, 3))
    if len(diff):
        extra = SD.backproject(np.array(sorted(diff)), depth.astype(np.float64), spec, *out["pose"])
        amb_pts = np.concatenate([amb_pts, extra])
    nn = np.sqrt(out["nn_d2"][ok])
    if len(amb_pts):
        da = np.sqrt(SD.min_dist2(og["mean"][ok], amb_pts))
        trust = da > nn * (1 + 1e-3)
    else:
        trust = np.ones(len(ok), bool)
    assert trust.mean() > 0.9
    np.testing.assert_allclose(new["log_scale"][gk][trust], og["log_scale"][ok][trust], atol=2e-3)
    return len(pairs)


@pytest.fixture(scope="module")
def small_room():
    spec = S.scale_camera(S.camera_room(), 320, 180)
    scene = S.room_scene(60_000, seed=100)
    q, t = S.submap_views()[1]
    rgb, depth, alpha_full = frame(scene, q, t, spec)
    rng = np.random.default_rng(3)
    half = rng.random(60_000) < 0.5
    existing = np.ascontiguousarray(scene["mean"][half])
    sub_scene = {k: v[half] for k, v in scene.items()}
    _, _, alpha_half = frame(sub_scene, q, t, spec)
    return spec, q, t, rgb, depth, alpha_half, existing


@pytest.mark.parametrize("first", [True, False])
def test_seed_keyframe_matches_oracle(small_room, first):
    from paper_2312_10070_gb300 import api
    spec, q, t, rgb, depth, alpha, existing = small_room
    cfg = api.SeedConfig(first_keyframe=first, m_u=6000, m_c=2000, m_k=4000, rho=0.01, s_max=0.1, seed=11)
    st, pix, keep, d2, new = run_gpu(spec, q, t, rgb, depth, None if first else alpha, existing, cfg)
    out = SD.seed_keyframe(rgb.astype(np.float64), depth.astype(np.float64), None if first else alpha, spec, q, t,
                           existing, first=first, m_u=6000, m_c=2000, m_k=4000, rho=0.01, s_max=0.1, seed=11)
    out["pose"] = (q, t)
    assert st["n_candidates"] == len(pix)
    if not first:
        assert np.all(alpha.ravel()[pix] < 0.6)
    n = compare(spec, rgb, depth, alpha, existing, cfg, out, st, pix, keep, d2, new, first)
    assert n > 500


def test_seed_first_keyframe_of_an_empty_sub_map():
    """Nothing to reject: every candidate is kept and scales come from the
    new points alone."""
    from paper_2312_10070_gb300 import api
    spec = S.scale_camera(S.camera_room(), 160, 90)
    scene = S.room_scene(30_000, seed=101)
    q, t = S.submap_views()[3]
    rgb, depth, _ = frame(scene, q, t, spec)
    cfg = api.SeedConfig(first_keyframe=True, m_u=3000, m_c=500, rho=0.01, s_max=0.1, seed=2)
    existing = np.zeros((0, 3), np.float32)
    st, pix, keep, d2, new = run_gpu(spec, q, t, rgb, depth, None, existing, cfg)
    out = SD.seed_keyframe(rgb.astype(np.float64), depth.astype(np.float64), None, spec, q, t, existing, first=True,
                           m_u=3000, m_c=500, rho=0.01, s_max=0.1, seed=2)
    out["pose"] = (q, t)
    assert keep.all() and np.isinf(d2).all()
    assert st["n_added"] == len(pix)
    compare(spec, rgb, depth, None, existing, cfg, out, st, pix, keep, d2, new, True)


def test_seed_capacity_error_writes_nothing():
    from paper_2312_10070_gb300 import api, _lib as L
    spec = S.scale_camera(S.camera_room(), 160, 90)
    scene = S.room_scene(30_000, seed=101)
    q, t = S.submap_views()[3]
    rgb, depth, _ = frame(scene, q, t, spec)
    ctx = api.Context()
    sub = api.SubMap(100)
    T = lambda a: torch.from_numpy(a).cuda()
    with pytest.raises(L.GsrError):
        api.seed_keyframe(ctx, sub, api.camera_from_spec(spec), api.make_pose(q, t), T(rgb), T(depth), None,
                          api.SeedConfig(m_u=3000, m_c=0))
    assert sub.n == 0 and float(sub.arrays.mean.abs().sum()) == 0.0


def test_seed_full_size_sampled():
    """1200x680 keyframe of the 500k-Gaussian room (sub-map view 5), all 500k
    means existing: candidate set exact; kept flags and scales on samples."""
    from paper_2312_10070_gb300 import api
    spec = S.camera_room()
    scene = S.room_scene(500_000, seed=3)
    q, t = S.submap_views()[S.HEADLINE_VIEW]
    rgb, depth, _ = frame(scene, q, t, spec)
    existing = np.ascontiguousarray(scene["mean"])
    cfg = api.SeedConfig(first_keyframe=True, m_u=100_000, m_c=50_000, rho=0.01, s_max=0.1, seed=5)
    st, pix, keep, d2, new = run_gpu(spec, q, t, rgb, depth, None, existing, cfg)
    ref_pix = SD.candidates(rgb.astype(np.float64), depth.astype(np.float64), None, True, 100_000, 50_000, 0, 0.6, 5)
    g2 = SD.gradient2(rgb.astype(np.float64)).ravel()
    valid = depth.ravel() > 0
    cut = np.sort(g2[valid])[::-1][50_000 - 1]
    amb_pix = set(np.nonzero(valid & (np.abs(g2 - cut) <= 1e-5 * cut + 1e-12))[0].tolist())
    assert (set(pix.tolist()) ^ set(ref_pix.tolist())) <= amb_pix
    rng = np.random.default_rng(0)
    sample = rng.choice(len(pix), 400, replace=False)
    pts = SD.backproject(pix[sample], depth.astype(np.float64), spec, q, t)
    od2 = SD.min_dist2(pts, existing)
    amb = np.abs(od2 - 1e-4) <= 5e-3 * 1e-4
    assert not ((keep[sample] != (od2 >= 1e-4)) & ~amb).any()
    # property at any size: each sampled new Gaussian's scale is its clamped
    # nearest-neighbour distance within the sub-map the call produced
    union = np.concatenate([existing.astype(np.float64), new["mean"].astype(np.float64)])
    ks = rng.choice(len(new["mean"]), 200, replace=False)
    for k in ks:
        dd = ((union - union[len(existing) + k]) ** 2).sum(axis=1)
        dd[len(existing) + k] = np.inf
        ref = np.log(np.clip(np.sqrt(dd.min()), 1e-4, 0.1))
        assert abs(new["log_scale"][k, 0] - ref) <= 2e-3, (k, new["log_scale"][k, 0], ref)
    assert np.all(new["log_scale"][:, 0] == new["log_scale"][:, 1])
    print("candidates", st["n_candidates"], "added", st["n_added"])
