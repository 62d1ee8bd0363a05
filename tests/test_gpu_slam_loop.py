"""End-to-end online SLAM on a synthetic RGB-D sequence: starting from an
empty map and the first frame's pose, the loop (tracking, keyframes every 5th
frame, seeding, sub-map optimisation with pruning, sub-map switching) keeps
the camera-centre error small.  The paper's own accuracy figures need its
datasets and are not reproduced here (parity unpinned); this is a functional
bound on a room_scene sequence.

Frames: renders of room_scene(300k, seed 100) along room_trajectory(seed 100,
40 frames, ~2 cm / <= 1.5 degrees apart); sensor depth = rendered depth / alpha
where alpha >= 0.5 (else invalid), then N(0, 0.01) colour noise and 1 % depth
noise.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def make_frames(scene, poses, spec, seed=0):
    from paper_2312_10070_gb300 import api, synth as S
    ctx = api.Context()
    g = api.GaussianParams.from_numpy(scene)
    cam = api.camera_from_spec(spec)
    frames = []
    for i, (q, t) in enumerate(zip(*poses)):
        r = api.render_forward(ctx, g, cam, api.make_pose(q, t))
        a = r["alpha"].cpu().numpy()
        d = np.where(a >= 0.5, r["depth"].cpu().numpy() / np.maximum(a, 1e-6), 0.0)
        rgb, dn = S.add_sensor_noise(r["rgb"].cpu().numpy(), d, None, seed=seed + i)
        frames.append((torch.from_numpy(rgb).cuda(), torch.from_numpy(dn).cuda()))
    return frames


def test_online_slam_tracks_a_room_sequence(tmp_path):
    from paper_2312_10070_gb300 import api, slam, synth as S
    spec = S.camera_room()
    scene = S.room_scene(300_000, seed=100)
    qs, ts = S.room_trajectory(seed=100, n_frames=40, step_m=0.02, max_step_deg=1.5)
    frames = make_frames(scene, (qs, ts), spec, seed=500)
    cfg = slam.SLAMConfig(track_iters=60, map_iters_first=100, map_iters=40, capacity=1_500_000,
                          seed=api.SeedConfig(m_u=100_000, m_c=50_000, m_k=30_000))
    s = slam.GaussianSLAM(spec, cfg)
    for i, (rgb, depth) in enumerate(frames):
        s.step(rgb, depth, init_pose=(qs[0], ts[0]) if i == 0 else None)
    gt = [(np.asarray(q, np.float64), np.asarray(t, np.float64)) for q, t in zip(qs, ts)]
    ate = slam.ate_rmse(s.poses, gt)
    path = sum(np.linalg.norm(slam.camera_centre(*gt[i + 1]) - slam.camera_centre(*gt[i])) for i in range(39))
    print("ATE RMSE (m)", ate, "path (m)", path, "sub-maps", len(s.submaps) + 1, s.log)
    assert ate < 0.02
    assert len(s.log) == 8 and all(e["seeded"] > 0 for e in s.log)
    if path > 0.6:
        assert len(s.submaps) >= 1
    # global map: merge the sub-maps (also through a save / load round trip), refine colours
    subs = slam.all_submaps(s)
    path_npz = str(tmp_path / "submaps.npz")
    slam.save_submaps(path_npz, subs)
    loaded = slam.load_submaps(path_npz)
    assert len(loaded) == len(subs)
    for a, b in zip(subs, loaded):
        for k in a:
            np.testing.assert_array_equal(a[k], b[k])
    g = slam.global_map(s.ctx, loaded)
    assert len(subs[0]["mean"]) <= g.n <= sum(len(x["mean"]) for x in subs)
    p0 = slam.psnr(s.ctx, g, s.cam, s.keyframes)
    before = {k: t[:g.n].clone() for k, t in zip(api.GaussianParams.NAMES, g.arrays.tensors())}
    slam.refine_colours(s.ctx, g, s.cam, s.keyframes, iters=150)
    p1 = slam.psnr(s.ctx, g, s.cam, s.keyframes)
    print("global map", g.n, "PSNR before / after colour refinement", p0, p1)
    assert p1 > p0
    for k, t in zip(api.GaussianParams.NAMES, g.arrays.tensors()):
        if k != "rgb":
            assert torch.equal(t[:g.n], before[k]), k
