"""The seeded synthetic workloads follow their stated recipe (CPU; the
oracle's projection decides visibility): the 500k-Gaussian sub-map of the
mapping workload has flat surfels on the room's faces with the stated
scales and opacity logits, and its 8 keyframes see between 60k and 450k
Gaussians (the batched mapping configuration's range), the headline view
about 326k; the unit scene's Gaussians are uniform in the stated box."""
import numpy as np

import oracle as O
from paper_2312_10070_gb300 import synth as S


def test_submap_scene_and_keyframe_visibility():
    n = 500_000
    sc = S.room_scene(n, seed=3)
    assert sc["mean"].shape == (n, 3) and all(v.dtype == np.float32 for v in sc.values())
    m = sc["mean"].astype(np.float64)
    assert m.min(axis=0).min() >= -1e-6 and np.all(m.max(axis=0) <= np.array(S.ROOM) + 1e-6)
    ls = sc["log_scale"].astype(np.float64)
    assert np.allclose(ls[:, 2], np.log(1e-3), atol=1e-6)      # 1 mm along the normal
    assert np.allclose(ls[:, 0], ls[0, 0]) and 0.01 < np.exp(ls[0, 0]) < 0.03   # ~2 cm tangent
    lg = sc["opacity_logit"].astype(np.float64)
    assert abs(lg.mean() - 2.0) < 0.01 and abs(lg.std() - 0.5) < 0.01
    # every surfel's normal axis (local z) is a coordinate axis: surfaces are axis-aligned
    q = sc["quat"].astype(np.float64)
    w, x, y, z = q.T
    nz = np.stack([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)], axis=1)
    assert np.allclose(np.abs(nz).max(axis=1), 1.0, atol=1e-5)
    spec = S.camera_room()
    cam = O.Camera(spec.width, spec.height, spec.fx, spec.fy, spec.cx, spec.cy)
    sc64 = O.Scene.from_dict(sc)
    vis = [int(O.project(sc64, qv, tv, cam)["visible"].sum()) for qv, tv in S.submap_views()]
    assert 60_000 <= min(vis) and max(vis) <= 450_000, vis
    assert abs(vis[S.HEADLINE_VIEW] - 326_000) < 2_000, vis


def test_unit_scene_recipe():
    sc = S.random_scene(5000, 1)
    m = sc["mean"].astype(np.float64)
    lo, hi = np.array([-1, -0.75, 1]), np.array([1, 0.75, 4])
    assert np.all(m >= lo) and np.all(m <= hi)
    assert np.all(np.abs(m.mean(axis=0) - (lo + hi) / 2) < 0.05 * (hi - lo))
    ls = sc["log_scale"].astype(np.float64)
    assert abs(ls.mean() + 3.0) < 0.02 and abs(ls.std() - 0.5) < 0.02
    assert np.all(sc["rgb"] >= 0) and np.all(sc["rgb"] <= 1)
    assert np.allclose(np.linalg.norm(sc["quat"].astype(np.float64), axis=1), 1.0, atol=1e-6)


def test_trajectories_perturbations_and_sensor_noise():
    from paper_2312_10070_gb300 import slam
    # room trajectories: consecutive frames move about step_m or turn about max_step_deg, never much more
    for step, deg in ((0.015, 1.0), (0.02, 1.5), (0.04, 3.0)):
        qs, ts = S.room_trajectory(100, n_frames=30, step_m=step, max_step_deg=deg)
        assert len(qs) == 30
        for i in range(29):
            d, ang = slam.relative_motion(qs[i + 1], ts[i + 1], qs[i], ts[i])
            assert d <= step * 1.05 and ang <= deg * 1.05, (i, d, ang)
            assert d >= step * 0.99 or ang >= deg * 0.99, (i, d, ang)
            c = slam.camera_centre(qs[i], ts[i])
            assert np.all(c > 0) and np.all(c < np.array(S.ROOM))
    # target pose of the unit workload: within 2 cm per axis and 1 degree
    for seed in (2, 22, 42):
        q, t = S.perturbed_pose(seed)
        assert np.all(np.abs(t) <= 0.02 + 1e-7)
        _, ang = slam.relative_motion(q, np.zeros(3), np.array([1.0, 0, 0, 0]), np.zeros(3))
        assert ang <= 1.0 + 1e-4
    # sensor noise: N(0, 0.01) colour, 1 % depth, depth invalid where alpha < 0.5
    rng = np.random.default_rng(0)
    rgb = rng.random((3, 200, 300)).astype(np.float32)
    dep = rng.uniform(1, 4, (200, 300)).astype(np.float32)
    al = rng.random((200, 300)).astype(np.float32)
    rn, dn = S.add_sensor_noise(rgb, dep, al, seed=1)
    assert abs(float((rn - rgb).std()) - 0.01) < 5e-4 and abs(float((rn - rgb).mean())) < 2e-4
    ok = al >= 0.5
    assert np.all(dn[~ok] == 0) and np.all(dn[ok] > 0)
    rel = dn[ok] / dep[ok] - 1
    assert abs(float(rel.std()) - 0.01) < 5e-4
