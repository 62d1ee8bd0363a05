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
