"""Host-side scheduling logic of the online SLAM loop (CPU only)."""
import numpy as np

from paper_2312_10070_gb300 import slam


def _quat(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[np.cos(ang / 2)], np.sin(ang / 2) * a])


def test_constant_velocity_extrapolates_uniform_motion():
    # translation exactly; rotation about a fixed axis to second order in the step
    t2, t1 = np.array([0.0, 0.1, 0.2]), np.array([0.01, 0.12, 0.2])
    q2, q1 = _quat([0, 0, 1], 0.00), _quat([0, 0, 1], 0.01)
    q, t = slam.constant_velocity(q1, t1, q2, t2)
    np.testing.assert_allclose(t, [0.02, 0.14, 0.2])
    np.testing.assert_allclose(q, _quat([0, 0, 1], 0.02), atol=1e-5)
    # a sign-flipped previous quaternion describes the same rotation
    qq, _ = slam.constant_velocity(q1, t1, -q2, t2)
    np.testing.assert_allclose(qq, q)


def test_relative_motion_and_ate():
    q0 = _quat([1, 0, 0], 0.0)
    q1 = _quat([0, 1, 0], np.deg2rad(30.0))
    d, ang = slam.relative_motion(q1, np.zeros(3), q0, np.array([0.0, 0.0, 0.3]))
    assert abs(ang - 30.0) < 1e-9
    # centres: -R^T t -> (0,0,0) and (0,0,-0.3)
    assert abs(d - 0.3) < 1e-12
    est = [(q0, np.array([0.0, 0.0, 0.0])), (q0, np.array([0.0, 0.03, 0.0]))]
    gt = [(q0, np.zeros(3)), (q0, np.zeros(3))]
    assert abs(slam.ate_rmse(est, gt) - 0.03 / np.sqrt(2)) < 1e-12


def test_schedule_gives_the_new_keyframe_at_least_40_percent():
    s = object.__new__(slam.GaussianSLAM)
    s.cfg = slam.SLAMConfig()
    s.rng = np.random.default_rng(0)
    s.active = type("A", (), {"keyframes": [None] * 6})()
    sched = s._schedule(100)
    assert len(sched) == 100 and sched.count(5) >= 40 and max(sched) == 5 and min(sched) >= 0
    s.active.keyframes = [None]
    assert s._schedule(7) == [0] * 7


def test_submap_switch_at_half_a_metre_or_fifty_degrees():
    cfg = slam.SLAMConfig()
    q0, t0 = _quat([0, 0, 1], 0.0), np.zeros(3)
    # world-to-camera t = -R c: with R = I the camera centre is -t
    assert not slam.needs_new_submap((q0, np.array([0.49, 0.0, 0.0])), (q0, t0), cfg)
    assert slam.needs_new_submap((q0, np.array([0.0, 0.51, 0.0])), (q0, t0), cfg)
    assert not slam.needs_new_submap((_quat([1, 1, 0], np.deg2rad(49.5)), t0), (q0, t0), cfg)
    assert slam.needs_new_submap((_quat([1, 1, 0], np.deg2rad(50.5)), t0), (q0, t0), cfg)


def test_submap_save_load_round_trip(tmp_path):
    rng = np.random.default_rng(2)
    subs = [{k: rng.standard_normal(s) for k, s in (("mean", (n, 3)), ("log_scale", (n, 3)), ("quat", (n, 4)),
                                                      ("opacity_logit", (n,)), ("rgb", (n, 3)))}
            for n in (5, 0, 12)]
    path = str(tmp_path / "s.npz")
    slam.save_submaps(path, subs)
    back = slam.load_submaps(path)
    assert len(back) == 3
    for a, b in zip(subs, back):
        assert set(a) == set(b)
        for k in a:
            np.testing.assert_array_equal(a[k], b[k])
