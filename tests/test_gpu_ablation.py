"""The synthetic mask / L_reg ablations run end to end (20-frame sequence with
2 % gross depth outliers); the full configuration tracks within 3 cm.  The
printed table is the synthetic counterpart of the paper's ablations, not a
reproduction of its numbers."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_tracking_mask_and_lreg_ablations_run():
    from paper_2312_10070_gb300 import ablation, api, slam, synth as S
    spec = S.camera_room()
    scene = S.room_scene(300_000, seed=100)
    qs, ts = S.room_trajectory(seed=100, n_frames=20, step_m=0.02, max_step_deg=1.5)
    gt = [(np.asarray(q, np.float64), np.asarray(t, np.float64)) for q, t in zip(qs, ts)]
    frames = ablation.synthetic_frames(scene, (qs, ts), spec, seed=500, outlier_frac=0.02)
    base = slam.SLAMConfig(track_iters=60, map_iters_first=100, map_iters=40, capacity=1_500_000,
                           seed=api.SeedConfig(m_u=100_000, m_c=50_000, m_k=30_000))
    masks = ablation.tracking_mask_ablation(frames, gt, spec, base)
    lreg = ablation.lreg_ablation(frames, gt, spec, base)
    print(masks, lreg)
    assert [(r["alpha_mask"], r["inlier_mask"]) for r in masks] == list(ablation.MASK_VARIANTS)
    for r in masks + lreg:
        assert np.isfinite(r["ate_cm"]) and np.isfinite(r["psnr_db"])
    assert masks[-1]["ate_cm"] < 3.0 and lreg[0]["ate_cm"] < 3.0
