"""Synthetic counterparts of the paper's tracking-mask and L_reg ablations.

Sequences (ablation.ablations_over_seeds): room scenes of 300k Gaussians,
seeds 100-102, 24 frames each with about 3 cm / 2 degrees between frames (so
each frame shows regions the map has not seen yet, which the alpha mask is
there to discount), 2 % gross depth outliers and flying pixels at half of the
depth-edge pixels (which the inlier mask is there to reject).  Both
ablations run the online SLAM loop once per variant and seed.

Measured on GB300 (mean over the three seeds): the alpha mask raises the
merged map's PSNR in every seed, with and without the inlier mask; no
direction of the tracking error (ATE) or of the L_reg weight holds across
the seeds.  The test asserts what held: the alpha mask's mean PSNR gain, with
and without the inlier mask, and tracking within 3 cm in every run.  The
variants' tracking losses themselves are compared with the oracle in
test_gpu_loss.py."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_tracking_mask_and_lreg_ablations_over_seeds():
    from paper_2312_10070_gb300 import ablation
    per_seed, summary = ablation.ablations_over_seeds([100, 101, 102], n_frames=24)
    for k, v in summary.items():
        print(f"{k}: ATE {v['ate_cm_mean']:.2f} +- {v['ate_cm_std']:.2f} cm {np.round(v['ate_cm'], 2).tolist()}, "
              f"PSNR {v['psnr_db_mean']:.2f} +- {v['psnr_db_std']:.2f} dB {np.round(v['psnr_db'], 2).tolist()}")
    for p in per_seed:
        assert [(r["alpha_mask"], r["inlier_mask"]) for r in p["tracking_masks"]] == list(ablation.MASK_VARIANTS)
        for r in p["tracking_masks"] + p["l_reg"]:
            assert np.isfinite(r["ate_cm"]) and np.isfinite(r["psnr_db"]) and r["ate_cm"] < 3.0, (p["seed"], r)
    for inlier in (0, 1):
        off, on = summary[f"alpha=0,inlier={inlier}"], summary[f"alpha=1,inlier={inlier}"]
        assert on["psnr_db_mean"] > off["psnr_db_mean"], (inlier, off, on)
