"""Synthetic ablations of the paper's tracking masks and of the isotropic
regulariser, run with the online SLAM loop on synthetic room sequences.

- Tracking mask ablation (the paper's tracking-mask table on TUM-RGBD desk):
  the tracking loss with or without the soft alpha mask (alpha^3) and with or
  without the inlier mask (depth error <= 50 x median), four runs.
- L_reg ablation (the paper's isotropic-regularisation tables): mapping
  with the regulariser weight 1 or 0.
Each run reports the ATE RMSE (cm) of the tracked trajectory and the PSNR
(dB) of the merged global map at the keyframes.  The paper's datasets are not
available, so these numbers describe the synthetic sequences, not the
paper's tables.

The sequences are renders of room_scene along room_trajectory with sensor
noise; `outlier_frac` of the valid depth pixels are additionally scaled by a
factor drawn from U[0.3, 2.0] (gross depth outliers, which the inlier mask is
there to reject).

    python -m paper_2312_10070_gb300.ablation [--frames 60] [--outliers 0.02]
"""
from __future__ import annotations

import argparse
import json
from dataclasses import replace

import numpy as np
import torch

from . import api, slam, synth


def synthetic_frames(scene: dict, poses, spec, seed: int = 0, outlier_frac: float = 0.0, ctx: api.Context = None):
    """RGB-D frames: the render, depth = rendered depth / alpha where alpha >=
    0.5 (else invalid), N(0, 0.01) colour and 1 % depth noise, then gross
    depth outliers on a fraction of the valid pixels."""
    ctx = ctx or api.Context()
    g = api.GaussianParams.from_numpy(scene)
    cam = api.camera_from_spec(spec)
    rng = np.random.default_rng(seed)
    frames = []
    for i, (q, t) in enumerate(zip(*poses)):
        r = api.render_forward(ctx, g, cam, api.make_pose(q, t))
        a = r["alpha"].cpu().numpy()
        d = np.where(a >= 0.5, r["depth"].cpu().numpy() / np.maximum(a, 1e-6), 0.0)
        rgb, dn = synth.add_sensor_noise(r["rgb"].cpu().numpy(), d, None, seed=seed + i)
        if outlier_frac > 0:
            out = (rng.random(dn.shape) < outlier_frac) & (dn > 0)
            dn[out] *= rng.uniform(0.3, 2.0, int(out.sum())).astype(np.float32)
        frames.append((torch.from_numpy(rgb).cuda(), torch.from_numpy(dn).cuda()))
    return frames


def run(frames, gt, spec, cfg: slam.SLAMConfig):
    """One SLAM run: (ATE RMSE in cm, PSNR of the merged map in dB, the run)."""
    s = slam.GaussianSLAM(spec, cfg)
    for i, (rgb, depth) in enumerate(frames):
        s.step(rgb, depth, init_pose=gt[0] if i == 0 else None)
    ate = 100.0 * slam.ate_rmse(s.poses, gt)
    g = slam.global_map(s.ctx, slam.all_submaps(s))
    return ate, slam.psnr(s.ctx, g, s.cam, s.keyframes), s


MASK_VARIANTS = ((False, False), (True, False), (False, True), (True, True))


def tracking_mask_ablation(frames, gt, spec, base: slam.SLAMConfig):
    rows = []
    for alpha_mask, inlier_mask in MASK_VARIANTS:
        track = replace(base.track, alpha_pow=3.0 if alpha_mask else 0.0, k_median=50.0 if inlier_mask else 1e30)
        ate, psnr, _ = run(frames, gt, spec, replace(base, track=track))
        rows.append(dict(alpha_mask=alpha_mask, inlier_mask=inlier_mask, ate_cm=ate, psnr_db=psnr))
    return rows


def lreg_ablation(frames, gt, spec, base: slam.SLAMConfig):
    rows = []
    for w in (1.0, 0.0):
        mcfg = replace(base.map, adam=replace(base.map.adam, w_reg=w))
        ate, psnr, _ = run(frames, gt, spec, replace(base, map=mcfg))
        rows.append(dict(w_reg=w, ate_cm=ate, psnr_db=psnr))
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=60)
    ap.add_argument("--outliers", type=float, default=0.02)
    ap.add_argument("--scene-seed", type=int, default=100)
    ap.add_argument("--gaussians", type=int, default=300_000)
    args = ap.parse_args()
    spec = synth.camera_room()
    scene = synth.room_scene(args.gaussians, seed=args.scene_seed)
    qs, ts = synth.room_trajectory(seed=args.scene_seed, n_frames=args.frames, step_m=0.02, max_step_deg=1.5)
    gt = [(np.asarray(q, np.float64), np.asarray(t, np.float64)) for q, t in zip(qs, ts)]
    frames = synthetic_frames(scene, (qs, ts), spec, seed=500, outlier_frac=args.outliers)
    base = slam.SLAMConfig(track_iters=60, map_iters_first=100, map_iters=40, capacity=1_500_000,
                           seed=api.SeedConfig(m_u=100_000, m_c=50_000, m_k=30_000))
    out = dict(sequence=dict(frames=args.frames, outliers=args.outliers, scene_seed=args.scene_seed,
                             gaussians=args.gaussians),
               tracking_masks=tracking_mask_ablation(frames, gt, spec, base),
               l_reg=lreg_ablation(frames, gt, spec, base))
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
