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


def flying_pixels(depth: np.ndarray, rng, frac: float, jump: float = 0.1) -> np.ndarray:
    """Depth-edge artefacts of an RGB-D sensor: at pixels next to a depth
    discontinuity (a 4-neighbour differing by more than `jump` relative),
    a fraction `frac` take a depth drawn uniformly between the two sides
    ("flying pixels"); invalid (0) depths stay invalid."""
    d = depth.copy()
    valid = d > 0
    pad = np.pad(d, 1, mode="edge")
    H, W = d.shape
    nb = [pad[0:H, 1:W + 1], pad[2:H + 2, 1:W + 1], pad[1:H + 1, 0:W], pad[1:H + 1, 2:W + 2]]
    far = np.max(nb, axis=0)
    near = np.min(np.where(np.array(nb) > 0, nb, np.inf), axis=0)
    edge = valid & np.isfinite(near) & (far > (1 + jump) * np.maximum(near, 1e-6))
    pick = edge & (rng.random(d.shape) < frac)
    u = rng.random(int(pick.sum()))
    d[pick] = (near[pick] + u * (far[pick] - near[pick])).astype(np.float32)
    return d


def synthetic_frames(scene: dict, poses, spec, seed: int = 0, outlier_frac: float = 0.0, ctx: api.Context = None,
                     edge_frac: float = 0.0):
    """RGB-D frames: the render, depth = rendered depth / alpha where alpha >=
    0.5 (else invalid), N(0, 0.01) colour and 1 % depth noise, then gross
    depth outliers on a fraction of the valid pixels and flying pixels on a
    fraction `edge_frac` of the pixels at depth edges."""
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
        if edge_frac > 0:
            dn = flying_pixels(dn, rng, edge_frac)
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


def ablations_over_seeds(seeds, n_frames: int = 24, gaussians: int = 300_000, outliers: float = 0.02,
                         edge_frac: float = 0.5, step_m: float = 0.03, max_step_deg: float = 2.0):
    """Both ablations on one synthetic sequence per scene seed (faster motion
    than the default sequences, so that each frame shows regions the map has
    not seen yet; gross depth outliers and flying pixels at depth edges).
    Returns per-seed rows and, per variant, the mean and standard deviation
    over seeds of ATE (cm) and PSNR (dB)."""
    spec = synth.camera_room()
    base = slam.SLAMConfig(track_iters=60, map_iters_first=100, map_iters=40, capacity=1_500_000,
                           seed=api.SeedConfig(m_u=100_000, m_c=50_000, m_k=30_000))
    per_seed = []
    for sd in seeds:
        scene = synth.room_scene(gaussians, seed=sd)
        qs, ts = synth.room_trajectory(seed=sd, n_frames=n_frames, step_m=step_m, max_step_deg=max_step_deg)
        gt = [(np.asarray(q, np.float64), np.asarray(t, np.float64)) for q, t in zip(qs, ts)]
        frames = synthetic_frames(scene, (qs, ts), spec, seed=500 + sd, outlier_frac=outliers, edge_frac=edge_frac)
        per_seed.append(dict(seed=sd, tracking_masks=tracking_mask_ablation(frames, gt, spec, base),
                             l_reg=lreg_ablation(frames, gt, spec, base)))
        del frames
        torch.cuda.empty_cache()
    summary = {}
    for key, name in (("tracking_masks", lambda r: f"alpha={int(r['alpha_mask'])},inlier={int(r['inlier_mask'])}"),
                      ("l_reg", lambda r: f"w_reg={r['w_reg']:g}")):
        for i, r in enumerate(per_seed[0][key]):
            ate = [p[key][i]["ate_cm"] for p in per_seed]
            ps = [p[key][i]["psnr_db"] for p in per_seed]
            summary[name(r)] = dict(ate_cm_mean=float(np.mean(ate)), ate_cm_std=float(np.std(ate)),
                                    psnr_db_mean=float(np.mean(ps)), psnr_db_std=float(np.std(ps)), ate_cm=ate,
                                    psnr_db=ps)
    return per_seed, summary


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=60)
    ap.add_argument("--outliers", type=float, default=0.02)
    ap.add_argument("--scene-seed", type=int, default=100)
    ap.add_argument("--gaussians", type=int, default=300_000)
    ap.add_argument("--seeds", type=str, default="",
                    help="comma-separated scene seeds: run both ablations on one artefact-laden sequence per seed "
                         "(faster motion, outliers, flying pixels) and report mean and spread")
    args = ap.parse_args()
    if args.seeds:
        per_seed, summary = ablations_over_seeds([int(x) for x in args.seeds.split(",")], n_frames=args.frames,
                                                 gaussians=args.gaussians, outliers=args.outliers)
        print(json.dumps(dict(per_seed=per_seed, summary=summary), indent=1))
        return
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
