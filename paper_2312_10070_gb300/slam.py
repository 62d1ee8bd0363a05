"""The online Gaussian-SLAM loop (Sec. 3.2-3.5, Sec. 4, supplementary Sec. A)
assembled from the C ABI, and the global map built from its sub-maps.

Per frame: a constant-velocity initial pose (Sec. 3.5: additive on t and on
the quaternion, which is sign-aligned and renormalised), then frame-to-model
tracking against the active sub-map (gsr_track_step).  Every kf_every-th
frame is a keyframe:
  1. a new sub-map starts when the camera has moved more than d_thre or
     turned more than theta_thre since the active sub-map's first keyframe
     (Sec. 3.2; Sec. 4: 0.5 m, 50 degrees); the finished sub-map is kept on
     the host (it no longer needs device memory);
  2. the keyframe seeds Gaussians (gsr_seed_keyframe: M_u + M_c points on a
     sub-map's first keyframe, M_k points where the rendered alpha is below
     alpha_n on later ones);
  3. the sub-map is optimised over its keyframes, at least 40 % of the
     iterations on the new keyframe (Sec. 4), Gaussians with opacity below
     o_thre being pruned at the middle and the end of those iterations
     (supplementary Sec. A).
After the sequence, the sub-maps are merged in order into a global map with
the seeding rule (gsr_merge_submap) and its colours are refined over every
keyframe (supplementary Sec. A).  Sub-maps can be saved to and loaded from
.npz files.  Every numerical step runs in libgsr.so; this module only
schedules.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from . import api


@dataclass
class SLAMConfig:
    kf_every: int = 5
    track_iters: int = 100
    map_iters_first: int = 100
    map_iters: int = 100
    new_kf_fraction: float = 0.4
    d_thre: float = 0.5
    theta_thre_deg: float = 50.0
    o_thre: float = 0.1
    capacity: int = 2_000_000
    seed: api.SeedConfig = field(default_factory=api.SeedConfig)
    track: api.TrackConfig = field(default_factory=api.TrackConfig)
    map: api.MapConfig = field(default_factory=lambda: api.MapConfig(use_graph=False))
    schedule_seed: int = 0


def _rot(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def camera_centre(q, t):
    return -_rot(q).T @ np.asarray(t, np.float64)


def relative_motion(qa, ta, qb, tb):
    """(camera-centre distance in m, relative rotation angle in degrees) between two poses."""
    Ra, Rb = _rot(qa), _rot(qb)
    cos = np.clip((np.trace(Ra @ Rb.T) - 1.0) / 2.0, -1.0, 1.0)
    return float(np.linalg.norm(camera_centre(qa, ta) - camera_centre(qb, tb))), float(np.degrees(np.arccos(cos)))


def needs_new_submap(pose, first_pose, cfg: SLAMConfig) -> bool:
    """Sub-map switching rule (Sec. 3.2, thresholds of Sec. 4): a keyframe
    starts a new sub-map when its camera centre lies more than d_thre from
    that of the active sub-map's first keyframe, or its orientation differs
    by more than theta_thre_deg."""
    d, ang = relative_motion(*pose, *first_pose)
    return d > cfg.d_thre or ang > cfg.theta_thre_deg


def constant_velocity(q1, t1, q2, t2):
    """Initial pose of frame i from frames i-1 (q1, t1) and i-2 (q2, t2):
    T_i = T_{i-1} + (T_{i-1} - T_{i-2}) on t and on the sign-aligned
    quaternion, renormalised."""
    q1, q2 = np.asarray(q1, np.float64), np.asarray(q2, np.float64)
    if np.dot(q1, q2) < 0:
        q2 = -q2
    q = 2 * q1 - q2
    q /= np.linalg.norm(q)
    if q[0] < 0:
        q = -q
    return q, 2 * np.asarray(t1, np.float64) - np.asarray(t2, np.float64)


class ActiveSubMap:
    def __init__(self, capacity: int, first_pose):
        self.sub = api.SubMap(capacity)
        self.moments = api.AdamMoments(self.sub.arrays)
        self.keyframes = []  # (pose (q, t), rgb, depth)
        self.first_pose = first_pose

    def to_host(self) -> dict:
        p = self.sub.params()
        return {k: t.cpu().numpy() for k, t in zip(api.GaussianParams.NAMES, p.tensors())}


class GaussianSLAM:
    """Feed frames with step(); estimated poses accumulate in .poses."""

    def __init__(self, spec, cfg: SLAMConfig = None, ctx: api.Context = None):
        self.cfg = cfg or SLAMConfig()
        self.ctx = ctx or api.Context()
        self.spec = spec
        self.cam = api.camera_from_spec(spec)
        self.poses = []
        self.submaps = []  # finished sub-maps (host dicts)
        self.active = None
        self.n_frames = 0
        self.rng = np.random.default_rng(self.cfg.schedule_seed)
        self.log = []
        self.keyframes = []  # every keyframe of the run: (pose, rgb, depth)

    # -------------------------------------------------------------- mapping
    def _schedule(self, n_iters: int):
        """Keyframe index per iteration: the new keyframe (the last) on at least
        new_kf_fraction of them, a random earlier keyframe of the sub-map on the rest."""
        K = len(self.active.keyframes)
        n_new = n_iters if K == 1 else int(math.ceil(self.cfg.new_kf_fraction * n_iters))
        sched = [K - 1] * n_new + [int(self.rng.integers(0, K - 1)) for _ in range(n_iters - n_new)]
        self.rng.shuffle(sched)
        return sched

    def _map(self, n_iters: int):
        a = self.active
        sched = self._schedule(n_iters)
        half = n_iters // 2
        i = 0
        while i < n_iters:
            j = i
            stop = half if i < half else n_iters  # prune at the middle: never run across it
            while j < stop and sched[j] == sched[i]:
                j += 1
            pose, rgb, depth = a.keyframes[sched[i]]
            api.map_step(self.ctx, a.sub.params(), a.moments, self.cam, [(api.make_pose(*pose), rgb, depth)],
                         None, j - i, self.cfg.map, want_stats=False)
            i = j
            if i == half or i == n_iters:
                api.prune(self.ctx, a.sub, a.moments, self.cfg.o_thre)

    def _keyframe(self, pose, rgb, depth):
        cfg = self.cfg
        first = self.active is None
        if not first and needs_new_submap(pose, self.active.first_pose, cfg):
            self.submaps.append(self.active.to_host())
            first = True
        if first:
            self.active = ActiveSubMap(cfg.capacity, pose)
        a = self.active
        scfg = api.SeedConfig(**{**cfg.seed.__dict__, "first_keyframe": first,
                                 "seed": cfg.seed.seed + self.n_frames})
        alpha = None
        if not first:
            alpha = api.render_forward(self.ctx, a.sub.params(), self.cam, api.make_pose(*pose))["alpha"]
        st = api.seed_keyframe(self.ctx, a.sub, self.cam, api.make_pose(*pose), rgb, depth, alpha, scfg)
        a.keyframes.append((pose, rgb, depth))
        self.keyframes.append((pose, rgb, depth))
        self._map(cfg.map_iters_first if first else cfg.map_iters)
        self.log.append(dict(frame=self.n_frames, new_submap=first, seeded=st["n_added"], gaussians=a.sub.n))

    # ------------------------------------------------------------- per frame
    def step(self, rgb: torch.Tensor, depth: torch.Tensor, init_pose=None):
        """Process one RGB-D frame (device tensors [3,H,W], [H,W]); the first
        frame's pose is init_pose (world-to-camera (q, t)).  Returns the pose."""
        i = self.n_frames
        if i == 0:
            if init_pose is None:
                raise ValueError("the first frame needs its pose")
            pose = (np.asarray(init_pose[0], np.float64), np.asarray(init_pose[1], np.float64))
        else:
            if i == 1:
                q0, t0 = self.poses[-1]
            else:
                q0, t0 = constant_velocity(*self.poses[-1], *self.poses[-2])
            p, _ = api.track_step(self.ctx, self.active.sub.params(), self.cam, rgb, depth, api.make_pose(q0, t0),
                                  self.cfg.track_iters, self.cfg.track)
            pose = (np.array(p.q[:], np.float64), np.array(p.t[:], np.float64))
        self.poses.append(pose)
        if i % self.cfg.kf_every == 0:
            self._keyframe(pose, rgb.clone(), depth.clone())
        self.n_frames += 1
        return pose


def ate_rmse(est, gt):
    """Root-mean-square camera-centre error (m) of estimated vs true world-to-camera poses."""
    e = [np.linalg.norm(camera_centre(*a) - camera_centre(*b)) for a, b in zip(est, gt)]
    return float(np.sqrt(np.mean(np.square(e))))


# ------------------------------------------------------------ global map
def all_submaps(s: GaussianSLAM):
    """The finished sub-maps and the active one, as host dicts, in order."""
    return s.submaps + ([s.active.to_host()] if s.active is not None else [])


def save_submaps(path: str, submaps):
    np.savez(path, **{f"{i}_{k}": v for i, sm in enumerate(submaps) for k, v in sm.items()})


def load_submaps(path: str):
    z = np.load(path)
    out = {}
    for key in z.files:
        i, k = key.split("_", 1)
        out.setdefault(int(i), {})[k] = z[key]
    return [out[i] for i in sorted(out)]


def global_map(ctx: api.Context, submaps, rho: float = 0.01) -> api.SubMap:
    """Merge sub-maps in sequence (supplementary Sec. A): each Gaussian is
    added when no Gaussian already in the global map lies within rho."""
    cap = sum(len(sm["mean"]) for sm in submaps)
    g = api.SubMap(max(cap, 1))
    for sm in submaps:
        api.merge_submap(ctx, g, api.GaussianParams.from_numpy(sm), rho)
    return g


def refine_colours(ctx: api.Context, g: api.SubMap, cam, keyframes, iters: int, lr_rgb: float = 2.5e-3,
                   seed: int = 0):
    """Colour refinement of the global map (supplementary Sec. A): mapping
    iterations over randomly drawn keyframes with every learning rate but the
    colour one at zero (and no regulariser), so only RGB changes."""
    cfg = api.MapConfig(adam=api.AdamConfig(lr_mean=0.0, lr_log_scale=0.0, lr_quat=0.0, lr_opacity=0.0,
                                            lr_rgb=lr_rgb, w_reg=0.0), use_graph=False)
    moments = api.AdamMoments(g.arrays)
    rng = np.random.default_rng(seed)
    for _ in range(iters):
        pose, rgb, depth = keyframes[int(rng.integers(0, len(keyframes)))]
        api.map_step(ctx, g.params(), moments, cam, [(api.make_pose(*pose), rgb, depth)], None, 1, cfg,
                     want_stats=False)
    return g


def psnr(ctx: api.Context, g: api.SubMap, cam, keyframes) -> float:
    """Mean PSNR (dB, peak 1) of the map's renders against the keyframes' colours."""
    vals = []
    for pose, rgb, _ in keyframes:
        r = api.render_forward(ctx, g.params(), cam, api.make_pose(*pose))["rgb"]
        mse = float(torch.mean((r.clamp(0, 1) - rgb) ** 2))
        vals.append(10.0 * math.log10(1.0 / max(mse, 1e-12)))
    return float(np.mean(vals))
