"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data: Gaussian sets, cameras and poses.  It contains
none of the rasterizer's arithmetic (no projection, blending or losses) and
imports nothing else from this package, so the CUDA path and the FP64 oracle
can both consume the same inputs.  All draws use ``numpy.random.default_rng``
(PCG64) in float64 and are cast to float32 at the end.

Scenes are dicts of contiguous float32 arrays:
    mean [n,3], log_scale [n,3], quat [n,4] (w,x,y,z), opacity_logit [n], rgb [n,3]
Poses are world-to-camera (q (w,x,y,z), t); camera frame x right, y down, z forward.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class CameraSpec:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float


def camera_unit() -> CameraSpec:
    """160x120 pinhole, fx = fy = 150, principal point at the centre."""
    return CameraSpec(160, 120, 150.0, 150.0, 80.0, 60.0)


def camera_room() -> CameraSpec:
    """1200x680 RGB-D camera of the room workloads."""
    return CameraSpec(1200, 680, 600.0, 600.0, 600.0, 340.0)


def camera_hires() -> CameraSpec:
    """1752x1168 high-resolution camera."""
    return CameraSpec(1752, 1168, 1200.0, 1200.0, 876.0, 584.0)


def scale_camera(cam: CameraSpec, width: int, height: int) -> CameraSpec:
    sx, sy = width / cam.width, height / cam.height
    return CameraSpec(width, height, cam.fx * sx, cam.fy * sy, cam.cx * sx, cam.cy * sy)


IDENTITY_POSE = (np.array([1.0, 0.0, 0.0, 0.0], np.float32), np.zeros(3, np.float32))


def _finish(mean, log_scale, quat, logit, rgb) -> dict:
    return dict(mean=np.ascontiguousarray(mean, np.float32),
                log_scale=np.ascontiguousarray(log_scale, np.float32),
                quat=np.ascontiguousarray(quat, np.float32),
                opacity_logit=np.ascontiguousarray(logit, np.float32),
                rgb=np.ascontiguousarray(rgb, np.float32))


def _random_quats(rng, n):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def random_scene(n: int = 5000, seed: int = 1, box=((-1.0, 1.0), (-0.75, 0.75), (1.0, 4.0)),
                 log_scale=(-3.0, 0.5), logit=(0.0, 1.0)) -> dict:
    """Gaussians uniform in a box in front of an identity camera.

    Defaults: the 160x120 unit workload (2 x 1.5 x [1,4] m box, log-scales
    N(-3, 0.5), random unit quaternions, opacity logits N(0, 1), RGB U[0,1])."""
    rng = np.random.default_rng(seed)
    lo = np.array([b[0] for b in box])
    hi = np.array([b[1] for b in box])
    mean = lo + (hi - lo) * rng.random((n, 3))
    ls = rng.normal(log_scale[0], log_scale[1], (n, 3))
    quat = _random_quats(rng, n)
    lg = rng.normal(logit[0], logit[1], n)
    rgb = rng.random((n, 3))
    return _finish(mean, ls, quat, lg, rgb)


def hires_scene(n: int = 1_500_000, seed: int = 4) -> dict:
    """Deep-overlap scene of the high-resolution workload: means in
    [-2,2] x [-1.3,1.3] x [1,6] m, log-scales N(-4, 0.7), logits N(1, 1)."""
    return random_scene(n, seed, box=((-2.0, 2.0), (-1.3, 1.3), (1.0, 6.0)), log_scale=(-4.0, 0.7),
                        logit=(1.0, 1.0))


def _axis_angle_quat(axis, angle):
    axis = np.asarray(axis, np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[np.cos(angle / 2)], np.sin(angle / 2) * axis])


def _qmul(a, b):
    """Hamilton product of (w,x,y,z) quaternions, broadcasting over leading dims."""
    aw, ax, ay, az = np.moveaxis(np.asarray(a, np.float64), -1, 0)
    bw, bx, by, bz = np.moveaxis(np.asarray(b, np.float64), -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw], axis=-1)


def perturbed_pose(seed: int = 2, max_t: float = 0.02, max_deg: float = 1.0):
    """A small world-to-camera pose: t ~ U[-max_t, max_t]^3 m and a rotation
    about a uniform random axis by U[-max_deg, max_deg] degrees."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(-max_t, max_t, 3)
    axis = rng.standard_normal(3)
    ang = np.deg2rad(rng.uniform(-max_deg, max_deg))
    q = _axis_angle_quat(axis, ang)
    return q.astype(np.float32), t.astype(np.float32)


# ---------------------------------------------------------------- room scenes

ROOM = (6.0, 5.0, 3.0)

# quaternions turning the local +z axis onto each axis-aligned normal
_S = np.sqrt(0.5)
_NORMAL_QUAT = {
    (0, 0, 1): (1.0, 0.0, 0.0, 0.0),
    (0, 0, -1): (0.0, 1.0, 0.0, 0.0),
    (1, 0, 0): (_S, 0.0, _S, 0.0),
    (-1, 0, 0): (_S, 0.0, -_S, 0.0),
    (0, 1, 0): (_S, -_S, 0.0, 0.0),
    (0, -1, 0): (_S, _S, 0.0, 0.0),
}


def _room_faces(rng, n_boxes):
    """Axis-aligned rectangles (origin, edge u, edge v, normal) of the room's
    six inner walls and the five visible faces of each box."""
    X, Y, Z = ROOM
    faces = [
        ((0, 0, 0), (X, 0, 0), (0, Y, 0), (0, 0, 1)),     # floor
        ((0, 0, Z), (X, 0, 0), (0, Y, 0), (0, 0, -1)),    # ceiling
        ((0, 0, 0), (0, Y, 0), (0, 0, Z), (1, 0, 0)),     # wall x = 0
        ((X, 0, 0), (0, Y, 0), (0, 0, Z), (-1, 0, 0)),    # wall x = X
        ((0, 0, 0), (X, 0, 0), (0, 0, Z), (0, 1, 0)),     # wall y = 0
        ((0, Y, 0), (X, 0, 0), (0, 0, Z), (0, -1, 0)),    # wall y = Y
    ]
    for _ in range(n_boxes):
        sx, sy, sz = rng.uniform(0.2, 1.0, 3)
        cx = rng.uniform(sx / 2, X - sx / 2)
        cy = rng.uniform(sy / 2, Y - sy / 2)
        x0, x1, y0, y1 = cx - sx / 2, cx + sx / 2, cy - sy / 2, cy + sy / 2
        faces += [
            ((x0, y0, sz), (sx, 0, 0), (0, sy, 0), (0, 0, 1)),
            ((x0, y0, 0), (0, sy, 0), (0, 0, sz), (-1, 0, 0)),
            ((x1, y0, 0), (0, sy, 0), (0, 0, sz), (1, 0, 0)),
            ((x0, y0, 0), (sx, 0, 0), (0, 0, sz), (0, -1, 0)),
            ((x0, y1, 0), (sx, 0, 0), (0, 0, sz), (0, 1, 0)),
        ]
    return [tuple(np.asarray(v, np.float64) for v in f) for f in faces]


def room_scene(n: int = 300_000, seed: int = 100, n_boxes: int = 40) -> dict:
    """Surface Gaussians of a 6 x 5 x 3 m room (z up) plus `n_boxes` boxes
    resting on the floor.  Gaussians are spread over faces in proportion to
    area, flat (tangent scale sqrt(A/n), normal scale 1 mm), local z along the
    face normal, opacity logits N(2, 0.5), RGB = per-face base colour plus a
    0.25-amplitude sinusoidal texture, clipped to [0, 1]."""
    rng = np.random.default_rng(seed)
    faces = _room_faces(rng, n_boxes)
    areas = np.array([np.linalg.norm(u) * np.linalg.norm(v) for _, u, v, _ in faces])
    counts = np.floor(n * areas / areas.sum()).astype(np.int64)
    counts[np.argmax(areas)] += n - counts.sum()
    tangent = np.log(np.sqrt(areas.sum() / n))
    means, quats, rgbs = [], [], []
    for (o, u, v, nrm), k in zip(faces, counts):
        if k == 0:
            continue
        a, b = rng.random(k), rng.random(k)
        means.append(o + a[:, None] * u + b[:, None] * v)
        qn = np.array(_NORMAL_QUAT[tuple(int(x) for x in nrm)])
        psi = rng.uniform(0, 2 * np.pi, k)
        qz = np.stack([np.cos(psi / 2), np.zeros(k), np.zeros(k), np.sin(psi / 2)], axis=1)
        quats.append(_qmul(qn[None, :], qz))
        base = rng.random(3)
        kk = rng.uniform(1.0, 5.0, 2)
        ph = rng.uniform(0, 2 * np.pi, 3)
        su, sv = a * np.linalg.norm(u), b * np.linalg.norm(v)
        tex = np.sin(2 * np.pi * (kk[0] * su + kk[1] * sv)[:, None] + ph[None, :])
        rgbs.append(np.clip(base[None, :] + 0.25 * tex, 0.0, 1.0))
    mean = np.concatenate(means)
    quat = np.concatenate(quats)
    rgb = np.concatenate(rgbs)
    ls = np.empty((n, 3))
    ls[:, :2] = tangent
    ls[:, 2] = np.log(1e-3)
    logit = rng.normal(2.0, 0.5, n)
    perm = rng.permutation(n)
    return _finish(mean[perm], ls[perm], quat[perm], logit[perm], rgb[perm])


def look_at_pose(position, target, up=(0.0, 0.0, 1.0)):
    """World-to-camera (q, t) of a camera at `position` looking at `target`
    (camera x right, y down, z forward; world z up)."""
    p = np.asarray(position, np.float64)
    f = np.asarray(target, np.float64) - p
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    Rcw = np.stack([r, d, f])          # rows: camera axes in world coordinates
    t = -Rcw @ p
    return _rot_to_quat(Rcw).astype(np.float32), t.astype(np.float32)


def _rot_to_quat(R):
    tr = np.trace(R)
    if tr > 0:
        s = np.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = np.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2]) * 2
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif R[1, 1] > R[2, 2]:
        s = np.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2]) * 2
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        s = np.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1]) * 2
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    return q if q[0] >= 0 else -q


def _catmull_rom(pts, samples_per_seg):
    pts = np.asarray(pts, np.float64)
    P = np.concatenate([pts[:1], pts, pts[-1:]])
    out = []
    for i in range(1, len(P) - 2):
        p0, p1, p2, p3 = P[i - 1], P[i], P[i + 1], P[i + 2]
        s = np.linspace(0, 1, samples_per_seg, endpoint=False)[:, None]
        out.append(0.5 * ((2 * p1) + (-p0 + p2) * s + (2 * p0 - 5 * p1 + 4 * p2 - p3) * s ** 2
                          + (-p0 + 3 * p1 - 3 * p2 + p3) * s ** 3))
    out.append(P[-2][None, :])
    return np.concatenate(out)


def room_trajectory(seed: int = 100, n_frames: int = 50, step_m: float = 0.015,
                    max_step_deg: float = 1.0):
    """Smooth camera path inside the room: Catmull-Rom splines through 10
    control points for the position ([1,5] x [1,4] x [1.2,1.8] m) and for the
    look-at target, re-sampled so that consecutive frames move about `step_m`
    metres and turn at most `max_step_deg` degrees.  Returns lists (q, t)."""
    rng = np.random.default_rng(seed)
    ctrl = np.stack([rng.uniform(1, 5, 10), rng.uniform(1, 4, 10), rng.uniform(1.2, 1.8, 10)], 1)
    look = np.stack([rng.uniform(0.3, 5.7, 10), rng.uniform(0.3, 4.7, 10), rng.uniform(0.6, 2.0, 10)], 1)
    pos = _catmull_rom(ctrl, 4000)
    tgt = _catmull_rom(look, 4000)
    fwd = tgt - pos
    fwd /= np.linalg.norm(fwd, axis=1, keepdims=True)
    frames = [0]
    for i in range(1, len(pos)):
        j = frames[-1]
        dist = np.linalg.norm(pos[i] - pos[j])
        ang = np.degrees(np.arccos(np.clip(np.dot(fwd[i], fwd[j]), -1, 1)))
        if dist >= step_m or ang >= max_step_deg:
            frames.append(i)
            if len(frames) == n_frames:
                break
    qs, ts = [], []
    for i in frames:
        q, t = look_at_pose(pos[i], tgt[i])
        qs.append(q)
        ts.append(t)
    return qs, ts


# Keyframe views of the 500k-Gaussian sub-map workload (camera position,
# look-at target).  With room_scene(500_000, seed=3) they see about 70k, 105k,
# 150k, 196k, 262k, 326k, 401k and 417k Gaussians.
SUBMAP_VIEWS = (
    ((3.0, 2.5, 1.5), (3.0, 5.0, 1.2)),
    ((3.5, 2.5, 1.5), (0.0, 2.5, 1.3)),
    ((3.0, 1.5, 1.5), (3.0, 5.0, 1.2)),
    ((4.5, 3.8, 1.7), (2.0, 1.0, 0.8)),
    ((1.2, 1.0, 1.6), (4.5, 4.0, 0.9)),
    ((5.5, 4.5, 2.2), (1.0, 0.5, 0.5)),
    ((0.3, 0.3, 2.8), (5.0, 4.0, 0.0)),
    ((5.9, 4.9, 2.95), (0.5, 0.5, 0.0)),
)
# the single view of the 1200x680 / 500k fwd+bwd throughput workload (~326k visible)
HEADLINE_VIEW = 5


def submap_views():
    """The 8 keyframe poses (q, t) of the sub-map mapping workload."""
    return [look_at_pose(p, t) for p, t in SUBMAP_VIEWS]


def noisy_copy(scene: dict, seed: int = 3, mean_sigma=0.005, log_scale_sigma=0.1, rgb_sigma=0.05,
               logit_sigma=0.3) -> dict:
    """The optimised copy of a ground-truth sub-map: GT plus Gaussian noise."""
    rng = np.random.default_rng(seed)
    n = scene["mean"].shape[0]
    return _finish(scene["mean"] + rng.normal(0, mean_sigma, (n, 3)),
                   scene["log_scale"] + rng.normal(0, log_scale_sigma, (n, 3)),
                   scene["quat"],
                   scene["opacity_logit"] + rng.normal(0, logit_sigma, n),
                   np.clip(scene["rgb"] + rng.normal(0, rgb_sigma, (n, 3)), 0, 1))


def add_sensor_noise(rgb, depth, alpha=None, seed: int = 0, rgb_sigma=0.01, depth_rel=0.01,
                     alpha_invalid=0.5):
    """Noisy RGB-D target: rgb + N(0, rgb_sigma), depth * (1 + N(0, depth_rel)),
    depth set to 0 (invalid) where the clean render's alpha < alpha_invalid."""
    rng = np.random.default_rng(seed)
    rgb_n = (rgb + rng.normal(0, rgb_sigma, rgb.shape)).astype(np.float32)
    d_n = (depth * (1 + rng.normal(0, depth_rel, depth.shape))).astype(np.float32)
    if alpha is not None:
        d_n[alpha < alpha_invalid] = 0
    return rgb_n, d_n
