"""FP64 CPU oracle of sub-map seeding (Sec. 3.2 "densification", Sec. 4
implementation details, supplementary Sec. A).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): imported by tests/ and
bench.py's CPU legs, never by the product path.

A keyframe adds Gaussians to the active sub-map:
  1. candidate pixels: on the first keyframe of a sub-map, M_u pixels drawn
     uniformly plus the M_c pixels of highest colour gradient; on later
     keyframes, M_k pixels drawn uniformly among those whose rendered alpha is
     below alpha_n (Sec. 3.2, Sec. 4: alpha_n = 0.6).  Only pixels with a
     valid depth (> 0) are candidates.
  2. back-projection of the candidates into world space with the keyframe pose;
  3. a candidate is kept only if no Gaussian of the current sub-map lies within
     the search radius rho (Sec. 4: rho = 0.01 m);
  4. each kept point becomes a Gaussian with opacity 0.5, the pixel's colour,
     identity rotation and all three scales equal to its nearest-neighbour
     distance within the active sub-map (existing plus kept points), clamped
     to [s_min, s_max] (supplementary Sec. A).

Readings (the paper leaves them open; the CUDA path takes the same):
  - "drawn uniformly": the pixels with the M smallest keys
    (upper 32 bits of splitmix64(seed + pixel index), ties by pixel index),
    i.e. a uniform sample without replacement;
  - "high colour gradient": the squared central-difference gradient of the
    luminance Y = (R + G + B) / 3, g2 = gx^2 + gy^2 with
    gx = (Y[i, j+1] - Y[i, j-1]) / 2 (border pixels have g2 = 0); the M_c
    valid pixels with the largest g2, ties by pixel index;
  - a neighbour "within rho": squared distance < rho^2;
  - nearest-neighbour distance: over the other points of the sub-map after
    the keyframe's points are added; s_max when none is closer.
Pixel (i, j) has its centre at (j + 0.5, i + 0.5); depth is the camera z.

splitmix64 is Steele, Lea and Flood's SplitMix generator (OOPSLA 2014) as a
counter-based hash: x = seed + index; z = x + 0x9E3779B97F4A7C15;
z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) *
0x94D049BB133111EB; return z ^ (z >> 31) (all modulo 2^64).
"""
from __future__ import annotations

import numpy as np


def splitmix64(x):
    """Vectorised splitmix64 finaliser of uint64 counters (wrapping arithmetic)."""
    z = (np.asarray(x, np.uint64) + np.uint64(0x9E3779B97F4A7C15))
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def uniform_keys(n_pix: int, seed: int):
    """32-bit sampling key of every pixel index."""
    idx = np.arange(n_pix, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return (splitmix64(np.uint64(seed) + idx) >> np.uint64(32)).astype(np.uint64)


def sample_uniform(eligible, m: int, seed: int):
    """Indices (ascending) of the min(m, |eligible|) eligible pixels with the smallest keys."""
    eligible = np.asarray(eligible, bool).ravel()
    keys = uniform_keys(eligible.size, seed)
    cand = np.nonzero(eligible)[0]
    order = np.lexsort((cand, keys[cand]))  # by key, then pixel index
    return np.sort(cand[order[:min(m, cand.size)]])


def gradient2(rgb):
    """Squared central-difference gradient of the luminance; 0 on the border."""
    y = np.asarray(rgb, np.float64).mean(axis=0)
    g = np.zeros_like(y)
    gx = (y[1:-1, 2:] - y[1:-1, :-2]) / 2.0
    gy = (y[2:, 1:-1] - y[:-2, 1:-1]) / 2.0
    g[1:-1, 1:-1] = gx * gx + gy * gy
    return g


def sample_gradient(eligible, g2, m: int):
    """Indices (ascending) of the min(m, |eligible|) eligible pixels with the largest g2."""
    eligible = np.asarray(eligible, bool).ravel()
    g = np.asarray(g2, np.float64).ravel()
    cand = np.nonzero(eligible)[0]
    order = np.lexsort((cand, -g[cand]))
    return np.sort(cand[order[:min(m, cand.size)]])


def candidates(rgb, depth, alpha, first: bool, m_u: int, m_c: int, m_k: int, alpha_n: float, seed: int):
    """Candidate pixel indices (ascending, unique) of one keyframe."""
    depth = np.asarray(depth, np.float64)
    valid = depth > 0
    if first:
        u = sample_uniform(valid, m_u, seed)
        c = sample_gradient(valid, gradient2(rgb), m_c)
        return np.union1d(u, c)
    mask = valid & (np.asarray(alpha, np.float64) < alpha_n)
    return sample_uniform(mask, m_k, seed)


def _rot(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def backproject(pix, depth, cam, q, t):
    """World points of pixel indices: camera point ((x - cx) z / fx, (y - cy) z / fy, z)
    at the pixel centre, then p_w = R^T (p_c - t) for the world-to-camera pose (q, t)."""
    depth = np.asarray(depth, np.float64)
    H, W = depth.shape
    i, j = np.divmod(np.asarray(pix, np.int64), W)
    z = depth.ravel()[pix]
    pc = np.stack([(j + 0.5 - cam.cx) * z / cam.fx, (i + 0.5 - cam.cy) * z / cam.fy, z], axis=1)
    R = _rot(q)
    return (pc - np.asarray(t, np.float64)) @ R  # rows: R^T (p_c - t)


def min_dist2(queries, points, exclude_self: bool = False):
    """Brute-force squared distance from each query to its nearest point
    (exclude_self: queries are the points themselves, each skips its own index)."""
    queries = np.asarray(queries, np.float64).reshape(-1, 3)
    points = np.asarray(points, np.float64).reshape(-1, 3)
    out = np.full(len(queries), np.inf)
    qc, pc = 512, 8192
    for s in range(0, len(queries), qc):
        qd = queries[s:s + qc]
        for p0 in range(0, len(points), pc):
            d = ((qd[:, None, :] - points[None, p0:p0 + pc, :]) ** 2).sum(-1)
            if exclude_self:
                r = np.arange(s, s + len(qd))
                hit = (r >= p0) & (r < p0 + pc)
                d[np.nonzero(hit)[0], r[hit] - p0] = np.inf
            out[s:s + qc] = np.minimum(out[s:s + qc], d.min(axis=1))
    return out


def nn_dist2_self(points):
    """Squared distance from each point to its nearest other point of the set."""
    return min_dist2(points, points, exclude_self=True)


def seed_keyframe(rgb, depth, alpha, cam, q, t, existing_means, first: bool, m_u: int = 100_000, m_c: int = 50_000,
                  m_k: int = 100_000, alpha_n: float = 0.6, rho: float = 0.01, s_min: float = 1e-4,
                  s_max: float = 0.1, seed: int = 0):
    """All four steps.  Returns a dict with the candidate pixels, their world
    points, the kept mask, the squared distance to the nearest existing
    Gaussian (inf if none) and, for the kept points, the new Gaussians
    (mean, log_scale, quat, opacity_logit, rgb) in candidate order."""
    pix = candidates(rgb, depth, alpha, first, m_u, m_c, m_k, alpha_n, seed)
    pts = backproject(pix, depth, cam, q, t)
    d2_exist = min_dist2(pts, existing_means)
    keep = d2_exist >= rho * rho
    new = pts[keep]
    allp = np.concatenate([np.asarray(existing_means, np.float64).reshape(-1, 3), new])
    n_ex = len(allp) - len(new)
    d2 = np.full(len(new), np.inf)
    if len(new):
        # nearest other point of the sub-map after the addition
        d2 = np.minimum(min_dist2(new, allp[:n_ex]) if n_ex else d2, nn_dist2_self(new))
    s = np.clip(np.sqrt(d2), s_min, s_max)
    col = np.asarray(rgb, np.float64).reshape(3, -1)[:, pix[keep]].T
    n = len(new)
    gauss = dict(mean=new, log_scale=np.repeat(np.log(s)[:, None], 3, axis=1),
                 quat=np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)), opacity_logit=np.zeros(n), rgb=col)
    return dict(pix=pix, points=pts, keep=keep, d2_existing=d2_exist, nn_d2=d2, gaussians=gauss)


def prune(params: dict, min_opacity: float):
    """Supplementary Sec. A pruning: keep the Gaussians whose opacity
    sigmoid(logit) is at least min_opacity, in their original order."""
    o = 1.0 / (1.0 + np.exp(-np.asarray(params["opacity_logit"], np.float64)))
    keep = o >= min_opacity
    return {k: np.asarray(v)[keep] for k, v in params.items()}, keep


def merge(submaps, rho: float = 0.01):
    """Supplementary Sec. A global merge: sub-maps in sequence; a Gaussian is
    added when no Gaussian already in the global map lies at squared distance
    < rho^2 (Gaussians of the same sub-map do not reject each other).
    Returns the merged parameters and, per sub-map, the added mask."""
    out = {k: [] for k in submaps[0]}
    glob = np.zeros((0, 3))
    masks = []
    for sm in submaps:
        d2 = min_dist2(np.asarray(sm["mean"], np.float64), glob)
        add = d2 >= rho * rho
        masks.append(add)
        for k, v in sm.items():
            out[k].append(np.asarray(v)[add])
        glob = np.concatenate([glob, np.asarray(sm["mean"], np.float64)[add]])
    return {k: np.concatenate(v) for k, v in out.items()}, masks
