"""Shared helpers of the GPU parity tests: the same seeded inputs go to the
CUDA path (float32) and to the FP64 oracle (the float32 values promoted)."""
import numpy as np

import oracle as O
from paper_2312_10070_gb300 import synth as S


def ocam(spec, tile=(16, 16), **kw):
    return O.Camera(spec.width, spec.height, spec.fx, spec.fy, spec.cx, spec.cy, tile_w=tile[0], tile_h=tile[1],
                    **kw)


def grad_close(g, ref, rel=1e-3, floor=0.1, rel_l2=1e-4):
    """Gradient parity: elementwise |g - ref| <= rel (|ref| + floor max|ref|) and
    a per-tensor relative L2 error <= rel_l2.  FP32 sums of many contributions
    of both signs carry an error relative to the contributions, not to the sum,
    so the elementwise floor scales with the tensor's largest entry (1e-4 of it
    by default).  Returns (ok, worst elementwise ratio)."""
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.size == 0:
        return True, 0.0
    mx = np.abs(ref).max()
    tol = rel * (np.abs(ref) + floor * mx) + 1e-30
    ratio = np.abs(g - ref) / tol
    l2 = np.linalg.norm(g - ref) / (np.linalg.norm(ref) + 1e-30)
    return bool((ratio <= 1.0).all() and l2 <= rel_l2), float(max(ratio.max(), l2 / rel_l2))


def strict_pass_fraction(g, ref):
    """Fraction of entries within the stricter elementwise bar
    |g - ref| <= 1e-3 (|ref| + 1e-3 rms(ref)) (reported beside grad_close)."""
    g = np.asarray(g, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    if ref.size == 0:
        return 1.0
    rms = np.sqrt(np.mean(ref * ref))
    return float(np.mean(np.abs(g - ref) <= 1e-3 * (np.abs(ref) + 1e-3 * rms) + 1e-30))


def tile_sequences_match(ranges, gids, ref_start, ref_gid, near_tie, skip):
    """Per tile, the GPU list must equal the oracle list once Gaussians with an
    ambiguous projection (`skip`) are removed; runs of float-depth near-ties
    may be permuted.  Returns the number of mismatching tiles."""
    bad = 0
    for t in range(len(ranges)):
        a = gids[ranges[t, 0]:ranges[t, 1]]
        s, e = ref_start[t], ref_start[t + 1]
        b = ref_gid[s:e]
        tie = near_tie[s:e]
        a = [x for x in a if not skip[x]]
        keep = [i for i, x in enumerate(b) if not skip[x]]
        b = [b[i] for i in keep]
        tie = [tie[i] for i in keep]
        if len(a) != len(b):
            bad += 1
            continue
        # group oracle entries into runs joined by near ties
        i = 0
        ok = True
        while i < len(b):
            j = i + 1
            while j < len(b) and tie[j]:
                j += 1
            if sorted(a[i:j]) != sorted(b[i:j]):
                ok = False
                break
            i = j
        bad += 0 if ok else 1
    return bad


def unit_inputs(seed=1, pose_seed=2):
    sc = S.random_scene(5000, seed)
    q, t = S.perturbed_pose(pose_seed)
    return sc, S.camera_unit(), q, t


def last_gids(last_idx, starts, gids, tile, width):
    """Gaussian id of each pixel's last composited list entry (-1 if none):
    last_idx indexes the list of the pixel's tile, which starts at
    starts[tile] in gids."""
    last_idx = np.asarray(last_idx, np.int64)
    H, W = last_idx.shape
    ys, xs = np.mgrid[0:H, 0:W]
    tx = (width + tile[0] - 1) // tile[0]
    t = (ys // tile[1]) * tx + xs // tile[0]
    pos = np.asarray(starts, np.int64)[t] + last_idx
    if len(gids) == 0:
        return np.full_like(last_idx, -1)
    g = np.asarray(gids)[np.clip(pos, 0, len(gids) - 1)]
    return np.where(last_idx >= 0, g, -1)


def box_min_sigma(u, v, ca, cb, cc, x0, x1, y0, y1):
    """Exact (FP64) minimum over the box [x0, x1] x [y0, y1] of
    sigma = 0.5 ca dx^2 + cb dx dy + 0.5 cc dy^2, dx = x - u, dy = y - v
    (a convex quadratic: 0 if (u, v) is inside, else the least of the four
    edge minima, each at the clamped one-dimensional minimiser)."""
    X0, X1, Y0, Y1 = x0 - u, x1 - u, y0 - v, y1 - v

    def edge(X, lo, hi, a, b, c):
        y = np.clip(-b * X / c, lo, hi)
        return 0.5 * a * X * X + b * X * y + 0.5 * c * y * y
    m = np.minimum.reduce([edge(X0, Y0, Y1, ca, cb, cc), edge(X1, Y0, Y1, ca, cb, cc),
                           edge(Y0, X0, X1, cc, cb, ca), edge(Y1, X0, X1, cc, cb, ca)])
    inside = (X0 <= 0) & (X1 >= 0) & (Y0 <= 0) & (Y1 >= 0)
    return np.where(inside, 0.0, m)

