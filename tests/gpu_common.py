"""Shared helpers of the GPU parity tests: the same seeded inputs go to the
CUDA path (float32) and to the FP64 oracle (the float32 values promoted)."""
import numpy as np

import oracle as O
from paper_2312_10070_gb300 import synth as S

TOL_IMAGE = 2e-4  # max-abs bar of RGB, depth, alpha and final T against the FP64 oracle


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



def check_forward(ctx, out, sc64, q, t, oc, max_excluded=0.0, tol=TOL_IMAGE, label=""):
    """Forward parity of one render on context `ctx` (outputs `out` as numpy,
    with n_contrib) against the oracle at camera `oc` (same tile shape).

    Pixels where no decision is marginal must match the oracle's render:
    RGB, depth, alpha and final T within `tol`, n_contrib and the Gaussian
    of the last composited entry bit-exact (the GPU's last_idx is mapped to
    a Gaussian through its own tile lists, which may be culled).  At a pixel
    with marginal skip / stop decisions every branch is a valid float32
    result: the GPU's output must match one of the oracle's alternatives
    (render_alternatives) to the same bar.  Pixels with another kind of
    marginal decision (sigma sign, depth order, tile membership) are
    excluded; their fraction must not exceed `max_excluded`.  Returns
    (flips [H,W] uint32: the branches the GPU's output took, for the oracle's
    backward; excluded [H,W] bool; the oracle's render)."""
    from paper_2312_10070_gb300 import api
    ref = O.render(sc64, q, t, oc)
    H, W = oc.height, oc.width
    tx, ty = oc.tiles
    tile = (oc.tile_w, oc.tile_h)
    ranges, gids, _ = api.tile_lists(ctx, tx * ty, sc64.n)
    bins = O.bin_tiles(sc64, q, t, oc)
    g_gpu = last_gids(out["last_idx"], ranges[:, 0], gids, tile, W)
    g_ref = last_gids(ref["last_idx"], bins["start"][:-1], bins["gid"], tile, W)
    ok = ref["amb"] == 0
    for k in ("depth", "alpha", "final_T"):
        err = np.abs(out[k][ok] - ref[k][ok]).max() if ok.any() else 0.0
        assert err <= tol, (label, k, err)
    err = np.abs(out["rgb"][:, ok] - ref["rgb"][:, ok]).max() if ok.any() else 0.0
    assert err <= tol, (label, "rgb", err)
    assert np.array_equal(out["n_contrib"][ok], ref["n_contrib"][ok]), label
    assert np.array_equal(g_gpu[ok], g_ref[ok]), label
    flips = np.zeros(H * W, np.uint32)
    excluded = np.zeros(H * W, bool)
    fl = np.nonzero(~ok.ravel())[0]
    alt = O.render_alternatives(sc64, q, t, oc, fl)
    o_rgb = out["rgb"].reshape(3, -1)
    o_d, o_T, o_nc, o_g = out["depth"].ravel(), out["final_T"].ravel(), out["n_contrib"].ravel(), g_gpu.ravel()
    unmatched = []
    for i, p in enumerate(fl):
        if alt["amb"][i] & 8:
            excluded[p] = True
            continue
        c = alt["count"][i]
        good = ((alt["n_contrib"][i, :c] == o_nc[p]) & (alt["last_gid"][i, :c] == o_g[p])
                & (np.abs(alt["rgb"][i, :c] - o_rgb[:, p]).max(-1) <= tol)
                & (np.abs(alt["depth"][i, :c] - o_d[p]) <= tol) & (np.abs(alt["final_T"][i, :c] - o_T[p]) <= tol))
        k = np.nonzero(good)[0]
        if k.size == 0:
            unmatched.append(int(p))
            continue
        flips[p] = alt["flip"][i, k[0]]
    print(f"forward parity {label}: {H * W} pixels, {fl.size} with marginal decisions "
          f"({fl.size / (H * W):.4%}), matched to an alternative {fl.size - excluded.sum() - len(unmatched)}, "
          f"excluded {excluded.sum()} ({excluded.mean():.5%}), unmatched {len(unmatched)}")
    assert not unmatched, (label, unmatched[:10])
    assert excluded.mean() <= max_excluded, (label, excluded.mean())
    return flips.reshape(H, W), excluded.reshape(H, W), ref
