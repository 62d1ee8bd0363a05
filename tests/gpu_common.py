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
