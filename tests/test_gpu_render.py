"""GPU parity of the renderer: the CUDA path (through the C ABI) against the
FP64 oracle on the same seeded inputs.

Bars: tile keys / per-tile lists and per-pixel contributor counts bit-exact;
RGB / depth / alpha within max-abs 2e-4; gradients within 1e-3 relative,
|g - g_ref| <= 1e-3 |g_ref| + 1e-4 max|g_ref| elementwise and a per-tensor
relative L2 error <= 1e-4 (the count of entries within the stricter
1e-3 (|g| + 1e-3 rms) is printed).  Where the oracle finds a skip or stop
decision within the float32 error bound of its threshold, each branch is a
valid result: the GPU's pixel must equal one of the oracle's alternatives,
and the oracle's backward then takes the same branch.  Pixels with another
kind of marginal decision are excluded (none on the unit scenes, at most
0.1 % on the 1200x680 view); Gaussians with a marginal projection decision
are left out of the tile-list comparison.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2312_10070_gb300 import api, synth as S
from tests.gpu_common import (box_min_sigma, check_forward, grad_close, last_gids, ocam, strict_pass_fraction,
                              tile_sequences_match, unit_inputs)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context()
    yield c
    c.close()


def run_forward(ctx, sc, spec, q, t, tile=(16, 16)):
    g = api.GaussianParams.from_numpy(sc)
    cam = api.camera_from_spec(spec)
    pose = api.make_pose(q, t)
    out = api.render_forward(ctx, g, cam, pose, want_n_contrib=True)
    torch.cuda.synchronize()
    return g, cam, pose, {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}, out


def grads_match(grads, pose6, ref, label="", strict_min=0.995):
    """grad_close per parameter kind, and at least `strict_min` of the entries
    within the stricter elementwise bar 1e-3 (|g| + 1e-3 rms(g))."""
    for k in api.GaussianParams.NAMES:
        g = getattr(grads, k).cpu().numpy()
        ok, worst = grad_close(g, ref[k])
        strict = strict_pass_fraction(g, ref[k])
        print(f"{label} {k}: worst ratio {worst:.3f}, strict-floor pass {strict:.5f}")
        assert ok, (label, k, worst)
        assert strict >= strict_min, (label, k, strict)
    if pose6 is not None:
        ok, worst = grad_close(pose6.cpu().numpy(), ref["pose"])
        print(f"{label} pose: worst ratio {worst:.3f}")
        assert ok, (label, "pose", worst)


@pytest.mark.parametrize("seed,pose_seed", [(1, 2), (7, 8)])
def test_forward_unit_matches_oracle(ctx, seed, pose_seed):
    sc, spec, q, t = unit_inputs(seed, pose_seed)
    _, _, _, out, _ = run_forward(ctx, sc, spec, q, t)
    check_forward(ctx, out, O.Scene.from_dict(sc), q, t, ocam(spec), label=f"unit {seed}")


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 8), (32, 8)])
def test_tile_lists_bit_exact(tile):
    """Rectangle lists (rect_lists=1): the prior art's tiling, bit for bit."""
    c = api.Context(tile=tile, rect_lists=True)
    sc, spec, q, t = unit_inputs(3, 4)
    g, cam, pose, out, _ = run_forward(c, sc, spec, q, t)
    oc = ocam(spec, tile)
    sc64 = O.Scene.from_dict(sc)
    tx, ty = oc.tiles
    ranges, gids, dbits = api.tile_lists(c, tx * ty, sc64.n)
    ref = O.bin_tiles(sc64, q, t, oc)
    pr = O.project(sc64, q, t, oc)
    skip = (pr["amb"] & 1).astype(bool)
    print("Gaussians with a marginal projection decision:", skip.sum(), "depth near-ties:", ref["near_tie"].sum())
    assert skip.sum() <= 10
    assert tile_sequences_match(ranges, gids, ref["start"], ref["gid"], ref["near_tie"], skip) == 0
    # culling decisions and depth keys
    vis = dbits != 0xFFFFFFFF
    assert np.array_equal(vis[~skip], pr["visible"][~skip].astype(bool))
    f32 = pr["depth"].astype(np.float32).view(np.uint32).astype(np.int64)
    ulp = np.abs(dbits.astype(np.int64) - f32)[vis & ~skip]
    assert ulp.max() == 0, ulp.max()  # the depth keys are the correctly rounded camera depths
    # forward outputs at this tile size
    check_forward(c, out, sc64, q, t, oc, label=f"rect lists {tile}")
    c.close()


def test_backward_unit_matches_oracle(ctx):
    """dL/dpixel is nonzero at every pixel: at pixels with marginal decisions
    the oracle's backward takes the branches the GPU's forward took."""
    sc, spec, q, t = unit_inputs(1, 2)
    g, cam, pose, out, saved = run_forward(ctx, sc, spec, q, t)
    sc64 = O.Scene.from_dict(sc)
    flips, excl, _ = check_forward(ctx, out, sc64, q, t, ocam(spec), label="unit backward")
    rng = np.random.default_rng(5)
    H, W = spec.height, spec.width
    w = [rng.standard_normal((3, H, W)), rng.standard_normal((H, W)), rng.standard_normal((H, W))]
    for a in w:
        a[..., excl] = 0.0
    w = [a.astype(np.float32) for a in w]
    grads, pose6 = api.render_backward(ctx, g, cam, pose, saved, *[torch.from_numpy(a).cuda() for a in w])
    torch.cuda.synchronize()
    ref = O.render_backward(sc64, q, t, ocam(spec), *w, flips=flips)
    grads_match(grads, pose6, ref, "unit backward")


def test_pose_only_backward(ctx):
    sc, spec, q, t = unit_inputs(11, 12)
    g, cam, pose, out, saved = run_forward(ctx, sc, spec, q, t)
    sc64 = O.Scene.from_dict(sc)
    flips, excl, _ = check_forward(ctx, out, sc64, q, t, ocam(spec), label="pose-only")
    rng = np.random.default_rng(6)
    H, W = spec.height, spec.width
    d_rgb, d_dep = rng.standard_normal((3, H, W)), rng.standard_normal((H, W))
    d_rgb[:, excl] = 0
    d_dep[excl] = 0
    d_rgb, d_dep = d_rgb.astype(np.float32), d_dep.astype(np.float32)
    _, pose6 = api.render_backward(ctx, g, cam, pose, saved, torch.from_numpy(d_rgb).cuda(),
                                   torch.from_numpy(d_dep).cuda(), None, want_params=False)
    ref = O.render_backward(sc64, q, t, ocam(spec), d_rgb, d_dep, None, flips=flips)
    ok, worst = grad_close(pose6.cpu().numpy(), ref["pose"])
    assert ok, worst


def test_edge_cases(ctx):
    spec = S.CameraSpec(50, 37, 40.0, 40.0, 25.0, 18.5)  # ragged: 4 x 3 tiles, partial tiles
    cam = api.camera_from_spec(spec)
    pose = api.make_pose(*S.IDENTITY_POSE)
    # empty scene
    empty = {k: np.zeros((0,) + s, np.float32) for k, s in
             (("mean", (3,)), ("log_scale", (3,)), ("quat", (4,)), ("opacity_logit", ()), ("rgb", (3,)))}
    g = api.GaussianParams.from_numpy(empty)
    out = api.render_forward(ctx, g, cam, pose)
    assert float(out["rgb"].abs().max()) == 0.0 and float(out["final_T"].min()) == 1.0
    assert int(out["last_idx"].max()) == -1
    grads, pose6 = api.render_backward(ctx, g, cam, pose, out, torch.ones((3, 37, 50), device="cuda"))
    assert float(pose6.abs().max()) == 0.0
    # everything behind the camera: all culled
    sc = S.random_scene(300, 3, box=((-1, 1), (-1, 1), (-3, -1)))
    g = api.GaussianParams.from_numpy(sc)
    out = api.render_forward(ctx, g, cam, pose)
    assert float(out["alpha"].max()) == 0.0
    assert api.frame_stats(ctx)["n_visible"] == 0
    # ragged image against the oracle
    sc = S.random_scene(400, 4, box=((-0.6, 0.6), (-0.45, 0.45), (1, 3)), log_scale=(-3.0, 0.4))
    _, _, _, out, _ = run_forward(ctx, sc, spec, *S.IDENTITY_POSE)
    sc64 = O.Scene.from_dict(sc)
    check_forward(ctx, out, sc64, *S.IDENTITY_POSE, ocam(spec), label="ragged")


def test_memory_saving_mode_is_bit_identical():
    sc, spec, q, t = unit_inputs(1, 2)
    outs = []
    for ms in (False, True):
        c = api.Context(memory_saving=ms)
        g, cam, pose, out, saved = run_forward(c, sc, spec, q, t)
        # a second forward in between: default mode then rebuilds too
        d = torch.ones((3, spec.height, spec.width), device="cuda")
        grads, pose6 = api.render_backward(c, g, cam, pose, saved, d, d[0], None)
        torch.cuda.synchronize()
        outs.append((out, grads, pose6))
        c.close()
    for k in ("rgb", "depth", "alpha", "final_T", "last_idx", "n_contrib"):
        assert np.array_equal(outs[0][0][k], outs[1][0][k])
    for k in api.GaussianParams.NAMES:
        a, b = getattr(outs[0][1], k).cpu().numpy(), getattr(outs[1][1], k).cpu().numpy()
        ok, worst = grad_close(a, b)  # float atomics: summation order may differ
        assert ok, (k, worst)


@pytest.mark.parametrize("tile,batch,ppt", [((16, 16), 256, 0), ((8, 8), 128, 1), ((8, 8), 32, 2)])
def test_full_size_room_view_matches_oracle(tile, batch, ppt):
    """1200x680, 500k-Gaussian sub-map, the headline view, in the default
    launch configuration and in those the benchmark's autotuner picks (8x8
    tiles with staging batch 128 and one pixel per thread, or batch 32 and
    two pixels per thread)."""
    ctx = api.Context(tile=tile, batch=batch, pixels_per_thread=ppt)
    sc = S.room_scene(500_000, seed=3)
    spec = S.camera_room()
    q, t = S.submap_views()[S.HEADLINE_VIEW]
    g, cam, pose, out, saved = run_forward(ctx, sc, spec, q, t)
    sc64 = O.Scene.from_dict(sc)
    flips, excl, ref = check_forward(ctx, out, sc64, q, t, ocam(spec, tile), max_excluded=1e-3,
                                     label=f"1200x680 {tile} {batch} {ppt}")
    st = api.frame_stats(ctx)
    pr = O.project(sc64, q, t, ocam(spec))
    assert abs(st["n_visible"] - pr["visible"].sum()) <= (pr["amb"] & 1).sum()
    # backward on sampled outputs: dL/dpixel nonzero on a random 2% of the
    # pixels (those with marginal decisions included, at the GPU's branches)
    rng = np.random.default_rng(9)
    H, W = spec.height, spec.width
    mask = (rng.random((H, W)) < 0.02) & ~excl
    d_rgb = (rng.standard_normal((3, H, W)) * mask).astype(np.float32)
    d_dep = (rng.standard_normal((H, W)) * mask).astype(np.float32)
    grads, pose6 = api.render_backward(ctx, g, cam, pose, saved, torch.from_numpy(d_rgb).cuda(),
                                       torch.from_numpy(d_dep).cuda(), None)
    refb = O.render_backward(sc64, q, t, ocam(spec, tile), d_rgb, d_dep, None, flips=flips)
    grads_match(grads, pose6, refb, f"1200x680 {tile}")
    ctx.close()


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_pixels_per_thread_is_bit_identical(tile):
    """The blend kernels give each thread 1 or 2 pixels; per-pixel arithmetic
    is the same, so the forward is bit-identical and the backward agrees."""
    sc, spec, q, t = unit_inputs(5, 6)
    res = []
    for ppt in (1, 2):
        c = api.Context(tile=tile, pixels_per_thread=ppt)
        g, cam, pose, out, saved = run_forward(c, sc, spec, q, t)
        d = torch.ones((3, spec.height, spec.width), device="cuda")
        grads, pose6 = api.render_backward(c, g, cam, pose, saved, d, d[0] * 0.5, d[0] * -0.25)
        torch.cuda.synchronize()
        res.append((out, grads, pose6.cpu().numpy()))
        c.close()
    for k in ("rgb", "depth", "alpha", "final_T", "last_idx", "n_contrib"):
        assert np.array_equal(res[0][0][k], res[1][0][k]), k
    for k in api.GaussianParams.NAMES:
        ok, worst = grad_close(getattr(res[0][1], k).cpu().numpy(), getattr(res[1][1], k).cpu().numpy())
        assert ok, (k, worst)
    ok, worst = grad_close(res[0][2], res[1][2])
    assert ok, worst


def room_inputs():
    """Thin, oriented surfels: a 320x180 view of a 60k-Gaussian room."""
    spec = S.scale_camera(S.camera_room(), 320, 180)
    q, t = S.submap_views()[2]
    return S.room_scene(60_000, seed=7), spec, q, t


@pytest.mark.parametrize("tile,scene", [((16, 16), "unit"), ((8, 8), "unit"), ((8, 8), "room"), ((16, 8), "room")])
def test_culled_lists_keep_exactly_what_can_composite(tile, scene):
    """Default lists (rect_lists=0): each tile's list is its rectangle list
    with entries removed that cannot composite at any pixel centre of the
    tile.  Checked against FP64: an entry whose exact minimum of sigma over
    the tile's pixel centres is below the skip threshold ln(255 o) by a
    relative 1e-4 is kept; one whose exact minimum over the tile's
    pixel-centre box exceeds the kernels' skip test (ln(255 o) + 0.02, a
    margin above the float32 error of the exponential) by a relative 1e-3 is
    dropped; the order is the
    rectangle list's (the same GPU lists with rect_lists=1, filtered)."""
    sc, spec, q, t = unit_inputs(3, 4) if scene == "unit" else room_inputs()
    oc = ocam(spec, tile)
    sc64 = O.Scene.from_dict(sc)
    tx, ty = oc.tiles
    lists = {}
    for rect in (False, True):
        c = api.Context(tile=tile, rect_lists=rect)
        run_forward(c, sc, spec, q, t)
        lists[rect] = api.tile_lists(c, tx * ty, sc64.n)
        c.close()
    pr = O.project(sc64, q, t, oc)
    skip = (pr["amb"] & 1).astype(bool)
    u, v = pr["uv"][:, 0], pr["uv"][:, 1]
    ca, cb, cc = pr["conic"].T
    thr = np.log(255.0 * pr["opacity"])
    (rc, gc, _), (rr, gr, _) = lists[False], lists[True]
    n_rect = n_cull = 0
    for tl in range(tx * ty):
        full = gr[rr[tl, 0]:rr[tl, 1]]
        kept = gc[rc[tl, 0]:rc[tl, 1]]
        n_rect += len(full)
        n_cull += len(kept)
        assert list(kept) == [g for g in full if g in set(kept.tolist())], tl
        if len(full) == 0:
            continue
        X, Y = tl % tx, tl // tx
        x0, y0 = X * tile[0] + 0.5, Y * tile[1] + 0.5
        x1, y1 = min(X * tile[0] + tile[0], spec.width) - 0.5, min(Y * tile[1] + tile[1], spec.height) - 0.5
        f = full.astype(np.int64)
        px, py = np.meshgrid(np.arange(x0, x1 + 0.5), np.arange(y0, y1 + 0.5))
        dx = px.ravel()[None, :] - u[f][:, None]
        dy = py.ravel()[None, :] - v[f][:, None]
        sig = (0.5 * ca[f][:, None] * dx * dx + cb[f][:, None] * dx * dy + 0.5 * cc[f][:, None] * dy * dy).min(1)
        boxm = box_min_sigma(u[f], v[f], ca[f], cb[f], cc[f], x0, x1, y0, y1)
        must_keep = (sig < thr[f] - 1e-4 * np.abs(thr[f])) & ~skip[f]
        # the kernels' test keeps a margin e = 1e-6 kappa (kappa = the conic's
        # condition number) on both sides, and keeps everything when e >= 0.25
        thr_k = thr[f] + 0.02
        hd = 0.5 * (ca[f] - cc[f])
        lmax = 0.5 * (ca[f] + cc[f]) + np.sqrt(hd * hd + cb[f] ** 2)
        e = 1e-6 * lmax ** 2 / np.maximum(ca[f] * cc[f] - cb[f] ** 2, 1e-300)
        must_drop = ((boxm * (1 - e) > thr_k * (1 + e) + 1e-3 * np.abs(thr_k)) & (e < 0.2) & ~skip[f])
        ks = set(kept.tolist())
        assert all(g in ks for g in f[must_keep]), tl
        assert not any(g in ks for g in f[must_drop]), tl
    assert n_cull < n_rect
    print("instances: rectangle lists", n_rect, "culled lists", n_cull)


def test_culled_and_rect_lists_render_identically():
    """Culling changes the lists, not the result: images, contributor counts
    and the last composited Gaussian of every pixel are bit-identical, and
    the gradients agree (float atomics may sum in another order)."""
    sc, spec, q, t = unit_inputs(5, 6)
    res = []
    for rect in (False, True):
        c = api.Context(tile=(8, 8), batch=128, pixels_per_thread=1, rect_lists=rect)
        g, cam, pose, out, saved = run_forward(c, sc, spec, q, t)
        tx, ty = ocam(spec, (8, 8)).tiles
        ranges, gids, _ = api.tile_lists(c, tx * ty, len(sc["mean"]))
        d = torch.ones((3, spec.height, spec.width), device="cuda")
        grads, pose6 = api.render_backward(c, g, cam, pose, saved, d, d[0] * 0.5, d[0] * -0.25)
        torch.cuda.synchronize()
        res.append((out, last_gids(out["last_idx"], ranges[:, 0], gids, (8, 8), spec.width), grads,
                    pose6.cpu().numpy()))
        c.close()
    for k in ("rgb", "depth", "alpha", "final_T", "n_contrib"):
        assert np.array_equal(res[0][0][k], res[1][0][k]), k
    assert np.array_equal(res[0][1], res[1][1])
    for k in api.GaussianParams.NAMES:
        ok, worst = grad_close(getattr(res[0][2], k).cpu().numpy(), getattr(res[1][2], k).cpu().numpy())
        assert ok, (k, worst)
    ok, worst = grad_close(res[0][3], res[1][3])
    assert ok, worst

