"""Pins of the FP64 oracle to facts outside itself (CPU only).

Each test ties an oracle function to a closed form, a library routine, brute
force on a tiny input, or central finite differences, so that a dropped term,
a wrong sign or index, or a transposed operand fails here.
"""
import json
import os

import numpy as np
import pytest
from scipy import ndimage
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2312_10070_gb300 import synth as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def logit(o):
    return np.log(o / (1 - o))


def one_gaussian_scene(means, scales, opac, rgbs):
    n = len(means)
    return O.Scene(np.array(means, float), np.log(np.array(scales, float)).reshape(n, 1).repeat(3, 1),
                   np.tile([1.0, 0, 0, 0], (n, 1)), logit(np.array(opac, float)), np.array(rgbs, float))


ID_Q, ID_T = np.array([1.0, 0, 0, 0]), np.zeros(3)


# ----------------------------------------------------------- closed forms

def test_single_isotropic_gaussian_footprint():
    """On-axis isotropic Gaussian, eps = 0: Sigma^I = (f s / z)^2 I, so every
    pixel is rgb * o exp(-|Delta|^2 / (2 (f s/z)^2)) and D = z * alpha (Sec. 3.1)."""
    cam = O.Camera(64, 48, 100.0, 100.0, 32.0, 24.0, eps2d=0.0)
    z, s, o = 2.0, 0.022, 0.8
    sc = one_gaussian_scene([[0, 0, z]], [s], [o], [[0.2, 0.5, 0.9]])
    r = O.render(sc, ID_Q, ID_T, cam)
    sp = 100.0 * s / z
    iy, ix = np.mgrid[0:48, 0:64]
    d2 = (ix + 0.5 - 32.0) ** 2 + (iy + 0.5 - 24.0) ** 2
    a = o * np.exp(-d2 / (2 * sp * sp))
    a = np.where(a >= 1 / 255, a, 0.0)
    for ch, c in enumerate([0.2, 0.5, 0.9]):
        np.testing.assert_allclose(r["rgb"][ch], c * a, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r["depth"], z * a, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r["alpha"], a, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r["final_T"], 1 - a, rtol=0, atol=1e-13)
    assert (r["n_contrib"] == (a > 0)).all()


def test_near_plane_cull():
    """Gaussians at camera depth p_z <= z_near (0.2 m) are culled; just beyond
    it they render (Sec. 3.1's projection with the near plane read as z_near)."""
    cam = O.Camera(64, 48, 100.0, 100.0, 32.0, 24.0)
    for z, seen in ((0.15, False), (0.19, False), (0.21, True), (0.25, True)):
        sc = one_gaussian_scene([[0, 0, z]], [0.02 * z], [0.8], [[0.2, 0.5, 0.9]])
        pr = O.project(sc, ID_Q, ID_T, cam)
        r = O.render(sc, ID_Q, ID_T, cam)
        assert pr["visible"][0] == int(seen) and pr["amb"][0] == 0, z
        assert (r["alpha"].max() > 0.5) == seen and (r["alpha"].max() == 0.0) == (not seen), z


def test_off_axis_cov2d_closed_form():
    """Isotropic Sigma = s^2 I is rotation invariant, so Sigma^I = s^2 J J^T + eps I
    with the pinhole Jacobian J at p (Zwicker et al. EWA, Sec. 3.1)."""
    cam = O.Camera(320, 240, 300.0, 280.0, 160.0, 120.0, eps2d=0.3)
    rng = np.random.default_rng(5)
    pts = np.column_stack([rng.uniform(-0.5, 0.5, 20), rng.uniform(-0.4, 0.4, 20), rng.uniform(1, 3, 20)])
    s = rng.uniform(0.01, 0.05, 20)
    sc = O.Scene(pts, np.log(s)[:, None].repeat(3, 1), rng.standard_normal((20, 4)),
                 np.zeros(20), np.zeros((20, 3)))
    # arbitrary camera rotation: p = R mu + t; put the points in camera frame first
    qc = Rotation.random(random_state=3)
    Rcw = qc.as_matrix()
    tcw = np.array([0.1, -0.2, 0.3])
    mu = (pts - tcw) @ Rcw  # R^T (p - t)
    sc.mean = np.ascontiguousarray(mu)
    xyzw = qc.as_quat()
    pr = O.project(sc, [xyzw[3], *xyzw[:3]], tcw, cam)
    for i in range(20):
        x, y, z = pts[i]
        a = s[i] ** 2 * (300.0 ** 2 / z ** 2) * (1 + (x / z) ** 2) + 0.3
        b = s[i] ** 2 * 300.0 * 280.0 * (x / z) * (y / z) / z ** 2
        c = s[i] ** 2 * (280.0 ** 2 / z ** 2) * (1 + (y / z) ** 2) + 0.3
        np.testing.assert_allclose(pr["cov2d"][i], [a, b, c], rtol=1e-10)
        np.testing.assert_allclose(pr["uv"][i], [300 * x / z + 160, 280 * y / z + 120], rtol=1e-12)
        np.testing.assert_allclose(pr["depth"][i], z, rtol=1e-12)
        det = a * c - b * b
        np.testing.assert_allclose(pr["conic"][i], [c / det, -b / det, a / det], rtol=1e-10)


def test_pose_jacobian_textbook():
    """d(u, v)/d(xi) of a left-perturbed pose is the textbook pinhole Jacobian
    [f/z, 0, -f x/z^2, -f x y/z^2, f (1 + x^2/z^2), -f y/z] (and its v row)."""
    cam = O.Camera(640, 480, 500.0, 450.0, 320.0, 240.0)
    rng = np.random.default_rng(11)
    n = 8
    qc = Rotation.random(random_state=7)
    Rcw, tcw = qc.as_matrix(), np.array([0.3, 0.1, -0.2])
    p = np.column_stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(1.5, 3, n)])
    mu = (p - tcw) @ Rcw
    sc = O.Scene(mu, np.full((n, 3), np.log(0.01)), rng.standard_normal((n, 4)), np.zeros(n), np.zeros((n, 3)))
    xyzw = qc.as_quat()
    pq = [xyzw[3], *xyzw[:3]]
    fx, fy = 500.0, 450.0
    for i in range(n):
        for comp in (0, 1):
            g2 = np.zeros((n, 10))
            g2[i, comp] = 1.0
            g = O.project_backward(sc, pq, tcw, cam, g2)["pose"]
            x, y, z = p[i]
            if comp == 0:
                ref = [fx / z, 0, -fx * x / z ** 2, -fx * x * y / z ** 2, fx * (1 + x * x / z ** 2), -fx * y / z]
            else:
                ref = [0, fy / z, -fy * y / z ** 2, -fy * (1 + y * y / z ** 2), fy * x * y / z ** 2, fy * x / z]
            np.testing.assert_allclose(g, ref, rtol=1e-10, atol=1e-10)


def test_opaque_front_stack():
    """alpha = 0.99 (clamped), then 0.98 (T test 2e-4 >= 1e-4, composited), then 0.9
    (T test 2e-5 < 1e-4, stop).  Everything behind the second Gaussian leaves the
    pixel bit-identical and receives exactly zero gradient."""
    cam = O.Camera(64, 48, 100.0, 100.0, 32.5, 24.5, eps2d=0.3)
    zs = [1.0, 2.0, 3.0, 4.0, 5.0]
    sc = one_gaussian_scene([[0, 0, z] for z in zs], [0.1 * z for z in zs], [0.995, 0.98, 0.9, 0.7, 0.6],
                            [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1]])
    r = O.render(sc, ID_Q, ID_T, cam)
    px = (24, 32)
    assert r["n_contrib"][px] == 2 and r["last_idx"][px] == 1
    np.testing.assert_allclose(r["final_T"][px], 0.01 * 0.02, rtol=1e-12)
    np.testing.assert_allclose(r["rgb"][:, 24, 32], [0.99, 0.98 * 0.01, 0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(r["depth"][px], 0.99 * 1 + 2 * 0.98 * 0.01, rtol=1e-12)
    d_rgb = np.zeros((3, 48, 64))
    d_rgb[:, 24, 32] = [0.3, -0.7, 1.1]
    d_dep = np.zeros((48, 64))
    d_dep[px] = 0.5
    d_al = np.zeros((48, 64))
    d_al[px] = -0.2
    g = O.render_backward(sc, ID_Q, ID_T, cam, d_rgb, d_dep, d_al)
    for j in (2, 3, 4):
        assert np.all(g["g2d"][j] == 0) and np.all(g["mean"][j] == 0) and g["opacity_logit"][j] == 0
        assert np.all(g["rgb"][j] == 0) and np.all(g["log_scale"][j] == 0) and np.all(g["quat"][j] == 0)
    assert g["opacity_logit"][0] == 0.0  # clamp active: d min(0.99, .)/d. = 0
    assert g["opacity_logit"][1] != 0.0
    # change everything behind the stop: the pixel stays bit-identical
    sc2 = sc.copy()
    sc2.rgb[2:] = 0.123
    sc2.opacity_logit[2:] = logit(np.array([0.95, 0.5, 0.3]))
    sc2.log_scale[2:] += 0.2
    r2 = O.render(sc2, ID_Q, ID_T, cam)
    assert np.array_equal(r2["rgb"][:, 24, 32], r["rgb"][:, 24, 32])
    assert r2["depth"][px] == r["depth"][px] and r2["final_T"][px] == r["final_T"][px]


def test_depth_adjoint_matches_paper():
    """Sec. 3.4: dD/dalpha_j = z_j T_j - (sum_{u>j} z_u alpha_u T_u)/(1 - alpha_j).
    At the pixel under three on-axis Gaussians sigma = 0, so alpha_j = o_j and
    dD/dlogit_j = dD/dalpha_j o_j (1 - o_j); dD/dz_j = alpha_j T_j."""
    cam = O.Camera(64, 48, 100.0, 100.0, 32.5, 24.5, eps2d=0.3)
    zs = np.array([1.5, 2.5, 3.2])
    os_ = np.array([0.5, 0.6, 0.7])
    sc = one_gaussian_scene([[0, 0, z] for z in zs], [0.05 * z for z in zs], os_, np.zeros((3, 3)))
    d_dep = np.zeros((48, 64))
    d_dep[24, 32] = 1.0
    g = O.render_backward(sc, ID_Q, ID_T, cam, None, d_dep, None)
    T = np.array([1.0, 1 - os_[0], (1 - os_[0]) * (1 - os_[1])])
    for j in range(3):
        S_after = sum(zs[u] * os_[u] * T[u] for u in range(j + 1, 3))
        dDda = zs[j] * T[j] - S_after / (1 - os_[j])
        np.testing.assert_allclose(g["opacity_logit"][j], dDda * os_[j] * (1 - os_[j]), rtol=1e-12)
        np.testing.assert_allclose(g["mean"][j], [0, 0, os_[j] * T[j]], rtol=1e-12, atol=1e-14)


# ------------------------------------------------------------ brute force

def brute_render(sc: O.Scene, q, t, cam: O.Camera):
    """Per-pixel compositing without tiles: projection with scipy rotations,
    numpy matrix products, eigvalsh radius; then, per pixel, every Gaussian whose
    tile rectangle covers the pixel's tile, sorted by (float32 depth, index)."""
    q = np.asarray(q, float)
    Rcw = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Rg = Rotation.from_quat(sc.quat[:, [1, 2, 3, 0]]).as_matrix()
    s2 = np.exp(2 * sc.log_scale)
    Sig = np.einsum("nij,nj,nkj->nik", Rg, s2, Rg)
    p = sc.mean @ Rcw.T + np.asarray(t, float)
    op = 1 / (1 + np.exp(-sc.opacity_logit))
    tiles_x, tiles_y = cam.tiles
    recs = []
    for i in range(sc.n):
        x, y, z = p[i]
        if z <= cam.z_near:
            continue
        limx, limy = cam.guard * 0.5 * cam.width / cam.fx, cam.guard * 0.5 * cam.height / cam.fy
        tx, ty = np.clip(x / z, -limx, limx), np.clip(y / z, -limy, limy)
        J = np.array([[cam.fx / z, 0, -cam.fx * tx / z], [0, cam.fy / z, -cam.fy * ty / z]])
        cov = J @ Rcw @ Sig[i] @ Rcw.T @ J.T + cam.eps2d * np.eye(2)
        if np.linalg.det(cov) <= 0:
            continue
        r = int(np.ceil(3 * np.sqrt(np.linalg.eigvalsh(cov).max())))
        u, v = cam.fx * x / z + cam.cx, cam.fy * y / z + cam.cy
        if u + r < 0 or u - r >= cam.width or v + r < 0 or v - r >= cam.height:
            continue
        rect = (max(0, int(np.floor((u - r) / cam.tile_w))), max(0, int(np.floor((v - r) / cam.tile_h))),
                min(tiles_x - 1, int(np.floor((u + r) / cam.tile_w))),
                min(tiles_y - 1, int(np.floor((v + r) / cam.tile_h))))
        recs.append((np.float32(z), i, u, v, np.linalg.inv(cov), op[i], z, rect))
    recs.sort(key=lambda e: (e[0], e[1]))
    H, W = cam.height, cam.width
    img = np.zeros((3, H, W))
    dep = np.zeros((H, W))
    Tf = np.ones((H, W))
    nc = np.zeros((H, W), int)
    for iy in range(H):
        for ix in range(W):
            tx, ty = ix // cam.tile_w, iy // cam.tile_h
            T = 1.0
            for (_, i, u, v, Q, o, z, (x0, y0, x1, y1)) in recs:
                if not (x0 <= tx <= x1 and y0 <= ty <= y1):
                    continue
                d = np.array([ix + 0.5 - u, iy + 0.5 - v])
                sg = 0.5 * d @ Q @ d
                if sg < 0:
                    continue
                a = min(0.99, o * np.exp(-sg))
                if a < 1 / 255:
                    continue
                if T * (1 - a) < 1e-4:
                    break
                img[:, iy, ix] += sc.rgb[i] * a * T
                dep[iy, ix] += z * a * T
                T *= 1 - a
                nc[iy, ix] += 1
            Tf[iy, ix] = T
    return img, dep, Tf, nc


@pytest.mark.parametrize("seed", [21, 22])
def test_tiled_oracle_equals_brute_force(seed):
    cam = O.Camera(40, 28, 40.0, 40.0, 20.0, 14.0, tile_w=8, tile_h=8)
    sc = O.Scene.from_dict(S.random_scene(60, seed, box=((-0.8, 0.8), (-0.6, 0.6), (1.0, 3.0)),
                                          log_scale=(-2.6, 0.4)))
    q, t = S.perturbed_pose(seed + 100)
    r = O.render(sc, q, t, cam)
    img, dep, Tf, nc = brute_render(sc, q, t, cam)
    ok = r["amb"] == 0
    assert ok.mean() > 0.9
    np.testing.assert_allclose(r["rgb"][:, ok], img[:, ok], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["depth"][ok], dep[ok], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["final_T"][ok], Tf[ok], rtol=0, atol=1e-12)
    assert np.array_equal(r["n_contrib"][ok], nc[ok])


def test_tile_lists_are_depth_sorted_rect_members():
    cam = O.Camera(48, 40, 50.0, 50.0, 24.0, 20.0, tile_w=16, tile_h=8)
    sc = O.Scene.from_dict(S.random_scene(200, 8, log_scale=(-3.0, 0.4)))
    b = O.bin_tiles(sc, *S.IDENTITY_POSE, cam)
    pr = O.project(sc, *S.IDENTITY_POSE, cam)
    tiles_x, tiles_y = cam.tiles
    for tile in range(tiles_x * tiles_y):
        tx, ty = tile % tiles_x, tile // tiles_x
        lst = b["gid"][b["start"][tile]:b["start"][tile + 1]]
        members = [i for i in range(sc.n) if pr["visible"][i] and pr["rect"][i, 0] <= tx <= pr["rect"][i, 2]
                   and pr["rect"][i, 1] <= ty <= pr["rect"][i, 3]]
        ref = sorted(members, key=lambda i: (np.float32(pr["depth"][i]), i))
        assert list(lst) == ref


def test_permutation_invariance():
    cam = O.Camera(64, 48, 60.0, 60.0, 32.0, 24.0)
    d = S.random_scene(300, 31)
    sc = O.Scene.from_dict(d)
    perm = np.random.default_rng(0).permutation(300)
    sp = O.Scene(sc.mean[perm], sc.log_scale[perm], sc.quat[perm], sc.opacity_logit[perm], sc.rgb[perm])
    q, t = S.perturbed_pose(4)
    a, b = O.render(sc, q, t, cam), O.render(sp, q, t, cam)
    for k in ("rgb", "depth", "final_T", "n_contrib", "last_idx"):
        assert np.array_equal(a[k], b[k]), k
    rng = np.random.default_rng(1)
    dr, dd = rng.standard_normal((3, 48, 64)), rng.standard_normal((48, 64))
    ga, gb = O.render_backward(sc, q, t, cam, dr, dd), O.render_backward(sp, q, t, cam, dr, dd)
    for k in ("mean", "log_scale", "quat", "opacity_logit", "rgb"):
        np.testing.assert_allclose(gb[k], ga[k][perm], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(gb["pose"], ga["pose"], rtol=1e-11)


# ----------------------------------------------------- finite differences

def _fd_scene():
    cam = O.Camera(48, 32, 45.0, 45.0, 24.0, 16.0, tile_w=16, tile_h=16)
    sc = O.Scene.from_dict(S.random_scene(30, 41, box=((-0.8, 0.8), (-0.5, 0.5), (1.0, 3.0)),
                                          log_scale=(-2.5, 0.3)))
    q, t = S.perturbed_pose(42)
    return cam, sc, q, t


def _linear_loss(sc, q, t, cam, w):
    r = O.render(sc, q, t, cam)
    return (np.sum(w[0] * r["rgb"]) + np.sum(w[1] * r["depth"]) + np.sum(w[2] * r["alpha"])), r


def test_render_backward_matches_central_fd():
    cam, sc, q, t = _fd_scene()
    rng = np.random.default_rng(3)
    w = (rng.standard_normal((3, 32, 48)), rng.standard_normal((32, 48)), rng.standard_normal((32, 48)))
    L0, r0 = _linear_loss(sc, q, t, cam, w)
    g = O.render_backward(sc, q, t, cam, *w)
    h = 1e-6
    checked = 0
    for name, shape in (("mean", 3), ("log_scale", 3), ("quat", 4), ("opacity_logit", 1), ("rgb", 3)):
        arr = getattr(sc, name)
        garr = g[name].reshape(sc.n, -1)
        flat = arr.reshape(sc.n, -1)
        for i in range(sc.n):
            for k in range(shape):
                old = flat[i, k]
                flat[i, k] = old + h
                Lp, rp = _linear_loss(sc, q, t, cam, w)
                flat[i, k] = old - h
                Lm, rm = _linear_loss(sc, q, t, cam, w)
                flat[i, k] = old
                if not (np.array_equal(rp["n_contrib"], r0["n_contrib"]) and np.array_equal(rm["n_contrib"], r0["n_contrib"])):
                    continue
                fd = (Lp - Lm) / (2 * h)
                assert abs(garr[i, k] - fd) <= 1e-6 * (abs(fd) + 1.0), (name, i, k, garr[i, k], fd)
                checked += 1
    assert checked > 0.95 * sc.n * 14
    # pose: left perturbation T(h e_k) = exp(h e_k^) T
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        Lp, _ = _linear_loss(sc, *O.pose_retract(q, t, xi), cam, w)
        Lm, _ = _linear_loss(sc, *O.pose_retract(q, t, -xi), cam, w)
        fd = (Lp - Lm) / (2 * h)
        assert abs(g["pose"][k] - fd) <= 1e-6 * (abs(fd) + 1.0), (k, g["pose"][k], fd)


def test_guard_band_clamp_gradient_matches_central_fd():
    """Gaussians whose centres lie beyond the guard band (|p_x/p_z| > 1.3 x the
    half-FOV tangent, likewise y) but whose footprints reach into the image:
    J is evaluated at the clamped coordinate, which passes no gradient.  The
    analytic gradient of every parameter and of the pose against FP64 central
    differences of the same clamped forward."""
    cam = O.Camera(48, 32, 45.0, 45.0, 24.0, 16.0, tile_w=16, tile_h=16)
    limx, limy = 1.3 * 24.0 / 45.0, 1.3 * 16.0 / 45.0
    means = [[1.0, 0.05, 1.2], [-0.1, -0.72, 1.4], [0.15, 0.1, 2.0]]
    sc = one_gaussian_scene(means, [0.35, 0.3, 0.05], [0.7, 0.6, 0.8], [[0.9, 0.2, 0.1], [0.1, 0.8, 0.3],
                                                                           [0.3, 0.3, 0.9]])
    sc.quat = np.array([[0.9, 0.1, -0.2, 0.3], [0.8, -0.3, 0.1, 0.2], [1.0, 0.0, 0.0, 0.0]])
    sc.log_scale = sc.log_scale + np.array([[0.0, -0.4, -1.5], [-0.3, 0.0, -1.2], [0.0, 0.0, 0.0]])
    m = np.array(means)
    assert abs(m[0, 0] / m[0, 2]) > limx and abs(m[1, 1] / m[1, 2]) > limy   # both clamps active
    rng = np.random.default_rng(11)
    w = (rng.standard_normal((3, 32, 48)), rng.standard_normal((32, 48)), rng.standard_normal((32, 48)))
    L0, r0 = _linear_loss(sc, ID_Q, ID_T, cam, w)
    assert r0["alpha"][:, 40:].max() > 0.05 and r0["alpha"][:4, :].max() > 0.05  # the clamped ones are seen
    g = O.render_backward(sc, ID_Q, ID_T, cam, *w)
    h = 1e-6
    for name, shape in (("mean", 3), ("log_scale", 3), ("quat", 4), ("opacity_logit", 1)):
        flat = getattr(sc, name).reshape(sc.n, -1)
        garr = g[name].reshape(sc.n, -1)
        for i in range(2):
            for k in range(shape):
                old = flat[i, k]
                flat[i, k] = old + h
                Lp, rp = _linear_loss(sc, ID_Q, ID_T, cam, w)
                flat[i, k] = old - h
                Lm, rm = _linear_loss(sc, ID_Q, ID_T, cam, w)
                flat[i, k] = old
                assert np.array_equal(rp["n_contrib"], r0["n_contrib"]) and np.array_equal(rm["n_contrib"],
                                                                                          r0["n_contrib"])
                fd = (Lp - Lm) / (2 * h)
                assert abs(garr[i, k] - fd) <= 1e-6 * (abs(fd) + 1.0), (name, i, k, garr[i, k], fd)
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        Lp, _ = _linear_loss(sc, *O.pose_retract(ID_Q, ID_T, xi), cam, w)
        Lm, _ = _linear_loss(sc, *O.pose_retract(ID_Q, ID_T, -xi), cam, w)
        fd = (Lp - Lm) / (2 * h)
        assert abs(g["pose"][k] - fd) <= 1e-6 * (abs(fd) + 1.0), (k, g["pose"][k], fd)


def test_loss_map_gradient_fd_and_ssim_library():
    rng = np.random.default_rng(9)
    H, W = 14, 17
    a, b = rng.random((3, H, W)), rng.random((3, H, W))
    d, dt = rng.uniform(1, 3, (H, W)), rng.uniform(1, 3, (H, W))
    dt[rng.random((H, W)) < 0.2] = 0
    out = O.loss_map(a, d, b, dt)
    # SSIM map from scipy's Gaussian filter (sigma 1.5, radius 5, zero padding)
    gf = lambda x: ndimage.gaussian_filter(x, 1.5, truncate=5 / 1.5, mode="constant", cval=0.0)
    C1, C2 = 1e-4, 9e-4
    ref = []
    for ch in range(3):
        x, y = a[ch], b[ch]
        mx, my = gf(x), gf(y)
        sx, sy, sxy = gf(x * x) - mx * mx, gf(y * y) - my * my, gf(x * y) - mx * my
        ref.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sx + sy + C2)))
    np.testing.assert_allclose(out["ssim_map"], np.array(ref), rtol=1e-10, atol=1e-12)
    valid = dt > 0
    l1c, l1d = np.abs(a - b).mean(), np.abs(d - dt)[valid].mean()
    np.testing.assert_allclose(out["loss"], 0.8 * l1c + 0.2 * (1 - np.mean(ref)) + l1d, rtol=1e-12)
    h = 1e-6
    for ch, y, x in [(0, 0, 0), (1, 5, 7), (2, 13, 16), (0, 7, 3), (1, 2, 15)]:
        ap, am = a.copy(), a.copy()
        ap[ch, y, x] += h
        am[ch, y, x] -= h
        fd = (O.loss_map(ap, d, b, dt)["loss"] - O.loss_map(am, d, b, dt)["loss"]) / (2 * h)
        np.testing.assert_allclose(out["d_rgb"][ch, y, x], fd, rtol=1e-6, atol=1e-9)
    for y, x in [(1, 1), (6, 9), (13, 0)]:
        dp, dm = d.copy(), d.copy()
        dp[y, x] += h
        dm[y, x] -= h
        fd = (O.loss_map(a, dp, b, dt)["loss"] - O.loss_map(a, dm, b, dt)["loss"]) / (2 * h)
        np.testing.assert_allclose(out["d_depth"][y, x], fd, rtol=1e-6, atol=1e-9)


def test_ssim_identical_and_constant_offset():
    rng = np.random.default_rng(2)
    a = rng.random((3, 20, 20))
    d = np.ones((20, 20))
    out = O.loss_map(a, d, a, d)
    np.testing.assert_allclose(out["ssim_map"], 1.0, rtol=0, atol=1e-12)
    assert np.abs(out["d_rgb"]).max() < 1e-15  # L1 sign(0) = 0 and SSIM at its maximum
    # constant images k and k + c: interior pixels (window fully inside) reduce to
    # the luminance term (2 k (k+c) + C1) / (k^2 + (k+c)^2 + C1)
    k, c = 0.3, 0.25
    out = O.loss_map(np.full((3, 20, 20), k), d, np.full((3, 20, 20), k + c), d)
    lum = (2 * k * (k + c) + 1e-4) / (k * k + (k + c) ** 2 + 1e-4)
    np.testing.assert_allclose(out["ssim_map"][:, 5:15, 5:15], lum, rtol=1e-10)


def test_loss_track_brute_force_and_fd():
    rng = np.random.default_rng(4)
    H, W = 10, 13
    a, b = rng.random((3, H, W)), rng.random((3, H, W))
    d = rng.uniform(1, 3, (H, W))
    dt = d + rng.normal(0, 0.05, (H, W))
    dt[0, :4] = 0
    d[5, 5] = dt[5, 5] + 40.0  # an outlier beyond 50x the median
    al = rng.random((H, W))
    out = O.loss_track(a, d, al, b, dt)
    valid = dt > 0
    e = np.abs(d - dt)
    med = np.sort(e[valid])[(valid.sum() - 1) // 2]
    assert out["median"] == med
    inl = valid & (e <= 50 * med)
    assert not inl[5, 5] and np.array_equal(out["inlier"], inl)
    w = inl * al ** 3
    ref = np.sum(w * (0.5 * np.abs(a - b).sum(0) + 0.5 * e))
    np.testing.assert_allclose(out["loss"], ref, rtol=1e-12)
    # Sec. 3.5 weighs colour by lambda_c and depth by 1 - lambda_c for any lambda_c
    # (0.5 above hides a swap) and masks by alpha to any power
    o2 = O.loss_track(a, d, al, b, dt, 0.3, 50.0, 2.0)
    ref2 = np.sum(inl * al ** 2 * (0.3 * np.abs(a - b).sum(0) + 0.7 * e))
    np.testing.assert_allclose(o2["loss"], ref2, rtol=1e-12)
    h = 1e-7
    for ch, y, x in [(0, 3, 3), (2, 9, 12), (1, 5, 6)]:
        ap, am = a.copy(), a.copy()
        ap[ch, y, x] += h
        am[ch, y, x] -= h
        fd = (O.loss_track(ap, d, al, b, dt)["loss"] - O.loss_track(am, d, al, b, dt)["loss"]) / (2 * h)
        np.testing.assert_allclose(out["d_rgb"][ch, y, x], fd, rtol=1e-6, atol=1e-9)
    for y, x in [(2, 2), (7, 11)]:
        dp, dm = d.copy(), d.copy()
        dp[y, x] += h
        dm[y, x] -= h
        fd = (O.loss_track(a, dp, al, b, dt)["loss"] - O.loss_track(a, dm, al, b, dt)["loss"]) / (2 * h)
        np.testing.assert_allclose(out["d_depth"][y, x], fd, rtol=1e-6, atol=1e-9)


def test_lreg_fd_and_isotropic_zero():
    rng = np.random.default_rng(6)
    ls = rng.normal(-3, 0.5, (12, 3))
    L, g = O.lreg(ls)
    s = np.exp(ls)
    np.testing.assert_allclose(L, np.abs(s - s.mean(1, keepdims=True)).sum() / 12, rtol=1e-12)
    h = 1e-7
    for i, k in [(0, 0), (3, 2), (11, 1)]:
        lp, lm = ls.copy(), ls.copy()
        lp[i, k] += h
        lm[i, k] -= h
        fd = (O.lreg(lp)[0] - O.lreg(lm)[0]) / (2 * h)
        np.testing.assert_allclose(g[i, k], fd, rtol=1e-6, atol=1e-12)
    L, g = O.lreg(np.full((5, 3), -2.0))
    assert L == 0.0 and np.all(g == 0.0)


def test_adam_matches_torch_optimizer():
    import torch
    rng = np.random.default_rng(8)
    p0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(5)]
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for k, g in enumerate(grads):
        O.adam(p, g.copy(), m, v, k + 1, 1e-2, 0.9, 0.999, 1e-15)
        if k == 0:  # first step: theta - lr g/(|g| + eps)
            np.testing.assert_allclose(p, p0 - 1e-2 * g / (np.abs(g) + 1e-15), rtol=1e-12)
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    for g in grads:
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12)


def test_pose_retract_matches_matrix_exponential():
    rng = np.random.default_rng(12)
    for _ in range(5):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        t = rng.standard_normal(3)
        xi = rng.standard_normal(6) * 0.3
        qo, to = O.pose_retract(q, t, xi)
        Xi = np.zeros((4, 4))
        rho, phi = xi[:3], xi[3:]
        Xi[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
        Xi[:3, 3] = rho
        T = np.eye(4)
        T[:3, :3] = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        T[:3, 3] = t
        ref = expm(Xi) @ T
        np.testing.assert_allclose(Rotation.from_quat([qo[1], qo[2], qo[3], qo[0]]).as_matrix(), ref[:3, :3],
                                   atol=1e-12)
        np.testing.assert_allclose(to, ref[:3, 3], atol=1e-12)


def test_paper_constants_fixture():
    c = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    rng = np.random.default_rng(1)
    a, b = rng.random((3, 12, 12)), rng.random((3, 12, 12))
    d = np.ones((12, 12))
    out = O.loss_map(a, d, b, d)
    lam = c["lambda_ssim"]["value"]
    np.testing.assert_allclose(out["loss"], (1 - lam) * out["l1_color"] + lam * (1 - out["ssim"]), rtol=1e-12)
    assert O.loss_track.__defaults__[1] == c["inlier_median_factor"]["value"]
    assert O.loss_track.__defaults__[2] == c["alpha_mask_power"]["value"]


def test_tile_aligned_crop_renders_the_same_window():
    """Region-restricted rendering (used for finite differences at high
    resolution) reproduces the full render inside the window exactly."""
    sc = O.Scene.from_dict(S.random_scene(3000, 5))
    cs = S.camera_unit()
    cam = O.Camera(cs.width, cs.height, cs.fx, cs.fy, cs.cx, cs.cy)
    q, t = S.perturbed_pose(3)
    full = O.render(sc, q, t, cam)
    for tiles in ((3, 2, 6, 5), (0, 0, 1, 7), (8, 6, 9, 7)):
        cc = cam.crop(*tiles)
        cr = O.render(sc, q, t, cc)
        y0, x0 = tiles[1] * 16, tiles[0] * 16
        win = (slice(y0, y0 + cc.height), slice(x0, x0 + cc.width))
        np.testing.assert_allclose(cr["rgb"], full["rgb"][(slice(None),) + win], rtol=0, atol=1e-12)
        np.testing.assert_allclose(cr["depth"], full["depth"][win], rtol=0, atol=1e-12)
        assert np.array_equal(cr["n_contrib"], full["n_contrib"][win])


def _hat(xi):
    X = np.zeros((4, 4))
    rho, phi = xi[:3], xi[3:]
    X[:3, :3] = [[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]]
    X[:3, 3] = rho
    return X


def test_se3_left_jacobian_matches_matrix_log_differences():
    """J_l(xi) e = log(exp((xi + e)^) exp(xi^)^-1) to first order: each column
    against central differences of scipy's matrix exponential and logarithm,
    for small (series branch), moderate and large rotations."""
    from scipy.linalg import logm
    rng = np.random.default_rng(17)
    h = 1e-6
    for scale in (1e-3, 5e-3, 0.05, 0.4, 1.5):
        xi = rng.standard_normal(6)
        xi[3:] *= scale / np.linalg.norm(xi[3:])
        J = O.se3_left_jacobian(xi)
        Einv = np.linalg.inv(expm(_hat(xi)))
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            Mp = np.real(logm(expm(_hat(xi + e)) @ Einv))
            Mm = np.real(logm(expm(_hat(xi - e)) @ Einv))
            D = (Mp - Mm) / (2 * h)
            col = np.array([D[0, 3], D[1, 3], D[2, 3], D[2, 1], D[0, 2], D[1, 0]])
            np.testing.assert_allclose(J[:, k], col, atol=2e-7, err_msg=f"scale {scale} column {k}")


def test_twist_gradient_at_nonzero_twist_matches_central_fd():
    """dL/dxi of a render at exp(xi^) T for xi != 0: J_l(xi)^T times the
    left-perturbation gradient at exp(xi^) T, against central differences of
    the loss over xi itself (a plain left-perturbation gradient misses the
    J_l factor, an error of order |xi|)."""
    cam, sc, q, t = _fd_scene()
    rng = np.random.default_rng(23)
    w = (rng.standard_normal((3, 32, 48)), rng.standard_normal((32, 48)), rng.standard_normal((32, 48)))
    xi = np.array([0.02, -0.015, 0.03, 0.05, -0.04, 0.06])
    qx, tx = O.pose_retract(q, t, xi)
    g = O.render_backward(sc, qx, tx, cam, *w)
    an = O.twist_gradient(xi, g["pose"])
    h = 1e-6
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        Lp, _ = _linear_loss(sc, *O.pose_retract(q, t, xi + e), cam, w)
        Lm, _ = _linear_loss(sc, *O.pose_retract(q, t, xi - e), cam, w)
        fd = (Lp - Lm) / (2 * h)
        assert abs(an[k] - fd) <= 1e-6 * (abs(fd) + 1.0), (k, an[k], fd)
    # the factor matters at this twist: the bare left gradient is off by more than the bar
    assert np.abs(g["pose"] - an).max() > 1e-3 * (np.abs(an).max() + 1.0)


def test_marginal_decision_alternatives_take_the_other_branch():
    """A skip decision (alpha within its error bound of 1/255) and a stop
    decision (T (1 - alpha) within its bound of 1e-4) each yield two results:
    the oracle's own branch, and the other branch, which equals the render
    of the scene without that Gaussian (skip) or the render where it is
    composited (stop).  The flip masks of render_alternatives reproduce
    render(flips=...) and the backward takes the same branches."""
    cam = O.Camera(16, 16, 40.0, 40.0, 8.0, 8.0, tile_w=16, tile_h=16, eps2d=0.0)
    # skip decision at pixel (8, 8) (centre (8.5, 8.5)): a Gaussian centred
    # 0.3 px off it (sigma clearly positive) whose alpha there is 1/255 (1 + 1e-9)
    sc = one_gaussian_scene([[0.04, 0.025, 2.0], [0.05, 0.045, 3.0]], [0.05, 0.05], [0.5, 0.5],
                            [[1, 0, 0], [0, 1, 0]])
    pr = O.project(sc, ID_Q, ID_T, cam)
    dx, dy = 8.5 - pr["uv"][0, 0], 8.5 - pr["uv"][0, 1]
    a_, b_, c_ = pr["conic"][0]
    sig = 0.5 * (a_ * dx * dx + c_ * dy * dy) + b_ * dx * dy
    assert sig > 0.01
    o = O.ALPHA_MIN * (1 + 1e-9) * np.exp(sig)
    sc.opacity_logit[0] = logit(o)
    pix = np.array([8 * 16 + 8])
    r = O.render(sc, ID_Q, ID_T, cam)
    assert r["amb"][8, 8] & 1 and not r["amb"][8, 8] & 8 and r["n_contrib"][8, 8] == 2
    alt = O.render_alternatives(sc, ID_Q, ID_T, cam, pix)
    assert alt["count"][0] == 2
    without = O.Scene(sc.mean[1:], sc.log_scale[1:], sc.quat[1:], sc.opacity_logit[1:], sc.rgb[1:])
    r1 = O.render(without, ID_Q, ID_T, cam)
    assert alt["n_contrib"][0, 1] == 1 and alt["last_gid"][0, 1] == 1
    np.testing.assert_array_equal(alt["rgb"][0, 1], r1["rgb"][:, 8, 8])
    assert alt["depth"][0, 1] == r1["depth"][8, 8]
    fl = np.zeros((16, 16), np.uint32)
    fl[8, 8] = alt["flip"][0, 1]
    rf = O.render(sc, ID_Q, ID_T, cam, flips=fl)
    np.testing.assert_array_equal(rf["rgb"][:, 8, 8], r1["rgb"][:, 8, 8])
    # the backward with the flip gives the first Gaussian no gradient from that pixel
    w = np.zeros((3, 16, 16))
    w[:, 8, 8] = 1.0
    gb = O.render_backward(sc, ID_Q, ID_T, cam, w, None, None, flips=fl)
    g1 = O.render_backward(without, ID_Q, ID_T, cam, w, None, None)
    assert np.all(gb["rgb"][0] == 0) and np.allclose(gb["rgb"][1], g1["rgb"][0], rtol=0, atol=1e-15)
    # stop decision: alphas 0.95 and 0.9 leave T = 0.005; a third entry with
    # 1 - alpha = 0.02 (1 + 1e-9) brings T (1 - alpha) to 1e-4 (1 + 1e-9)
    # (each Gaussian 0.2-0.3 px off the pixel centre, opacities set so that
    # alpha at the pixel is exactly these values)
    sc = one_gaussian_scene([[0.03, 0.028, 2.0], [0.04, 0.035, 2.5], [0.045, 0.04, 3.0]], [0.05, 0.05, 0.05],
                            [0.5, 0.5, 0.5], [[1, 0, 0], [0, 1, 0], [0, 0, 1]])
    pr = O.project(sc, ID_Q, ID_T, cam)
    for i, al in enumerate((0.95, 0.9, 1 - 0.02 * (1 + 1e-9))):
        dx, dy = 8.5 - pr["uv"][i, 0], 8.5 - pr["uv"][i, 1]
        a_, b_, c_ = pr["conic"][i]
        sig = 0.5 * (a_ * dx * dx + c_ * dy * dy) + b_ * dx * dy
        assert 1e-3 < sig < -np.log(al)
        sc.opacity_logit[i] = logit(al * np.exp(sig))
    r = O.render(sc, ID_Q, ID_T, cam)
    assert r["amb"][8, 8] & 1 and not r["amb"][8, 8] & 8 and r["n_contrib"][8, 8] == 3
    alt = O.render_alternatives(sc, ID_Q, ID_T, cam, pix)
    assert alt["count"][0] == 2 and alt["n_contrib"][0, 1] == 2 and alt["last_gid"][0, 1] == 1
    without = O.Scene(sc.mean[:2], sc.log_scale[:2], sc.quat[:2], sc.opacity_logit[:2], sc.rgb[:2])
    np.testing.assert_array_equal(alt["rgb"][0, 1], O.render(without, ID_Q, ID_T, cam)["rgb"][:, 8, 8])
