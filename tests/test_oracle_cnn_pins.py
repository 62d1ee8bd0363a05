"""Pins of the FP64 warm-start CNN oracle (CPU only)."""
import numpy as np
from scipy import signal

from oracle import cnn as C


def he_params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in C.param_shapes():
        if name.endswith(".b"):
            p[name] = rng.normal(0, 0.05, shp)
        else:
            fan_in = int(np.prod(shp[1:]))
            p[name] = rng.normal(0, scale * np.sqrt(2.0 / fan_in), shp)
    return p


def test_conv_matches_scipy_correlation():
    """One 3x3 stride-2 zero-padded convolution: im2col + matmul against
    scipy.signal.correlate per (output, input) channel pair."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 13, 18, 5))
    w = rng.standard_normal((4, 3, 3, 5))
    cols, (B, Ho, Wo) = C._im2col(x)
    got = (cols @ w.reshape(4, -1).T).reshape(B, Ho, Wo, 4)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    for b in range(2):
        for co in range(4):
            ref = sum(signal.correlate(xp[b, :, :, ci], w[co, :, :, ci], mode="valid") for ci in range(5))
            np.testing.assert_allclose(got[b, :, :, co], ref[::2, ::2], rtol=1e-12, atol=1e-12)


def test_col2im_is_the_adjoint_of_im2col():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 15, 20, 3))
    cols, _ = C._im2col(x)
    c = rng.standard_normal(cols.shape)
    np.testing.assert_allclose(np.sum(cols * c), np.sum(x * C._col2im(c, x.shape)), rtol=1e-12)


def test_network_shapes_and_flatten_roundtrip():
    p = he_params()
    assert C.n_params() == sum(v.size for v in p.values())
    np.testing.assert_array_equal(C.flatten(C.unflatten(C.flatten(p))), C.flatten(p))
    x = np.random.default_rng(3).standard_normal((1, C.IN_H, C.IN_W, C.IN_C))
    out, _ = C.forward(p, x)
    assert out.shape == (1, 6)


def test_backward_matches_central_fd():
    rng = np.random.default_rng(4)
    p = he_params(5)
    x = rng.standard_normal((2, C.IN_H, C.IN_W, C.IN_C))
    d_out = rng.standard_normal((2, 6))
    out, cache = C.forward(p, x)
    g = C.backward(p, cache, d_out)
    h = 1e-6
    names = [n for n, _ in C.param_shapes()]
    for name in names:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, 3, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = np.sum(d_out * C.forward(p, x)[0])
            flat[idx] = old - h
            lm = np.sum(d_out * C.forward(p, x)[0])
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            ga = g[name].reshape(-1)[idx]
            assert abs(ga - fd) <= 1e-5 * (abs(fd) + 1e-3), (name, idx, ga, fd)


def test_loss_gradient_and_box_downsample():
    rng = np.random.default_rng(6)
    out, tgt, w = rng.standard_normal((4, 6)), rng.standard_normal((4, 6)), rng.random(6)
    L, d = C.loss(out, tgt, w)
    np.testing.assert_allclose(L, np.mean(np.sum(w * (out - tgt) ** 2, axis=1)))
    h = 1e-6
    o2 = out.copy()
    o2[1, 3] += h
    np.testing.assert_allclose((C.loss(o2, tgt, w)[0] - L) / h, d[1, 3], rtol=1e-4)
    # integer factors: box average = reshape-mean; invalid depth is excluded
    rgb = rng.random((3, 12, 16))
    dep = rng.uniform(1, 2, (12, 16))
    dep[0, 0] = 0.0
    r, dd = C.box_downsample(rgb, dep, 3, 4)
    np.testing.assert_allclose(r, rgb.reshape(3, 3, 4, 4, 4).mean(axis=(2, 4)))
    assert abs(dd[0, 0] - dep[0:4, 0:4][dep[0:4, 0:4] > 0].mean()) < 1e-12


def test_storage_rounding_hooks():
    """rnd = identity changes nothing; rnd = 0 leaves only the output bias and
    zeroes every gradient (it is applied to d_out and every stored activation)."""
    p = he_params(9)
    x = np.random.default_rng(10).standard_normal((2, C.IN_H, C.IN_W, C.IN_C))
    d_out = np.random.default_rng(11).standard_normal((2, 6))
    o0, c0 = C.forward(p, x)
    o1, c1 = C.forward(p, x, rnd=lambda a: a)
    np.testing.assert_array_equal(o0, o1)
    g0, g1 = C.backward(p, c0, d_out), C.backward(p, c1, d_out, rnd=lambda a: a)
    for k in g0:
        np.testing.assert_array_equal(g0[k], g1[k])
    zero = lambda a: np.zeros_like(a)
    oz, cz = C.forward(p, x, rnd=zero)
    np.testing.assert_array_equal(oz, np.broadcast_to(p["fc1.b"], (2, 6)))
    gz = C.backward(p, cz, d_out, rnd=zero)
    assert all(not np.any(v) for v in gz.values())


def test_residual_input_worked_example():
    """A render and a frame built so every channel is known: rendered RGB and
    depth / scale, frame minus render, depth residual / scale where both
    depths are valid and 0 where either is not; a doubled scale halves the
    depth channels."""
    H, W = 4, 5
    rgb_r = np.full((3, H, W), 0.25)
    rgb_r[1] = 0.5
    rgb_i = rgb_r + np.array([0.125, -0.25, 0.0])[:, None, None]
    d_r = np.full((H, W), 2.0)
    d_i = np.full((H, W), 2.5)
    d_r[0, 0] = 0.0           # render invalid
    d_i[1, 2] = 0.0           # frame invalid
    x = C.residual_input(rgb_r, d_r, rgb_i, d_i, depth_scale=5.0)
    assert x.shape == (H, W, 8)
    np.testing.assert_array_equal(x[..., 0:3], np.moveaxis(rgb_r, 0, -1))
    np.testing.assert_array_equal(x[..., 3], d_r / 5.0)
    np.testing.assert_allclose(x[..., 4:7], np.broadcast_to([0.125, -0.25, 0.0], (H, W, 3)))
    expect = np.full((H, W), 0.1)
    expect[0, 0] = expect[1, 2] = 0.0
    np.testing.assert_allclose(x[..., 7], expect, atol=1e-15)
    y = C.residual_input(rgb_r, d_r, rgb_i, d_i, depth_scale=10.0)
    np.testing.assert_allclose(y[..., [3, 7]], x[..., [3, 7]] / 2, atol=1e-15)
    z = C.residual_input(rgb_r, d_r, rgb_r, d_r)      # frame == render
    assert np.all(z[..., 4:] == 0)
