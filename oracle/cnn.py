"""FP64 CPU oracle of the tracking warm-start CNN.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The network has no
counterpart in the paper: it predicts the 6-DoF correction of a tracking
initialisation from the rendered-versus-input RGB-D residual.  This module
computes it the plain way, in float64 with numpy: zero-padded im2col and a
matrix product per 3x3 stride-2 convolution, then two dense layers, and the
exact backward of each step by the chain rule.

Layouts (shared with the CUDA path's import/export of weights):
    input        x  [B, 120, 160, 8]   (NHWC)
    conv l       W  [C_out, 3, 3, C_in],  b [C_out]; ReLU after each conv
    dense 1      W  [256, 1536] (input flattened in (y, x, c) order), b [256], ReLU
    dense 2      W  [6, 256], b [6]
    output       [B, 6] = (rho, phi) twist
"""
from __future__ import annotations

import numpy as np

CONV = ((8, 32), (32, 64), (64, 128), (128, 128), (128, 256), (256, 256))
DENSE = ((1536, 256), (256, 6))
IN_H, IN_W, IN_C = 120, 160, 8


def param_shapes():
    shapes = []
    for ci, co in CONV:
        shapes += [(f"conv{len(shapes) // 2}.w", (co, 3, 3, ci)), (f"conv{len(shapes) // 2}.b", (co,))]
    for k, (ni, no) in enumerate(DENSE):
        shapes += [(f"fc{k}.w", (no, ni)), (f"fc{k}.b", (no,))]
    return shapes


def unflatten(flat):
    """Flat float vector (the order of param_shapes) -> dict of arrays."""
    out, o = {}, 0
    for name, shp in param_shapes():
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def flatten(params):
    return np.concatenate([params[name].reshape(-1) for name, _ in param_shapes()])


def n_params():
    return sum(int(np.prod(s)) for _, s in param_shapes())


def _im2col(x):
    """x [B, H, W, C] -> columns [B*Ho*Wo, 9*C] in (ky, kx, c) order, zero padding 1, stride 2."""
    B, H, W, C = x.shape
    Ho, Wo = (H - 1) // 2 + 1, (W - 1) // 2 + 1
    xp = np.zeros((B, H + 2, W + 2, C))
    xp[:, 1:H + 1, 1:W + 1, :] = x
    cols = np.empty((B, Ho, Wo, 3, 3, C))
    for ky in range(3):
        for kx in range(3):
            cols[:, :, :, ky, kx, :] = xp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :]
    return cols.reshape(B * Ho * Wo, 9 * C), (B, Ho, Wo)


def _col2im(dcols, shape_in):
    """Adjoint of _im2col: scatter-add columns back to [B, H, W, C]."""
    B, H, W, C = shape_in
    Ho, Wo = (H - 1) // 2 + 1, (W - 1) // 2 + 1
    d = dcols.reshape(B, Ho, Wo, 3, 3, C)
    dxp = np.zeros((B, H + 2, W + 2, C))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + 2 * Ho:2, kx:kx + 2 * Wo:2, :] += d[:, :, :, ky, kx, :]
    return dxp[:, 1:H + 1, 1:W + 1, :]


def _identity(a):
    return a


def forward(params, x, rnd=None):
    """Returns the output [B, 6] and a cache for backward.

    rnd (optional) is applied to every stored activation (each ReLU output):
    a network that keeps its activations in a narrower type than it
    accumulates in is this function with rnd = rounding to that type."""
    rnd = rnd or _identity
    a = np.asarray(x, np.float64)
    cache = []
    for li in range(len(CONV)):
        w, b = params[f"conv{li}.w"], params[f"conv{li}.b"]
        cols, (B, Ho, Wo) = _im2col(a)
        z = cols @ w.reshape(w.shape[0], -1).T + b
        y = rnd(np.maximum(z, 0.0)).reshape(B, Ho, Wo, -1)
        cache.append((a.shape, cols, z))
        a = y
    B = a.shape[0]
    h = a.reshape(B, -1)
    z1 = h @ params["fc0.w"].T + params["fc0.b"]
    h1 = rnd(np.maximum(z1, 0.0))
    out = h1 @ params["fc1.w"].T + params["fc1.b"]
    return out, (cache, h, z1, h1)


def backward(params, cache_all, d_out, rnd=None):
    """Gradients of sum(d_out * out) with respect to every parameter.

    rnd (optional) is applied to every stored upstream gradient: d_out and
    each gradient after a ReLU mask (the GEMM operands of the backward)."""
    rnd = rnd or _identity
    cache, h, z1, h1 = cache_all
    d_out = rnd(np.asarray(d_out, np.float64))
    g = {}
    g["fc1.w"] = d_out.T @ h1
    g["fc1.b"] = d_out.sum(0)
    dh1 = d_out @ params["fc1.w"]
    dz1 = rnd(dh1 * (z1 > 0))
    g["fc0.w"] = dz1.T @ h
    g["fc0.b"] = dz1.sum(0)
    dh = dz1 @ params["fc0.w"]
    da = dh.reshape(h.shape[0], 2, 3, -1)
    for li in reversed(range(len(CONV))):
        shape_in, cols, z = cache[li]
        w = params[f"conv{li}.w"]
        dz = rnd(da.reshape(z.shape) * (z > 0))
        g[f"conv{li}.w"] = (dz.T @ cols).reshape(w.shape)
        g[f"conv{li}.b"] = dz.sum(0)
        if li > 0:
            dcols = dz @ w.reshape(w.shape[0], -1)
            da = _col2im(dcols, shape_in)
    return g


def loss(out, target, weights):
    """L = (1/B) sum_b sum_c w_c (out - target)^2 and dL/dout."""
    out = np.asarray(out, np.float64)
    r = out - np.asarray(target, np.float64)
    w = np.asarray(weights, np.float64)
    B = out.shape[0]
    return float(np.sum(w * r * r) / B), 2.0 * w * r / B


def residual_input(rgb_r, depth_r, rgb_i, depth_i, depth_scale=5.0):
    """Network input [H, W, 8] from a render (rgb [3,H,W], depth [H,W]) and a
    frame: (rendered rgb, rendered depth / scale, input - rendered rgb,
    (input - rendered depth) / scale where both depths are valid, else 0)."""
    rgb_r, rgb_i = np.asarray(rgb_r, np.float64), np.asarray(rgb_i, np.float64)
    d_r, d_i = np.asarray(depth_r, np.float64), np.asarray(depth_i, np.float64)
    valid = (d_r > 0) & (d_i > 0)
    ch = [rgb_r[0], rgb_r[1], rgb_r[2], d_r / depth_scale, rgb_i[0] - rgb_r[0], rgb_i[1] - rgb_r[1],
          rgb_i[2] - rgb_r[2], np.where(valid, (d_i - d_r) / depth_scale, 0.0)]
    return np.stack(ch, axis=-1)


def box_downsample(rgb, depth, H, W):
    """Box average of a [3, h, w] / [h, w] frame to H x W: output pixel (i, j)
    averages the input pixels whose index lies in [floor(i h/H), floor((i+1) h/H))
    (same for columns); depth averages only valid (> 0) pixels, 0 if none."""
    rgb, depth = np.asarray(rgb, np.float64), np.asarray(depth, np.float64)
    h, w = depth.shape
    out_rgb, out_d = np.zeros((3, H, W)), np.zeros((H, W))
    for i in range(H):
        y0, y1 = (i * h) // H, ((i + 1) * h) // H
        for j in range(W):
            x0, x1 = (j * w) // W, ((j + 1) * w) // W
            out_rgb[:, i, j] = rgb[:, y0:y1, x0:x1].mean(axis=(1, 2))
            dv = depth[y0:y1, x0:x1]
            m = dv > 0
            out_d[i, j] = dv[m].mean() if m.any() else 0.0
    return out_rgb, out_d
