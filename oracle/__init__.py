"""FP64 CPU oracle of the Gaussian-SLAM differentiable rasterizer (arXiv 2312.10070).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import this package.  The product path
(``paper_2312_10070_gb300``) never imports it, and it imports nothing from the
product path.

The arithmetic lives in ``gsr_oracle.c`` (plain C, double precision, one
function per step of Sec. 3.1, 3.4 and 3.5 of the paper); this module only
compiles it with gcc and marshals numpy arrays through ctypes.  Inputs are
promoted to float64; outputs are float64 / int32 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsr_oracle.c")
_SO = os.path.join(_HERE, "libgsr_oracle.so")
_lib = None

# Fixed readings of points the paper leaves open.
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_STOP = 1e-4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Cam(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("z_near", ctypes.c_double), ("eps2d", ctypes.c_double),
                ("guard", ctypes.c_double), ("amb_rel", ctypes.c_double), ("guard_y", ctypes.c_double)]


@dataclass
class Camera:
    """Pinhole camera (x right, y down, z forward) and rasterizer settings."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    z_near: float = 0.2
    eps2d: float = 0.3
    guard: float = 1.3
    tile_w: int = 16
    tile_h: int = 16
    amb_rel: float = 0.0
    guard_y: float = 0.0

    def c(self) -> _Cam:
        return _Cam(self.width, self.height, self.tile_w, self.tile_h, self.fx, self.fy, self.cx,
                    self.cy, self.z_near, self.eps2d, self.guard, self.amb_rel, self.guard_y)

    def crop(self, tx0, ty0, tx1, ty1):
        """Camera of the tile-aligned window of tiles [tx0, tx1] x [ty0, ty1]:
        same projection, tiles and guard-band limits, fewer pixels."""
        x0, y0 = tx0 * self.tile_w, ty0 * self.tile_h
        w = min((tx1 + 1) * self.tile_w, self.width) - x0
        h = min((ty1 + 1) * self.tile_h, self.height) - y0
        gx = (self.guard * self.width) / w
        gy = ((self.guard_y or self.guard) * self.height) / h
        return Camera(w, h, self.fx, self.fy, self.cx - x0, self.cy - y0, self.z_near, self.eps2d, gx,
                      self.tile_w, self.tile_h, self.amb_rel, gy)

    @property
    def tiles(self):
        return ((self.width + self.tile_w - 1) // self.tile_w,
                (self.height + self.tile_h - 1) // self.tile_h)


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)


def _load():
    global _lib
    if _lib is None:
        # GSR_ORACLE_LIB names another build of gsr_oracle.c to load instead:
        # the mutation tests load copies with one planted mistake each
        lib = ctypes.CDLL(os.environ.get("GSR_ORACLE_LIB") or build())
        P = ctypes.c_void_p
        lib.orc_project.restype = ctypes.c_int64
        lib.orc_project.argtypes = [ctypes.c_int64] + [P] * 6 + [ctypes.POINTER(_Cam)] + [P] * 9
        lib.orc_bin.restype = ctypes.c_int64
        lib.orc_bin.argtypes = [ctypes.c_int64] + [P] * 6 + [ctypes.POINTER(_Cam), ctypes.c_int64, P, P, P]
        lib.orc_render.restype = ctypes.c_int
        lib.orc_render.argtypes = [ctypes.c_int64] + [P] * 7 + [ctypes.POINTER(_Cam)] + [P] * 9
        lib.orc_render_backward.restype = ctypes.c_int
        lib.orc_render_backward.argtypes = ([ctypes.c_int64] + [P] * 7 + [ctypes.POINTER(_Cam)]
                                            + [P] * 3 + [P] * 7 + [P])
        lib.orc_render_alternatives.restype = ctypes.c_int
        lib.orc_render_alternatives.argtypes = ([ctypes.c_int64] + [P] * 7 + [ctypes.POINTER(_Cam), P,
                                                ctypes.c_int64, ctypes.c_int, ctypes.c_int] + [P] * 8)
        lib.orc_project_backward.restype = ctypes.c_int
        lib.orc_project_backward.argtypes = ([ctypes.c_int64] + [P] * 6 + [ctypes.POINTER(_Cam)]
                                             + [P] * 7)
        lib.orc_loss_map.restype = ctypes.c_double
        lib.orc_loss_map.argtypes = ([ctypes.c_int, ctypes.c_int] + [P] * 4
                                     + [ctypes.c_double] * 3 + [P] * 4)
        lib.orc_loss_track.restype = ctypes.c_double
        lib.orc_loss_track.argtypes = ([ctypes.c_int, ctypes.c_int] + [P] * 5
                                       + [ctypes.c_double] * 3 + [P] * 4)
        lib.orc_lreg.restype = ctypes.c_double
        lib.orc_lreg.argtypes = [ctypes.c_int64, P, ctypes.c_double, P]
        lib.orc_adam.restype = None
        lib.orc_adam.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int64] + [ctypes.c_double] * 4
        lib.orc_pose_retract.restype = None
        lib.orc_pose_retract.argtypes = [P] * 5
        lib.orc_error_model.restype = None
        lib.orc_error_model.argtypes = [P]
        lib.orc_se3_left_jacobian.restype = None
        lib.orc_se3_left_jacobian.argtypes = [P] * 2
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_set_num_threads.restype = None
        lib.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Thread count of the oracle's OpenMP loops (for timing runs)."""
    _load().orc_set_num_threads(int(n))


class Scene:
    """FP64 copy of a Gaussian set: mean [n,3], log_scale [n,3], quat [n,4]
    (w,x,y,z), opacity_logit [n], rgb [n,3]."""

    def __init__(self, mean, log_scale, quat, opacity_logit, rgb):
        self.mean = _f64(mean).reshape(-1, 3)
        self.log_scale = _f64(log_scale).reshape(-1, 3)
        self.quat = _f64(quat).reshape(-1, 4)
        self.opacity_logit = _f64(opacity_logit).reshape(-1)
        self.rgb = _f64(rgb).reshape(-1, 3)
        self.n = self.mean.shape[0]

    @classmethod
    def from_dict(cls, d):
        return cls(d["mean"], d["log_scale"], d["quat"], d["opacity_logit"], d["rgb"])

    def copy(self):
        return Scene(self.mean.copy(), self.log_scale.copy(), self.quat.copy(),
                     self.opacity_logit.copy(), self.rgb.copy())

    def params(self):
        return self.mean, self.log_scale, self.quat, self.opacity_logit


def _pose(pose_q, pose_t):
    return _f64(pose_q).reshape(4), _f64(pose_t).reshape(3)


def project(scene: Scene, pose_q, pose_t, cam: Camera) -> dict:
    """Sec. 3.1 projection of every Gaussian (mean, EWA covariance, cull, tiles)."""
    lib = _load()
    n = scene.n
    q, t = _pose(pose_q, pose_t)
    out = dict(visible=np.zeros(n, np.int32), uv=np.zeros((n, 2)), depth=np.zeros(n),
               cov2d=np.zeros((n, 3)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
               radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
               amb=np.zeros(n, np.int32))
    c = cam.c()
    total = lib.orc_project(n, *[_p(a) for a in scene.params()], _p(q), _p(t), ctypes.byref(c),
                            *[_p(out[k]) for k in ("visible", "uv", "depth", "cov2d", "conic",
                                                   "opacity", "radius", "rect", "amb")])
    out["n_instances"] = int(total)
    return out


def bin_tiles(scene: Scene, pose_q, pose_t, cam: Camera) -> dict:
    """Per-tile Gaussian lists ordered by (float32 depth, index)."""
    lib = _load()
    q, t = _pose(pose_q, pose_t)
    total = project(scene, pose_q, pose_t, cam)["n_instances"]
    tx, ty = cam.tiles
    start = np.zeros(tx * ty + 1, np.int64)
    gid = np.zeros(max(total, 1), np.int32)
    tie = np.zeros(max(total, 1), np.int32)
    c = cam.c()
    got = lib.orc_bin(scene.n, *[_p(a) for a in scene.params()], _p(q), _p(t), ctypes.byref(c),
                      max(total, 1), _p(start), _p(gid), _p(tie))
    assert got == total
    return dict(start=start, gid=gid[:total], near_tie=tie[:total].astype(bool))


def render(scene: Scene, pose_q, pose_t, cam: Camera, flips=None) -> dict:
    """Forward render: rgb [3,H,W], depth, alpha, final_T, last_idx, n_contrib,
    amb (per-pixel ambiguity flags: bit 0 a marginal decision, bit 1 a marginal
    alpha cap, bit 3 a marginal decision other than a skip or stop) and n_eval
    (list entries visited).  flips (uint32 [H,W], optional): per pixel, the
    branches taken at its marginal skip / stop decisions."""
    lib = _load()
    q, t = _pose(pose_q, pose_t)
    H, W = cam.height, cam.width
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), alpha=np.zeros((H, W)),
               final_T=np.zeros((H, W)), last_idx=np.zeros((H, W), np.int32),
               n_contrib=np.zeros((H, W), np.int32), amb=np.zeros((H, W), np.int32))
    ne = np.zeros(1, np.int64)
    c = cam.c()
    fl = None if flips is None else np.ascontiguousarray(np.asarray(flips, np.uint32).reshape(H, W))
    lib.orc_render(scene.n, *[_p(a) for a in scene.params()], _p(scene.rgb), _p(q), _p(t),
                   ctypes.byref(c), *[_p(out[k]) for k in ("rgb", "depth", "alpha", "final_T",
                                                           "last_idx", "n_contrib", "amb")], _p(ne), _p(fl))
    out["n_eval"] = int(ne[0])
    return out


def render_backward(scene: Scene, pose_q, pose_t, cam: Camera, d_rgb=None, d_depth=None,
                    d_alpha=None, flips=None) -> dict:
    """Exact gradient of sum(d_rgb*rgb + d_depth*depth + d_alpha*alpha) with respect
    to every Gaussian parameter and the pose twist (rho, phi) of a left perturbation.
    flips (uint32 [H,W], optional): per pixel, the branches taken at its marginal
    skip / stop decisions (the flip mask of one of render_alternatives' results)."""
    lib = _load()
    q, t = _pose(pose_q, pose_t)
    n = scene.n
    d_rgb = None if d_rgb is None else _f64(d_rgb)
    d_depth = None if d_depth is None else _f64(d_depth)
    d_alpha = None if d_alpha is None else _f64(d_alpha)
    g = dict(mean=np.zeros((n, 3)), log_scale=np.zeros((n, 3)), quat=np.zeros((n, 4)),
             opacity_logit=np.zeros(n), rgb=np.zeros((n, 3)), pose=np.zeros(6),
             g2d=np.zeros((n, 10)))
    c = cam.c()
    fl = None if flips is None else np.ascontiguousarray(np.asarray(flips, np.uint32).reshape(cam.height, cam.width))
    lib.orc_render_backward(n, *[_p(a) for a in scene.params()], _p(scene.rgb), _p(q), _p(t),
                            ctypes.byref(c), _p(d_rgb), _p(d_depth), _p(d_alpha),
                            *[_p(g[k]) for k in ("mean", "log_scale", "quat", "opacity_logit",
                                                 "rgb", "pose", "g2d")], _p(fl))
    return g


def render_alternatives(scene: Scene, pose_q, pose_t, cam: Camera, pixels, max_bits=4, kmax=16) -> dict:
    """Every result a float32 implementation may produce at the given pixel
    indices (row-major): per pixel up to kmax alternatives that take either
    branch of its marginal skip / stop decisions.  Arrays [npix, kmax]:
    rgb [npix, kmax, 3], depth, final_T, last_gid, n_contrib, flip; count
    [npix]; amb [npix]."""
    lib = _load()
    q, t = _pose(pose_q, pose_t)
    pix = np.ascontiguousarray(np.asarray(pixels, np.int64).reshape(-1))
    m = pix.size
    out = dict(rgb=np.zeros((m, kmax, 3)), depth=np.zeros((m, kmax)), final_T=np.zeros((m, kmax)),
               last_gid=np.full((m, kmax), -2, np.int32), n_contrib=np.zeros((m, kmax), np.int32),
               flip=np.zeros((m, kmax), np.uint32), count=np.zeros(m, np.int32), amb=np.zeros(m, np.int32))
    if m == 0:
        return out
    c = cam.c()
    lib.orc_render_alternatives(scene.n, *[_p(a) for a in scene.params()], _p(scene.rgb), _p(q), _p(t),
                                ctypes.byref(c), _p(pix), m, int(max_bits), int(kmax),
                                *[_p(out[k]) for k in ("rgb", "depth", "final_T", "last_gid", "n_contrib", "flip",
                                                       "count", "amb")])
    return out


def project_backward(scene: Scene, pose_q, pose_t, cam: Camera, g2d) -> dict:
    """Chain given image-space gradients [n,10] = (u, v, conic a, b, c, opacity,
    r, g, b, depth) back to the parameters and the pose twist."""
    lib = _load()
    q, t = _pose(pose_q, pose_t)
    n = scene.n
    g2d = _f64(g2d).reshape(n, 10)
    g = dict(mean=np.zeros((n, 3)), log_scale=np.zeros((n, 3)), quat=np.zeros((n, 4)),
             opacity_logit=np.zeros(n), rgb=np.zeros((n, 3)), pose=np.zeros(6))
    c = cam.c()
    lib.orc_project_backward(n, *[_p(a) for a in scene.params()], _p(q), _p(t), ctypes.byref(c),
                             _p(g2d), *[_p(g[k]) for k in ("mean", "log_scale", "quat",
                                                           "opacity_logit", "rgb", "pose")])
    return g


def loss_map(rgb, depth, rgb_t, depth_t, lam=0.2, w_color=1.0, w_depth=1.0) -> dict:
    """Mapping loss of Eq. (joint_loss) without L_reg; returns loss, gradients,
    SSIM map and parts (l1_color, ssim, l1_depth, n_valid)."""
    lib = _load()
    rgb, depth, rgb_t, depth_t = _f64(rgb), _f64(depth), _f64(rgb_t), _f64(depth_t)
    _, H, W = rgb.shape
    d_rgb = np.zeros_like(rgb)
    d_depth = np.zeros_like(depth)
    smap = np.zeros_like(rgb)
    parts = np.zeros(4)
    L = lib.orc_loss_map(H, W, _p(rgb), _p(depth), _p(rgb_t), _p(depth_t), lam, w_color, w_depth,
                         _p(d_rgb), _p(d_depth), _p(smap), _p(parts))
    return dict(loss=float(L), d_rgb=d_rgb, d_depth=d_depth, ssim_map=smap,
                l1_color=parts[0], ssim=parts[1], l1_depth=parts[2], n_valid=int(parts[3]))


def loss_track(rgb, depth, alpha, rgb_t, depth_t, lam_c=0.5, k_med=50.0, apow=3.0) -> dict:
    """Tracking loss of Sec. 3.5 with the alpha^3 and inlier masks."""
    lib = _load()
    rgb, depth, alpha, rgb_t, depth_t = (_f64(a) for a in (rgb, depth, alpha, rgb_t, depth_t))
    _, H, W = rgb.shape
    d_rgb = np.zeros_like(rgb)
    d_depth = np.zeros_like(depth)
    inl = np.zeros((H, W), np.int32)
    med = np.zeros(1)
    L = lib.orc_loss_track(H, W, _p(rgb), _p(depth), _p(alpha), _p(rgb_t), _p(depth_t), lam_c,
                           k_med, apow, _p(d_rgb), _p(d_depth), _p(inl), _p(med))
    return dict(loss=float(L), d_rgb=d_rgb, d_depth=d_depth, inlier=inl.astype(bool),
                median=float(med[0]))


def lreg(log_scale, w=1.0):
    """Isotropic regulariser L_reg and w * dL_reg/dlog_scale."""
    lib = _load()
    ls = _f64(log_scale).reshape(-1, 3)
    g = np.zeros_like(ls)
    L = lib.orc_lreg(ls.shape[0], _p(ls), w, _p(g))
    return float(L), g


def adam(param, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-15):
    """In-place Adam step on float64 arrays (step is 1-based)."""
    lib = _load()
    for a in (param, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib.orc_adam(param.size, _p(param), _p(grad), _p(m), _p(v), step, lr, b1, b2, eps)


def pose_retract(pose_q, pose_t, xi):
    """T <- exp(xi^) T for a world-to-camera pose (q, t), xi = (rho, phi)."""
    lib = _load()
    q, t = _pose(pose_q, pose_t)
    xi = _f64(xi).reshape(6)
    qo, to = np.zeros(4), np.zeros(3)
    lib.orc_pose_retract(_p(q), _p(t), _p(xi), _p(qo), _p(to))
    return qo, to


def se3_left_jacobian(xi):
    """SE(3) left Jacobian J_l(xi) (6x6, xi = (rho, phi)): to first order
    exp((xi + e)^) = exp((J_l e)^) exp(xi^)."""
    lib = _load()
    xi = _f64(xi).reshape(6)
    J = np.zeros((6, 6))
    lib.orc_se3_left_jacobian(_p(xi), _p(J))
    return J


def twist_gradient(xi, pose_grad):
    """dL/dxi of a loss of T(xi) = exp(xi^) T, from the left-perturbation pose
    gradient at T(xi): J_l(xi)^T pose_grad."""
    return se3_left_jacobian(xi).T @ _f64(pose_grad).reshape(6)


def error_model() -> dict:
    """The float32 error bounds behind the ambiguity flags (see gsr_oracle.c):
    unit roundoff u; compensated transform bound; u, v ratio and rounding
    factors; conic quadratic-form factor (x u sqrt(kappa)); sigmoid factor;
    sigma evaluation factor; relative error of the exponential."""
    c = np.zeros(8)
    _load().orc_error_model(_p(c))
    return dict(zip(("u", "df", "ratio", "round", "conic", "opacity", "sigma", "exp"), c.tolist()))
