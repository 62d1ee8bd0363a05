"""Python binding of the C ABI (include/gsr.h) over PyTorch tensors.

Functions carry the names of the C entry points (without the ``gsr_``
prefix).  PyTorch supplies device memory and the current CUDA stream; all
computation happens in libgsr.so.  Tensors must be float32 (int32 where
stated), contiguous and on the context's CUDA device.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """Owns a gsr_ctx (scratch, tile lists, graphs) on the current device."""

    def __init__(self, tile=(16, 16), batch=256, memory_saving=False, fixed_capacity=False, max_gaussians=0,
                 max_instances=0, pixels_per_thread=0, ppt_fwd=0, ppt_bwd=0, rect_lists=False):
        if not torch.cuda.is_available():
            raise RuntimeError("the GB300 rasterizer needs a CUDA device; there is no CPU fallback")
        self.lib = L.load()
        o = L.Options()
        self.lib.gsr_default_options(ctypes.byref(o))
        o.tile_w, o.tile_h = tile
        o.batch = batch
        o.memory_saving = int(memory_saving)
        o.fixed_capacity = int(fixed_capacity)
        o.max_gaussians = max_gaussians
        o.max_instances = max_instances
        o.ppt_fwd = ppt_fwd or pixels_per_thread
        o.ppt_bwd = ppt_bwd or pixels_per_thread
        o.rect_lists = int(rect_lists)
        self.options = o
        h = ctypes.c_void_p()
        L.check(self.lib.gsr_create(ctypes.byref(h), ctypes.byref(o)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gsr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status):
        L.check(status, self.handle)

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.gsr_kernel_launches(self.handle))


PHASES = ("bin", "blend_fwd", "loss", "blend_bwd", "project_bwd", "adam")


def profile_enable(ctx: Context, on: bool = True):
    ctx.check(ctx.lib.gsr_profile_enable(ctx.handle, int(on)))


def profile_read(ctx: Context) -> dict:
    """Elapsed ms of each phase in its latest execution (gsr_profile_read)."""
    ms = (ctypes.c_float * len(PHASES))()
    ctx.check(ctx.lib.gsr_profile_read(ctx.handle, ms, len(PHASES), _stream()))
    return {k: float(v) for k, v in zip(PHASES, ms)}


def make_camera(width, height, fx, fy, cx, cy, z_near=0.2, eps2d=0.3) -> L.Camera:
    return L.Camera(int(width), int(height), float(fx), float(fy), float(cx), float(cy), float(z_near), float(eps2d))


def camera_from_spec(spec, **kw) -> L.Camera:
    return make_camera(spec.width, spec.height, spec.fx, spec.fy, spec.cx, spec.cy, **kw)


def make_pose(q, t) -> L.Pose:
    q = [float(x) for x in np.asarray(q, np.float64).reshape(4)]
    t = [float(x) for x in np.asarray(t, np.float64).reshape(3)]
    return L.Pose((ctypes.c_float * 4)(*q), (ctypes.c_float * 3)(*t))


@dataclass
class GaussianParams:
    """Gaussian parameters (SoA, float32, CUDA)."""
    mean: torch.Tensor
    log_scale: torch.Tensor
    quat: torch.Tensor
    opacity_logit: torch.Tensor
    rgb: torch.Tensor

    NAMES = ("mean", "log_scale", "quat", "opacity_logit", "rgb")
    ROW_SHAPES = ((3,), (3,), (4,), (), (3,))

    def check(self):
        """Raises ValueError unless every array is float32 with the layout
        gsr_gaussians documents ([n,3], [n,3], [n,4], [n], [n,3]): the C ABI
        reads them as such and cannot tell."""
        n = self.n
        for k, row in zip(self.NAMES, self.ROW_SHAPES):
            t = getattr(self, k)
            if t.dtype != torch.float32 or tuple(t.shape) != (n,) + row:
                raise ValueError(f"{k}: expected float32 {[n, *row]}, got {t.dtype} {list(t.shape)}")
        return self

    @classmethod
    def from_numpy(cls, d: dict, device="cuda"):
        return cls(*[torch.as_tensor(np.ascontiguousarray(d[k]), dtype=torch.float32, device=device)
                     for k in cls.NAMES])

    @property
    def n(self) -> int:
        return int(self.mean.shape[0])

    def tensors(self):
        return [getattr(self, k) for k in self.NAMES]

    def clone(self):
        return GaussianParams(*[t.clone() for t in self.tensors()])

    def zeros_like(self):
        return GaussianParams(*[torch.zeros_like(t) for t in self.tensors()])

    def c(self) -> L.Gaussians:
        return L.Gaussians(*[_ptr(t) for t in self.check().tensors()], self.n)

    def c_mut(self) -> L.GaussiansMut:
        return L.GaussiansMut(*[_ptr(t) for t in self.check().tensors()], self.n)

    def c_grads(self) -> L.GaussianGrads:
        return L.GaussianGrads(*[_ptr(t) for t in self.check().tensors()])


def render_forward(ctx: Context, g: GaussianParams, cam: L.Camera, pose: L.Pose, want_n_contrib=False,
                   xi: torch.Tensor = None) -> dict:
    """gsr_render_forward: rgb [3,H,W], depth, alpha, final_T, last_idx (int32).
    With a device twist xi (float32 [6]): gsr_render_forward_xi, the render at
    exp(xi^) T formed on the device."""
    H, W = cam.height, cam.width
    dev = g.mean.device
    out = dict(rgb=torch.empty((3, H, W), device=dev), depth=torch.empty((H, W), device=dev),
               alpha=torch.empty((H, W), device=dev), final_T=torch.empty((H, W), device=dev),
               last_idx=torch.empty((H, W), dtype=torch.int32, device=dev),
               n_contrib=torch.empty((H, W), dtype=torch.int32, device=dev) if want_n_contrib else None)
    ro = L.RenderOut(*[_ptr(out[k]) for k in ("rgb", "depth", "alpha", "final_T", "last_idx", "n_contrib")])
    if xi is None:
        ctx.check(ctx.lib.gsr_render_forward(ctx.handle, ctypes.byref(g.c()), ctypes.byref(cam), ctypes.byref(pose),
                                             ctypes.byref(ro), _stream()))
    else:
        ctx.check(ctx.lib.gsr_render_forward_xi(ctx.handle, ctypes.byref(g.c()), ctypes.byref(cam),
                                                ctypes.byref(pose), _twist(xi), ctypes.byref(ro), _stream()))
    return out


def _twist(xi):
    if xi.dtype != torch.float32 or xi.numel() != 6:
        raise ValueError("the twist must be a float32 tensor of 6 elements (rho, phi)")
    return _ptr(xi)


def frame_stats(ctx: Context) -> dict:
    st = L.FrameStats()
    ctx.check(ctx.lib.gsr_frame_stats_get(ctx.handle, ctypes.byref(st), _stream()))
    return dict(n_visible=st.n_visible, n_instances=st.n_instances, n_tiles=st.n_tiles,
                capacity_instances=st.capacity_instances)


def check_wait_timeout(ctx: Context, polls: int = 4096):
    """gsr_check_wait_timeout: a bounded device wait on a word nothing
    publishes; raises GsrError(GSR_ERR_TIMEOUT) once it has expired."""
    ctx.check(ctx.lib.gsr_check_wait_timeout(ctx.handle, int(polls), _stream()))


def tile_lists(ctx: Context, n_tiles: int, n_gaussians: int, capacity: int = None):
    """gsr_tile_lists_get: (ranges uint32 [n_tiles, 2], gids int32 [I], depth bits uint32 [n])."""
    st = frame_stats(ctx)
    cap = int(st["n_instances"]) if capacity is None else capacity
    ranges = np.zeros((n_tiles, 2), np.uint32)
    gids = np.zeros(max(cap, 1), np.int32)
    dbits = np.zeros(max(n_gaussians, 1), np.uint32)
    ni = ctypes.c_int64()
    ctx.check(ctx.lib.gsr_tile_lists_get(ctx.handle, ranges.ctypes.data_as(ctypes.c_void_p),
                                         gids.ctypes.data_as(ctypes.c_void_p), cap,
                                         dbits.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ni), _stream()))
    return ranges, gids[:ni.value], dbits[:n_gaussians]


def records(ctx: Context, n: int):
    """gsr_records_get: (rec float32 [n, 12], visible bool [n]) of the last
    forward: u, v, conic (a, b, c), opacity, depth, ... per Gaussian."""
    rec = np.zeros((max(n, 1), 12), np.float32)
    vis = np.zeros(max(n, 1), np.uint32)
    ctx.check(ctx.lib.gsr_records_get(ctx.handle, rec.ctypes.data_as(ctypes.c_void_p),
                                      vis.ctypes.data_as(ctypes.c_void_p), int(n), _stream()))
    return rec[:n], vis[:n].astype(bool)


def render_backward(ctx: Context, g: GaussianParams, cam: L.Camera, pose: L.Pose, saved: dict, d_rgb=None,
                    d_depth=None, d_alpha=None, want_params=True, want_pose=True, out: GaussianParams = None,
                    xi: torch.Tensor = None):
    """gsr_render_backward: returns (GaussianParams of gradients or None, pose6 tensor or None).
    With a device twist xi: gsr_render_backward_xi, and pose6 is dL/dxi."""
    grads = None
    if want_params:
        grads = out if out is not None else g.zeros_like()
    pose6 = torch.empty(6, device=g.mean.device) if want_pose else None
    ro = L.RenderOut(None, None, None, _ptr(saved["final_T"]), _ptr(saved["last_idx"]), None)
    gg = grads.c_grads() if grads is not None else None
    if xi is None:
        ctx.check(ctx.lib.gsr_render_backward(ctx.handle, ctypes.byref(g.c()), ctypes.byref(cam), ctypes.byref(pose),
                                              ctypes.byref(ro), _ptr(d_rgb), _ptr(d_depth), _ptr(d_alpha),
                                              ctypes.byref(gg) if gg is not None else None, _ptr(pose6), _stream()))
    else:
        ctx.check(ctx.lib.gsr_render_backward_xi(ctx.handle, ctypes.byref(g.c()), ctypes.byref(cam),
                                                 ctypes.byref(pose), _twist(xi), ctypes.byref(ro), _ptr(d_rgb),
                                                 _ptr(d_depth), _ptr(d_alpha),
                                                 ctypes.byref(gg) if gg is not None else None, _ptr(pose6),
                                                 _stream()))
    return grads, pose6


def loss_map(ctx: Context, rgb, depth, rgb_t, depth_t, lambda_ssim=0.2, w_color=1.0, w_depth=1.0, scale=1.0):
    """gsr_loss_map: returns (loss [1] device tensor, d_rgb, d_depth)."""
    _, H, W = rgb.shape
    d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
    loss = torch.empty(1, device=rgb.device)
    ctx.check(ctx.lib.gsr_loss_map(ctx.handle, W, H, _ptr(rgb), _ptr(depth), _ptr(rgb_t), _ptr(depth_t),
                                   lambda_ssim, w_color, w_depth, scale, _ptr(d_rgb), _ptr(d_depth), _ptr(loss),
                                   _stream()))
    return loss, d_rgb, d_depth


def loss_track(ctx: Context, rgb, depth, alpha, rgb_t, depth_t, lambda_c=0.5, k_median=50.0, alpha_pow=3.0):
    """gsr_loss_track: returns (loss [1], median [1], d_rgb, d_depth)."""
    _, H, W = rgb.shape
    d_rgb, d_depth = torch.empty_like(rgb), torch.empty_like(depth)
    loss = torch.empty(1, device=rgb.device)
    med = torch.empty(1, device=rgb.device)
    ctx.check(ctx.lib.gsr_loss_track(ctx.handle, W, H, _ptr(rgb), _ptr(depth), _ptr(alpha), _ptr(rgb_t),
                                     _ptr(depth_t), lambda_c, k_median, alpha_pow, _ptr(d_rgb), _ptr(d_depth),
                                     _ptr(loss), _ptr(med), _stream()))
    return loss, med, d_rgb, d_depth


@dataclass
class AdamConfig:
    """Learning rates per parameter group (the paper names none; these are
    configurable defaults), betas, eps and the L_reg weight (1, Sec. 4)."""
    lr_mean: float = 1e-4
    lr_log_scale: float = 5e-3
    lr_quat: float = 1e-3
    lr_opacity: float = 5e-2
    lr_rgb: float = 2.5e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    w_reg: float = 1.0

    def c(self) -> L.AdamOpts:
        return L.AdamOpts(self.lr_mean, self.lr_log_scale, self.lr_quat, self.lr_opacity, self.lr_rgb,
                          self.beta1, self.beta2, self.eps, self.w_reg)


class AdamMoments:
    """First/second moments (same layout as the parameters) and a device step."""

    def __init__(self, g: GaussianParams):
        self.m = g.zeros_like()
        self.v = g.zeros_like()
        self.step = torch.zeros(1, dtype=torch.int32, device=g.mean.device)

    def c(self) -> L.AdamState:
        return L.AdamState(*[_ptr(t) for t in self.m.tensors()], *[_ptr(t) for t in self.v.tensors()],
                           _ptr(self.step))


def adam_step(ctx: Context, g: GaussianParams, grads: GaussianParams, state: AdamMoments, cfg: AdamConfig,
              loss_reg=None):
    """gsr_adam_step (in place).  loss_reg: optional [1] tensor that receives += w_reg L_reg."""
    ctx.check(ctx.lib.gsr_adam_step(ctx.handle, ctypes.byref(g.c_mut()), ctypes.byref(grads.c_grads()),
                                    ctypes.byref(state.c()), ctypes.byref(cfg.c()), _ptr(loss_reg), _stream()))


@dataclass
class TrackConfig:
    lambda_c: float = 0.5
    k_median: float = 50.0
    alpha_pow: float = 3.0
    lr_rho: float = 2e-3
    lr_phi: float = 2e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    use_graph: bool = True

    def c(self) -> L.TrackOpts:
        return L.TrackOpts(self.lambda_c, self.k_median, self.alpha_pow, self.lr_rho, self.lr_phi, self.beta1,
                           self.beta2, self.eps, int(self.use_graph))


def track_step(ctx: Context, g: GaussianParams, cam: L.Camera, rgb_in, depth_in, pose: L.Pose, n_iters: int,
               cfg: TrackConfig = None):
    """gsr_track_step: returns (pose after tracking, dict of stats).  Synchronising."""
    cfg = cfg or TrackConfig()
    p = L.Pose(pose.q, pose.t)
    st = L.TrackStats()
    ctx.check(ctx.lib.gsr_track_step(ctx.handle, ctypes.byref(g.c()), ctypes.byref(cam), _ptr(rgb_in),
                                     _ptr(depth_in), ctypes.byref(p), int(n_iters), ctypes.byref(cfg.c()),
                                     ctypes.byref(st), _stream()))
    return p, dict(loss_first=st.loss_first, loss_last=st.loss_last, iters=st.iters)


@dataclass
class MapConfig:
    lambda_ssim: float = 0.2
    w_color: float = 1.0
    w_depth: float = 1.0
    adam: AdamConfig = field(default_factory=AdamConfig)
    use_graph: bool = True

    def c(self) -> L.MapOpts:
        return L.MapOpts(self.lambda_ssim, self.w_color, self.w_depth, self.adam.c(), int(self.use_graph))


def map_step(ctx: Context, g: GaussianParams, state: AdamMoments, cam: L.Camera, keyframes, weights=None,
             n_iters: int = 1, cfg: MapConfig = None, want_stats=True):
    """gsr_map_step over keyframes = [(pose, rgb [3,H,W], depth [H,W]), ...]."""
    cfg = cfg or MapConfig()
    kfs = (L.Keyframe * len(keyframes))()
    for i, (pose, rgb, depth) in enumerate(keyframes):
        kfs[i] = L.Keyframe(pose, _ptr(rgb), _ptr(depth))
    w = None
    if weights is not None:
        w = (ctypes.c_float * len(keyframes))(*[float(x) for x in weights])
    st = L.MapStats()
    ctx.check(ctx.lib.gsr_map_step(ctx.handle, ctypes.byref(g.c_mut()), ctypes.byref(state.c()), ctypes.byref(cam),
                                   kfs, len(keyframes), ctypes.cast(w, ctypes.c_void_p) if w is not None else None,
                                   int(n_iters), ctypes.byref(cfg.c()), ctypes.byref(st) if want_stats else None,
                                   _stream()))
    return dict(loss_last=st.loss_last, iters=st.iters) if want_stats else None


def map_loss(ctx: Context, out: torch.Tensor = None) -> torch.Tensor:
    """gsr_map_loss: the last map step's loss, copied on the current stream
    into a device scalar (no synchronisation)."""
    out = out if out is not None else torch.empty((), dtype=torch.float32, device="cuda")
    ctx.check(ctx.lib.gsr_map_loss(ctx.handle, ctypes.c_void_p(out.data_ptr()), _stream()))
    return out


# ------------------------------------------------------------- seeding
class SubMap:
    """Gaussian arrays of a sub-map with room for `capacity` Gaussians, the
    first `n` in use (`params()` views them)."""

    def __init__(self, capacity: int, device="cuda"):
        self.capacity = int(capacity)
        self.n = 0
        z = lambda *shape: torch.zeros(shape, dtype=torch.float32, device=device)
        self.arrays = GaussianParams(z(capacity, 3), z(capacity, 3), z(capacity, 4), z(capacity), z(capacity, 3))

    def params(self) -> GaussianParams:
        return GaussianParams(*[t[:self.n] for t in self.arrays.tensors()])

    def append(self, g: GaussianParams):
        m = g.n
        if self.n + m > self.capacity:
            raise ValueError("sub-map capacity exceeded")
        for dst, src in zip(self.arrays.tensors(), g.tensors()):
            dst[self.n:self.n + m].copy_(src)
        self.n += m


@dataclass
class SeedConfig:
    first_keyframe: bool = True
    m_u: int = 100_000
    m_c: int = 50_000
    m_k: int = 100_000
    alpha_n: float = 0.6
    rho: float = 0.01
    s_min: float = 1e-4
    s_max: float = 0.1
    seed: int = 0

    def c(self) -> L.SeedOpts:
        return L.SeedOpts(int(self.first_keyframe), self.m_u, self.m_c, self.m_k, self.alpha_n, self.rho, self.s_min,
                          self.s_max, self.seed)


def seed_keyframe(ctx: Context, sub: SubMap, cam: L.Camera, pose: L.Pose, rgb, depth, alpha=None,
                  cfg: SeedConfig = None) -> dict:
    """gsr_seed_keyframe: appends the keyframe's new Gaussians to `sub`.  Synchronising."""
    cfg = cfg or SeedConfig()
    st = L.SeedStats()
    gm = sub.arrays.c_mut()
    ctx.check(ctx.lib.gsr_seed_keyframe(ctx.handle, ctypes.byref(cam), ctypes.byref(pose), _ptr(rgb), _ptr(depth),
                                        _ptr(alpha), ctypes.byref(cfg.c()), ctypes.byref(gm), sub.n, sub.capacity,
                                        ctypes.byref(st), _stream()))
    sub.n += int(st.n_added)
    return dict(n_candidates=int(st.n_candidates), n_added=int(st.n_added))


def seed_candidates(ctx: Context, capacity: int):
    """The last seeding's candidates: (pixel index, kept flag, squared distance to the sub-map) tensors."""
    n = ctypes.c_int64()
    pix = torch.empty(capacity, dtype=torch.int32, device="cuda")
    keep = torch.empty(capacity, dtype=torch.int32, device="cuda")
    d2 = torch.empty(capacity, dtype=torch.float32, device="cuda")
    ctx.check(ctx.lib.gsr_seed_candidates_get(ctx.handle, _ptr(pix), _ptr(keep), _ptr(d2), capacity,
                                              ctypes.byref(n), _stream()))
    k = int(n.value)
    return pix[:k], keep[:k], d2[:k]


def prune(ctx: Context, sub: SubMap, state: "AdamMoments" = None, min_opacity: float = 0.1) -> int:
    """gsr_prune: drops sub-map Gaussians with opacity below min_opacity (and
    their Adam moments), keeping the order.  Returns the new count."""
    n = ctypes.c_int64()
    gm = sub.arrays.c_mut()
    gm.n = sub.n
    st = ctypes.byref(state.c()) if state is not None else None
    ctx.check(ctx.lib.gsr_prune(ctx.handle, ctypes.byref(gm), st, float(min_opacity), ctypes.byref(n), _stream()))
    sub.n = int(n.value)
    return sub.n


def merge_submap(ctx: Context, global_map: SubMap, sub: GaussianParams, rho: float = 0.01) -> int:
    """gsr_merge_submap: appends the Gaussians of `sub` that have no global-map
    mean within rho.  Returns the number added."""
    n = ctypes.c_int64()
    ctx.check(ctx.lib.gsr_merge_submap(ctx.handle, ctypes.byref(global_map.arrays.c_mut()), global_map.n,
                                       global_map.capacity, ctypes.byref(sub.c()), float(rho), ctypes.byref(n),
                                       _stream()))
    global_map.n += int(n.value)
    return int(n.value)


# ------------------------------------------------------ throughput probes
def probe_peaks(blocks: int = 152 * 8, iters: int = 16384, reps: int = 5):
    """Measured FP32 FMA rate (TFLOP/s) and base-2 exponential rate (G/s) of
    the current device (gsr_probe_fma / gsr_probe_exp), best of `reps`
    launches timed with CUDA events on the current stream."""
    lib = L.load()
    out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    res = {}
    for name, fn, per in (("fp32_tflops", lib.gsr_probe_fma, 16), ("exp_gps", lib.gsr_probe_exp, 8)):
        L.check(fn(ctypes.c_void_p(out.data_ptr()), blocks, 32, _stream()))  # warm-up
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            L.check(fn(ctypes.c_void_p(out.data_ptr()), blocks, iters, _stream()))
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        ops = blocks * 256 * iters * per
        res[name] = ops / best / (1e12 if name == "fp32_tflops" else 1e9)
    return res


# ----------------------------------------------------------- pose helpers
def pose_retract(pose: L.Pose, xi: torch.Tensor, out: torch.Tensor = None) -> torch.Tensor:
    """gsr_pose_retract: (q', t') of exp(xi^) T as a device float32 [7]
    tensor (stream-ordered; xi is a device float32 [6] twist (rho, phi))."""
    out = out if out is not None else torch.empty(7, dtype=torch.float32, device=xi.device)
    L.check(L.load().gsr_pose_retract(ctypes.byref(pose), _twist(xi.contiguous()), _ptr(out), _stream()))
    return out


def pose_from_tensor(p: torch.Tensor) -> L.Pose:
    """A (q, t) float32 [7] tensor (e.g. from pose_retract) as a host pose
    (reads it back, synchronising)."""
    h = p.detach().cpu().numpy().astype(np.float64)
    return make_pose(h[:4], h[4:7])


def autotune(ctx: Context, g: GaussianParams, cam: L.Camera, poses, reps: int = 3):
    """gsr_autotune: times render fwd+bwd at `poses` for every tile shape x
    batch x pixels-per-thread and keeps the fastest on `ctx`.
    Returns (best dict, list of all timings)."""
    n = len(poses)
    arr = (L.Pose * n)(*[L.Pose(p.q, p.t) for p in poses])
    best = L.TuneResult()
    allr = (L.TuneResult * 32)()
    ctx.check(ctx.lib.gsr_autotune(ctx.handle, ctypes.byref(g.c()), ctypes.byref(cam), arr, n, int(reps),
                                   ctypes.byref(best), allr, 32, _stream()))
    conv = lambda r: dict(tile=(r.tile_w, r.tile_h), batch=r.batch, ppt_fwd=r.ppt_fwd, ppt_bwd=r.ppt_bwd,
                          ms_fwd=r.ms_fwd, ms_bwd=r.ms_bwd, ms=r.ms)
    return conv(best), [conv(r) for r in allr if r.batch > 0]
