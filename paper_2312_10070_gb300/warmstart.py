"""Python binding of the learned tracking warm-start (include/gsr_warmstart.h).

The network predicts the left-multiplied twist xi = (rho, phi) that moves an
initial world-to-camera pose (the constant-velocity guess of the tracker) to
the true one, from a 160 x 120 residual between a render at the initial pose
and the input frame.  All arithmetic runs in libgsr.so; PyTorch provides
device memory and the current stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from .api import _ptr, _stream

IN_H, IN_W, IN_C, N_OUT = 120, 160, 8, 6
CONV = ((8, 32), (32, 64), (64, 128), (128, 128), (128, 256), (256, 256))  # 3x3 stride-2 layers (in, out)
DENSE = ((1536, 256), (256, 6))


@dataclass
class WarmstartConfig:
    lr: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    weights: tuple = (1.0, 1.0, 1.0, 1.0, 1.0, 1.0)

    def c(self) -> L.WarmstartOpts:
        o = L.WarmstartOpts()
        o.lr, o.beta1, o.beta2, o.eps = self.lr, self.beta1, self.beta2, self.eps
        for i, w in enumerate(self.weights):
            o.w[i] = w
        return o


def num_params() -> int:
    return int(L.load().gsr_warmstart_num_params())


class WarmStartNet:
    """Owns a gsr_warmstart (FP32 masters, BF16 copies, Adam moments, scratch)."""

    def __init__(self, max_batch: int = 256, seed: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("the warm-start network needs a CUDA device; there is no CPU fallback")
        self.lib = L.load()
        self.max_batch = max_batch
        h = ctypes.c_void_p()
        L.check(self.lib.gsr_warmstart_create(ctypes.byref(h), max_batch, seed))
        self.handle = h
        self.n_params = int(self.lib.gsr_warmstart_num_params())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.gsr_warmstart_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status):
        if status != 0:
            msg = self.lib.gsr_warmstart_last_error(self.handle).decode()
            raise L.GsrError(status, msg)

    def set_kernels(self, tcgen05_min_k: int):
        """Forward products with reduction length >= tcgen05_min_k on tcgen05,
        the rest on the mma.sync kernel (negative: none on tcgen05)."""
        self.check(self.lib.gsr_warmstart_set_kernels(self.handle, int(tcgen05_min_k)))

    def check_status(self):
        """Synchronise; raise if a tensor-core kernel reported an expired wait."""
        self.check(self.lib.gsr_warmstart_check(self.handle, _stream()))

    def get_params(self) -> torch.Tensor:
        p = torch.empty(self.n_params, device="cuda")
        self.check(self.lib.gsr_warmstart_get_params(self.handle, _ptr(p), _stream()))
        return p

    def set_params(self, p: torch.Tensor):
        p = p.to(device="cuda", dtype=torch.float32).contiguous()
        if p.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {p.numel()}")
        self.check(self.lib.gsr_warmstart_set_params(self.handle, _ptr(p), _stream()))

    def _batch(self, x):
        if x.dtype != torch.float32 or tuple(x.shape[1:]) != (IN_H, IN_W, IN_C):
            raise ValueError("x must be float32 [B, 120, 160, 8]")
        return x.shape[0]

    def forward(self, x: torch.Tensor, out: torch.Tensor = None) -> torch.Tensor:
        b = self._batch(x)
        if out is None:
            out = torch.empty(b, N_OUT, device="cuda")
        self.check(self.lib.gsr_warmstart_forward(self.handle, _ptr(x), b, _ptr(out), _stream()))
        return out

    def backward(self, d_out: torch.Tensor) -> torch.Tensor:
        """Gradient of sum(d_out * out) of the last forward, as a flat vector."""
        d_out = d_out.to(device="cuda", dtype=torch.float32).contiguous()
        g = torch.empty(self.n_params, device="cuda")
        self.check(self.lib.gsr_warmstart_backward(self.handle, _ptr(d_out), d_out.shape[0], _ptr(g), _stream()))
        return g

    def train_step(self, x: torch.Tensor, target: torch.Tensor, cfg: WarmstartConfig = None) -> torch.Tensor:
        """One Adam step on the weighted squared twist error; returns the loss (device scalar)."""
        b = self._batch(x)
        target = target.to(device="cuda", dtype=torch.float32).contiguous()
        loss = torch.empty(1, device="cuda")
        o = (cfg or WarmstartConfig()).c()
        self.check(self.lib.gsr_warmstart_train_step(self.handle, _ptr(x), _ptr(target), b, ctypes.byref(o),
                                                     _ptr(loss), _stream()))
        return loss


def make_input(rgb_r, depth_r, rgb_i, depth_i, depth_scale: float = 5.0, out=None) -> torch.Tensor:
    """Network input [120, 160, 8] from a 160 x 120 render and a frame of any size >= 160 x 120."""
    lib = L.load()
    h, w = depth_i.shape
    if out is None:
        out = torch.empty(IN_H, IN_W, IN_C, device="cuda")
    st = lib.gsr_warmstart_make_input(_ptr(rgb_r), _ptr(depth_r), _ptr(rgb_i), _ptr(depth_i), h, w, depth_scale,
                                      _ptr(out), _stream())
    L.check(st)
    return out


# ------------------------------------------------------------ training data
# Samples are (network input at an initial pose, twist from that pose to the
# true one).  The initial pose is the true pose moved by a random twist of up
# to max_t metres / max_deg degrees (the error of a constant-velocity guess
# under inter-frame motion up to that size); the label is the exact inverse
# twist, since the synthetic ground truth is known.

def random_twist(rng, max_t: float, max_deg: float):
    """xi = (rho, phi): rho uniform in the ball of radius max_t (m), phi about
    a uniform random axis with angle uniform in [0, max_deg] degrees."""
    d = rng.standard_normal(3)
    rho = d / np.linalg.norm(d) * max_t * rng.random() ** (1.0 / 3.0)
    a = rng.standard_normal(3)
    phi = a / np.linalg.norm(a) * np.deg2rad(max_deg) * rng.random()
    return np.concatenate([rho, phi])


def _rot(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def pose_error(q, t, q_gt, t_gt):
    """(camera-centre distance in m, relative rotation angle in degrees)."""
    R, Rg = _rot(q), _rot(q_gt)
    c, cg = -R.T @ np.asarray(t, np.float64), -Rg.T @ np.asarray(t_gt, np.float64)
    cos = np.clip((np.trace(R @ Rg.T) - 1.0) / 2.0, -1.0, 1.0)
    return float(np.linalg.norm(c - cg)), float(np.degrees(np.arccos(cos)))


@dataclass
class Frame:
    q_gt: np.ndarray
    t_gt: np.ndarray
    rgb: torch.Tensor    # [3, H, W] noisy input frame
    depth: torch.Tensor  # [H, W], 0 = invalid


class Samples:
    """Network inputs x [N, 120, 160, 8] and labels y [N, 6] on the device,
    filled in a random slot order so that contiguous windows are shuffled
    batches; per slot the initial pose and the index of its frame."""

    def __init__(self, capacity: int, seed: int = 0):
        self.x = torch.empty(capacity, IN_H, IN_W, IN_C, device="cuda")
        self._y = np.zeros((capacity, N_OUT), np.float32)
        self.slots = np.random.default_rng(seed).permutation(capacity)
        self.init = [None] * capacity
        self.frame = [None] * capacity
        self.frames = []
        self.n = 0

    @property
    def y(self) -> torch.Tensor:
        return torch.from_numpy(self._y).cuda()

    def full(self) -> bool:
        return self.n == len(self.slots)


def low_res_camera(spec):
    from . import synth
    return synth.scale_camera(spec, IN_W, IN_H)


def add_frames(data: Samples, ctx_full, ctx_low, g, spec, poses, per_frame: int, rng, max_t: float = 0.05,
               max_deg: float = 3.0, noise_seed: int = 0, depth_scale: float = 5.0, keep_frames: bool = True):
    """Render each true pose at full resolution (plus sensor noise) and, for
    `per_frame` random initial poses per frame, the 160 x 120 render at the
    initial pose; writes network inputs and labels into free slots of `data`.
    keep_frames=False keeps only each frame's true pose (no images), for
    training sets too large to keep every full-resolution frame."""
    from . import api, synth
    cam_f = api.camera_from_spec(spec)
    cam_l = api.camera_from_spec(low_res_camera(spec))
    for i, (q, t) in enumerate(zip(*poses)):
        if data.full():
            break
        r = api.render_forward(ctx_full, g, cam_f, api.make_pose(q, t))
        rgb_n, d_n = synth.add_sensor_noise(r["rgb"].cpu().numpy(), r["depth"].cpu().numpy(),
                                            r["alpha"].cpu().numpy(), seed=noise_seed + i)
        fr = Frame(np.asarray(q, np.float64), np.asarray(t, np.float64), torch.from_numpy(rgb_n).cuda(),
                   torch.from_numpy(d_n).cuda())
        data.frames.append(fr if keep_frames else Frame(fr.q_gt, fr.t_gt, None, None))
        for _ in range(per_frame):
            if data.full():
                break
            k = int(data.slots[data.n])
            xi = random_twist(rng, max_t, max_deg)
            pi = api.pose_retract(api.make_pose(q, t), torch.tensor(xi, dtype=torch.float32, device="cuda"))
            qi, ti = _host_pose(pi)
            lo = api.render_forward(ctx_low, g, cam_l, api.make_pose(qi, ti))
            make_input(lo["rgb"], lo["depth"], fr.rgb, fr.depth, depth_scale, out=data.x[k])
            data._y[k] = -xi
            data.init[k] = (qi, ti)
            data.frame[k] = len(data.frames) - 1
            data.n += 1
    torch.cuda.synchronize()


def train(net: WarmStartNet, data: Samples, steps: int, batch: int = 64, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Adam on the per-component variance-normalised squared twist error.
    Each batch is a contiguous window of the samples at a random offset (no
    gather: the network reads the window in place)."""
    rng = np.random.default_rng(seed)
    if not data.full():
        raise ValueError("the sample set is not full")
    x, y = data.x, data.y
    var = np.maximum(data._y.astype(np.float64).var(axis=0), 1e-12)
    cfg = WarmstartConfig(lr=lr, weights=tuple(float(1.0 / v) for v in var))
    n = x.shape[0]
    batch = min(batch, n)
    losses = []
    for s in range(steps):
        o = int(rng.integers(0, n - batch + 1))
        loss = net.train_step(x[o:o + batch], y[o:o + batch], cfg)
        if log_every and (s % log_every == 0 or s == steps - 1):
            losses.append((s, loss.item()))
    return losses


def predict(net: WarmStartNet, x: torch.Tensor, batch: int = 0) -> torch.Tensor:
    batch = batch or net.max_batch
    out = torch.empty(x.shape[0], N_OUT, device="cuda")
    for i in range(0, x.shape[0], batch):
        net.forward(x[i:i + batch], out=out[i:i + batch])
    return out


def _host_pose(p: torch.Tensor):
    """(q, t) float64 arrays of a device (q, t) float32 [7] pose (synchronising)."""
    h = p.cpu().numpy().astype(np.float64)
    return h[:4], h[4:7]


def corrected_poses(data: Samples, pred: torch.Tensor):
    """exp(pred_i^) T_i for every sample's initial pose T_i (gsr_pose_retract)."""
    from . import api
    pred = pred.to(torch.float32).contiguous()
    out = torch.empty((len(data.init), 7), dtype=torch.float32, device=pred.device)
    for i, (q, t) in enumerate(data.init):
        api.pose_retract(api.make_pose(q, t), pred[i], out=out[i])
    return [_host_pose(p) for p in out]


def pose_errors(data: Samples, poses):
    out = []
    for (q, t), f in zip(poses, data.frame):
        fr = data.frames[f]
        out.append(pose_error(q, t, fr.q_gt, fr.t_gt))
    return np.array(out)


# ------------------------------------------------------- warm-started tracking
def track_from(ctx, g, spec, frame: Frame, q, t, n_iters: int, cfg=None):
    """Run the tracker for n_iters from (q, t); returns ((q, t), stats)."""
    from . import api
    p, st = api.track_step(ctx, g, api.camera_from_spec(spec), frame.rgb, frame.depth, api.make_pose(q, t),
                           n_iters, cfg)
    return (np.array(p.q[:], np.float64), np.array(p.t[:], np.float64)), st


def iterations_to_converge(ctx, g, spec, frame: Frame, q, t, budgets=(10, 20, 40, 80, 160), tol_m: float = 0.01,
                           tol_deg: float = 0.5, cfg=None):
    """Smallest budget (tracker iterations from (q, t)) whose result is within
    tol_m / tol_deg of the true pose (None if none is), the tracking loss at
    (q, t), and the pose errors at the largest budget run."""
    loss0, err = None, None
    for n in budgets:
        (qe, te), st = track_from(ctx, g, spec, frame, q, t, n, cfg)
        loss0 = st["loss_first"]
        err = pose_error(qe, te, frame.q_gt, frame.t_gt)
        if err[0] <= tol_m and err[1] <= tol_deg:
            return n, loss0, err
    return None, loss0, err


def warm_start_pose(net: WarmStartNet, ctx_low, g, spec, frame: Frame, q, t, depth_scale: float = 5.0):
    """One network correction of the initial pose (q, t) for `frame`."""
    from . import api
    cam_l = api.camera_from_spec(low_res_camera(spec))
    lo = api.render_forward(ctx_low, g, cam_l, api.make_pose(q, t))
    x = make_input(lo["rgb"], lo["depth"], frame.rgb, frame.depth, depth_scale).unsqueeze(0)
    xi = net.forward(x)[0].contiguous()
    return _host_pose(api.pose_retract(api.make_pose(q, t), xi))
