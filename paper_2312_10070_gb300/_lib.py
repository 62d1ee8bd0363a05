"""ctypes mirror of include/gsr.h and loader of the in-tree libgsr.so.

Argument marshalling only: every step of the rasterizer runs in the CUDA
kernels of libgsr.so.  There is no fallback; if the library is missing or
cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsr.so")

c_f = ctypes.c_float
c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
P_f = ctypes.POINTER(c_f)
P_i32 = ctypes.POINTER(c_i32)
c_vp = ctypes.c_void_p

GSR_OK = 0
NOALLOC_MAX_PIXELS = 921600  # GSR_NOALLOC_MAX_PIXELS of gsr.h (1280 x 720)
STATUS = {0: "GSR_OK", -1: "GSR_ERR_INVALID_ARG", -2: "GSR_ERR_CUDA", -3: "GSR_ERR_OOM",
          -4: "GSR_ERR_CAPACITY", -5: "GSR_ERR_TIMEOUT", -6: "GSR_ERR_NONFINITE", -7: "GSR_ERR_STATE"}


class Options(ctypes.Structure):
    _fields_ = [("tile_w", c_i32), ("tile_h", c_i32), ("batch", c_i32), ("memory_saving", c_i32),
                ("fixed_capacity", c_i32), ("max_gaussians", c_i64), ("max_instances", c_i64),
                ("max_pixels", c_i64), ("ppt_fwd", c_i32), ("ppt_bwd", c_i32), ("rect_lists", c_i32)]


class Camera(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f),
                ("z_near", c_f), ("eps2d", c_f)]


class Pose(ctypes.Structure):
    _fields_ = [("q", c_f * 4), ("t", c_f * 3)]


class Gaussians(ctypes.Structure):
    _fields_ = [("mean", c_vp), ("log_scale", c_vp), ("quat", c_vp), ("opacity_logit", c_vp), ("rgb", c_vp),
                ("n", c_i64)]


class GaussianGrads(ctypes.Structure):
    _fields_ = [("mean", c_vp), ("log_scale", c_vp), ("quat", c_vp), ("opacity_logit", c_vp), ("rgb", c_vp)]


class RenderOut(ctypes.Structure):
    _fields_ = [("rgb", c_vp), ("depth", c_vp), ("alpha", c_vp), ("final_T", c_vp), ("last_idx", c_vp),
                ("n_contrib", c_vp)]


class FrameStats(ctypes.Structure):
    _fields_ = [("n_visible", c_i64), ("n_instances", c_i64), ("n_tiles", c_i64), ("capacity_instances", c_i64)]


class AdamOpts(ctypes.Structure):
    _fields_ = [("lr_mean", c_f), ("lr_log_scale", c_f), ("lr_quat", c_f), ("lr_opacity", c_f), ("lr_rgb", c_f),
                ("beta1", c_f), ("beta2", c_f), ("eps", c_f), ("w_reg", c_f)]


class AdamState(ctypes.Structure):
    _fields_ = [("m_mean", c_vp), ("m_log_scale", c_vp), ("m_quat", c_vp), ("m_opacity_logit", c_vp),
                ("m_rgb", c_vp), ("v_mean", c_vp), ("v_log_scale", c_vp), ("v_quat", c_vp),
                ("v_opacity_logit", c_vp), ("v_rgb", c_vp), ("step", c_vp)]


class GaussiansMut(ctypes.Structure):
    _fields_ = [("mean", c_vp), ("log_scale", c_vp), ("quat", c_vp), ("opacity_logit", c_vp), ("rgb", c_vp),
                ("n", c_i64)]


class TrackOpts(ctypes.Structure):
    _fields_ = [("lambda_c", c_f), ("k_median", c_f), ("alpha_pow", c_f), ("lr_rho", c_f), ("lr_phi", c_f),
                ("beta1", c_f), ("beta2", c_f), ("eps", c_f), ("use_graph", c_i32)]


class TrackStats(ctypes.Structure):
    _fields_ = [("loss_first", c_f), ("loss_last", c_f), ("iters", c_i32)]


class Keyframe(ctypes.Structure):
    _fields_ = [("pose", Pose), ("rgb", c_vp), ("depth", c_vp)]


class MapOpts(ctypes.Structure):
    _fields_ = [("lambda_ssim", c_f), ("w_color", c_f), ("w_depth", c_f), ("adam", AdamOpts), ("use_graph", c_i32)]


class MapStats(ctypes.Structure):
    _fields_ = [("loss_last", c_f), ("iters", c_i32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("tile_w", c_i32), ("tile_h", c_i32), ("batch", c_i32), ("ppt_fwd", c_i32), ("ppt_bwd", c_i32),
                ("ms_fwd", c_f), ("ms_bwd", c_f), ("ms", c_f)]


class SeedOpts(ctypes.Structure):
    _fields_ = [("first_keyframe", c_i32), ("m_u", c_i64), ("m_c", c_i64), ("m_k", c_i64), ("alpha_n", c_f),
                ("rho", c_f), ("s_min", c_f), ("s_max", c_f), ("seed", ctypes.c_uint64)]


class SeedStats(ctypes.Structure):
    _fields_ = [("n_candidates", c_i64), ("n_added", c_i64)]


class WarmstartOpts(ctypes.Structure):
    _fields_ = [("lr", c_f), ("beta1", c_f), ("beta2", c_f), ("eps", c_f), ("w", c_f * 6)]


# name -> (restype, argtypes); every symbol include/gsr.h and include/gsr_warmstart.h declare
PROTOTYPES = {
    "gsr_default_options": (None, [ctypes.POINTER(Options)]),
    "gsr_default_camera": (None, [ctypes.POINTER(Camera), c_i32, c_i32, c_f, c_f, c_f, c_f]),
    "gsr_create": (c_i32, [ctypes.POINTER(c_vp), ctypes.POINTER(Options)]),
    "gsr_destroy": (None, [c_vp]),
    "gsr_last_error": (ctypes.c_char_p, [c_vp]),
    "gsr_status_string": (ctypes.c_char_p, [c_i32]),
    "gsr_kernel_launches": (c_i64, [c_vp]),
    "gsr_profile_enable": (c_i32, [c_vp, c_i32]),
    "gsr_profile_read": (c_i32, [c_vp, c_vp, c_i32, c_vp]),
    "gsr_render_forward": (c_i32, [c_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), ctypes.POINTER(Pose),
                                   ctypes.POINTER(RenderOut), c_vp]),
    "gsr_frame_stats_get": (c_i32, [c_vp, ctypes.POINTER(FrameStats), c_vp]),
    "gsr_check_wait_timeout": (c_i32, [c_vp, c_i32, c_vp]),
    "gsr_tile_lists_get": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp, ctypes.POINTER(c_i64), c_vp]),
    "gsr_render_backward": (c_i32, [c_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), ctypes.POINTER(Pose),
                                    ctypes.POINTER(RenderOut), c_vp, c_vp, c_vp, ctypes.POINTER(GaussianGrads),
                                    c_vp, c_vp]),
    "gsr_render_forward_xi": (c_i32, [c_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), ctypes.POINTER(Pose),
                                      c_vp, ctypes.POINTER(RenderOut), c_vp]),
    "gsr_render_backward_xi": (c_i32, [c_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), ctypes.POINTER(Pose),
                                       c_vp, ctypes.POINTER(RenderOut), c_vp, c_vp, c_vp,
                                       ctypes.POINTER(GaussianGrads), c_vp, c_vp]),
    "gsr_pose_retract": (c_i32, [ctypes.POINTER(Pose), c_vp, c_vp, c_vp]),
    "gsr_records_get": (c_i32, [c_vp, c_vp, c_vp, c_i64, c_vp]),
    "gsr_probe_expf": (c_i32, [c_vp, c_vp, c_i64, c_vp]),
    "gsr_loss_map": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_f, c_f, c_f, c_f, c_vp, c_vp, c_vp,
                             c_vp]),
    "gsr_loss_track": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_f, c_f, c_f, c_vp, c_vp,
                               c_vp, c_vp, c_vp]),
    "gsr_loss_track_noalloc": (c_i32, [c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_f, c_f, c_f, c_vp, c_vp, c_vp,
                                       c_vp, c_vp]),
    "gsr_adam_step": (c_i32, [c_vp, ctypes.POINTER(GaussiansMut), ctypes.POINTER(GaussianGrads),
                              ctypes.POINTER(AdamState), ctypes.POINTER(AdamOpts), c_vp, c_vp]),
    "gsr_track_step": (c_i32, [c_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), c_vp, c_vp,
                               ctypes.POINTER(Pose), c_i32, ctypes.POINTER(TrackOpts), ctypes.POINTER(TrackStats),
                               c_vp]),
    "gsr_map_step": (c_i32, [c_vp, ctypes.POINTER(GaussiansMut), ctypes.POINTER(AdamState), ctypes.POINTER(Camera),
                             ctypes.POINTER(Keyframe), c_i32, c_vp, c_i32, ctypes.POINTER(MapOpts),
                             ctypes.POINTER(MapStats), c_vp]),
    "gsr_autotune": (c_i32, [c_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), ctypes.POINTER(Pose), c_i32,
                             c_i32, ctypes.POINTER(TuneResult), ctypes.POINTER(TuneResult), c_i32, c_vp]),
    "gsr_default_seed_opts": (None, [ctypes.POINTER(SeedOpts)]),
    "gsr_seed_keyframe": (c_i32, [c_vp, ctypes.POINTER(Camera), ctypes.POINTER(Pose), c_vp, c_vp, c_vp,
                                  ctypes.POINTER(SeedOpts), ctypes.POINTER(GaussiansMut), c_i64, c_i64,
                                  ctypes.POINTER(SeedStats), c_vp]),
    "gsr_seed_candidates_get": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64), c_vp]),
    "gsr_prune": (c_i32, [c_vp, ctypes.POINTER(GaussiansMut), ctypes.POINTER(AdamState), c_f, ctypes.POINTER(c_i64),
                          c_vp]),
    "gsr_merge_submap": (c_i32, [c_vp, ctypes.POINTER(GaussiansMut), c_i64, c_i64, ctypes.POINTER(Gaussians), c_f,
                                 ctypes.POINTER(c_i64), c_vp]),
    "gsr_map_loss": (c_i32, [c_vp, c_vp, c_vp]),
    "gsr_probe_fma": (c_i32, [c_vp, c_i32, c_i32, c_vp]),
    "gsr_probe_exp": (c_i32, [c_vp, c_i32, c_i32, c_vp]),
    "gsr_warmstart_num_params": (c_i64, []),
    "gsr_warmstart_create": (c_i32, [ctypes.POINTER(c_vp), c_i32, ctypes.c_uint64]),
    "gsr_warmstart_destroy": (None, [c_vp]),
    "gsr_warmstart_last_error": (ctypes.c_char_p, [c_vp]),
    "gsr_warmstart_set_params": (c_i32, [c_vp, c_vp, c_vp]),
    "gsr_warmstart_get_params": (c_i32, [c_vp, c_vp, c_vp]),
    "gsr_warmstart_forward": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp]),
    "gsr_warmstart_backward": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp]),
    "gsr_warmstart_default_opts": (None, [ctypes.POINTER(WarmstartOpts)]),
    "gsr_warmstart_set_kernels": (c_i32, [c_vp, c_i32]),
    "gsr_warmstart_check": (c_i32, [c_vp, c_vp]),
    "gsr_warmstart_train_step": (c_i32, [c_vp, c_vp, c_vp, c_i32, ctypes.POINTER(WarmstartOpts), c_vp, c_vp]),
    "gsr_warmstart_make_input": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32, c_i32, c_f, c_vp, c_vp]),
}

_lib = None


def load(build_if_missing: bool = True):
    """Load libgsr.so (building it first when missing).  Raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH) and build_if_missing:
        from . import _build
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgsr.so not found at {LIB_PATH}; run paper_2312_10070_gb300._build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GsrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status: int, ctx_handle=None):
    if status != GSR_OK:
        msg = ""
        if ctx_handle:
            m = load().gsr_last_error(ctx_handle)
            msg = m.decode() if m else ""
        raise GsrError(status, msg)
