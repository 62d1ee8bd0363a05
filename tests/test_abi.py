"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
symbol include/gsr.h declares, and the ctypes mirror matches the header's
struct layouts (checked against gcc's own sizeof/offsetof).  No compute call
is made here."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2312_10070_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsr.h")
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    names = set()
    for h in HEADERS:
        names |= set(re.findall(r"^GSR_API\s+[\w\s\*]+?\b(gsr_\w+)\s*\(", open(h).read(), flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _lib.load(build_if_missing=False)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.PROTOTYPES), set(names) ^ set(_lib.PROTOTYPES)


def test_library_has_sm103a_code_and_no_torch_types():
    for h in HEADERS:
        txt = open(h).read()
        assert "torch" not in txt.lower().replace("pytorch type", ""), h
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)


STRUCTS = {
    "gsr_options": _lib.Options, "gsr_camera": _lib.Camera, "gsr_pose": _lib.Pose,
    "gsr_gaussians": _lib.Gaussians, "gsr_gaussian_grads": _lib.GaussianGrads, "gsr_render_out": _lib.RenderOut,
    "gsr_frame_stats": _lib.FrameStats, "gsr_adam_opts": _lib.AdamOpts, "gsr_adam_state": _lib.AdamState,
    "gsr_gaussians_mut": _lib.GaussiansMut, "gsr_track_opts": _lib.TrackOpts, "gsr_track_stats": _lib.TrackStats,
    "gsr_keyframe": _lib.Keyframe, "gsr_map_opts": _lib.MapOpts, "gsr_map_stats": _lib.MapStats,
    "gsr_tune_result": _lib.TuneResult, "gsr_warmstart_opts": _lib.WarmstartOpts,
    "gsr_seed_opts": _lib.SeedOpts, "gsr_seed_stats": _lib.SeedStats,
}


def test_struct_layouts_match_header(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"',
             f'#include "{os.path.join(ROOT, "include", "gsr_warmstart.h")}"', "int main(void){"]
    for cname, py in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append('printf("GSR_NOALLOC_MAX_PIXELS value %d\\n", (int)GSR_NOALLOC_MAX_PIXELS);')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)]).decode().split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        if cname == "GSR_NOALLOC_MAX_PIXELS":
            assert _lib.NOALLOC_MAX_PIXELS == int(val)
            continue
        py = STRUCTS[cname]
        if field == "size":
            assert ctypes.sizeof(py) == int(val), cname
        else:
            assert getattr(py, field).offset == int(val), (cname, field)


def test_default_options_without_gpu(lib):
    o = _lib.Options()
    lib.gsr_default_options(ctypes.byref(o))
    assert (o.tile_w, o.tile_h, o.batch) == (16, 16, 256)
    c = _lib.Camera()
    lib.gsr_default_camera(ctypes.byref(c), 160, 120, 150.0, 150.0, 80.0, 60.0)
    assert abs(c.z_near - 0.2) < 1e-7 and abs(c.eps2d - 0.3) < 1e-7
    assert lib.gsr_status_string(-4) == b"GSR_ERR_CAPACITY"


def test_invalid_arguments_are_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    o = _lib.Options()
    lib.gsr_default_options(ctypes.byref(o))
    o.tile_w = 12
    assert lib.gsr_create(ctypes.byref(h), ctypes.byref(o)) == -1
    assert not h.value
    o.tile_w, o.batch = 16, 100
    assert lib.gsr_create(ctypes.byref(h), ctypes.byref(o)) == -1
    assert lib.gsr_create(None, None) == -1
    # stream-ordered loss readout: NULL arguments are rejected before any CUDA call
    assert lib.gsr_map_loss(None, None, None) == -1
    # bounded-wait check: a NULL context is rejected before any launch
    assert lib.gsr_check_wait_timeout(None, 100, None) == -1
    # throughput probes: sizes are checked before any launch
    assert lib.gsr_probe_fma(None, 1, 32, None) == -1
    assert lib.gsr_probe_exp(None, 1, 32, None) == -1
    buf = ctypes.c_void_p(16)  # never dereferenced: the checks below fail first
    assert lib.gsr_probe_fma(buf, 0, 32, None) == -1
    assert lib.gsr_probe_fma(buf, 1, 33, None) == -1
    assert lib.gsr_probe_exp(buf, 1, 0, None) == -1


def test_warmstart_layout_and_argument_checks_without_gpu(lib):
    from oracle import cnn
    assert lib.gsr_warmstart_num_params() == cnn.n_params()
    o = _lib.WarmstartOpts()
    lib.gsr_warmstart_default_opts(ctypes.byref(o))
    assert abs(o.lr - 1e-3) < 1e-9 and list(o.w) == [1.0] * 6
    h = ctypes.c_void_p()
    assert lib.gsr_warmstart_create(None, 4, 0) == -1
    assert lib.gsr_warmstart_create(ctypes.byref(h), 0, 0) == -1
    assert lib.gsr_warmstart_create(ctypes.byref(h), 5000, 0) == -1
    assert lib.gsr_warmstart_make_input(None, None, None, None, 120, 160, 5.0, None, None) == -1
