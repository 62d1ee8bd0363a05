"""Host logic of bench.py, without a GPU: the lookup of committed DRAM
traffic per launch configuration, the derived FP32 peak, and the JSON line of
the reference arm (the FP64 oracle on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def tuned(tile, batch, ppt):
    return dict(tile=tile, batch=batch, ppt_fwd=ppt, ppt_bwd=ppt)


def test_traffic_lookup_prefers_the_captured_configuration(monkeypatch):
    entries = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["blend_bwd"]
    # the lookup logic, with the sources as they were at capture time
    shas = {tuple(e["sources"]): e["sources_sha256"] for e in entries}
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda files: shas.get(tuple(files), "0" * 64))
    by_cfg = {(e["config"]["batch"], e["config"]["ppt"]): e["dram_bytes_per_launch"] for e in entries}
    for (batch, ppt), b in by_cfg.items():
        got, cfg = bench.measured_traffic("blend_bwd", tuned((8, 8), batch, ppt))
        assert got == b and cfg["batch"] == batch and cfg["ppt"] == ppt
    # another batch / pixels per thread with the same tile shape: a capture of that tile
    got, cfg = bench.measured_traffic("blend_bwd", tuned((8, 8), 32, 2))
    assert got in by_cfg.values() and list(cfg["tile"]) == [8, 8]
    # no capture of another tile shape, of an uncaptured kernel
    assert bench.measured_traffic("blend_bwd", tuned((16, 16), 128, 1)) == (None, None)
    assert bench.measured_traffic("no_such_kernel") == (None, None)


def test_traffic_is_dropped_when_the_kernel_sources_change(monkeypatch):
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda files: "0" * 64)
    assert bench.measured_traffic("blend_bwd", tuned((8, 8), 64, 2)) == (None, None)


def test_derived_fp32_peak():
    # 152 SMs x 128 FP32 lanes x 2 flops per FMA x 2070 MHz
    assert bench.fp32_peak_tflops(2070.0) == pytest.approx(80.54784)


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "iters/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == dict(value=line["value"], unit="iters/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    assert line["dtype"] == "f64" and line["steps"] == 1 and line["warmup"] == 1


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT,
                       env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_extra_workloads_namespace_has_every_argument_the_workloads_read():
    """The default bench line runs the other workloads with a namespace of
    its own: every args.<name> those functions read must be in it (a missing
    one crashes the default run only on a GPU machine)."""
    import ast
    import inspect
    import re
    import bench
    src = inspect.getsource(bench.extra_workloads)
    call = next(n for n in ast.walk(ast.parse(src)) if isinstance(n, ast.Call)
                and getattr(n.func, "attr", "") == "Namespace")
    given = {kw.arg for kw in call.keywords}
    for fn in (bench.run_track, bench.run_map8, bench.run_hires, bench.run_warmstart):
        read = set(re.findall(r"\bargs\.([a-z_]+)", inspect.getsource(fn)))
        assert read <= given, (fn.__name__, sorted(read - given))
