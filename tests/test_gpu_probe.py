"""The throughput probes that give the measured ALU-roofline denominators
(gsr_probe_fma / gsr_probe_exp) run and report rates that are physically
possible on one GB300: FP32 FMA throughput at most the 152 SMs x 128 lanes x
2 FLOP x 2.07 GHz = 80.5 TFLOP/s the hardware can issue (plus timer slack),
and above a quarter of it; the exp2 rate positive and below 64 per SM per
clock."""
import pytest

torch = pytest.importorskip("torch")

from paper_2312_10070_gb300 import api

pytestmark = pytest.mark.gpu


def test_probes_report_plausible_rates():
    r = api.probe_peaks(blocks=152 * 4, iters=4096, reps=3)
    assert 0.25 * 80.5 < r["fp32_tflops"] < 1.05 * 80.5, r
    assert 0 < r["exp_gps"] < 64 * 152 * 2.07, r
