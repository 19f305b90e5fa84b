"""The bench's roofline arithmetic (host logic, no GPU): each kernel class's algorithmic work
per unit times the plan's unit counts, over the class's time, against the measured peak."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

# the 64-water plan's unit counts and the measured peaks
INFO = {"sum_mn": 2.451e9, "sum_mn2": 9.557e11, "sum_ms": 9.615e8, "sum_n2": 5.071e9}
PEAKS = {"hbm_gbs": 6687.1, "bf16_tflops": 1936.0}
ALU = {"fp32_tflops": 78.4, "fp64_tflops": 1.254, "source": "measured"}


def _r(kind, ms, form="mixed"):
    return bench.roofline(kind, ms, form, INFO, PEAKS, "measured", ALU)


def test_contractions_at_the_split_bf16_count_and_issued():
    r = _r("vgemm", 35.1)
    assert r["bound"] == "tensor"
    assert abs(r["achieved"] - 3 * 2 * 9.557e11 / 35.1e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 1936.0) < 1e-12
    assert abs(r["issued"]["frac"] - 5 * r["frac"]) < 1e-12   # 15 slice products against 3


def test_float64_contractions_against_the_float64_pipe():
    r = _r("xgemm", 183.0, "fp64")
    assert r["bound"] == "alu" and r["peak"] == 1.254
    assert abs(r["achieved"] - 2 * 9.557e11 / 0.183 / 1e12) < 1e-9


def test_streaming_kernels_at_their_stored_widths():
    # rho_mixed reads X (8 B), Phi (8 B) and grad Phi (12 + 6 B); z_slice reads Phi (8 B) and
    # the grad Phi hi words (12 B) and writes the Z slices (5 x 2 B)
    assert abs(_r("rho_z", 14.5)["achieved"] - 34 * 2.451e9 / 14.5e-3 / 1e9) < 1e-6
    assert abs(_r("vslice", 14.8)["achieved"] - 30 * 2.451e9 / 14.8e-3 / 1e9) < 1e-6
    assert abs(_r("pgather", 11.5)["achieved"] - 8 * 5.071e9 / 11.5e-3 / 1e9) < 1e-6


def test_collocation_against_the_float32_pipe():
    r = _r("colloc", 28.1)
    assert r["bound"] == "alu" and r["peak"] == 78.4
    assert abs(r["achieved"] - 28 * 9.615e8 / 28.1e-3 / 1e12) < 1e-12


def test_unknown_or_untimed_class_has_no_roofline():
    assert _r("weights", 5.0)["frac"] is None
    assert _r("vgemm", 0.0)["frac"] is None
