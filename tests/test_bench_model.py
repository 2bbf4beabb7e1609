"""Host logic of bench.py: the algorithmic byte model behind the roofline
fraction, checked against per-sweep byte counts written out by hand
(a whole smoothing sweep moves x twice, b once and every stored coefficient
array once; a colour pass is charged 1/C of a sweep), and the half-size
traffic scaling."""
import json
import os

import pytest

import bench

N2 = 128 * 128 * 256          # the 128 x 128 x 256 bench grid
N2C = 64 * 128 * 256          # its first coarse level (radius halved)


def test_sweep_bytes_follow_the_table():
    # x read + written, b read, coefficients: 7 points FP32 4+4+4+12
    assert bench.sweep_bytes_per_cell(7, 1) == 24
    assert bench.sweep_bytes_per_cell(19, 1, ncomp=9) == 48        # 4+4+4+36
    assert bench.sweep_bytes_per_cell(19, 2, ncomp=9) == 30        # FP16 coefficients 4+4+4+18
    assert bench.sweep_bytes_per_cell(7, 0) == 48                  # FP64
    assert bench.sweep_bytes_per_cell(19, 0, ncomp=9) == 96
    # the axisymmetric operator stores five arrays
    assert bench.sweep_bytes_per_cell(19, 1, axi=True) == 32
    assert bench.sweep_bytes_per_cell(19, 2, axi=True) == 22


def test_colour_pass_is_a_fraction_of_the_sweep():
    # 7 points: two colour passes per sweep, 12 B per cell each
    assert bench.algorithmic_bytes("smooth0", 7, 1, N2, N2C) == pytest.approx(12 * N2)
    assert bench.algorithmic_bytes("smooth0", 7, 1, N2, N2C) == pytest.approx(50.331648e6)
    # a one-pass sweep is charged the whole sweep
    assert bench.algorithmic_bytes("smooth0", 7, 1, N2, N2C, passes_per_sweep=1) == pytest.approx(24 * N2)
    # 19 points: four colour passes
    assert bench.algorithmic_bytes("smooth0", 19, 1, N2, N2C) == pytest.approx(12 * N2)
    assert bench.algorithmic_bytes("smooth0", 19, 1, N2, N2C, axi=True) == pytest.approx(8 * N2)
    assert bench.algorithmic_bytes("smooth0", 19, 2, N2, N2C, axi=True) == pytest.approx(5.5 * N2)


def test_line_pass_adds_the_factors():
    base = bench.algorithmic_bytes("smooth0", 7, 1, N2, N2C)
    line = bench.algorithmic_bytes("smooth0", 7, 1, N2, N2C, smoother=2)
    assert line - base == pytest.approx(3 * 4 * N2 / 2)


def test_outer_residual_bytes():
    # x64 8 + b64 8 + FP64 coefficients + r32 4
    # FP32 cycles: + the FP32 residual written and the fine correction cleared
    assert bench.algorithmic_bytes("residual", 7, 1, N2, N2C) == pytest.approx(N2 * (8 + 8 + 24 + 8))
    assert bench.algorithmic_bytes("residual", 19, 1, N2, N2C) == pytest.approx(N2 * (8 + 8 + 72 + 8))
    assert bench.algorithmic_bytes("residual", 19, 1, N2, N2C, axi=True) == pytest.approx(N2 * (8 + 8 + 40 + 8))
    assert bench.algorithmic_bytes("residual", 7, 0, N2, N2C) == pytest.approx(N2 * (8 + 8 + 24))


def test_transfer_and_update_bytes():
    # residual + restriction: x, b, coefficients, coarse right side (20.5 B per fine cell at FP32)
    assert bench.algorithmic_bytes("restrict0", 7, 1, N2, N2C) == pytest.approx(N2 * (8 + 12) + 4 * N2C)
    assert bench.algorithmic_bytes("prolong0", 7, 1, N2, N2C) == pytest.approx(8 * N2 + 4 * N2C)
    assert bench.algorithmic_bytes("update", 7, 1, N2, N2C) == pytest.approx(20 * N2)


def test_traffic_lookup_scales_a_half_size_capture():
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    d = json.load(open(path))
    e = d.get("single_oblate_256/2/fp32/smooth0")
    if not e or e.get("source_hash") != bench.kernel_source_hash(tuple(e.get("sources", bench.BATCH_SOURCES))):
        pytest.skip("no capture for the current kernel sources")
    assert bench.ncu_traffic("single_oblate_256", "fp32", "smooth0") == pytest.approx(8 * e["dram_bytes_per_launch"])


def test_event_cross_check_uses_the_same_bytes():
    """The CUDA-event figure beside the clocks: the same algorithmic bytes over
    the events' mean launch time."""
    roof = {"algorithmic_bytes_per_launch": 50.0e6, "peak": 5000.0}
    prof = {"events": {"smooth0": {"avg_ms": 0.02}, "residual": {"avg_ms": None}}}
    bench.add_event_check(roof, prof, "smooth0")
    assert roof["avg_launch_ms_events"] == 0.02
    assert roof["frac_events"] == pytest.approx(50.0e6 / 20e-6 / 1e9 / 5000.0)
    roof2 = {"algorithmic_bytes_per_launch": 1.0, "peak": 1.0}
    bench.add_event_check(roof2, prof, "residual")    # no events figure: nothing added
    assert "frac_events" not in roof2
