"""Host logic of bench.py: the algorithmic byte model behind the roofline
fraction (each array a launch needs moved once), checked against the counts
written out by hand, and the half-size traffic scaling."""
import json
import os

import pytest

import bench

N2 = 128 * 128 * 256          # the 128 x 128 x 256 bench grid
N2C = 64 * 128 * 256          # its first coarse level (radius halved)


def test_seven_point_colour_pass_bytes():
    # x read (4 B) + b and x of the updated half (2 x 4 B / 2) + three G arrays (12 B)
    assert bench.algorithmic_bytes("smooth0", 7, 1, N2, N2C) == pytest.approx(N2 * (4 + 4 + 12))
    assert bench.algorithmic_bytes("smooth0", 7, 1, N2, N2C) == pytest.approx(83.886080e6)


def test_nineteen_point_colour_pass_bytes():
    # 18 coefficients of the updated quarter, or 10 with the axisymmetric operator
    full = bench.algorithmic_bytes("smooth0", 19, 1, N2, N2C)
    axi = bench.algorithmic_bytes("smooth0", 19, 1, N2, N2C, axi=True)
    assert full == pytest.approx(N2 * (4 + 2 + 18))
    assert axi == pytest.approx(N2 * (4 + 2 + 10))


def test_line_pass_adds_the_factors_of_the_updated_cells():
    base = bench.algorithmic_bytes("smooth0", 7, 1, N2, N2C)
    line = bench.algorithmic_bytes("smooth0", 7, 1, N2, N2C, smoother=2)
    assert line - base == pytest.approx(3 * 4 * N2 / 2)


def test_outer_residual_bytes():
    # x 8 + b 8 + FP64 rows + r32 4: 7-point rows = 3 faces + centre
    assert bench.algorithmic_bytes("residual", 7, 1, N2, N2C) == pytest.approx(N2 * (8 + 8 + 32 + 4))
    assert bench.algorithmic_bytes("residual", 19, 1, N2, N2C) == pytest.approx(N2 * (8 + 8 + 152 + 4))
    assert bench.algorithmic_bytes("residual", 19, 1, N2, N2C, axi=True) == pytest.approx(N2 * (8 + 8 + 88 + 4))
    assert bench.algorithmic_bytes("residual", 7, 0, N2, N2C) == pytest.approx(N2 * (8 + 8 + 32))


def test_transfer_and_update_bytes():
    assert bench.algorithmic_bytes("restrict0", 7, 1, N2, N2C) == pytest.approx(N2 * (8 + 12) + 8 * N2C)
    assert bench.algorithmic_bytes("prolong0", 7, 1, N2, N2C) == pytest.approx(8 * N2 + 4 * N2C)
    assert bench.algorithmic_bytes("update", 7, 1, N2, N2C) == pytest.approx(20 * N2)


def test_traffic_lookup_scales_a_half_size_capture():
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    d = json.load(open(path))
    e = d.get("single_oblate_256/2/fp32/smooth0")
    if not e or e.get("source_hash") != bench.kernel_source_hash():
        pytest.skip("no capture for the current kernel sources")
    assert bench.ncu_traffic("single_oblate_256", "fp32", "smooth0") == pytest.approx(8 * e["dram_bytes_per_launch"])
