"""Accounting of the benchmark (no GPU needed): the per-element counts behind
the metric and the rooflines, against the closed forms they stand for."""

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_dof_per_element_closed_form():
    # D_e = 3 N3(p) + 3 N3(p-1): 90, 165, 420 at p = 3, 4, 6 (E of degree p, H of degree p-1)
    assert [bench.dof_per_elem(p) for p in (3, 4, 6)] == [90, 165, 420]
    assert bench.n3(6) == 84 and bench.n3(5) == 56 and bench.n2(6) == 28


def test_dense_flops_per_element_step():
    # 24 N3(p-1) N3(p) + 32 (N2(p) N3(p) + N2(p-1) N3(p-1)); 225,792 at p = 6
    assert bench.flops_per_elem_step(6) == 24 * 56 * 84 + 32 * (28 * 84 + 21 * 56) == 225792
    # per DoF: about 146, 242 and 538 flop at p = 3, 4, 6
    per_dof = [bench.flops_per_elem_step(p) / bench.dof_per_elem(p) for p in (3, 4, 6)]
    assert [round(x) for x in per_dof] == [146, 242, 538]


def test_alu_roofline_arithmetic():
    class W:
        nt, p = 196608, 6
    r = bench.alu_roofline(W, 83.76)
    assert r["dense_equivalent"]["flops_per_element_step"] == 225792
    expect = W.nt * 225792 / 83.76e-3 / 1e12
    assert abs(r["achieved"] - expect) < 1e-12 and r["unit"] == "TFLOP/s" and r["bound"] == "alu"
    assert abs(r["frac"] - expect / r["peak"]) < 1e-12
    # without a GPU the measurement fails and the nominal rate is used, saying so
    if "measured" not in r["peak_source"]:
        assert r["peak"] == bench.FP64_NOMINAL_TFLOPS and "nominal" in r["peak_source"]


def test_measured_hbm_peak_is_read_from_the_measurement_file():
    peak, src = bench.measured_peak_hbm()
    if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")):
        assert src == "measured" and peak > 1000
    else:
        assert src == "fallback" and peak == 6800.0


def test_phase_bytes_at_the_default_workload():
    # planewave_n32_p6 in fp32 state: 478.9 MB per H-phase, 545.0 MB per E-phase
    bh, be = bench.phase_bytes(196608, 6, 4)
    assert bh == 196608 * (4 * (3 * 84 + 6 * 56) + 84) and round(bh / 1e6, 1) == 478.9
    assert be == 196608 * (4 * (6 * 84 + 3 * 56) + 84) and round(be / 1e6, 1) == 545.0
    # one step: 3 b D_e + 2 (g + c) per element
    assert bh + be == 196608 * (3 * 4 * bench.dof_per_elem(6) + 2 * 84)


def test_executed_flops_of_the_trace_buffer_kernels():
    # p = 6 dense: 2 x (2 x 6 x 56 x 84 + 20 x 21 x (56 + 84)) = 230,496 flops per element and step
    assert bench.executed_flops_per_elem_step(6, False) == 2 * (2 * 6 * 56 * 84 + 20 * 21 * 140) == 230496
