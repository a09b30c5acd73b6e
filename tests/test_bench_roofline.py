"""The benchmark's roofline arithmetic on CPU: the algorithmic bytes of a CG
apply (read x, write y: 24 B per node; the modulus: 4 B per element), the
achieved bandwidth and its fraction of the peak, the executed-operation FP32
floor, and which kernel and operation count each operator choice reports."""
import pytest

import bench
from paper_2605_04735_gb300 import inputs as I


def test_operator_bytes_count_nodes_and_elements():
    w = I.WORKLOADS["mbb_96x32x32"]
    assert w.n_nodes == 97 * 33 * 33 and w.n_elem == 96 * 32 * 32
    assert bench.operator_bytes(w) == 24 * 97 * 33 * 33 + 4 * 96 * 32 * 32


def test_hbm_roofline_is_bytes_over_time_over_peak():
    w = I.WORKLOADS["mbb_96x32x32"]
    peaks = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}
    nbytes, ms = 3.0e6, 0.002  # 3 MB in 2 us: 1.5 TB/s
    r = bench.hbm_roofline("k", w, nbytes, ms, 1.0, peaks, "measured", traffic=3.1e6, ops=250.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(1500.0)
    assert r["frac"] == pytest.approx(0.25)
    assert r["hbm_floor_us"] == pytest.approx(0.5)
    assert r["traffic"] == 3.1e6
    # 98,304 elements x 250 lane-operations over 152 SMs x 128 lanes x 2 GHz
    floor_us = w.n_elem * 250.0 / (152 * 128 * 2.0e9) * 1e6
    assert r["alu_view"]["executed_floor_us"] == pytest.approx(floor_us)
    assert r["alu_view"]["executed_frac_of_fp32_pipe"] == pytest.approx(floor_us / 2.0)
    # no operation count: no executed floor
    assert "executed_floor_us" not in bench.hbm_roofline("k", w, nbytes, ms, 1.0, peaks,
                                                         "measured")["alu_view"]


def test_executed_operation_counts_follow_the_kernel_choice():
    small, large = 96, 320  # the one-column and the paired kernel (nx >= 150)
    assert bench.exec_ops(0, small, "cheb_step") == bench.EXEC_FP32_OPS_PER_ELEM["cheb_step"]
    assert bench.exec_ops(0, small, "cg_apply") == bench.EXEC_FP32_OPS_PER_ELEM["cg_apply_tma"]
    assert bench.exec_ops(0, large, "cg_apply") == bench.EXEC_FP32_OPS_PER_ELEM["cg_apply_pair"]
    assert bench.exec_ops(0, large, "cheb_step") is None  # not counted for the paired kernel
    for op in (1, 2, 3, 4, 5):  # the other forms are not counted
        assert bench.exec_ops(op, small, "cg_apply") is None
    assert bench.operator_kernel(0, small).startswith("k_modal_tma")
    assert bench.operator_kernel(0, large).startswith("k_modal_pair")
    assert bench.operator_kernel(4, small).startswith("k_tc_tma")
    assert "cluster" in bench.operator_kernel(5, small)


def test_clock_summary_reads_clocks_reasons_and_power():
    """nvidia-smi CSV rows (index, SM clock, max SM clock, power, active
    reasons, then the four reasons the timing rules name) become the median
    and minimum SM clock, the reasons seen active and the power figures;
    malformed rows are skipped."""
    clk = bench.ClockSampler(0)
    clk.lines = [
        "0, 2070, 2070, 800.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 850.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1965, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    s = clk.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_min_mhz"] == 1965.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert s["power_w_median"] == pytest.approx(850.0) and s["power_w_max"] == 900.0
    empty = bench.ClockSampler(0).summary()
    assert empty["reasons"] == ["unsampled"] and empty["sm_mhz"] is None


def test_reference_arm_prints_one_line_of_the_contract(capsys):
    """`bench.py --impl reference` on the smallest workload: one JSON line
    with the metric, unit and config of our arm, the oracle as its
    cpu_baseline, an e2e of the same value with no host-device bytes, and
    no GPU launch (the oracle is host code)."""
    import argparse
    import json
    w = I.WORKLOADS["cantilever_24x12x12"]
    bench.run_reference(argparse.Namespace(steps=1, warmup=0), w)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["gpu_launches"] == 0
    assert line["config"]["workload"] == w.name
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
