"""CPU checks of the benchmark line's derived fields (no GPU): the roofline
object for each kind of dominant kernel class and the clock-sample summary."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6797.9, "bf16_tflops": 1885.0, "bf16_tflops_sustained": 1715.4}


def _res(dominant, ms=7.2, panel=8):
    prof = {k: (0.1, 5) for k in ("partition", "stage", "kbuild", "potrf", "trsm", "update", "matvec", "precond",
                                  "pcgvec", "predict", "select")}
    prof[dominant] = (ms * 5, 5 * (62 if dominant == "update" else 1))
    w = dict(X=np.zeros((65536, 90)), Xt=np.zeros((8192, 90)), p=16, sigmas=[1.0, 4.0, 16.0],
             lambdas=[1e-6, 1e-4], workload="bkrr2_n65536_t8192_d90_p16")
    return dict(prof=prof, w=w, sizes=[4096] * 16, clocks={"sm_mhz": 2070.0}, panel_width=panel)


def test_roofline_alu_for_the_prediction():
    r = bench.roofline(_res("predict"), 5, PEAKS)
    assert r["kernel"] == "predict" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    peak = 152 * 128 * 2070e6 / 1e12
    assert r["peak"] == pytest.approx(peak)
    pairs = 8192 * 65536
    per_pair = 22 + 3 * (7 + 41) + 6 * 12
    assert r["achieved"] == pytest.approx(pairs * per_pair / 7.2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == bench.TRAFFIC[("predict", "bkrr2_n65536_t8192_d90_p16", 8)]


def test_roofline_tensor_for_the_update_and_traffic_only_at_the_captured_width():
    r = bench.roofline(_res("update", ms=5.3), 5, PEAKS)
    assert r["bound"] == "tensor"
    assert r["peak"] == pytest.approx(1715.4 * 1.1 / 2.25)
    flops = 6 * 16 * 4096 ** 3 / 3.0  # per step: G x p x m^3/3
    assert r["achieved"] == pytest.approx(flops / 5.3e-3 / 1e12)
    assert r["traffic"] is not None
    assert bench.roofline(_res("update", ms=5.3, panel=4), 5, PEAKS)["traffic"] is None


def test_roofline_hbm_for_a_memory_bound_class():
    r = bench.roofline(_res("precond", ms=2.7), 5, PEAKS)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == pytest.approx(6797.9)
    assert 0 < r["frac"] and r["traffic"] is None


def test_host_cpu_reads_x86_and_arm_cpuinfo(tmp_path):
    import bench
    x86 = tmp_path / "x86"
    x86.write_text("processor\t: 0\nmodel name\t: Some CPU @ 2.0GHz\nprocessor\t: 1\nmodel name\t: Some CPU @ 2.0GHz\n")
    arm = tmp_path / "arm"
    arm.write_text("processor\t: 0\nCPU implementer\t: 0x41\nCPU architecture: 8\nCPU part\t: 0xd4f\n")
    assert bench.host_cpu(str(x86))["model"] == "Some CPU @ 2.0GHz"
    assert bench.host_cpu(str(arm))["model"] == "implementer 0x41 part 0xd4f"
    h = bench.host_cpu(str(tmp_path / "missing"))
    assert "model" not in h and h["nproc"] >= 1
