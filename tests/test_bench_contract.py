"""CPU checks of the benchmark line's derived fields (no GPU): the roofline
object for each kind of dominant kernel class and the clock-sample summary."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6797.9, "bf16_tflops": 1885.0, "bf16_tflops_sustained": 1715.4}


def _res(dominant, ms=7.2, classes=None):
    prof = {k: (0.1 * 5, 5) for k in ("partition", "stage", "kbuild", "potrf", "trsm", "update", "matvec",
                                      "precond", "pcgvec", "predict", "select")}
    prof[dominant] = (ms * 5, 5 * (62 if dominant == "update" else 1))
    w = dict(X=np.zeros((65536, 90)), Xt=np.zeros((8192, 90)), p=16, sigmas=[1.0, 4.0, 16.0],
             lambdas=[1e-6, 1e-4], workload="bkrr2_n65536_t8192_d90_p16")
    cls = np.array(classes if classes is not None else [1] * 96, np.int32)
    return dict(prof=prof, nprof=5, w=w, sizes=[4096] * 16, clocks={"sm_mhz": 2070.0}, panel_width=8,
                classes=cls)


def test_prediction_stage_against_section_8d_work(monkeypatch):
    res = _res("predict")
    st = bench.stage_rooflines(res, PEAKS)["predict"]
    pairs = 8192 * 65536
    sec = 7.2e-3
    assert st["tensor_frac"] == pytest.approx(pairs * 180 / sec / 1e12 / 1885.0)
    mufu = 152 * 16 * 2070e6 / 1e9
    assert st["mufu_frac"] == pytest.approx(pairs * 3 / sec / 1e9 / mufu)
    assert st["hbm_frac"] == pytest.approx((16 * 8192 + 65536) * 90 * 8 / sec / 1e9 / 6797.9)
    assert st["binding"] == "mufu" and st["frac"] == pytest.approx(st["mufu_frac"])
    r = bench.roofline(res, bench.stage_rooflines(res, PEAKS), PEAKS)
    assert r["kernel"] == "predict" and r["bound"] == "alu" and r["unit"] == "Gexp/s"
    assert r["frac"] == pytest.approx(st["mufu_frac"])
    assert r["impl_alu_frac"] == pytest.approx(pairs * 238 / sec / (152 * 128 * 2070e6))
    # the captured traffic is used only for the kernel source it was taken on
    key = ("predict", "bkrr2_n65536_t8192_d90_p16", bench._source_sha("predict"))
    assert r["traffic"] == bench.TRAFFIC.get(key)
    monkeypatch.setattr(bench, "_source_sha", lambda kind: "0" * 16)
    assert bench.roofline(res, bench.stage_rooflines(res, PEAKS), PEAKS)["traffic"] is None


def test_factor_stage_charges_each_solve_at_its_class_peak():
    cls = [1] * 80 + [3] * 16
    res = _res("update", ms=5.3, classes=cls)
    st = bench.stage_rooflines(res, PEAKS)["factor"]
    m = 4096
    need = 80 * (m ** 3 / 3) / 1885e12 + 16 * (m ** 3 / 3) / (1885e12 * 1.1 / 2.25)
    sec = (0.1 + 0.1 + 5.3) / 1e3
    assert st["frac"] == pytest.approx(need / sec)
    assert st["classes"] == {"1": 80, "3": 16}
    r = bench.roofline(res, bench.stage_rooflines(res, PEAKS), PEAKS)
    assert r["bound"] == "tensor" and r["kernel"] == "update"
    tot, potrf, trsm, upd = bench.factor_flops(m)
    assert tot == pytest.approx(potrf + trsm + upd)
    assert r["achieved"] == pytest.approx(96 * upd / 5.3e-3 / 1e12)
    upd_need = 80 * upd / 1885e12 + 16 * upd / (1885e12 * 1.1 / 2.25)
    assert r["frac"] == pytest.approx(upd_need / 5.3e-3)


def test_kernel_build_stage_and_unmeasured_classes():
    res = _res("kbuild", ms=2.2)
    st = bench.stage_rooflines(res, PEAKS)["kbuild"]
    ent = 16 * 4096 ** 2 / 2 * 3
    assert st["hbm_frac"] == pytest.approx(ent * 4 / 2.2e-3 / 1e9 / 6797.9)
    r = bench.roofline(res, bench.stage_rooflines(res, PEAKS), PEAKS)
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(st["hbm_frac"])
    r2 = bench.roofline(_res("precond", ms=2.7), {}, PEAKS)
    assert r2["frac"] is None and r2["traffic"] is None


def test_traffic_is_dropped_when_the_kernel_source_changes(monkeypatch):
    res = _res("predict")
    sha = bench._source_sha("predict")
    monkeypatch.setitem(bench.TRAFFIC, ("predict", "bkrr2_n65536_t8192_d90_p16", sha), 123)
    assert bench.roofline(res, bench.stage_rooflines(res, PEAKS), PEAKS)["traffic"] == 123
    monkeypatch.setattr(bench, "_source_sha", lambda k: "0" * 16)
    assert bench.roofline(res, bench.stage_rooflines(res, PEAKS), PEAKS)["traffic"] is None


def test_accuracy_vs_oracle_reports_the_worst_sampled_solve():
    pairs = [(0, 1), (1, 0)]
    refs = [dict(alpha=np.array([1.0, 2.0]), yhat=np.array([1.0, -1.0]), mse=0.5, kappa=10.0),
            dict(alpha=np.array([4.0]), yhat=np.array([2.0, 2.0]), mse=0.25, kappa=1e6)]
    gpu = {"tf32": {"failed": 0, (0, 1): (np.array([1.0, 2.0 + 2e-7]), np.array([1.0, -1.0]), 0.5),
                    (1, 0): (np.array([4.0 + 4e-6]), np.array([2.0, 2.0 + 2e-9]), 0.25 * (1 + 3e-8))}}
    acc = bench.accuracy_vs_oracle(gpu, refs, pairs)["tf32"]
    assert acc["max_rel_err_alpha"] == pytest.approx(1e-6)
    assert acc["max_rel_err_pred"] == pytest.approx(1e-9)
    assert acc["max_rel_err_mse"] == pytest.approx(3e-8)
    assert acc["worst_alpha_model"] == [1, 0] and acc["worst_alpha_kappa"] == 1e6


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
