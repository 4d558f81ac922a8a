"""bench.py's roofline bookkeeping on the host: the integral kernel's bound
weighs compensated and plain-FP32 multiply-adds by their share of the flops,
and roofline.traffic comes from the committed ncu capture only while the
integral kernel's source is the captured one."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def fake_stats(f32_share=0.25):
    return {"flops_eri": 1.0e12, "flops_eri_f32": f32_share * 1.0e12, "eri_values": 1_000_000,
            "flops_half1": 2.0e12, "flops_half2": 1.0e11}


def test_integral_roofline_mix_and_traffic(monkeypatch):
    from paper_2606_04316_gb300 import qdt
    monkeypatch.setattr(qdt, "alu_peak", lambda device, kind: 78.0 if kind == "fp32" else 1.25)
    avg = {"ms_eri": 500.0, "ms_half1": 100.0, "ms_half2": 10.0}
    r = bench.roofline(fake_stats(0.25), avg, qdt.SPLIT, {"sm_mhz": 2070.0}, {"bf16_tflops_sustained": 1700.0},
                       "measured", 0, ["coulomb", "gaunt", "gauge"])
    assert r["kernel"] == "eri_rows_kernel" and r["bound"] == "alu"
    ops = 12 * 0.75 + 1 * 0.25
    assert abs(r["peak"] - 78.0 / ops) < 1e-12
    assert abs(r["achieved"] - 1.0e12 / 0.5 / 1e12) < 1e-12
    per_value, _ = bench.traffic_per_value("eri_rows_kernel")
    if per_value is None:                 # the kernel changed since the capture: no traffic figure
        assert r["traffic"] is None
    else:
        assert abs(r["traffic"] - per_value * 1_000_000) < 1e-6
    assert r["launches_per_step"] == 2


def test_traffic_is_null_for_another_kernel_version(monkeypatch, tmp_path):
    src = tmp_path / "eri.cu"
    src.write_text("// not the captured kernel\n")
    monkeypatch.setattr(bench, "ERI_SOURCE", str(src))
    assert bench.traffic_per_value("eri_rows_kernel") == (None, None)


def test_fp64_form_uses_fp64_peak(monkeypatch):
    from paper_2606_04316_gb300 import qdt
    monkeypatch.setattr(qdt, "alu_peak", lambda device, kind: 78.0 if kind == "fp32" else 1.25)
    avg = {"ms_eri": 500.0, "ms_half1": 100.0, "ms_half2": 10.0}
    r = bench.roofline(fake_stats(), avg, qdt.FP64, {"sm_mhz": 2070.0}, {"bf16_tflops_sustained": 1700.0},
                       "measured", 0, ["coulomb"])
    assert r["peak"] == 1.25 and r["launches_per_step"] == 1
