"""Host-side arithmetic of bench.py (no GPU): the per-class roofline figures
derived from the library profiler's (ms, launches, work) records."""
import pytest

import bench

PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2000.0, "_source": "test"}


def test_class_rooflines_bounds_and_units():
    n, nrhs = 16384, 1
    prof = {
        "panel": (40.0, 683, 4.0e10),        # flops
        "update": (10.0, 42, 2.9e12),        # flops of the FP32-equivalent product
        "trsv": (4.0, 16, 16 * 4.0 * n * n),  # bytes
        "residual": (5.0, 8, 8 * (8.0 * n * n)),
        "rowmoves": (0.0, 0, 0.0),           # not timed: left out
    }
    r = bench.class_rooflines(prof, PEAKS, "fp16x3", n, nrhs)
    assert set(r) == {"panel", "update", "trsv", "residual"}
    fp32 = 152 * 128 * 2 * 2000.0e6 / 1e12
    assert r["panel"]["bound"] == "alu" and r["panel"]["peak"] == pytest.approx(fp32)
    assert r["panel"]["achieved"] == pytest.approx(4.0e10 / 0.040 / 1e12)
    # fp16x3 issues three tensor products per FP32-equivalent one
    assert r["update"]["bound"] == "tensor"
    assert r["update"]["achieved"] == pytest.approx(3 * 2.9e12 / 0.010 / 1e12)
    assert r["trsv"]["bound"] == "hbm" and r["trsv"]["unit"] == "GB/s"
    assert r["trsv"]["achieved"] == pytest.approx(16 * 4.0 * n * n / 0.004 / 1e9)
    # residual: 2 n^2 nrhs FP64 flops per launch against the FP64 pipe
    assert r["residual"]["peak"] == bench.FP64_NOMINAL_TFLOPS
    assert r["residual"]["achieved"] == pytest.approx(8 * 2.0 * n * n / 0.005 / 1e12)
    for v in r.values():
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"])


def test_class_rooflines_fp32_update_is_alu():
    r = bench.class_rooflines({"update": (100.0, 64, 2.9e12)}, PEAKS, "fp32", 16384, 1)
    assert r["update"]["bound"] == "alu"


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """The traffic figure of a class is read from the profile table only while
    the kernel's source file still has the hash recorded at capture time; once
    the file changes, the bench reports no traffic and says why."""
    src = tmp_path / "paper_0808_2794_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "panel.cu").write_text("// kernel source at capture time\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.source_sha16("paper_0808_2794_gb300/csrc/panel.cu")
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.md").write_text(
        "| class | kernel | source | sha16 | workload | launches | bytes/launch |\n|---|---|---|---|---|---|---|\n"
        f"| panel | panel_getf2_kernel | paper_0808_2794_gb300/csrc/panel.cu | {sha} | test | 3 | 2.5e+06 |\n")
    value, why = bench.recorded_traffic("panel")
    assert value == 2.5e6 and "test" in why
    (src / "panel.cu").write_text("// kernel source changed since\n")
    value, why = bench.recorded_traffic("panel")
    assert value is None and "changed" in why
    assert bench.recorded_traffic("no_such_class") == (None, None)
