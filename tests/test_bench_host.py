"""CPU checks of the benchmark's host-side bookkeeping: the clock log summary
(median SM clock, throttle reasons), the roofline peak lookup and the rule
that the ncu traffic figure is reported only for the kernel source it was
measured on."""
import json
import os

import bench


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.out = "\n".join(lines)
    return s


def test_clock_summary_median_max_and_reasons():
    na = "Not Active"
    rows = [
        f"0, 2070, 2070, 900.1, 0x0, {na}, {na}, {na}, {na}",
        f"0, 1980, 2070, 1400.0, 0x4, {na}, {na}, {na}, Active",
        f"0, 2055, 2070, 1200.5, 0x0, {na}, {na}, {na}, {na}",
        "",
        "0, [N/A], 2070, [N/A], 0x0, [N/A], [N/A], [N/A], [N/A]",   # unreadable sample
        "garbage",
    ]
    out = _sampler(rows).summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_hw_slowdown():
    na = "Not Active"
    rows = [f"0, 1500, 2070, 800, 0x8, Active, {na}, Active, {na}"]
    out = _sampler(rows).summary()
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    out = _sampler([]).summary()
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_peak_is_the_measured_copy_bandwidth(tmp_path, monkeypatch):
    val, kind = bench._peaks()
    d = json.load(open(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")))
    assert (val, kind) == (float(d["hbm_gbs"]), "measured")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")


def test_code_digest_ignores_comments_and_whitespace_only(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("// header\n__global__ void k(float* x) { x[0] = 1.0f; }  /* a\nb */\n")
    b = tmp_path / "b.cu"
    b.write_text("// another header\n__global__ void k(float* x)\n{\n    x[0] = 1.0f;   // set\n}\n")
    c = tmp_path / "c.cu"
    c.write_text("__global__ void k(float* x) { x[0] = 2.0f; }\n")
    assert bench.code_digest(a) == bench.code_digest(b)
    assert bench.code_digest(a) != bench.code_digest(c)


def test_traffic_record_only_for_the_measured_source(tmp_path, monkeypatch):
    src = tmp_path / "paper_1606_04004_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "apply_h.cu").write_text("// kernel v1\nint k;\n")
    rec = {"apply_code_sha256": bench.apply_digest(str(tmp_path)),
           "dram_bytes_per_coef": 100.0}
    (tmp_path / "profiles" / "apply_h_hh6d_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_record()["dram_bytes_per_coef"] == 100.0
    (src / "apply_h.cu").write_text("// kernel v1, comment edited\nint  k;\n")
    assert bench._traffic_record()["dram_bytes_per_coef"] == 100.0
    (src / "apply_h.cu").write_text("// kernel v2\nint k2;\n")      # code changed since
    assert bench._traffic_record() is None
    os.remove(tmp_path / "profiles" / "apply_h_hh6d_traffic.json")
    assert bench._traffic_record() is None


def test_committed_traffic_record_matches_the_kernel_source():
    # the committed counters were taken on the H.psi kernels as they are now
    rec = bench._traffic_record()
    assert rec is not None, ("the H.psi sources changed since the ncu traffic capture: "
                             "re-take it, or the bench reports traffic as null")
    assert 20 < rec["dram_bytes_per_coef"] < 200


def test_algorithmic_bytes_per_coefficient():
    # psi read + H.psi write + index: 8 + 8 + 4 (complex64), 16 + 16 + 4 (complex128)
    assert bench.BYTES_PER_COEF == {"fp32mix": 20, "fp64": 36}
