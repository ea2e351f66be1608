"""bench.py's host side on CPU: the reference arm (the CPU oracle) prints the
run contract's single JSON line, and the roofline helpers read the measured
peaks when the file is there and fall back to the stated figures otherwise."""
import json

import bench


def test_reference_arm_prints_one_contract_line(capsys):
    rc = bench.main(["--impl", "reference", "--n", "4000", "--per-object", "200", "--nq", "64",
                     "--k", "10", "--steps", "2", "--warmup", "1", "--ref-sample", "4",
                     "--cpu-sample", "4"])
    assert rc == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["config"]["n_db"] == 4000 and d["config"]["n_queries"] == 64
    assert d["config"]["workload"] == bench.workload_name(bench.parse_args(["--n", "4000",
                                                                            "--per-object", "200",
                                                                            "--nq", "64"]))


def test_peaks_fall_back_then_read_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk = bench.peaks()
    assert pk["kind"] == "fallback"
    assert (pk["hbm_gbs"], pk["bf16_tflops"], pk["bf16_tflops_sustained"]) == (6800.0, 1900.0, 1700.0)
    assert bench.fp8_peak(sustained=True)[0] == 3400.0
    assert bench.fp8_peak(sustained=False)[0] == 3800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(
        json.dumps({"hbm_gbs": 7000, "bf16_tflops": 2000, "bf16_tflops_sustained": 1800}))
    pk = bench.peaks()
    assert pk["kind"] == "measured" and pk["hbm_gbs"] == 7000.0
    peak, kind = bench.fp8_peak(sustained=True)
    assert peak == 3600.0 and "measured" in kind
    assert bench.fp8_peak(sustained=False)[0] == 4000.0


def test_tree_scan_traffic_scales_with_the_rows():
    t, note = bench.tree_scan_traffic(bench.parse_args(["--n", "10000000"]))
    assert t == bench.TREE_SCAN_TRAFFIC["bytes_per_row"] * 10_000_000
    assert "scaled by rows" in note
    # another query batch or k: no capture covers it
    assert bench.tree_scan_traffic(bench.parse_args(["--nq", "5000"])) == (None, None)
    assert bench.tree_scan_traffic(bench.parse_args(["--k", "1"])) == (None, None)
