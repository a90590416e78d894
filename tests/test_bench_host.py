"""CPU tests of bench.py's host logic: workload specs, the traffic record's guards, peaks,
the fixed-tuning option and the whole-job arithmetic (no GPU)."""
import argparse
import hashlib
import os

import pytest

import bench


def _args(**kw):
    base = dict(workload="grid3d", size=0, k=0, iters=0, dtype="", tuning="")
    base.update(kw)
    return argparse.Namespace(**base)


def test_default_workload_is_the_400_cubed_grid():
    spec = bench.workload_spec(_args())
    assert (spec["N"], spec["b"], spec["k"], spec["iters"], spec["rescale"], spec["dtype"]) == (400, 4096, 16, 20, True, "f32")
    assert bench.workload_key(spec) == "grid3d N=400 k=16 f32 rescale=1"
    r = bench.workload_spec(_args(workload="rmat"))
    assert (r["N"], r["b"], r["k"], r["iters"], r["dtype"]) == (23, 8192, 128, 8, "bf16")


def test_traffic_record_matches_source_and_workload():
    spec = bench.workload_spec(_args())
    tr = bench.kernel_traffic(bench.workload_key(spec))
    digest = bench.kernel_source_digest()
    if tr is None:
        pytest.skip("traffic record taken on another kernel source")      # reported as null then
    assert tr["kernel_source_sha256_16"] == digest
    dram = float(tr["dram_bytes_per_launch_full_size"])
    alg = float(tr["algorithmic_bytes_per_launch_full_size"])
    assert dram == pytest.approx(float(tr["dram_bytes_read_per_launch_full_size"]) +
                                 float(tr["dram_bytes_write_per_launch_full_size"]), rel=1e-6)
    assert 0.5 < dram / alg < 1.5
    # any other workload (or size) gets no traffic figure
    for other in (_args(size=200), _args(k=32), _args(workload="grid2d")):
        assert bench.kernel_traffic(bench.workload_key(bench.workload_spec(other))) is None


def test_traffic_guard_rejects_a_changed_source(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("// another kernel\n")
    monkeypatch.setattr(bench, "KERNEL_SRCS", [str(src)])
    assert bench.kernel_traffic("grid3d N=400 k=16 f32 rescale=1") is None
    assert bench.kernel_traffic("rmat N=23 k=128 bf16 rescale=0") is None


def test_traffic_record_blocks_are_parsed_per_workload(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    d = bench.kernel_source_digest()
    (prof / "arrow_rows_traffic.txt").write_text(
        "# header\nworkload: A\nkernel_source_sha256_16: %s\ndram_bytes_per_launch_full_size: 1\n"
        "workload: B\nkernel_source_sha256_16: 0000\ndram_bytes_per_launch_full_size: 2\n"
        "workload: C\nkernel_source_sha256_16: %s\ndram_bytes_per_launch_full_size: 3\n" % (d, d))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("A")["dram_bytes_per_launch_full_size"] == "1"
    assert bench.kernel_traffic("B") is None                          # taken on another source
    assert bench.kernel_traffic("C")["dram_bytes_per_launch_full_size"] == "3"
    assert bench.kernel_traffic("D") is None


def test_fixed_tuning_parse():
    assert bench.fixed_tuning(_args()) is None
    assert bench.fixed_tuning(_args(tuning="384,3072,3,85")) == (384, 3072, 3, 85)
    with pytest.raises(SystemExit):
        bench.fixed_tuning(_args(tuning="384,3072"))


def test_peaks_and_job_value():
    peak, kind = bench.load_peaks()
    assert peak > 1000 and kind in ("measured", "fallback")
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured"
    # whole-job throughput: every rank's units over the slowest rank's time
    assert bench.job_value(20, 4, 100.0) == pytest.approx(800.0)
    assert bench.max_over_ranks(None, 3.5) == 3.5


def test_reference_arm_prints_the_contract_line():
    # the reference arm times the CPU oracle only: it runs here, without a GPU, and prints one
    # JSON line with the keys the benchmark contract names
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "grid2d", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                         cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_subrecords_collect_child_lines_and_errors(monkeypatch):
    # the default run attaches the other configurations by running bench.py as child processes;
    # here the children are the CPU-only reference arm (a line comes back) and an unknown option
    # (the error is recorded, not raised)
    monkeypatch.setattr(bench, "SUBRECORDS", [
        ("ok", ["--impl", "reference", "--workload", "grid2d", "--steps", "1", "--warmup", "0"]),
        ("bad", ["--no-such-option"]),
        ("skipped", ["--impl", "reference"]),
    ])
    recs = bench.run_subrecords(["ok", "bad"], timeout_s=600)
    assert set(recs) == {"ok", "bad"}
    assert recs["ok"]["impl"] == "reference" and recs["ok"]["value"] > 0 and recs["ok"]["wall_s"] > 0
    assert "error" in recs["bad"] and recs["bad"]["error"].startswith("rc=")


def test_every_default_subrecord_is_a_known_workload():
    # the children's arguments parse: each names a workload bench.py knows
    for key, args in bench.SUBRECORDS:
        wl = args[args.index("--workload") + 1]
        assert wl in ("grid2d", "rmat", "batch", "serve", "predicates"), (key, wl)
    assert [k for k, _ in bench.SUBRECORDS] == ["grid2d", "rmat", "batch", "serve", "predicates"]
