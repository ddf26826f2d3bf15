"""The JSON line of `bench.py --impl reference` (the FP64 oracle timed on
the host cores), run on CPU: one line with the keys a reader of the bench
output relies on, its end-to-end figure equal to its own value, and no
host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_complete_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small",
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == "MLUPS" and line["unit"] == "MLUPS"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 0
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert line["config"]["workload"] and line["config"]["cells"] == 32 ** 3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    e = line["e2e"]
    assert e["value"] == line["value"] and e["unit"] == line["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_l2_note_tells_resident_from_streamed_inputs():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.l2_note(4194304 * 19 * 4).startswith("inputs larger than L2")    # 256x128x128 FP32: 319 MB
    assert bench.l2_note(4194304 * 19 * 2).startswith("inputs larger than L2")    # FP16 offsets: 159 MB
    assert bench.l2_note(32768 * 19 * 8).startswith("inputs fit in L2")           # 32^3 FP64: 5 MB


def test_recorded_sweep_traffic_matches_its_profile():
    """Every recorded DRAM traffic figure names a committed profile summary
    that states the same per-launch bytes (to the summary's precision)."""
    sys.path.insert(0, ROOT)
    import bench
    for (workload, prec), rec in bench.SWEEP_TRAFFIC.items():
        path = os.path.join(ROOT, rec["profile"])
        assert os.path.isfile(path), rec["profile"]
        text = open(path).read()
        mb = rec["bytes"] / 1e6
        shown = {f"{mb:.1f} MB", f"{mb / 1e3:.2f} GB"}
        assert any(s in text for s in shown), (workload, prec, shown)
        assert len(rec["src"]) == 16 and int(rec["src"], 16) >= 0
