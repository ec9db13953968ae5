"""The benchmark's host-side contract, on the CPU: the reference arm (the FP64 oracle on the host
cores) prints one JSON line with the keys the driver reads, and the tile-kernel traffic record is
keyed to band.cu's code with comments ignored."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "c1", "--steps", "2",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


def test_code_hash_ignores_comments_and_blank_lines(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f() {\n    return 1;  // one\n}\n")
    b.write_text("// header\n\nint f() {\n    return 1;\n\n}\n")
    assert bench.code_hash(str(a)) == bench.code_hash(str(b))
    b.write_text("int f() {\n    return 2;\n}\n")
    assert bench.code_hash(str(a)) != bench.code_hash(str(b))
    # the recorded traffic belongs to the current tile kernel source, else it is not reported
    rec = bench.TILE_TRAFFIC["c2"]
    current = bench.code_hash(os.path.join(ROOT, "paper_1903_00353_gb300", "csrc", "band.cu"))
    assert (bench.tile_traffic("c2", True) == rec["bytes"]) == (current == rec["band_cu_code_hash"])
    assert bench.tile_traffic("c2", False) is None
