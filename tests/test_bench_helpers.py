"""Host-side helpers of bench.py: the kernel-code digest that keys the
recorded DRAM traffic, and the lookup of that record.  No GPU needed."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_digest_ignores_comments_and_whitespace():
    a = bench.code_digest(["int f(int x) { return x + 1; }\n"])
    b = bench.code_digest(["// a note\nint f(int x)\n{\n    return x + 1;   /* another\n note */\n}\n"])
    assert a == b


def test_digest_follows_code():
    a = bench.code_digest(["int f(int x) { return x + 1; }"])
    assert a != bench.code_digest(["int f(int x) { return x + 2; }"])
    assert a != bench.code_digest(["int f(int x) { return x + 1; }", "int g;"])


def test_digest_keeps_the_boundary_between_tokens():
    # a comment between two tokens must not glue them together
    assert bench.code_digest(["int/**/x;"]) == bench.code_digest(["int x;"])
    assert bench.code_digest(["int x;"]) != bench.code_digest(["intx;"])


def test_traffic_lookup_matches_kernel_and_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    want = bench.kernel_source_hash()
    (prof / "traffic.txt").write_text(
        "# comment line\n"
        f"sweep_tiled_kernel<5,64,16>@512 {want} 2100000000 ncu-test\n"
        f"sweep_tiled_kernel<5,64,16,__half>@512 0000000000000000 1500000000 ncu-stale\n")
    # the lookup reads the record under ROOT, the hash from the real sources
    real_hash = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: real_hash)
    assert bench.profiled_traffic("sweep_tiled_kernel<5,64,16>@512") == (2100000000.0, "ncu-test")
    # another kernel's line, taken on other code: no traffic
    assert bench.profiled_traffic("sweep_tiled_kernel<5,64,16,__half>@512") == (None, None)
    assert bench.profiled_traffic("sweep_tiled_kernel<4,64,16>@512") == (None, None)


def test_recorded_traffic_is_near_the_algorithmic_bytes():
    """Every line of the committed record: DRAM bytes of one 512^3 launch
    within 10 % of the kernel's algorithmic bytes (16 B per point for FP32,
    12 B for the 16-bit storage)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    n = 512 ** 3
    seen = 0
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if line.startswith("#") or len(parts) < 4:
                continue
            tag, _, traffic = parts[0], parts[1], float(parts[2])
            per = 12.0 if ("__half" in tag or "bfloat16" in tag) else 16.0
            assert tag.endswith("@512")
            assert abs(traffic / (per * n) - 1.0) < 0.10, tag
            seen += 1
    assert seen >= 1


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) on a
    small shot: one JSON line with the contract's keys, its cpu_baseline and
    e2e describing the same run, and a sample no longer than the shot."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "24",
                        "--timesteps", "4", "--steps", "2", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["sample_timesteps_per_step"] == 4
    assert "first 4 of 4" in line["cpu_baseline"]["sample"]
