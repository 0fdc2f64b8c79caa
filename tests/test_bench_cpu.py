"""bench.py's reference arm (the CPU oracle on a bounded sample of the cycle)
prints one JSON line with the contract's keys and the GPU arm's metric and
workload (no GPU)."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-budget", "2"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    cfg = line["config"]
    assert cfg["n"] == 1024 * 1024 and cfg["s"] == 8 and cfg["restart_blocks"] == 30
    assert cfg["workload"].startswith("block-GMRes restart cycle")


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun the reference arm runs on rank 0 alone: any other rank
    exits 0 without work and prints no JSON line."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0", "--cpu-budget", "2"], capture_output=True, text=True,
                         timeout=300, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.strip().startswith("{")], out.stdout


def test_strip_comments_keeps_code_and_literals():
    """The traffic capture is keyed by the kernel's source without comments."""
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    src = 'int a = 1; // note\n/* block\n comment */ const char* s = "x//y  /*z*/"; char q = \'"\';\n'
    assert bench.strip_comments(src) == 'int a = 1; const char* s = "x//y  /*z*/"; char q = \'"\';'
    assert bench.strip_comments("a /* c */ b") == bench.strip_comments("a\n  b  // d")
    assert bench.strip_comments("a /* c */ b") != bench.strip_comments("a b c")
