"""The benchmark's command-line contract, on the CPU: the reference arm (the
CPU oracle) prints one JSON line with the required keys, and the library arm
fails loudly instead of falling back to the CPU when there is no GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric": str, "value": float, "unit": str, "n_gpus": int, "steps": int, "warmup": int,
        "ms_per_step": float, "higher_is_better": bool, "scaling": str, "dtype": str, "data": str,
        "config": dict, "impl": str, "cpu_baseline": dict, "e2e": dict}


def _bench(*args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_json_line():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k, t in KEYS.items():
        assert isinstance(d[k], t), (k, d.get(k))
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"]["workload"] == "hbm_2^28" and d["vs_baseline"] is None
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_library_arm_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _bench("--steps", "1", "--warmup", "3", "--no-cpu", "--no-e2e", timeout=300)
    assert r.returncode != 0
    assert not any(ln.startswith("{") for ln in r.stdout.splitlines())


def test_profile_counters_follow_the_kernel_code(tmp_path):
    """roofline.traffic comes from a committed ncu summary only while the
    kernel's code is the one the summary was taken on: editing a comment keeps
    the digest, editing code changes it."""
    sys.path.insert(0, ROOT)
    import bench

    src = tmp_path / "k.cu"
    src.write_text("// a kernel\n__global__ void k(int* p)\n{\n    // store\n    p[0] = 1;\n}\n")
    d0 = bench.kernel_code_digest(str(src))
    src.write_text("// a kernel, reworded\n__global__ void k(int* p)   \n{\n        // the store\n    p[0] = 1;\n}\n")
    assert bench.kernel_code_digest(str(src)) == d0
    src.write_text("// a kernel\n__global__ void k(int* p)\n{\n    // store\n    p[0] = 2;\n}\n")
    assert bench.kernel_code_digest(str(src)) != d0
    # the committed summaries resolve against the sources they name
    for workload in ("hbm_2^28", "plain_2^24"):
        for storage in ("pingpong", "vm"):
            t = bench.traffic_from_profile(workload, storage)
            assert t is None or t > 0
