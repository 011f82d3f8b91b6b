"""bench.py's contract on a machine without a GPU: the reference arm (the oracle on
the host cores) prints one JSON line with the contract's keys; the GPU arm refuses
to run without a device instead of falling back to anything."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1305_3440_gb300 import build
    build.build()


def _run(args, timeout=300):
    env = dict(os.environ, PYTHONPATH=ROOT)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          timeout=timeout, env=env, cwd=ROOT)


def test_reference_arm_prints_the_contract_line(built):
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_gpu_arm_refuses_without_a_device(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run(["--steps", "1", "--warmup", "0"], timeout=120)
    assert r.returncode != 0 and "CUDA GPU" in (r.stdout + r.stderr)


def test_traffic_record_is_tied_to_the_kernel_sources(tmp_path, monkeypatch):
    """bench.py uses an ncu traffic record only while the kernel sources hash to
    the value stored with it."""
    sys.path.insert(0, ROOT)
    import bench
    h = bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.md").write_text(
        f"    traffic-record: kernel=k_sweep_f32 config=7 bytes_per_launch=123 sources={h}\n"
        "    traffic-record: kernel=k_sweep_f32 config=8 bytes_per_launch=456 sources=0000000000000000\n")
    for rel in bench.KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, rel), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("k_sweep_f32", 7) == 123
    assert bench.recorded_traffic("k_sweep_f32", 8) is None  # recorded for other sources
    assert bench.recorded_traffic("k_sweep_anchor", 0) is None
