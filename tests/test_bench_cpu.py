"""The benchmark's reference arm (the FP64 oracle timed on the host cores) on
CPU: one JSON line with the contract's keys from rank 0, nothing from the
other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    return [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = _run({})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Gvis/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Gvis/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same config dictionary as the GPU arm prints for its headline workload
    sys.path.insert(0, ROOT)
    import bench
    from paper_1709_08681_gb300 import inputs as I
    assert d["config"] == bench.config_for(I.make_workload("drift197_l128ch"))


def test_reference_arm_is_silent_on_other_ranks():
    assert _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}) == []


def test_our_arm_refuses_to_run_without_a_gpu():
    """No CPU fallback: without a CUDA device the benchmark exits non-zero."""
    import pytest
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    out = subprocess.run([sys.executable, "bench.py", "--steps", "1", "--warmup", "3"], cwd=ROOT,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode != 0
    assert "needs a CUDA device" in out.stderr + out.stdout
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
