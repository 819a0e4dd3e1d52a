"""The JSON line of `bench.py --impl reference` (the FP64 oracle timed on the host cores)
against the benchmark contract, on CPU: one line with the required keys and types, the
same metric, unit and workload configuration as the GPU arm, and the e2e and cpu_baseline
objects describing this run."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def line(tmp_path_factory):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env,
                       cwd=str(tmp_path_factory.mktemp("bench")), timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_required_keys_and_types(line):
    want = {"metric": str, "value": float, "unit": str, "n_gpus": int, "steps": int, "warmup": int,
            "ms_per_step": float, "higher_is_better": bool, "scaling": str, "dtype": str, "data": str,
            "config": dict, "e2e": dict, "cpu_baseline": dict, "impl": str}
    for k, t in want.items():
        assert isinstance(line[k], t), (k, line.get(k))
    assert "vs_baseline" in line and line["vs_baseline"] is None
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 0
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]


def test_same_metric_and_workload_as_the_gpu_arm(line):
    sys.path.insert(0, ROOT)
    import bench
    assert line["metric"] == "particles_per_s" and line["unit"] == "particles/s"
    gpu_config = bench.workload_config(1)
    for k, v in gpu_config.items():
        assert line["config"][k] == v, k
    assert "sample" in line["config"]
