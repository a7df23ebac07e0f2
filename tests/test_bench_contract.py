"""The benchmark's output contract, checked on the CPU through its reference
arm (the FP64 oracle timed on the host cores, which needs no GPU): one JSON
line with the metric, the unit and direction, the step's configuration, a
cpu_baseline describing the sample that was timed and an e2e entry with no
host-device copies; under torchrun only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env_extra=None, timeout=600):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_json_line():
    p = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "coupled sample-steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "large32_1024"
    assert d["config"]["levels"] == [32, 64, 128, 256, 512, 1024]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert 1 <= cb["cores"] <= cb["nproc"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # ms_per_step is the whole step's oracle time: value = sample-steps per step / step time
    sps = d["config"]["sample_steps_per_step"]
    assert abs(sps / (d["ms_per_step"] * 1e-3) - d["value"]) <= 1e-9 * d["value"]


def test_reference_arm_other_ranks_exit_without_work():
    p = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0"],
               {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
