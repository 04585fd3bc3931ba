"""bench.py's output contract, through its reference arm (the CPU oracle on
the bench workload; no device needed): one JSON line with the keys a
benchmark consumer reads, consistent with each other, and silence with exit
status 0 on ranks other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_complete_line():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--rk", "2"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["unit"] == "DoF-steps/s" and line["higher_is_better"] is True
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 1, 0)
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["workload"] == "cell40_p3_256x256" and line["config"]["p"] == 3
    # value = DoF per density x RK steps / time: one density, R RK steps per bench step
    dof = line["config"]["active_elements"] * 16
    R = line["config"]["rk_steps_per_bench_step"]
    assert R == 2 and line["config"]["densities_per_gpu"] == 64
    assert abs(line["value"] * line["ms_per_step"] * 1e-3 / (dof * R) - 1) < 1e-9
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert cb["cores"] <= (os.cpu_count() or 1) and "logical CPUs" in cb["cpu"]
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_is_silent_on_other_ranks():
    r = _bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--gpus", "2"],
               {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
