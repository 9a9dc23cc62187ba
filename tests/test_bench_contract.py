"""bench.py's reference arm (the FP64 oracle on the host cores) prints one JSON
line with the keys and types the benchmark contract names; runs on CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-seconds", "1"], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "walker-moves/s" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_gpus_flag_starts_one_rank_per_gpu_dry_run():
    """`--gpus 2` outside torchrun relaunches itself as two ranks; the CPU dry run
    checks the plumbing: disjoint walker keys, one histogram exchange per step, the
    slowest rank's time, and one line from rank 0 with n_gpus = 2."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--dry-run-cpu", "--steps", "3",
                        "--warmup", "1", "--walkers", "64"], capture_output=True, text=True, timeout=300, cwd=ROOT,
                       env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["dry_run"] is True and d["n_gpus"] == 2 and d["exchanges_per_step"] == 1.0
    assert d["key_ranges"] == [[0, 63], [64, 127]]
    assert d["max_ms"] == max(d["rank_ms"]) and len(d["rank_ms"]) == 2   # the slowest rank's time


def test_oracle_sample_of_a_small_system_runs_several_sweeps_per_task():
    """The CPU baseline of a small system: each thread-pool task carries a walker
    through k sweeps, enough for about 10 ms of work, so that the pool's per-task
    overhead does not set the figure; the eight 55-mers keep one sweep a task."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1702_01770_gb300 import inputs
    v, pev, n, dt, k = bench.oracle_walker_moves_per_s(inputs.config0(), 0.3, 2)
    assert k > 1 and n >= 2 and dt > 0.0
    assert v > 0.0 and pev > 0.0
    s4 = inputs.config4(walkers=1)
    v4, pev4, n4, dt4, k4 = bench.oracle_walker_moves_per_s(s4, 0.01, 1)
    assert k4 == 1 and n4 >= 1 and pev4 / v4 > 100.0   # hundreds of pair evaluations per move
