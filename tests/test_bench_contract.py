"""The benchmark's reference arm (the FP64 oracle on the host cores) runs on the
CPU and prints the one-line JSON contract; a non-zero rank prints nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, env_extra=None):
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip()


def test_reference_arm_prints_the_contract_line():
    out = run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-sample", "256"])
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["vs_baseline"] is None and d["steps"] == 1
    assert d["warmup"] == 3  # at least three warm-up steps, whatever is asked
    assert "workload" in d["config"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    out = run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-sample", "64"],
              {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert out == ""


def test_kernel_count_per_step_follows_the_launch_rules():
    """gpu_launches counts the kernels one gs_solve_grad call launches: the
    starting-step pass, the record, the t1-save pass (FP64, no shared weights,
    k = 1, last save at t1), the reverse sweep, and the weight reduction of
    shared-weight problems."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2609_02876_gb300 import workloads as W
    lor = W.make("lorenz", 4)
    assert bench.launches_per_step("lorenz", "fp64", 1, lor) == 4
    assert bench.launches_per_step("lorenz", "fp32_mixed", 1, lor) == 3
    assert bench.launches_per_step("lorenz", "fp64", 11, lor) == 3  # k > 1: no t1-save pass
    assert bench.launches_per_step("lorenz", "fp64", 1, dict(lor, save_t=lor["save_t"][:-1])) == 3
    assert bench.launches_per_step("lv_ude", "fp32_mixed", 1, W.make("lv_ude", 4)) == 4
