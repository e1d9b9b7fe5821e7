"""bench.py's reference arm on the CPU: one JSON line with the keys of the benchmark contract (the
oracle timed on a seeded sample of the workload's columns), and no output on ranks other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--workload", "diamond_64", "--steps", "1", "--warmup", "1",
                           "--cpu-sample", "16"], capture_output=True, text=True, env=env, cwd=ROOT,
                          timeout=600)


def test_reference_line_has_the_contract_keys():
    res = _run({"RANK": "0"})
    assert res.returncode == 0, res.stderr
    lines = [l for l in res.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["unit"] == "columns/s" and d["dtype"] == "f64" and d["extrapolated"] is True
    assert d["config"]["workload"].startswith("diamond_64") and d["config"]["columns_per_step"] == 256
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "16 seeded" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "columns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_other_ranks_print_nothing():
    res = _run({"RANK": "1"})
    assert res.returncode == 0 and res.stdout.strip() == ""


def test_both_arms_name_a_batch_size_set_on_the_command_line():
    """--batch-atoms changes the workload's batches, so both arms' config says so (and leaves it
    out when the library chooses them)."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as wl
    w = wl.make("diamond_64")
    saved = sys.argv
    try:
        sys.argv = ["bench.py", "--workload", "diamond_64", "--batch-atoms", "16"]
        args = bench.parse()
        assert bench.bench_config(args, w, 1)["batch_atoms"] == 16
        sys.argv = ["bench.py", "--workload", "diamond_64"]
        args = bench.parse()
        assert "batch_atoms" not in bench.bench_config(args, w, 1)
    finally:
        sys.argv = saved
