"""bench.py's reference arm: the CPU oracle timed on a bounded sample of the
headline workload.  Its one JSON line carries the keys, metric, unit and
workload of the GPU arm, and under torchrun the ranks other than 0 exit
without work.  Also the host side of the headline's fault injection (the
Poisson draws, sites and magnitudes bench.py passes to the kernels).  Runs on
the CPU."""
import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def _bench_module():
    spec = importlib.util.spec_from_file_location("bench_under_test", BENCH)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _reference(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, BENCH, "--impl", "reference", "--steps", "1", "--warmup", "0"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def test_reference_arm_prints_one_complete_line():
    p = _reference()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["data"] == "synthetic"

    # the same metric, unit and workload as the GPU arm's line
    b = _bench_module()
    assert d["metric"] == b.METRIC and d["unit"] == "TFLOP/s"
    assert d["config"] == b.workload_config(16384, "block")
    assert d["config"]["schedule"]["k_tb"] == b.SCHED["k_tb"]

    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_no_work():
    p = _reference({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_headline_fault_draws():
    # the bench's faults: a Poisson count at 200 per minute of kernel time,
    # sites inside the headline tiling (at most one per tile and period), and
    # magnitudes log-uniform in [1e-2, 1e3] x the expected tile maximum
    import math
    import numpy as np
    b = _bench_module()
    n, t_kernel = 16384, 0.14
    ksteps = n // b.SCHED["k_tb"]
    tiles = n // b.SCHED["m_tb"]
    tile_max = 4.0 * math.sqrt(n / 9.0)
    counts, deltas = [], []
    for s in range(3000):
        f = b.make_faults(1000 + 17 * s, t_kernel, n, ksteps)
        counts.append(len(f))
        units = set()
        for tm, tn, ks, r, c, d in f:
            assert 0 <= tm < tiles and 0 <= tn < tiles and 0 <= ks < ksteps
            assert 0 <= r < b.SCHED["m_tb"] and 0 <= c < b.SCHED["n_tb"]
            units.add((tm, tn, ks // b.SCHED["cadence"]))
            deltas.append(d)
        assert len(units) == len(f)
    lam = b.FAULTS_PER_MIN / 60.0 * t_kernel
    assert abs(np.mean(counts) - lam) < 5 * math.sqrt(lam / len(counts))
    mags = np.abs(np.array(deltas)) / tile_max
    assert mags.min() >= 1e-2 * (1 - 1e-6) and mags.max() <= 1e3 * (1 + 1e-6)
    assert 0.4 < np.mean(np.array(deltas) > 0) < 0.6
    assert b.make_faults(4242, t_kernel, n, ksteps) == b.make_faults(4242, t_kernel, n, ksteps)
