"""bench.py's reference arm (the FP64 oracle timed on host cores) runs without
a GPU: its JSON line carries every key of the bench contract, and under a
multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, timeout=600):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout,
                          stdin=subprocess.DEVNULL)


def test_reference_line_has_the_contract_keys():
    r = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "unit", "ms_per_step", "higher_is_better", "scaling", "dtype", "data", "config"):
        assert key in d, key
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["dtype"] == "f64"
    assert d["config"]["workload"] and "model" not in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # ms per extrapolated full ID agrees with the rate
    assert abs(1000.0 / d["ms_per_step"] - d["value"]) <= 1e-9 * d["value"] + 1e-12


def test_reference_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_oracle_timer_over_worker_processes():
    """The batched CPU baseline's timer: every worker runs its share of the
    oracle IDs and reports its compute time; a failing worker raises."""
    import numpy as np
    import pytest

    sys.path.insert(0, ROOT)
    import bench

    rng = np.random.default_rng(0)
    mats = [rng.standard_normal((20 + 3 * i, 50)) for i in range(6)]
    ks = [5] * 6
    t1 = bench.time_oracle_many(mats, ks, 1)
    t3 = bench.time_oracle_many(mats, ks, 3)
    assert t1 > 0 and t3 > 0
    assert bench.time_oracle_many(mats[:2], ks[:2], 8) > 0          # more workers than matrices
    grads = [rng.standard_normal((5, 50)) for _ in range(6)]           # forward ID plus gradient per matrix
    assert bench.time_oracle_many(mats, ks, 2, grads=grads) > 0
    with pytest.raises(RuntimeError):
        bench.time_oracle_many([rng.standard_normal((10, 20))], [11], 1)   # k > min(m, n): the oracle refuses


def test_a_failing_side_workload_is_reported_not_fatal(capsys):
    sys.path.insert(0, ROOT)
    import bench

    assert bench.guarded("ok", lambda a, b: a + b, 2, 3) == 5

    def boom():
        raise ValueError("no device")

    out = bench.guarded("side", boom)
    assert out["workload"] == "side" and "no device" in out["error"]
    assert "side workload side failed" in capsys.readouterr().err


def test_algorithmic_units_match_the_stated_figures():
    """The roofline's work units: the flop convention 4 (m-j)(n-j) per step plus
    k^2 (n-k), the algorithmic bytes s sum (m-j)(n-j) + s m n, and the FP64
    operations the left-looking form executes, at 4096 x 8192, k = 256."""
    import pytest

    sys.path.insert(0, ROOT)
    import bench

    assert bench.flops_cpqr(4096, 8192, 256) == pytest.approx(3.28e10, rel=2e-3)
    assert bench.flops_solve(8192, 256) == pytest.approx(5.2e8, rel=1e-2)
    assert bench.bytes_cpqr(4096, 8192, 256, 8) == pytest.approx(65.8e9, rel=2e-3)
    assert bench.bytes_cpqr(4096, 8192, 256, 4) == pytest.approx(32.9e9, rel=2e-3)
    assert bench.fp64_flops_executed(4096, 8192, 256) == pytest.approx(1.79e10, rel=3e-3)
    # closed forms of the sums on a small case
    m, n, k = 7, 11, 5
    assert bench.flops_cpqr(m, n, k) == sum(4 * (m - j) * (n - j) for j in range(k))
    assert bench.bytes_cpqr(m, n, k, 8) == 8 * (sum((m - j) * (n - j) for j in range(k)) + m * n)
