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


def test_reference_line_has_the_contract_keys(monkeypatch, capsys):
    """run_reference on a shrunken copy of the headline workload (the full
    16384 x 32768 inputs are generated on the GPU machine): one JSON line with the
    contract's keys, the GPU arm's config dict, and a rate that is the
    sample's scaled by the column ratio."""
    import argparse

    sys.path.insert(0, ROOT)
    import bench

    for name, val in (("RM", 256), ("RN", 1024), ("RK", 32), ("RL", 42), ("RID_CPU_COLS", 128)):
        monkeypatch.setattr(bench, name, val)
    monkeypatch.setattr(bench, "RWORKLOAD", "rid_256x1024_k32_l42")
    for k, v in (("RANK", "0"), ("WORLD_SIZE", "1"), ("LOCAL_RANK", "0")):
        monkeypatch.setenv(k, v)
    args = argparse.Namespace(gpus=1, steps=1, warmup=3, impl="reference", no_cpu_baseline=False, only="all")
    assert bench.run_reference(args) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "unit", "ms_per_step", "higher_is_better", "scaling", "dtype", "data", "config"):
        assert key in d, key
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["dtype"] == "f64"
    assert d["config"] == bench.rid_config(1) and "model" not in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # ms_per_step is one sample; the rate scales it by the column ratio
    assert abs(bench.rid_oracle_rate(d["ms_per_step"] / 1000.0) - d["value"]) <= 1e-9 * d["value"]


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


def test_headline_units_match_the_stated_figures():
    """The headline's work units at 16384 x 32768, k = 512, l = 522: sketch
    2 l m n = 5.6e11, CPQR of the sketch 1.78e10, solve 8.5e9, refinement
    2mk(n-k) + 4mk^2 + 2k^2(n-k) = 5.75e11 flop; the sketch CPQR's algorithmic
    bytes 4 sum (l-j)(n-j) + 4 l n = 17.9 GB."""
    import pytest

    sys.path.insert(0, ROOT)
    import bench

    f = bench.rid_flops()
    assert f["sketch"] == pytest.approx(5.6e11, rel=1e-2)
    assert f["cpqr"] == pytest.approx(1.78e10, rel=1e-2)
    assert f["solve"] == pytest.approx(8.5e9, rel=1e-2)
    # 2mk(n-k) = 5.4e11 is the convention's leading term; 4mk^2 + 2k^2(n-k) add 3.4e10
    assert f["refine"] == pytest.approx(2.0 * 16384 * 512 * (32768 - 512) + 4.0 * 16384 * 512 ** 2
                                        + 2.0 * 512 ** 2 * (32768 - 512))
    assert 2.0 * 16384 * 512 * (32768 - 512) == pytest.approx(5.4e11, rel=1e-2)
    assert bench.bytes_cpqr(522, 32768, 512, 4) == pytest.approx(17.9e9, rel=1e-2)
    assert bench.rid_oracle_rate(1.0) == pytest.approx(bench.RID_CPU_COLS / bench.RN)


def test_roofline_is_the_longest_single_kernel():
    """The line's roofline is the CPQR kernel's (one launch per ID), even when
    the refinement stage, spread over many launches, takes longer; its achieved
    figure is the CPQR's algorithmic bytes over that launch's time."""
    sys.path.insert(0, ROOT)
    import bench

    per = {"cpqr": 7.5, "refine": 8.7, "sketch": 0.95}
    out, dom = bench.rid_rooflines(per, 6774.0, "measured")
    assert dom == "cpqr"
    r = out["cpqr"]
    assert r["achieved"] == bench.bytes_cpqr(bench.RL, bench.RN, bench.RK, 4) / 7.5e-3 / 1e9
    assert abs(r["frac"] - r["achieved"] / 6774.0) < 1e-12 and r["unit"] == "GB/s"
    assert set(out) == {"cpqr", "refine", "sketch"}
