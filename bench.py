"""Throughput of the GB300 interpolative decomposition on the 4096 x 8192, k = 256 workload.

One step = one rank-256 ID (column-pivoted QR stopped after 256 pivots,
back substitution, Z assembly) of a 4096 x 8192 matrix A = U diag(s) V^T with
Haar U, V and s_i = exp(-i/64). The headline is the FP64 ID; the FP32 ID of
the same matrix is measured in the same run and reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbid|reference]

Multi-GPU (N > 1, launched by torchrun): every rank decomposes its own copy
(independent replicas, no collective on the data path); value = total IDs/s.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only) and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, K_RANK = 4096, 8192, 256
WORKLOAD = "id_4096x8192_k256"
METRIC = "IDs/s and effective TFLOP/s at stated rel. Frobenius error vs FP64 plain ID"
UNIT = "IDs/s"
REF_SAMPLE_STEPS = 4           # pivot steps per --impl reference step


def flops_cpqr(m, n, k):
    """Flop convention of the ID: 4 (m-j)(n-j) per pivot step (a GEMV and a rank-1 update)."""
    return sum(4.0 * (m - j) * (n - j) for j in range(k))


def flops_solve(n, k):
    return float(k) * k * (n - k)


def bytes_cpqr(m, n, k, s):
    """Algorithmic bytes: one read of A plus the trailing block once per pivot step."""
    return s * sum((m - j) * (n - j) for j in range(k)) + s * m * n


def fp64_flops_executed(m, n, k):
    """FP64 operations the left-looking CPQR performs: per step j the trailing
    product 2 (m-j)(n-j-1), the F corrections 4 (n-j-1) j and the pivot
    column update + aux 4 (m-j) j (panel = all k steps)."""
    return sum(2.0 * (m - j) * (n - j - 1) + 4.0 * (n - j - 1) * j + 4.0 * (m - j) * j for j in range(k))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# FP64 ALU peak: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz (a DFMA
# microbenchmark on this GPU measured 1.196 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.rows = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_input(device, dtype):
    import torch

    import synth

    A = synth.lowrank(M, N, synth.spectrum("exp64", M), 2, device=device)
    return A.to(dtype).contiguous()


# ---------------------------------------------------------------- oracle CPU --
ORACLE_SNIPPET = r"""
import sys, time, json
import numpy as np
sys.path.insert(0, sys.argv[1])
from oracle import id_oracle as orc
A = np.load(sys.argv[2])
s = int(sys.argv[3])
reps = int(sys.argv[4])
full = sys.argv[5] == "full"
out = []
for _ in range(reps):
    t0 = time.perf_counter()
    if full:
        orc.interp_decomp(A, s)
    else:
        orc.cpqr(A, s)
    out.append(time.perf_counter() - t0)
print(json.dumps(out))
"""


def time_oracle(A_cpu_np, steps, reps, full=False):
    """Seconds per call of the oracle (its first `steps` pivot steps, or a whole rank-`steps` ID
    when `full`), single-threaded, in a fresh process."""
    import numpy as np

    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "A.npy")
        np.save(path, A_cpu_np)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", ORACLE_SNIPPET, ROOT, path, str(steps), str(reps),
                            "full" if full else "steps"],
                           capture_output=True, text=True, env=env, timeout=1800)
        if r.returncode != 0:
            raise RuntimeError(r.stderr[-2000:])
        return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_ids_per_s(sample_seconds, steps):
    """Full-ID rate extrapolated from `steps` pivot steps by the CPQR flop count."""
    scale = flops_cpqr(M, N, K_RANK) / flops_cpqr(M, N, steps)
    return 1.0 / (sample_seconds * scale)


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    import numpy as np
    import torch

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A = make_input(dev, torch.float64).cpu().numpy()
    total = args.warmup + args.steps
    secs = time_oracle(A, REF_SAMPLE_STEPS, total)[args.warmup:]
    per = statistics.mean(secs)
    value = oracle_ids_per_s(per, REF_SAMPLE_STEPS)
    sample = (f"first {REF_SAMPLE_STEPS} of {K_RANK} pivot steps of the FP64 oracle per step, "
              f"extrapolated to a full ID by the CPQR flop count")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3 * flops_cpqr(M, N, K_RANK) /
        flops_cpqr(M, N, REF_SAMPLE_STEPS), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "k": K_RANK, "spectrum": "s_i = exp(-i/64)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm --
def time_gpu(gbid, A, steps, warmup, flush, trace=True):
    """Per-step device times (ms) of id_decompose on resident inputs, L2 flushed between steps."""
    import torch

    m, n = A.shape
    ws = gbid.Workspace.for_problem(A.dtype, m, n, K_RANK, device=A.device)
    J = torch.empty(K_RANK, dtype=torch.int32, device=A.device)
    Z = torch.empty(K_RANK, max(m, n), dtype=A.dtype, device=A.device)
    for _ in range(warmup):
        gbid.id_decompose(A, K_RANK, workspace=ws, out=(J, Z), sync=False)
    torch.cuda.synchronize()
    if trace:
        gbid.trace_enable(4 * steps + 8)
    times = []
    s = torch.cuda.current_stream()
    for _ in range(steps):
        flush.fill_(1.0)                       # evict L2 (buffer larger than L2), outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        gbid.id_decompose(A, K_RANK, workspace=ws, out=(J, Z), sync=False)
        e1.record(s)
        times.append((e0, e1))
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in times]
    tr = gbid.trace_read() if trace else {}
    if trace:
        gbid.trace_enable(0)
    info = gbid.read_info(ws)
    return ms, tr, info, J, Z


def rel_error_gpu(A, J, Z):
    import torch

    A64 = A.double()
    C = A64[:, J.long()]
    return (torch.linalg.norm(A64 - C @ Z.double()) / torch.linalg.norm(A64)).item()


def e2e_rate(gbid, A, steps):
    """IDs/s through the host-buffer C entry point: H2D copy of A, ID, D2H of J and Z, all timed."""
    import torch

    Ah = A.cpu().pin_memory()
    m, n = Ah.shape
    ws = gbid.Workspace.for_problem(A.dtype, m, n, K_RANK, device=A.device, host_io=True)
    Jh = torch.empty(K_RANK, dtype=torch.int32, pin_memory=True)
    Zh = torch.empty(K_RANK, max(m, n), dtype=A.dtype, pin_memory=True)
    gbid.id_decompose_host(Ah, K_RANK, workspace=ws, out=(Jh, Zh))
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        gbid.id_decompose_host(Ah, K_RANK, workspace=ws, out=(Jh, Zh))
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    h2d = Ah.numel() * Ah.element_size()
    d2h = Jh.numel() * 4 + Zh.numel() * Zh.element_size()
    return 1000.0 / ms, h2d, d2h


def run_gbid(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__ as ge

    ge.build()
    import paper_2105_07076_gb300 as gbid

    dev = torch.device("cuda", local)
    hbm_peak, peak_src = load_peaks()
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2
    results = {}
    clocks = None
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        A = make_input(dev, dt)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if name == "f64":
            with ClockSampler(local) as cs:
                ms, tr, info, J, Z = time_gpu(gbid, A, args.steps, args.warmup, flush)
            clocks = cs.summary()
        else:
            ms, tr, info, J, Z = time_gpu(gbid, A, args.steps, args.warmup, flush)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        mean_ms = statistics.mean(ms)
        t = torch.tensor([mean_ms], device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        mean_ms = t.item()
        err = rel_error_gpu(A, J, Z)
        cp_ms, cp_n = tr.get("cpqr", (0.0, 0))
        cp_avg = cp_ms / cp_n if cp_n else float("nan")
        s = A.element_size()
        if name == "f64":
            achieved = fp64_flops_executed(M, N, K_RANK) / (cp_avg * 1e-3) / 1e12
            roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "k_cpqr<double>",
                    "kernel_ms": cp_avg,
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (DFMA probe: 1.196)"}
        else:
            achieved = bytes_cpqr(M, N, K_RANK, s) / (cp_avg * 1e-3) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": None, "kernel": "k_cpqr<float>", "kernel_ms": cp_avg,
                    "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                    else "fallback"}
        eff = (flops_cpqr(M, N, K_RANK) + flops_solve(N, K_RANK)) / (mean_ms * 1e-3) / 1e12
        results[name] = {"ms_per_step": mean_ms, "value": world * 1000.0 / mean_ms, "eff_tflops": eff,
                         "rel_err": err, "status": info["status_name"], "roofline": roof,
                         "solve_ms": (tr.get("solve", (0.0, 1))[0] / max(tr.get("solve", (0, 1))[1], 1)),
                         "launches_per_step": gbid.launch_count(dt, M, N, K_RANK), "A": A}
    e2e_v, h2d, d2h = e2e_rate(gbid, results["f64"]["A"], max(2, min(args.steps, 5)))
    if world > 1:
        t = torch.tensor([1.0 / e2e_v], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_v = world / t.item()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        A_np = results["f64"]["A"].cpu().numpy()
        secs = time_oracle(A_np, K_RANK, 1, full=True)
        cpu = {"value": 1.0 / secs[0], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one complete rank-{K_RANK} ID of the same 4096 x 8192 FP64 matrix by the oracle "
                         f"({secs[0]:.1f} s, numpy, one thread)"}
    if world > 1 and dist.is_initialized():
        dist.barrier()
    if rank != 0:
        return 0
    import synth

    tail = synth.tail_bound(synth.spectrum("exp64", M), K_RANK)
    r64, r32 = results["f64"], results["f32"]
    line = {
        "metric": METRIC, "value": r64["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r64["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "k": K_RANK, "spectrum": "s_i = exp(-i/64)",
                   "inputs": "A = U diag(s) V^T, Haar U, V (seed 2)", "parallelism": f"replicas x{world}",
                   "l2": "256 MB buffer written between timed steps (A + working copy also exceed L2)"},
        "eff_tflops": r64["eff_tflops"], "rel_err": r64["rel_err"], "tail_bound": tail, "status": r64["status"],
        "roofline": r64["roofline"],
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": r64["launches_per_step"] * args.steps,
        "clocks": clocks,
        "f32": {"value": r32["value"], "unit": UNIT, "ms_per_step": r32["ms_per_step"], "eff_tflops": r32["eff_tflops"],
                "rel_err": r32["rel_err"], "status": r32["status"], "roofline": r32["roofline"],
                "speedup_vs_f64": r32["value"] / r64["value"]},
        "solve_ms": {"f64": r64["solve_ms"], "f32": r32["solve_ms"]},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbid", choices=["gbid", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gbid(args)


if __name__ == "__main__":
    sys.exit(main())
