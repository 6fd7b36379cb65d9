"""Throughput of the GB300 interpolative decomposition on its headline workload.

One step = one randomized rank-512 ID of a 16384 x 32768 FP32 matrix
A = U diag(s) V^T (Haar U, V, s_i = (1+i)^-1.5): the Gaussian sketch
Y = Omega A (Omega 522 x 16384, N(0,1) rounded to BF16) on the tensor cores,
k = 512 steps of column-pivoted QR of Y (FP32 matrix, FP64 norm downdate,
the compact-WY update on the tensor cores), the sketch's T, and one
least-squares refinement of Z against A (3xTF32 products on the tensor
cores). Inputs stay resident in HBM; A (2.15 GB) exceeds L2, so no flush is
needed between steps. The line carries the roofline of the dominant kernel
in SURVEY-convention units, the end-to-end rate with host buffers, the
oracle's rate on a bounded sample (cpu_baseline), and, under "compare", the
plain FP64 GPU ID of the same matrix and the FP64 batched launch beside the
mixed-precision and FP32 batched forms at their reconstruction errors.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbid|reference]

Side workloads in the same line: "deterministic" (the 4096 x 8192, k = 256 ID
in FP64 and FP32, s_i = exp(-i/64)), "batched" (4096 uneven FP32 IDs in one
persistent launch, tile shape picked by the library's tuner), "latency"
(back-to-back 200 x 400 FP64 IDs, k = 20), "differentiable" (256 IDs of
512 x 1024 at k = 64, forward and backward), "sampled" (the paper's
column-sampling Optim RID of the 4096 x 8192 matrices), "listing" (Z from the
normal equations, approx = C @ Z), "two_sided" and "sparse" (a 4096 x 8192
CSR matrix). --only randomized runs the headline alone; --only id the
headline and the deterministic block; --only batched / latency /
differentiable / compare one side workload alone.

Multi-GPU (N > 1, launched by torchrun): every rank decomposes its own copy
(independent replicas, no collective on the data path); value = total IDs/s.
--impl reference times the FP64 CPU oracle on a bounded sample of the
headline workload (rank 0 only) and prints the same JSON line with
"impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, K_RANK = 4096, 8192, 256
WORKLOAD = "id_4096x8192_k256"
# the headline: the randomized ID of a 16384 x 32768 FP32 matrix, k = 512, l = k + 10
RM, RN, RK, RL = 16384, 32768, 512, 522
RWORKLOAD = f"rid_{RM}x{RN}_k{RK}_l{RL}"
RID_CPU_COLS = 1024            # columns of A in one oracle sample of the headline workload
METRIC = "IDs/s and effective TFLOP/s at stated rel. Frobenius error vs FP64 plain ID"
UNIT = "IDs/s"
BATCHED_CPU_SAMPLE = 1024      # problems of the uneven batch the oracle decomposes for its CPU baseline
DIFF_CPU_SAMPLE = 64           # forward + gradient problems of the differentiable workload for its CPU baseline


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


# dram__bytes_read.sum + dram__bytes_write.sum of one k_cpqr launch on this
# workload, from the ncu capture summarised in profiles/ (bytes per launch).
# Set to None whenever k_cpqr changes until it is captured again.
NCU_TRAFFIC = {"f64": 49.62e9, "f32": 11.95e9}

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


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of the ranks' values (the slowest rank's time): an all-reduce MAX."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def aggregate_rate(ms_slowest: float, world: int) -> float:
    """Whole-job IDs/s of independent replicas: every rank decomposes one matrix
    per step and the job's step lasts as long as its slowest rank's."""
    return world * 1000.0 / ms_slowest


def make_input(device, dtype):
    import torch

    import synth

    A = synth.lowrank(M, N, synth.spectrum("exp64", M), 2, device=device)
    return A.to(dtype).contiguous()


# ---------------------------------------------------------------- oracle CPU --
ORACLE_SNIPPET = r"""
import io, sys, time, json
import numpy as np
sys.path.insert(0, sys.argv[1])
from oracle import id_oracle as orc
A = np.load(io.BytesIO(sys.stdin.buffer.read()))
s = int(sys.argv[2])
reps = int(sys.argv[3])
full = sys.argv[4] == "full"
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


ONE_THREAD = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def _npy_bytes(save, *args, **kw) -> bytes:
    import io

    buf = io.BytesIO()
    save(buf, *args, **kw)
    return buf.getvalue()


def time_oracle(A_cpu_np, steps, reps, full=False):
    """Seconds per call of the oracle (its first `steps` pivot steps, or a whole rank-`steps` ID
    when `full`), single-threaded, in a fresh process (the matrix goes through its stdin)."""
    import numpy as np

    r = subprocess.run([sys.executable, "-c", ORACLE_SNIPPET, ROOT, str(steps), str(reps),
                        "full" if full else "steps"],
                       input=_npy_bytes(np.save, A_cpu_np), capture_output=True, env=dict(os.environ, **ONE_THREAD),
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(r.stderr.decode(errors="replace")[-2000:])
    return json.loads(r.stdout.decode().strip().splitlines()[-1])


MANY_SNIPPET = r"""
import io, sys, time, json
import numpy as np
sys.path.insert(0, sys.argv[1])
from oracle import id_oracle as orc
d = np.load(io.BytesIO(sys.stdin.buffer.read()))
ks = d["ks"]
grad = sys.argv[2] == "grad"
t0 = time.perf_counter()
for i in range(len(ks)):
    A = d["A%d" % i]
    J, Z, _ = orc.interp_decomp(A, int(ks[i]))
    if grad:
        J = np.asarray(J, dtype=np.int64)
        perm = np.concatenate([J, np.setdiff1d(np.arange(A.shape[1]), J)])
        orc.id_grad(A, J, perm, d["G%d" % i])
print(json.dumps(time.perf_counter() - t0))
"""


def time_oracle_many(mats, ks, workers, grads=None):
    """Seconds for the oracle's complete IDs of the FP64 numpy matrices `mats`
    (and, with `grads`, the gradient of <grads[i], Z> with the skeleton frozen)
    on `workers` single-threaded processes that run at the same time, worker w
    taking matrices w, w + workers, ...: the largest of their compute times
    (process start and data transfer excluded)."""
    import numpy as np

    procs = []
    for w in range(min(workers, len(mats))):
        idx = list(range(w, len(mats), workers))
        arrays = {f"A{j}": mats[i] for j, i in enumerate(idx)}
        if grads is not None:
            arrays.update({f"G{j}": grads[i] for j, i in enumerate(idx)})
        payload = _npy_bytes(np.savez, ks=np.array([ks[i] for i in idx], dtype=np.int64), **arrays)
        p = subprocess.Popen([sys.executable, "-c", MANY_SNIPPET, ROOT, "grad" if grads is not None else "id"],
                             stdin=subprocess.PIPE,
                             stdout=subprocess.PIPE, stderr=subprocess.STDOUT, env=dict(os.environ, **ONE_THREAD))
        procs.append((p, payload))
    # each worker reads all of its input before it starts computing, so writing
    # the inputs one after the other still lets the workers overlap
    for p, payload in procs:
        p.stdin.write(payload)
        p.stdin.close()
    secs = []
    for p, _ in procs:
        out = p.stdout.read().decode(errors="replace")
        if p.wait(timeout=1800) != 0:
            raise RuntimeError(out[-2000:])
        secs.append(float(json.loads(out.strip().splitlines()[-1])))
    return max(secs)


def run_reference(args):
    """The oracle, as it stands, on the host cores: each step is one oracle
    randomized ID of the headline matrix's first RID_CPU_COLS columns (same
    Omega and k), and the rate is scaled to the whole matrix by the column ratio.
    Rank 0 alone runs and prints; the other ranks exit without work."""
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    import torch

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A, om = rid_inputs(dev)
    secs = rid_oracle_seconds(A, om, args.warmup + args.steps)[args.warmup:]
    per = statistics.mean(secs)
    value = rid_oracle_rate(per)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": rid_config(max(world, args.gpus)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": RID_SAMPLE + f"; ms_per_step is one sample ({per:.2f} s)"},
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




def rid_config(world):
    return {"workload": RWORKLOAD, "m": RM, "n": RN, "k": RK, "l": RL, "spectrum": "s_i = (1+i)^-1.5",
            "inputs": "A = U diag(s) V^T with Haar U, V (seed 3), FP32; Omega N(0,1) rounded to BF16 (seed 33)",
            "form": "randomized ID: BF16 sketch on the tensor cores, FP32 CPQR of the sketch with FP64 norms and "
                    "tensor-core WY updates, one least-squares refinement of Z against A (3xTF32 tensor-core products)",
            "parallelism": f"replicas x{world}",
            "l2": "no flush: A (2.15 GB) exceeds L2 (129 MB) and is read in full every step"}


def rid_flops():
    """The flop convention of one randomized ID (sketch, CPQR of Y, solve, refinement)."""
    f_sketch = 2.0 * RL * RM * RN
    f_cpqr = flops_cpqr(RL, RN, RK)
    f_solve = flops_solve(RN, RK)
    f_refine = 2.0 * RM * RK * (RN - RK) + 4.0 * RM * RK * RK + 2.0 * RK * RK * (RN - RK)
    return {"sketch": f_sketch, "cpqr": f_cpqr, "solve": f_solve, "refine": f_refine}


def rid_inputs(dev):
    import torch

    import synth

    A = synth.lowrank(RM, RN, synth.spectrum("poly1.5", RM), 3, device=dev, dtype=torch.float32,
                      gen_dtype=torch.float32)
    om = synth.gaussian_sketch_bf16(RL, RM, seed=33, device=dev)
    return A, om


def rid_time(gbid, A, om, steps, warmup, world, local):
    """Per-step device times (ms) of the randomized ID on resident inputs, the
    per-stage kernel times of the library's trace, the clocks during the timed
    region, and the last step's J, Z and status."""
    import torch
    import torch.distributed as dist

    dev = A.device
    ws = gbid.rid_workspace(RM, RN, RL, RK, device=dev)
    J = torch.empty(RK, dtype=torch.int32, device=dev)
    Z = torch.empty(RK, RN, dtype=torch.float32, device=dev)
    for _ in range(warmup):
        gbid.id_decompose_randomized(A, om, RK, workspace=ws, out=(J, Z), sync=False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    gbid.trace_enable(64 * steps + 64)
    s = torch.cuda.current_stream()
    ev = []
    with ClockSampler(local) as cs:
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            gbid.id_decompose_randomized(A, om, RK, workspace=ws, out=(J, Z), sync=False)
            e1.record(s)
            ev.append((e0, e1))
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    tr = gbid.trace_read()
    gbid.trace_enable(0)
    per = {k: v[0] / v[1] for k, v in tr.items() if v[1]}
    return ms, per, cs.summary(), gbid.read_info(ws), J, Z


def rid_error(A, J, Z):
    """||A - A[:, J] Z||_F / ||A||_F in FP64 sums, 4096 columns at a time."""
    import torch

    C = A[:, J.long()].double()
    num = den = 0.0
    for c0 in range(0, A.shape[1], 4096):
        Ac = A[:, c0:c0 + 4096].double()
        num += torch.sum((Ac - C @ Z[:, c0:c0 + 4096].double()) ** 2).item()
        den += torch.sum(Ac ** 2).item()
    return math.sqrt(num / den)


def rid_rooflines(per, hbm_peak, peak_src):
    """Per-stage rooflines in the SURVEY's units: the CPQR of the sketch against
    HBM (its algorithmic bytes, the trailing block read once per pivot step),
    the sketch and the refinement against the tensor peak of their input type."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
        bsrc = "of measured: MEASURED_PEAKS.json bf16_tflops (burst)"
    except Exception:
        bf16, bsrc = 1900.0, "of fallback"
    tf32 = bf16 * 1.1 / 2.25          # nominal dense TF32 / BF16 ratio
    fl = rid_flops()
    out = {}
    cp = per.get("cpqr")
    if cp:
        b = bytes_cpqr(RL, RN, RK, 4)
        ach = b / (cp * 1e-3) / 1e9
        out["cpqr"] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                       "traffic": None,
                       "kernel": "k_cpqr_short (one persistent launch per ID: all 512 steps, tcgen05 WY updates inside; "
                                 "522 x 32768 sketch)",
                       "kernel_ms": cp, "algorithmic_bytes": b,
                       "peak_source": f"of {peak_src}: MEASURED_PEAKS.json hbm_gbs" if peak_src == "measured"
                       else "of fallback",
                       "note": "the 68 MB sketch stays in L2; its trailing reads are counted against HBM"}
    sk = per.get("sketch")
    if sk:
        ach = fl["sketch"] / (sk * 1e-3) / 1e12
        out["sketch"] = {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                         "traffic": None, "kernel": "k_sketch (BF16 tcgen05)", "kernel_ms": sk, "peak_source": bsrc}
    rf = per.get("refine")
    if rf:
        executed = 3.0 * 2.0 * 2.0 * RM * RK * RN      # C Z and C^T R, three TF32 products each
        ach = executed / (rf * 1e-3) / 1e12
        out["refine"] = {"bound": "tensor", "achieved": ach, "peak": tf32, "unit": "TFLOP/s", "frac": ach / tf32,
                         "traffic": None, "kernel": "k_gemm_tf32x3 (3xTF32 tcgen05) + skeleton factorisation",
                         "kernel_ms": rf, "convention_tflops": fl["refine"] / (rf * 1e-3) / 1e12,
                         "peak_source": bsrc + " x the nominal TF32/BF16 ratio 1.1/2.25",
                         "note": "achieved counts the executed 3xTF32 products of the residual and C^T R"}
    # The dominant kernel is the longest single kernel of the launch list: the CPQR of the sketch is
    # one launch per ID, while the refinement's time spreads over some 260 launches of several kernels
    # (its largest, the residual product, takes under half of the stage).
    dom = "cpqr" if "cpqr" in out else (max(out, key=lambda k: out[k]["kernel_ms"]) if out else None)
    return out, dom


def rid_e2e(gbid, A, om, steps):
    """IDs/s through the public host-buffer entry point for a stream of IDs
    (id_rid_pipe): every ID copies its A and Omega from pinned host memory and
    its J, Z and status back; the copies of neighbouring IDs overlap the current
    ID on the device. Timed on the host clock from the first submit until the
    last ID's outputs are on the host (the copy streams are the pipe's own), so
    the first ID's input copy, which nothing overlaps, is inside."""
    import ctypes
    import time

    import torch

    Ah = A.cpu().pin_memory()
    Oh = om.cpu().pin_memory()
    Jh = torch.empty(RK, dtype=torch.int32, pin_memory=True)
    Zh = torch.empty(RK, RN, dtype=torch.float32, pin_memory=True)
    pipe = gbid.RandomizedPipeline(RM, RN, RL, RK, device=A.device)
    for _ in range(2):   # warm-up: both slots once
        pipe.submit(Ah, Oh, Jh, Zh)
    pipe.synchronize()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        pipe.submit(Ah, Oh, Jh, Zh)
    infos = pipe.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / steps
    pipe.close()
    if any(i["status"] != gbid.ID_OK for i in infos):
        raise RuntimeError(f"pipelined ID status {[i['status_name'] for i in infos]}")
    h2d = Ah.numel() * 4 + Oh.numel() * 2
    d2h = Jh.numel() * 4 + Zh.numel() * 4 + ctypes.sizeof(gbid.IdInfo)
    del Ah, Oh
    return 1000.0 / ms, h2d, d2h


RID_ORACLE_SNIPPET = r"""
import io, sys, time, json
import numpy as np
sys.path.insert(0, sys.argv[1])
from oracle import id_oracle as orc
d = np.load(io.BytesIO(sys.stdin.buffer.read()))
k, reps = int(sys.argv[2]), int(sys.argv[3])
out = []
for _ in range(reps):
    t0 = time.perf_counter()
    orc.randomized_interp_decomp(d["A"], d["om"], k)
    out.append(time.perf_counter() - t0)
print(json.dumps(out))
"""


def rid_oracle_seconds(A, om, reps):
    """Seconds per oracle randomized ID (sketch, CPQR of Y, refinement, FP64) of the
    first RID_CPU_COLS columns of A with the same Omega and k, single-threaded, in a
    fresh process (the sample goes through its stdin)."""
    import numpy as np

    Ah = A[:, :RID_CPU_COLS].double().cpu().numpy()
    Oh = om.double().cpu().numpy()
    r = subprocess.run([sys.executable, "-c", RID_ORACLE_SNIPPET, ROOT, str(RK), str(reps)],
                       input=_npy_bytes(np.savez, A=Ah, om=Oh), capture_output=True,
                       env=dict(os.environ, **ONE_THREAD), timeout=3600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr.decode(errors="replace")[-2000:])
    return json.loads(r.stdout.decode().strip().splitlines()[-1])


def rid_oracle_rate(secs):
    """IDs/s of the whole workload from the sample: every stage's work grows
    linearly with the number of columns (the sketch, the refinement, and the
    CPQR of Y for n >> k), so one ID takes RN / RID_CPU_COLS samples' time."""
    return RID_CPU_COLS / (RN * secs)


RID_SAMPLE = (f"oracle randomized ID (FP64, numpy, one thread) of the first {RID_CPU_COLS} of the {RN} columns of the "
              f"same A with the same Omega and k = {RK}, scaled to all columns by the column ratio")


def sampled_block(gbid, dev, steps, mats):
    """The column-sampling Optim RID (Sec. 2.2) of the headline matrices: p =
    k + floor(0.2 k) = 307 columns drawn without replacement (seed 7), CPQR of
    the 4096 x 307 sample, Z from the normal equations against all of A. ms per
    ID, the stage split, and the error on A beside the deterministic ID's."""
    import numpy as np
    import torch

    p = K_RANK + int(0.2 * K_RANK)
    idx = np.random.default_rng(7).choice(N, size=p, replace=False).astype(np.int32)
    out = {"workload": f"optim_rid_{M}x{N}_k{K_RANK}_p{p}"}
    for name, A in mats.items():
        ws = gbid.sampled_workspace(A.dtype, M, N, p, K_RANK, device=dev)
        for _ in range(3):
            gbid.id_decompose_sampled(A, idx, K_RANK, workspace=ws, sync=False)
        torch.cuda.synchronize()
        gbid.trace_enable(4 * steps + 8)
        s = torch.cuda.current_stream()
        ev = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            J, Z, _ = gbid.id_decompose_sampled(A, idx, K_RANK, workspace=ws, sync=False)
            e1.record(s)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        tr = gbid.trace_read()
        gbid.trace_enable(0)
        info = gbid.read_info(ws)
        out[name] = {"ms_per_step": ms, "value": 1000.0 / ms, "unit": UNIT, "status": info["status_name"],
                     "kernel_ms": {k: v[0] / v[1] for k, v in tr.items() if v[1]},
                     "rel_err": rel_error_gpu(A, J, Z)}
    return out


def listing_block(gbid, dev, steps, mats):
    """The paper's listing outputs on the headline matrices: Z from the normal
    equations R_k^T R_k Z = C^T A (Eq. final_eq) instead of the back
    substitution, and approx = C @ Z. ms per ID (normal-equation route), ms per
    reconstruction, and the error of approx."""
    import torch

    out = {"workload": f"listing_{M}x{N}_k{K_RANK}"}
    for name, A in mats.items():
        ws = gbid.Workspace.for_problem(A.dtype, M, N, K_RANK, device=dev, normal_eq=True)
        J = torch.empty(K_RANK, dtype=torch.int32, device=dev)
        Z = torch.empty(K_RANK, N, dtype=A.dtype, device=dev)
        approx = torch.empty(M, N, dtype=A.dtype, device=dev)
        rws = gbid.reconstruct_workspace(A.dtype, M, N, K_RANK, device=dev)
        for _ in range(3):
            gbid.id_decompose(A, K_RANK, normal_eq=True, workspace=ws, out=(J, Z), sync=False)
            gbid.id_reconstruct(A, J, Z, out=approx, workspace=rws, sync=False)
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        ev = []
        for _ in range(steps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(s)
            gbid.id_decompose(A, K_RANK, normal_eq=True, workspace=ws, out=(J, Z), sync=False)
            e[1].record(s)
            gbid.id_reconstruct(A, J, Z, out=approx, workspace=rws, sync=False)
            e[2].record(s)
            ev.append(e)
        torch.cuda.synchronize()
        id_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in ev)
        rc_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in ev)
        info = gbid.read_info(ws)
        err = (torch.linalg.norm(A.double() - approx.double()) / torch.linalg.norm(A.double())).item()
        out[name] = {"id_ms": id_ms, "reconstruct_ms": rc_ms, "value": 1000.0 / (id_ms + rc_ms), "unit": UNIT,
                     "status": info["status_name"], "rel_err": err}
    return out


def two_sided_block(gbid, dev, steps, mats):
    """The two-sided ID X^T A[I, J] Z (Sec. 1.2 footnote) of the headline
    matrices, and the row ID at scale: the 8192 x 4096 transpose of the FP64
    matrix (the m > n route), whose pivots and Z must equal the column ID's."""
    import torch

    out = {"workload": f"two_sided_{M}x{N}_k{K_RANK}; row_id_{N}x{M}_k{K_RANK}"}
    s = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            ev.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b) for a, b in ev)

    for name, A in mats.items():
        ws = gbid.two_sided_workspace(A.dtype, M, N, K_RANK, device=dev)
        I = torch.empty(K_RANK, dtype=torch.int32, device=dev)
        J = torch.empty(K_RANK, dtype=torch.int32, device=dev)
        X = torch.empty(K_RANK, M, dtype=A.dtype, device=dev)
        Z = torch.empty(K_RANK, N, dtype=A.dtype, device=dev)
        ms = timed(lambda: gbid.id_decompose_two_sided(A, K_RANK, workspace=ws, out=(I, J, X, Z), sync=False))
        _, _, _, _, infos = gbid.id_decompose_two_sided(A, K_RANK, workspace=ws, out=(I, J, X, Z))
        A64 = A.double()
        approx = X.double().T @ A64[I.long()][:, J.long()] @ Z.double()
        err = (torch.linalg.norm(A64 - approx) / torch.linalg.norm(A64)).item()
        out[name] = {"ms_per_step": ms, "value": 1000.0 / ms, "unit": UNIT, "rel_err": err,
                     "status": [i["status_name"] for i in infos]}
    At = mats["f64"].T.contiguous()
    ws = gbid.Workspace.for_problem(At.dtype, N, M, K_RANK, device=dev)
    Jr = torch.empty(K_RANK, dtype=torch.int32, device=dev)
    Zr = torch.empty(K_RANK, N, dtype=At.dtype, device=dev)
    ms = timed(lambda: gbid.id_decompose(At, K_RANK, workspace=ws, out=(Jr, Zr), sync=False))
    info = gbid.read_info(ws)
    out["row_id_f64"] = {"ms_per_step": ms, "value": 1000.0 / ms, "unit": UNIT, "status": info["status_name"],
                         "transposed": info["transposed"]}
    del At
    return out


def sparse_block(gbid, dev, steps):
    """Sparse input (CSR) at the headline size: 4096 x 8192, 1% nonzeros with
    power-law column degrees, U(0,1) values (seed 6), k = 256, FP64; ms per ID
    from device-resident CSR arrays, and the dense ID of the same matrix."""
    import numpy as np
    import torch

    import synth

    rowptr, colind, vals = synth.sparse_powerlaw_csr(M, N, 0.01, 6)
    r = torch.as_tensor(rowptr, device=dev)
    c = torch.as_tensor(colind, device=dev)
    v = torch.as_tensor(vals, dtype=torch.float64, device=dev)
    ws = gbid.csr_workspace(torch.float64, M, N, K_RANK, device=dev)
    J = torch.empty(K_RANK, dtype=torch.int32, device=dev)
    Z = torch.empty(K_RANK, N, dtype=torch.float64, device=dev)
    for _ in range(3):
        gbid.id_decompose_csr(r, c, v, (M, N), K_RANK, workspace=ws, out=(J, Z), sync=False)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ev = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        gbid.id_decompose_csr(r, c, v, (M, N), K_RANK, workspace=ws, out=(J, Z), sync=False)
        e1.record(s)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    info = gbid.read_info(ws)
    A = torch.zeros(M, N, dtype=torch.float64, device=dev)
    rows = torch.repeat_interleave(torch.arange(M, device=dev), torch.diff(r))
    A.index_put_((rows, c.long()), v, accumulate=True)
    err = rel_error_gpu(A, J, Z)
    return {"workload": f"csr_{M}x{N}_density0.01_k{K_RANK}_f64", "nnz": int(vals.size), "ms_per_step": ms,
            "value": 1000.0 / ms, "unit": UNIT, "status": info["status_name"], "rel_err": err}


BATCH_COUNT = 4096


def differentiable_block(gbid, dev, steps, cpu_sample=0):
    """The differentiable form: 256 FP32 matrices 512 x 1024, s_i = (1+i)^-2,
    k = 64 (seed 5): forward by one batched launch, then dL/dA for
    L = <G, Z> (G ~ N(0,1), seed 5) by id_backward per matrix, the 256 backward
    calls spread over 16 streams (one workspace each) and replayed from one
    CUDA graph."""
    import torch

    import synth

    nb, m, n, k = 256, 512, 1024, 64
    s_ = synth.spectrum("poly2", m)
    mats = [synth.lowrank(m, n, s_, 5000 + b, device=dev, dtype=torch.float32, gen_dtype=torch.float32)
            for b in range(nb)]
    g = torch.Generator(device=dev).manual_seed(5)
    Gs = [torch.randn(k, n, generator=g, device=dev) for _ in range(nb)]
    plan = gbid.BatchedPlan(mats, [k] * nb, autotune=True)     # tile shape tuned here, before timing
    bplan = gbid.BackwardPlan(m, n, k, streams=16, device=dev)
    dAs = [torch.empty(m, n, device=dev) for _ in range(nb)]

    def backward_all():
        bplan.run(mats, plan.J, plan.Z, Gs, dAs)

    plan.run()
    backward_all()
    torch.cuda.synchronize()
    graph = None
    try:
        graph = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            with torch.cuda.graph(graph, stream=cs):
                backward_all()
        torch.cuda.current_stream().wait_stream(cs)
        torch.cuda.synchronize()
    except Exception as exc:
        print(f"backward graph capture: {exc}", file=sys.stderr)
        graph = None
        torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ev = []
    for _ in range(max(3, min(steps, 10))):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        plan.run()
        e1.record(st)
        if graph is not None:
            graph.replay()
        else:
            backward_all()
        e2.record(st)
        ev.append((e0, e1, e2))
    torch.cuda.synchronize()
    fwd = statistics.mean(a.elapsed_time(b) for a, b, _ in ev)
    bwd = statistics.mean(b.elapsed_time(c) for _, b, c in ev)
    infos = plan.read_infos()
    ok = sum(1 for i in infos if i["status_name"] == "ID_OK")
    cpu = None
    if cpu_sample > 0:
        sample = [A.double().cpu().numpy() for A in mats[:cpu_sample]]
        grads = [G.double().cpu().numpy() for G in Gs[:cpu_sample]]
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        t1 = time_oracle_many(sample, [k] * len(sample), 1, grads=grads)
        tp = time_oracle_many(sample, [k] * len(sample), cores, grads=grads)
        what = (f"forward ID and gradient of the first {len(sample)} of the {nb} problems (FP32 values in FP64) by "
                f"the oracle, numpy")
        cpu = {"value": len(sample) / t1, "unit": "IDs/s (forward + backward)", "cores": 1, "kind": "oracle",
               "sample": f"{what}, one thread ({t1:.1f} s)",
               "all_cores": {"value": len(sample) / tp, "unit": "IDs/s (forward + backward)", "cores": cores,
                             "kind": "oracle", "sample": f"{what}, {cores} single-threaded processes ({tp:.1f} s)"}}
    return {"workload": "diff_256x512x1024_k64_f32", "fwd_ms": fwd, "bwd_ms": bwd, "cpu_baseline": cpu,
            "value": nb * 1000.0 / (fwd + bwd), "unit": "IDs/s (forward + backward)",
            "bwd_graph": graph is not None, "statuses_ok": ok,
            "fwd_tuned_instance": gbid.batched_configs(torch.float32)[plan.config]}


def latency_block(gbid, dev, steps):
    """The small-ID latency workload: 200 x 400 FP64, s_i = 2^(-i/2), k = 20
    (seed 1), back-to-back IDs in one stream (A is 640 KB and stays in L2).
    Reported plainly and replayed from a CUDA graph of 20 IDs."""
    import torch

    import synth

    A = synth.lowrank(200, 400, synth.spectrum("pow2_half", 200), 1, device=dev)
    k = 20
    ws = gbid.Workspace.for_problem(A.dtype, 200, 400, k, device=dev)
    J = torch.empty(k, dtype=torch.int32, device=dev)
    Z = torch.empty(k, 400, dtype=A.dtype, device=dev)
    for _ in range(5):
        gbid.id_decompose(A, k, workspace=ws, out=(J, Z), sync=False)
    torch.cuda.synchronize()
    reps = max(50, 20 * steps)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        gbid.id_decompose(A, k, workspace=ws, out=(J, Z), sync=False)
    e1.record(s)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / reps
    us_graph = None
    try:
        g = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            with torch.cuda.graph(g, stream=cs):
                for _ in range(20):
                    gbid.id_decompose(A, k, workspace=ws, out=(J, Z), sync=False)
        torch.cuda.current_stream().wait_stream(cs)
        g.replay()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(max(3, reps // 20)):
            g.replay()
        e1.record(s)
        torch.cuda.synchronize()
        us_graph = e0.elapsed_time(e1) * 1e3 / (20 * max(3, reps // 20))
    except Exception as exc:                 # capture refused: report the stream-ordered figure only
        print(f"latency graph capture: {exc}", file=sys.stderr)
        torch.cuda.synchronize()
    best = us_graph if us_graph is not None else us
    info = gbid.read_info(ws)
    err = rel_error_gpu(A, J, Z)
    trail = sum((200 - j) * (400 - j) for j in range(k)) * 8
    # the same matrix in FP32, which the default sends to the thread-block-cluster kernel
    A32 = A.float()
    ws32 = gbid.Workspace.for_problem(A32.dtype, 200, 400, k, device=dev)
    Z32 = torch.empty(k, 400, dtype=A32.dtype, device=dev)
    for _ in range(5):
        gbid.id_decompose(A32, k, workspace=ws32, out=(J, Z32), sync=False)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        gbid.id_decompose(A32, k, workspace=ws32, out=(J, Z32), sync=False)
    e1.record(s)
    torch.cuda.synchronize()
    us32 = e0.elapsed_time(e1) * 1e3 / reps
    info32 = gbid.read_info(ws32)
    return {"workload": "id_200x400_k20_f64", "us_per_id": us, "us_per_id_graph": us_graph,
            "value": 1e6 / best, "unit": UNIT, "rel_err": err, "tail_bound": 2.0 ** -10,
            "status": info["status_name"],
            "f32": {"us_per_id": us32, "engine": info32["engine"], "rel_err": rel_error_gpu(A32, J, Z32)},
            "engine": info["engine"],
            "l2_gbs_trailing_bytes": trail / (best * 1e-6) / 1e9,
            "note": "trailing-GEMV bytes s*sum_j (m-j)(n-j) over the best per-ID time (A stays in L2)"}


def batched_block(gbid, dev, steps, cpu_sample=0):
    """The batched form: 4096 FP32 matrices, m ~ U[32, 256], n ~ U[m, 4m],
    k ~ U[8, 64], s_i = exp(-8 i / m), 10% non-negative sparse (seed 4), all
    decomposed by one persistent launch. The inputs plus scratch (about 1.7 GB)
    exceed L2, so no flush is needed between launches. With cpu_sample > 0 the
    oracle decomposes the first cpu_sample problems on the host, on one core
    and on every core (one single-threaded process per core)."""
    import torch

    import synth

    probs = synth.batched_uneven(BATCH_COUNT, 4, dtype=torch.float32, device=dev)
    mats = [p["A"] for p in probs]
    ks = [p["k"] for p in probs]
    plan = gbid.BatchedPlan(mats, ks, autotune=True)            # tile shape tuned here, before timing
    for _ in range(3):
        plan.run()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ev = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        plan.run()
        e1.record(s)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    infos = plan.read_infos()
    flops = sum(flops_cpqr(min(p["m"], p["n"]), max(p["m"], p["n"]), p["k"]) +
                flops_solve(max(p["m"], p["n"]), p["k"]) for p in probs)
    ratios = []
    for p, J, Z in zip(probs, plan.J, plan.Z):
        if p["kind"] != "lowrank":
            continue
        A64 = p["A"].double()
        err = (torch.linalg.norm(A64 - A64[:, J.long()] @ Z.double()) / torch.linalg.norm(A64)).item()
        tail = synth.tail_bound(synth.spectrum("exp8m", min(p["m"], p["n"]), m=p["m"]), p["k"])
        if tail > 1e-5:        # below that the FP32 rounding of the input dominates the floor
            ratios.append(err / tail)
    statuses = {}
    for i in infos:
        statuses[i["status_name"]] = statuses.get(i["status_name"], 0) + 1
    cpu = None
    if cpu_sample > 0:
        sample = [p["A"].double().cpu().numpy() for p in probs[:cpu_sample]]
        ks_s = ks[:cpu_sample]
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        t1 = time_oracle_many(sample, ks_s, 1)
        tp = time_oracle_many(sample, ks_s, cores)
        what = (f"complete IDs of the first {len(sample)} of the {BATCH_COUNT} problems (FP32 values in FP64) "
                f"by the oracle, numpy")
        cpu = {"value": len(sample) / t1, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{what}, one thread ({t1:.1f} s)",
               "all_cores": {"value": len(sample) / tp, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{what}, {cores} single-threaded processes ({tp:.1f} s)"}}
    return {"workload": f"batched_{BATCH_COUNT}_uneven_f32", "ms_per_launch": ms,
            "value": BATCH_COUNT * 1000.0 / ms, "unit": UNIT, "eff_tflops": flops / (ms * 1e-3) / 1e12,
            "launches_per_step": 1, "statuses": statuses,
            "tuner": {"chosen": gbid.batched_configs(torch.float32)[plan.config],
                      "ms_per_instance": [round(x, 3) for x in plan.tune_ms]},
            "err_over_tail": {"median": statistics.median(ratios), "max": max(ratios)}, "cpu_baseline": cpu}


def compare_block(gbid, dev, steps):
    """The mixed-precision and batched forms beside the plain FP64 GPU ID at
    their reconstruction errors: the randomized ID of the 16384 x 32768 FP32
    matrix against the deterministic FP64 ID of the same matrix (promoted; the
    FP64 CPQR at 16384 rows runs k_cpqr's one-CTA-per-SM configuration, which
    the tall-matrix parity tests cover), and the FP32 batched launch against the
    FP64 batched launch of the same 4096 problems."""
    import torch

    import synth

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            out = fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    out = {"workload": "same-error comparisons"}
    A, om = rid_inputs(dev)
    ws = gbid.rid_workspace(RM, RN, RL, RK, device=dev)
    ms_r, (J, Z, _) = timed(lambda: gbid.id_decompose_randomized(A, om, RK, workspace=ws, sync=False), max(2, steps))
    err_r = rid_error(A, J, Z)
    del ws, J, Z
    A64 = A.double()
    ws64 = gbid.Workspace.for_problem(torch.float64, RM, RN, RK, device=dev)
    ms_d, (J, Z, _) = timed(lambda: gbid.id_decompose(A64, RK, workspace=ws64, sync=False), 2)
    info = gbid.read_info(ws64)
    err_d = rid_error(A64, J, Z)
    out["randomized_vs_fp64"] = {"matrix": f"{RM}x{RN} k={RK}", "randomized_ms": ms_r, "randomized_rel_err": err_r,
                                 "randomized_ids_per_s": 1000.0 / ms_r, "fp64_ms": ms_d, "fp64_rel_err": err_d,
                                 "fp64_ids_per_s": 1000.0 / ms_d, "fp64_status": info["status_name"],
                                 "speedup": ms_d / ms_r, "err_ratio": err_r / err_d,
                                 "tail_bound": synth.tail_bound(synth.spectrum("poly1.5", RM), RK)}
    del A, A64, J, Z, ws64
    torch.cuda.empty_cache()
    probs = synth.batched_uneven(BATCH_COUNT, 4, dtype=torch.float32, device=dev)
    res = {}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        mats = [p["A"].to(dt) for p in probs]
        plan = gbid.BatchedPlan(mats, [p["k"] for p in probs], autotune=True)
        ms, _ = timed(plan.run, steps)
        ratios = []
        for p, A_, J_, Z_ in zip(probs, mats, plan.J, plan.Z):
            if p["kind"] == "lowrank":
                A_64 = A_.double()
                ratios.append((torch.linalg.norm(A_64 - A_64[:, J_.long()] @ Z_.double()) /
                               torch.linalg.norm(A_64)).item())
        res[name] = {"ms_per_launch": ms, "IDs_per_s": BATCH_COUNT * 1000.0 / ms,
                     "median_rel_err": statistics.median(ratios), "instance": batched_configs_of(gbid, dt, plan)}
    res["speedup_f32_over_f64"] = res["f64"]["ms_per_launch"] / res["f32"]["ms_per_launch"]
    out["batched_f32_vs_f64"] = res
    return out


def batched_configs_of(gbid, dt, plan):
    return gbid.batched_configs(dt)[plan.config]


def guarded(name, fn, *a):
    """fn(*a), or {"error": ...} with the traceback on stderr if it raises."""
    import traceback

    try:
        return fn(*a)
    except Exception as exc:                      # noqa: BLE001 - reported in the JSON line
        traceback.print_exc()
        print(f"side workload {name} failed: {exc!r}", file=sys.stderr, flush=True)
        return {"workload": name, "error": repr(exc)[:500]}


def deterministic_block(gbid, dev, args, world, hbm_peak, peak_src, cpu_ok):
    """The deterministic ID of the 4096 x 8192 matrix (s_i = exp(-i/64), k = 256)
    in FP64 and FP32: per-step device times with L2 flushed between steps, the
    error, rooflines of k_cpqr in the SURVEY's units (algorithmic bytes against
    HBM; FP64 also the flop convention and the executed FP64 operations against
    the FP64 peak), the end-to-end rate through the host-buffer entry point and
    one complete oracle ID of the FP64 matrix on one core. Returns (block, matrices)."""
    import torch

    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)   # 256 MB > L2
    res = {}
    mats = {}
    for name, dt in (("f64", torch.float64), ("f32", torch.float32)):
        A = make_input(dev, dt)
        ms, tr, info, J, Z = time_gpu(gbid, A, args.steps, args.warmup, flush)
        mean_ms = max_over_ranks(statistics.mean(ms), world, dev)
        cp_ms, cp_n = tr.get("cpqr", (0.0, 0))
        cp = cp_ms / cp_n if cp_n else float("nan")
        s = A.element_size()
        b = bytes_cpqr(M, N, K_RANK, s)
        ach = b / (cp * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
                "traffic": NCU_TRAFFIC[name], "kernel": f"k_cpqr<{'double' if s == 8 else 'float'}>", "kernel_ms": cp,
                "algorithmic_bytes": b,
                "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs" if peak_src == "measured" else "of fallback"}
        if s == 8:
            conv = flops_cpqr(M, N, K_RANK) / (cp * 1e-3) / 1e12
            exe = fp64_flops_executed(M, N, K_RANK) / (cp * 1e-3) / 1e12
            roof["fp64"] = {"bound": "alu", "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                            "convention_achieved": conv, "convention_frac": conv / FP64_PEAK_TFLOPS,
                            "executed_achieved": exe, "executed_frac": exe / FP64_PEAK_TFLOPS,
                            "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (a DFMA probe: 1.196)",
                            "note": "the convention counts 4 (m-j)(n-j) per step; the left-looking form executes fewer"}
        eff = (flops_cpqr(M, N, K_RANK) + flops_solve(N, K_RANK)) / (mean_ms * 1e-3) / 1e12
        res[name] = {"ms_per_step": mean_ms, "value": aggregate_rate(mean_ms, world), "unit": UNIT, "eff_tflops": eff,
                     "rel_err": rel_error_gpu(A, J, Z), "status": info["status_name"], "roofline": roof,
                     "launches_per_step": gbid.launch_count(dt, M, N, K_RANK)}
        mats[name] = A
    del flush
    e2e_v, h2d, d2h = e2e_rate(gbid, mats["f64"], max(2, min(args.steps, 5)))
    res["f64"]["e2e"] = {"value": aggregate_rate(max_over_ranks(1000.0 / e2e_v, world, dev), world), "unit": UNIT,
                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    res["f32"]["speedup_vs_f64"] = res["f32"]["value"] / res["f64"]["value"]
    res["tail_bound"] = __import__("synth").tail_bound(__import__("synth").spectrum("exp64", M), K_RANK)
    res["workload"] = WORKLOAD
    if cpu_ok:
        def one_oracle_id():
            secs = time_oracle(mats["f64"].cpu().numpy(), K_RANK, 1, full=True)
            return {"value": 1.0 / secs[0], "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"one complete rank-{K_RANK} ID of the same 4096 x 8192 FP64 matrix by the oracle "
                              f"({secs[0]:.1f} s, numpy, one thread)"}

        res["cpu_baseline"] = guarded("cpu_baseline", one_oracle_id)
    return res, mats


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
    import synth

    dev = torch.device("cuda", local)
    cpu_ok = rank == 0 and world == 1 and not args.no_cpu_baseline
    if args.only in ("batched", "latency", "differentiable", "compare"):  # one side workload alone
        if args.only == "compare":
            side = compare_block(gbid, dev, max(3, min(args.steps, 10)))
        elif args.only == "latency":
            side = latency_block(gbid, dev, args.steps)
        elif args.only == "differentiable":
            side = differentiable_block(gbid, dev, args.steps, DIFF_CPU_SAMPLE if cpu_ok else 0)
        else:
            side = batched_block(gbid, dev, max(3, min(args.steps, 10)), BATCHED_CPU_SAMPLE if cpu_ok else 0)
        if rank == 0:
            print(json.dumps(dict(side, n_gpus=world, steps=args.steps, warmup=args.warmup)), flush=True)
        return 0
    hbm_peak, peak_src = load_peaks()

    # ---- the headline: the randomized ID of the 16384 x 32768 matrix
    A, om = rid_inputs(dev)
    ms, per, clocks, info, J, Z = rid_time(gbid, A, om, args.steps, args.warmup, world, local)
    mean_ms = max_over_ranks(statistics.mean(ms), world, dev)
    err = rid_error(A, J, Z)
    kernels, dom = rid_rooflines(per, hbm_peak, peak_src)
    fl = rid_flops()
    eff = sum(fl.values()) / (mean_ms * 1e-3) / 1e12
    e2e_v, h2d, d2h = rid_e2e(gbid, A, om, max(3, min(2 * args.steps, 20)))
    e2e_v = aggregate_rate(max_over_ranks(1000.0 / e2e_v, world, dev), world)
    cpu = None
    if cpu_ok:
        def oracle_sample():
            secs = rid_oracle_seconds(A, om, 2)
            return {"value": rid_oracle_rate(statistics.mean(secs)), "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": RID_SAMPLE + f" ({statistics.mean(secs):.1f} s per sample, 2 samples)"}

        cpu = guarded("cpu_baseline", oracle_sample)
    tail = synth.tail_bound(synth.spectrum("poly1.5", RM), RK)
    del A, om, J, Z
    torch.cuda.empty_cache()

    # ---- side workloads: a failure in one is reported in the line, not fatal to the headline
    side_steps = max(3, min(args.steps, 10))
    with_det = args.only in ("all", "id", "sampled")
    with_sampled = args.only in ("all", "sampled")
    with_all = args.only == "all"
    det, mats = None, None
    if with_det:
        try:
            det, mats = deterministic_block(gbid, dev, args, world, hbm_peak, peak_src, cpu_ok)
        except Exception as exc:                  # noqa: BLE001 - reported in the JSON line
            import traceback

            traceback.print_exc()
            det = {"workload": WORKLOAD, "error": repr(exc)[:500]}
    samp = guarded("sampled", sampled_block, gbid, dev, side_steps, mats) if with_sampled and mats else None
    lst = guarded("listing", listing_block, gbid, dev, side_steps, mats) if with_sampled and mats else None
    two = guarded("two_sided", two_sided_block, gbid, dev, side_steps, mats) if with_sampled and mats else None
    spa = guarded("sparse", sparse_block, gbid, dev, side_steps) if with_sampled else None
    mats = None
    torch.cuda.empty_cache()
    bat = guarded("batched", batched_block, gbid, dev, side_steps, BATCHED_CPU_SAMPLE if cpu_ok else 0) \
        if with_all else None
    lat = guarded("latency", latency_block, gbid, dev, args.steps) if with_all else None
    dif = guarded("differentiable", differentiable_block, gbid, dev, args.steps, DIFF_CPU_SAMPLE if cpu_ok else 0) \
        if with_all else None
    cmp = guarded("compare", compare_block, gbid, dev, side_steps) if with_all else None
    if world > 1 and dist.is_initialized():
        dist.barrier()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": aggregate_rate(mean_ms, world), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "precision": "BF16 sketch (FP32 accumulation), FP32 CPQR with FP64 norms, FP32 solve of the sketch's T, "
                     "3xTF32 refinement products, FP64 Gram factor",
        "data": "synthetic", "config": rid_config(max(world, args.gpus)),
        "eff_tflops": eff, "flops_convention": fl, "rel_err": err, "tail_bound": tail, "status": info["status_name"],
        "roofline": dict(kernels[dom], stage=dom) if dom else None,
        "kernels": kernels, "kernel_ms": per,
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": gbid.rid_launch_count(RM, RN, RL, RK) * args.steps,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "compare": cmp,
        "deterministic": det,
        "sampled": samp,
        "listing": lst,
        "two_sided": two,
        "sparse": spa,
        "batched": bat,
        "latency": lat,
        "differentiable": dif,
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
    ap.add_argument("--only", default="all",
                    choices=["all", "randomized", "id", "sampled", "batched", "latency", "differentiable", "compare"],
                    help="randomized: the headline alone; id: the headline and the 4096 x 8192 deterministic ID; "
                         "sampled: those and the column-sampling RID, the listing outputs, the two-sided ID and the "
                         "sparse ID; batched / latency / differentiable / compare: that side workload alone")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gbid(args)


if __name__ == "__main__":
    sys.exit(main())
