"""Oracle work for the GPU parity tests, run in worker processes.

The full-size checks (every pivot and all of Z at 4096 x 8192, every step of
the 16384 x 32768 sketch's CPQR, all 4096 problems of the uneven batch) are
CPU-bound in the FP64 oracle; they run here in a pool of spawned processes
(spawn: the parent already holds a CUDA context, which a forked child must
not inherit). Nothing here computes anything but calls into ``oracle/``.
"""
from __future__ import annotations

import contextlib
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np

from oracle import id_oracle as orc

_BLAS_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


@contextlib.contextmanager
def oracle_pool(workers: int, blas_threads: int):
    """A spawn pool whose workers each use ``blas_threads`` BLAS threads (the
    variables are set while the workers start and restored afterwards; the
    parent's own BLAS is already loaded and keeps its setting)."""
    saved = {v: os.environ.get(v) for v in _BLAS_VARS}
    for v in _BLAS_VARS:
        os.environ[v] = str(max(1, blas_threads))
    try:
        with ProcessPoolExecutor(max_workers=max(1, workers), mp_context=mp.get_context("spawn")) as ex:
            yield ex
    finally:
        for v, old in saved.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def forced_id(A: np.ndarray, k: int, J: np.ndarray) -> dict:
    """The oracle's ID of A with the GPU's pivots forced (m > n: the row ID).

    Returns Z, the per-step shortfall of each forced pivot against the greedy
    rule (1 - nu / top, what verify_pivots reports, from the same pass), the
    numerical rank of the forced run and cond(X[:, J])."""
    _, Z, info = orc.interp_decomp(A, k, pivots=J)
    X = A.T if info["transposed"] else A
    top = info["top"]
    short = np.where(top > 0, 1.0 - info["nu"] / np.where(top > 0, top, 1.0), 0.0)
    return {"Z": Z, "short": short, "rank": int(info["rank"]), "cond": float(np.linalg.cond(X[:, J]))}


def ls_z(A: np.ndarray, J: np.ndarray) -> np.ndarray:
    """The oracle's least-squares Z for the skeleton J."""
    return orc.ls_interp(A, J)
