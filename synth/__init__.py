"""Seeded synthetic inputs for the interpolative-decomposition workloads.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests. It holds no arithmetic of the method itself (no pivoting, no reflectors,
no triangular solves): it only draws random numbers and assembles matrices of a
prescribed singular spectrum, so that both sides are fed identical inputs.

Workloads (names state what they are; sizes are part of the name):

* ``id_200x400_k20_f64``     A = U diag(s) V^T, s_i = 2^(-i/2), rank 20, FP64.
* ``id_4096x8192_k256``      s_i = exp(-i/64), rank 256, FP64 and FP32, plus an
                             exact-rank-256 variant (s_i = 0 for i >= 256).
* ``rid_16384x32768_k512``   s_i = (1+i)^-1.5, FP32, Gaussian sketch of
                             (k+10) rows rounded to BF16.
* ``batched_4096_uneven``    4096 FP32 matrices, m ~ U[32,256], n ~ U[m,4m],
                             k ~ U[8,64], s_i = exp(-8i/m); 10 % of them are
                             non-negative sparse (density 5 %, entries U(0,1)).
* ``diff_256x512x1024_k64``  256 FP32 matrices 512x1024, s_i = (1+i)^-2, k=64,
                             cotangent G ~ N(0,1).

U and V are Haar-distributed: the Q factor of a QR of an N(0,1) matrix with
its columns multiplied by sign(diag R) (Mezzadri, "How to generate random
matrices from the classical compact groups", 2007). Indices of s are 0-based.

The paper's own synthetic datasets (Sec. 3, Appendix A: Boolean, Gaussian and
Uniform matrices of size 784x1000) are reproduced by ``paper_dataset``.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

__all__ = [
    "haar",
    "lowrank",
    "spectrum",
    "tail_bound",
    "paper_dataset",
    "gaussian_sketch_bf16",
    "batched_uneven",
    "WORKLOADS",
]


def _preload_cuda_linalg(device) -> None:
    """Load torch's CUDA linear-algebra library by absolute path.

    torch opens it lazily by bare name on the first GPU QR; under a profiler
    that injects itself into the process that lookup can fail, so the
    generators load it explicitly first.
    """
    if torch.device(device).type != "cuda":
        return
    path = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
    if os.path.exists(path):
        ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed))
    return g


def haar(rows: int, cols: int, seed: int, device="cpu", dtype=torch.float64) -> torch.Tensor:
    """rows x cols matrix with Haar-distributed orthonormal columns (rows >= cols)."""
    assert rows >= cols
    _preload_cuda_linalg(device)
    g = _gen(seed, device)
    G = torch.randn(rows, cols, generator=g, device=device, dtype=dtype)
    Q, R = torch.linalg.qr(G, mode="reduced")
    d = torch.sign(torch.diagonal(R))
    d = torch.where(d == 0, torch.ones_like(d), d)
    return Q * d.unsqueeze(0)


def spectrum(kind: str, r: int, *, rank: int | None = None, m: int | None = None) -> np.ndarray:
    """Singular values s_0..s_{r-1} (0-based index i) of a named spectrum."""
    i = np.arange(r, dtype=np.float64)
    if kind == "pow2_half":          # s_i = 2^(-i/2)
        s = 2.0 ** (-i / 2.0)
    elif kind == "exp64":            # s_i = exp(-i/64)
        s = np.exp(-i / 64.0)
    elif kind == "poly1.5":          # s_i = (1+i)^-1.5
        s = (1.0 + i) ** -1.5
    elif kind == "poly2":            # s_i = (1+i)^-2
        s = (1.0 + i) ** -2.0
    elif kind == "exp8m":            # s_i = exp(-8 i / m)
        assert m is not None
        s = np.exp(-8.0 * i / float(m))
    else:
        raise ValueError(kind)
    if rank is not None:
        s[rank:] = 0.0
    return s


def tail_bound(s: np.ndarray, k: int) -> float:
    """sqrt(sum_{i>=k} s_i^2 / sum_i s_i^2): the rank-k Eckart-Young floor."""
    s2 = np.asarray(s, dtype=np.float64) ** 2
    return float(math.sqrt(s2[k:].sum() / s2.sum()))


def lowrank(m: int, n: int, s: np.ndarray, seed: int, device="cpu", dtype=torch.float64,
            gen_dtype=torch.float64) -> torch.Tensor:
    """A = U diag(s) V^T (m x n, row-major) with Haar U (m x r) and V (n x r), r = min(m, n).

    U uses seed ``2*seed`` and V seed ``2*seed+1`` so the two factors are drawn
    from independent streams. ``gen_dtype`` is the precision of the assembly.
    """
    r = min(m, n)
    s = np.asarray(s, dtype=np.float64)
    assert s.shape == (r,)
    U = haar(m, r, 2 * seed, device, gen_dtype)
    V = haar(n, r, 2 * seed + 1, device, gen_dtype)
    st = torch.as_tensor(s, dtype=gen_dtype, device=device)
    A = (U * st.unsqueeze(0)) @ V.T
    return A.to(dtype).contiguous()


def paper_dataset(name: str, seed: int, m: int = 784, n: int = 1000) -> np.ndarray:
    """The paper's synthetic dense datasets (Appendix A), as FP64 numpy arrays.

    boolean: entries drawn uniformly from {0, 1}; gaussian: standard normal;
    uniform: uniform on [0, 1).
    """
    rng = np.random.default_rng(seed)
    if name == "boolean":
        return rng.integers(0, 2, size=(m, n)).astype(np.float64)
    if name == "gaussian":
        return rng.standard_normal((m, n))
    if name == "uniform":
        return rng.random((m, n))
    raise ValueError(name)


def gaussian_sketch_bf16(l: int, m: int, seed: int, device="cpu") -> torch.Tensor:
    """l x m test matrix with N(0,1) entries rounded to BF16 (returned as bfloat16)."""
    g = _gen(seed, device)
    return torch.randn(l, m, generator=g, device=device, dtype=torch.float32).to(torch.bfloat16)


def batched_uneven(count: int, seed: int, *, m_range=(32, 256), k_range=(8, 64), sparse_frac=0.1,
                   density=0.05, dtype=torch.float32, device="cpu"):
    """Uneven batch of low-rank matrices (hierarchical-compression use case).

    Returns a list of dicts ``{"m", "n", "k", "A"}``. m ~ U[m_lo, m_hi],
    n ~ U[m, 4m], k ~ U[k_lo, min(k_hi, m)], s_i = exp(-8 i / m); a
    ``sparse_frac`` share of the matrices are instead non-negative sparse with
    the given density and U(0,1) entries (stored dense).
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        n = int(rng.integers(m, 4 * m + 1))
        k = int(rng.integers(k_range[0], min(k_range[1], m) + 1))
        sub = int(rng.integers(0, 2**31 - 1))
        if rng.random() < sparse_frac:
            r2 = np.random.default_rng(sub)
            mask = r2.random((m, n)) < density
            vals = r2.random((m, n))
            A = torch.as_tensor(np.where(mask, vals, 0.0), dtype=dtype, device=device)
            kind = "sparse"
        else:
            A = lowrank(m, n, spectrum("exp8m", min(m, n), m=m), sub, device=device).to(dtype=dtype)
            kind = "lowrank"
        out.append({"m": m, "n": n, "k": k, "A": A.contiguous(), "kind": kind})
    return out


def sparse_powerlaw_csr(m: int, n: int, density: float, seed: int, *, alpha: float = 1.2):
    """Seeded sparse m x n matrix in CSR form with a power-law column degree
    distribution (column l gets a share proportional to (1 + r_l)^-alpha of the
    density * m * n nonzeros, r a random permutation; capped at m), rows drawn
    uniformly per column, values U(0, 1) (non-negative, like the paper's
    sparse and Boolean data). Returns (rowptr int64 (m+1), colind int32,
    values float64), rows sorted, column indices sorted within a row."""
    rng = np.random.default_rng(seed)
    w = (1.0 + rng.permutation(n)) ** -alpha
    deg = np.minimum(rng.multinomial(int(density * m * n), w / w.sum()), m)
    rows, cols = [], []
    for l in np.flatnonzero(deg):
        r = rng.choice(m, size=int(deg[l]), replace=False)
        rows.append(r)
        cols.append(np.full(r.size, l))
    rows = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    cols = np.concatenate(cols) if cols else np.zeros(0, np.int64)
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    vals = rng.random(rows.size)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    return np.cumsum(rowptr), cols.astype(np.int32), vals


# name -> (m, n, k, spectrum kind, seed)
WORKLOADS = {
    "id_200x400_k20_f64": dict(m=200, n=400, k=20, spec="pow2_half", seed=1),
    "id_4096x8192_k256": dict(m=4096, n=8192, k=256, spec="exp64", seed=2),
    "rid_16384x32768_k512": dict(m=16384, n=32768, k=512, spec="poly1.5", seed=3, oversample=10),
    "diff_256x512x1024_k64": dict(m=512, n=1024, k=64, spec="poly2", seed=5, batch=256),
}
