"""Python binding of the GB300 interpolative-decomposition library (libgbid.so).

Argument marshalling only: every step of the decomposition runs in the CUDA
kernels behind the C ABI declared in include/gbid.h. PyTorch supplies device
memory (outputs and workspace) and the current stream. There is no CPU
fallback: if the library is not built, or a tensor is not on a CUDA device,
the call raises.

Method (Advani & O'Hagan, arXiv 2105.07076): rank-k interpolative
decomposition A ~= A[:, J] Z from a column-pivoted Householder QR stopped
after k pivots (Sec. 2.1, Sec. 4.1), with Z P = [I  R11^{-1} R12]; for m > n
the method runs on A^T and returns a row ID A ~= Z^T A[J, :] (Sec. 2 footnote).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgbid.so")

ID_OK = 0
ID_RANK_DEFICIENT = 1
ID_EINVAL = -1
ID_ENOMEM = -2
ID_ECUDA = -3
ID_ENONFINITE = -4
ID_ETIMEOUT = -5
STATUS_NAMES = {0: "ID_OK", 1: "ID_RANK_DEFICIENT", -1: "ID_EINVAL", -2: "ID_ENOMEM", -3: "ID_ECUDA",
                -4: "ID_ENONFINITE", -5: "ID_ETIMEOUT"}

ID_F64 = 0
ID_F32 = 1
ENGINE_AUTO, ENGINE_GRID, ENGINE_CLUSTER = 0, 1, 2
ENGINE_NAMES = {1: "grid", 2: "cluster", 3: "batched"}
_DTYPES = {torch.float64: ID_F64, torch.float32: ID_F32}


class IdOpts(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int32), ("refine", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("zsolve", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class IdInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("rank", ctypes.c_int32), ("transposed", ctypes.c_int32),
                ("n_recompute", ctypes.c_int32), ("n_gt2", ctypes.c_int64), ("max_abs_z", ctypes.c_double),
                ("r00", ctypes.c_double), ("nb", ctypes.c_int32), ("refined", ctypes.c_int32),
                ("engine", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("err_est", ctypes.c_double)]

    def as_dict(self):
        return {"status": self.status, "status_name": STATUS_NAMES.get(self.status, str(self.status)),
                "rank": self.rank, "transposed": bool(self.transposed), "n_recompute": self.n_recompute,
                "n_gt2": self.n_gt2, "max_abs_z": self.max_abs_z, "r00": self.r00, "nb": self.nb,
                "refined": bool(self.refined), "engine": ENGINE_NAMES.get(self.engine, self.engine),
                "err_est": self.err_est}


# Return codes that mean the call itself failed; device-detected conditions
# (ID_RANK_DEFICIENT, ID_ENONFINITE, ID_ETIMEOUT) come back in the info dict.
_CALL_ERRORS = (ID_EINVAL, ID_ENOMEM, ID_ECUDA)


class IdError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")
        self.status = status


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIG = {
    "id_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64, _P]),
    "id_cpqr_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64, _I64, _P]),
    "id_decompose_host_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64, _P]),
    "id_decompose": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _P, _I64, _P,
                                    ctypes.c_size_t, _P, _P]),
    "id_decompose_host": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _P, _I64, _P,
                                         ctypes.c_size_t, _P, _P]),
    "id_cpqr": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _P, _P, ctypes.c_size_t, _P, _P]),
    "id_solve": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _P, _I64, _P]),
    "id_info_read": (ctypes.c_int, [_P, _P, _P]),
    "id_decompose_noalloc": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _P, _I64, _P, _P]),
    "id_sketch_workspace_size": (ctypes.c_size_t, []),
    "id_sketch_scratch_size": (ctypes.c_size_t, [ctypes.c_int64, ctypes.c_int64]),
    "id_sketch": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _P, _I64, _I64, _P, _I64, _P, ctypes.c_size_t, _P,
                                 _P]),
    "id_rid_workspace_size": (ctypes.c_size_t, [_I64, _I64, _I64, _I64, _P]),
    "id_decompose_randomized": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _P, _I64, _I64, _I64, _P, _P, _P,
                                               _I64, _P, ctypes.c_size_t, _P, _P]),
    "id_rid_pipe_workspace_size": (ctypes.c_size_t, [_I64, _I64, _I64, _I64, _P]),
    "id_rid_pipe_create": (ctypes.c_int, [_P, _I64, _I64, _I64, _I64, _P, _P, ctypes.c_size_t]),
    "id_rid_pipe_submit": (ctypes.c_int, [_P, _P, _I64, _P, _I64, _P, _P, _I64, _P, _P]),
    "id_rid_pipe_sync": (ctypes.c_int, [_P]),
    "id_rid_pipe_destroy": (None, [_P]),
    "id_batched_problem_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64]),
    "id_decompose_batched": (ctypes.c_int, [_P, _I64, ctypes.c_int, _P, ctypes.c_size_t, _P, _P]),
    "id_batched_config_count": (ctypes.c_int, [ctypes.c_int]),
    "id_batched_config_get": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P]),
    "id_decompose_batched_with": (ctypes.c_int, [_P, _I64, ctypes.c_int, _P, ctypes.c_size_t, _P, ctypes.c_int, _P]),
    "id_batched_autotune": (ctypes.c_int, [_P, _I64, ctypes.c_int, _P, ctypes.c_size_t, _P, ctypes.c_int, _P, _P,
                                           _P]),
    "id_sampled_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64, _I64, _P]),
    "id_reconstruct_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64, ctypes.c_int32]),
    "id_two_sided_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64, _P]),
    "id_csr_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64, _P]),
    "id_decompose_csr": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _P, _I64, _P,
                                        ctypes.c_size_t, _P, _P]),
    "id_decompose_two_sided": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _P, _P, _I64, _P, _I64,
                                              _P, ctypes.c_size_t, _P, _P]),
    "id_reconstruct": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _I64, ctypes.c_int32, _P, _I64,
                                      _P, ctypes.c_size_t, _P, _P]),
    "id_decompose_sampled": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _P, _I64, _I64, _P, _P, _P, _I64, _P,
                                            ctypes.c_size_t, _P, _P]),
    "id_refine_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64]),
    "id_backward_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64]),
    "id_backward": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _I64, _P, _I64, _P, _I64, _P,
                                   ctypes.c_size_t, _P, _P]),
    "id_refine": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _I64, _P, ctypes.c_size_t, _P, _P]),
    "id_launch_count": (ctypes.c_int64, [ctypes.c_int, _I64, _I64, _I64, _P]),
    "id_rid_launch_count": (ctypes.c_int64, [_I64, _I64, _I64, _I64, _P]),
    "id_cpqr_timeline": (ctypes.c_int, [_P, ctypes.c_int]),
    "id_cpqr_residual_norms": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I64, _I64, _I64, _P, _P, _P]),
    "id_selftest_bounded_wait": (ctypes.c_int, [_P, ctypes.c_size_t, _P, _P]),
    "id_trace_enable": (ctypes.c_int, [ctypes.c_int]),
    "id_trace_read": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "id_version": (ctypes.c_char_p, []),
    "id_gemm_workspace_size": (ctypes.c_size_t, [ctypes.c_int, _I64, _I64, _I64]),
    "id_gemm": (ctypes.c_int, [ctypes.c_int, ctypes.c_int32, ctypes.c_int32, _I64, _I64, _I64, ctypes.c_double, _P, _I64,
                               _P, _I64, ctypes.c_double, _P, _I64, _P, ctypes.c_size_t, _P, _P]),
}

TRACE_KINDS = ("cpqr", "solve", "sketch", "copy_in", "scatter", "batched", "refine", "sampled_z")


def lib():
    """The loaded libgbid.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIG.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIG)


def _opts(nb: int, refine: bool = True, engine: int = 0, zsolve: int = 0):
    o = IdOpts()
    o.nb = int(nb)
    o.refine = 0 if refine else -1
    o.engine = int(engine)
    o.zsolve = int(zsolve)
    return o


def _stream(dev) -> int:
    return torch.cuda.current_stream(dev).cuda_stream


def _check_cuda_matrix(A: torch.Tensor, name: str):
    if not isinstance(A, torch.Tensor) or not A.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU fallback)")
    if A.dtype not in _DTYPES:
        raise ValueError(f"{name} must be float32 or float64")
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError(f"{name} must be 2-D with unit column stride (row-major)")


def workspace_size(dtype: torch.dtype, m: int, n: int, k: int, nb: int = 0) -> int:
    o = _opts(nb)
    return int(lib().id_workspace_size(_DTYPES[dtype], m, n, k, ctypes.byref(o)))


@dataclass
class Workspace:
    """Device scratch for id_decompose (reusable across calls of the same size)."""
    buf: torch.Tensor

    @staticmethod
    def for_problem(dtype, m, n, k, nb=0, device="cuda", host_io=False, normal_eq=False):
        o = _opts(nb, zsolve=1 if normal_eq else 0)
        if host_io:
            nbytes = int(lib().id_decompose_host_workspace_size(_DTYPES[dtype], m, n, k, ctypes.byref(o)))
        else:
            nbytes = int(lib().id_workspace_size(_DTYPES[dtype], m, n, k, ctypes.byref(o)))
        if nbytes == 0:
            raise IdError(ID_EINVAL, "workspace size")
        return Workspace(torch.empty(nbytes, dtype=torch.uint8, device=device))


def id_decompose(A: torch.Tensor, k: int, *, nb: int = 0, engine: int = ENGINE_AUTO, normal_eq: bool = False,
                 workspace: Workspace | None = None, out: tuple | None = None, sync: bool = True):
    """Rank-k ID of a CUDA matrix A (m x n, row-major, float32/float64).

    Returns (J, Z, info): J int32 (k,), Z (k, max(m,n)) of A's dtype, info a
    dict (when sync) or None. m <= n: A ~= A[:, J] @ Z; m > n: A ~= Z.T @ A[J, :].
    With sync=False nothing waits for the GPU (usable inside CUDA-graph capture);
    read the status later with ``read_info(workspace)``. engine: ENGINE_AUTO
    (small problems on one thread-block cluster, others on the persistent grid),
    ENGINE_GRID or ENGINE_CLUSTER. normal_eq: Z from the paper's normal
    equations R_k^T R_k Z = C^T A (column IDs, grid engine) instead of the back
    substitution with R.
    """
    _check_cuda_matrix(A, "A")
    m, n = A.shape
    nz = max(m, n)
    dev = A.device
    if workspace is None:
        workspace = Workspace.for_problem(A.dtype, m, n, k, nb, dev, normal_eq=normal_eq)
    if out is None:
        J = torch.empty(k, dtype=torch.int32, device=dev)
        Z = torch.empty(k, nz, dtype=A.dtype, device=dev)
    else:
        J, Z = out
    o = _opts(nb, engine=engine, zsolve=1 if normal_eq else 0)
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_decompose(A.data_ptr(), _DTYPES[A.dtype], m, n, A.stride(0), k, ctypes.byref(o),
                                J.data_ptr(), Z.data_ptr(), Z.stride(0), workspace.buf.data_ptr(),
                                workspace.buf.numel(), ctypes.byref(info) if sync else None, _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_decompose")
    return J, Z, (info.as_dict() if sync else None)


NOALLOC_SCRATCH_BYTES = 32 << 20   # ID_NOALLOC_SCRATCH_BYTES in gbid.h


def id_decompose_noalloc(A: torch.Tensor, k: int, *, nb: int = 0, out: tuple | None = None, sync: bool = True):
    """The ID with the library's fixed scratch instead of a workspace, for callers that
    cannot allocate device memory (only J and Z are allocated here, unless ``out`` is given).

    sync=False passes no info pointer, so nothing waits for the stream (the form to use
    while the stream is being captured); the third result is then None."""
    _check_cuda_matrix(A, "A")
    m, n = A.shape
    dev = A.device
    if out is None:
        J = torch.empty(k, dtype=torch.int32, device=dev)
        Z = torch.empty(k, max(m, n), dtype=A.dtype, device=dev)
    else:
        J, Z = out
    o = _opts(nb)
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_decompose_noalloc(A.data_ptr(), _DTYPES[A.dtype], m, n, A.stride(0), k, ctypes.byref(o),
                                        J.data_ptr(), Z.data_ptr(), Z.stride(0),
                                        ctypes.byref(info) if sync else None, _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_decompose_noalloc")
    return J, Z, (info.as_dict() if sync else None)


def id_sketch(A: torch.Tensor, omega: torch.Tensor, *, out: torch.Tensor | None = None, sync: bool = True):
    """Y = omega @ A on the tensor cores (A FP32 m x n rounded to BF16 in shared memory,
    omega BF16 l x m, FP32 accumulation). Returns (Y, info)."""
    _check_cuda_matrix(A, "A")
    if A.dtype != torch.float32:
        raise ValueError("A must be float32")
    if not omega.is_cuda or omega.dtype != torch.bfloat16 or omega.dim() != 2 or omega.stride(1) != 1:
        raise ValueError("omega must be a row-major CUDA bfloat16 matrix")
    m, n = A.shape
    l = omega.shape[0]
    if omega.shape[1] != m:
        raise ValueError("omega must have A.shape[0] columns")
    dev = A.device
    Y = out if out is not None else torch.empty(l, n, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        # with the scratch of the last wave's split: Y is bit-identical to the randomized ID's sketch
        nbytes = int(lib().id_sketch_workspace_size()) + int(lib().id_sketch_scratch_size(n, l))
    work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_sketch(A.data_ptr(), ID_F32, m, n, A.stride(0), omega.data_ptr(), l, omega.stride(0),
                             Y.data_ptr(), Y.stride(0), work.data_ptr(), work.numel(),
                             ctypes.byref(info) if sync else None, _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_sketch")
    return Y, (info.as_dict() if sync else None)


def rid_workspace(m: int, n: int, l: int, k: int, nb: int = 0, device="cuda", refine: bool = True) -> Workspace:
    o = _opts(nb, refine)
    nbytes = int(lib().id_rid_workspace_size(m, n, l, k, ctypes.byref(o)))
    if nbytes == 0:
        raise IdError(ID_EINVAL, "id_rid_workspace_size")
    return Workspace(torch.empty(nbytes, dtype=torch.uint8, device=device))


def id_decompose_randomized(A: torch.Tensor, omega: torch.Tensor, k: int, *, nb: int = 0, refine: bool = True,
                            workspace: Workspace | None = None, out: tuple | None = None, sync: bool = True):
    """Randomized rank-k ID from the sketch Y = omega @ A (A FP32 m x n, m <= n;
    omega BF16 l x m). Returns (J, Z, info) with A ~= A[:, J] @ Z. With refine
    (the default) Z gets one least-squares refinement against A_J."""
    _check_cuda_matrix(A, "A")
    if A.dtype != torch.float32 or omega.dtype != torch.bfloat16 or not omega.is_cuda or omega.stride(1) != 1:
        raise ValueError("A must be float32 and omega a row-major CUDA bfloat16 matrix")
    m, n = A.shape
    l = omega.shape[0]
    dev = A.device
    if workspace is None:
        workspace = rid_workspace(m, n, l, k, nb, dev, refine)
    if out is None:
        J = torch.empty(k, dtype=torch.int32, device=dev)
        Z = torch.empty(k, n, dtype=torch.float32, device=dev)
    else:
        J, Z = out
    o = _opts(nb, refine)
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_decompose_randomized(A.data_ptr(), ID_F32, m, n, A.stride(0), omega.data_ptr(), l,
                                           omega.stride(0), k, ctypes.byref(o), J.data_ptr(), Z.data_ptr(),
                                           Z.stride(0), workspace.buf.data_ptr(), workspace.buf.numel(),
                                           ctypes.byref(info) if sync else None, _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_decompose_randomized")
    return J, Z, (info.as_dict() if sync else None)


def sampled_workspace(dtype: torch.dtype, m: int, n: int, p: int, k: int, *, nb: int = 0,
                      device=None) -> Workspace:
    """Workspace for id_decompose_sampled with p sampled columns."""
    o = _opts(nb)
    nbytes = int(lib().id_sampled_workspace_size(_DTYPES[dtype], m, n, p, k, ctypes.byref(o)))
    if nbytes == 0:
        raise IdError(ID_EINVAL, "id_sampled_workspace_size")
    return Workspace(torch.empty(nbytes, dtype=torch.uint8, device=device))


def id_decompose_sampled(A: torch.Tensor, idx, k: int, *, nb: int = 0, workspace: Workspace | None = None,
                         sync: bool = True):
    """The paper's Optim RID: CPQR of the sampled columns A[:, idx] (idx: p distinct
    column indices, host sequence), J = idx[P_k], Z from the normal equations against
    all of A. Returns (J, Z, info) with A ~= A[:, J] @ Z."""
    _check_cuda_matrix(A, "A")
    import numpy as _np

    ih = _np.ascontiguousarray(_np.asarray(idx, dtype=_np.int32))
    m, n = A.shape
    p = ih.size
    dev = A.device
    o = _opts(nb)
    if workspace is None:
        workspace = sampled_workspace(A.dtype, m, n, p, k, nb=nb, device=dev)
    J = torch.empty(k, dtype=torch.int32, device=dev)
    Z = torch.empty(k, n, dtype=A.dtype, device=dev)
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_decompose_sampled(A.data_ptr(), _DTYPES[A.dtype], m, n, A.stride(0),
                                        ih.ctypes.data_as(ctypes.c_void_p), p, k, ctypes.byref(o), J.data_ptr(),
                                        Z.data_ptr(), Z.stride(0), workspace.buf.data_ptr(), workspace.buf.numel(),
                                        ctypes.byref(info) if sync else None, _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_decompose_sampled")
    return J, Z, (info.as_dict() if sync else None)


def csr_workspace(dtype: torch.dtype, m: int, n: int, k: int, *, nb: int = 0, device=None) -> Workspace:
    o = _opts(nb)
    nbytes = int(lib().id_csr_workspace_size(_DTYPES[dtype], m, n, k, ctypes.byref(o)))
    if nbytes == 0:
        raise IdError(ID_EINVAL, "id_csr_workspace_size")
    return Workspace(torch.empty(nbytes, dtype=torch.uint8, device=device))


def id_decompose_csr(rowptr: torch.Tensor, colind: torch.Tensor, values: torch.Tensor, shape, k: int, *,
                     nb: int = 0, workspace: Workspace | None = None, out: tuple | None = None, sync: bool = True):
    """Rank-k ID of a sparse CUDA matrix in CSR form (rowptr int64 (m+1),
    colind int32, values float32/float64, all on the GPU). Same outputs as
    id_decompose; the skeleton A[:, J] keeps A's sparsity."""
    m, n = (int(shape[0]), int(shape[1]))
    if not (rowptr.is_cuda and colind.is_cuda and values.is_cuda):
        raise ValueError("rowptr, colind and values must be CUDA tensors (no CPU fallback)")
    if rowptr.dtype != torch.int64 or colind.dtype != torch.int32 or values.dtype not in _DTYPES:
        raise ValueError("rowptr int64, colind int32, values float32/float64")
    if rowptr.numel() != m + 1 or colind.numel() != values.numel():
        raise ValueError("rowptr must have m + 1 entries and colind as many as values")
    dev = values.device
    if workspace is None:
        workspace = csr_workspace(values.dtype, m, n, k, nb=nb, device=dev)
    nz = max(m, n)
    if out is None:
        J = torch.empty(k, dtype=torch.int32, device=dev)
        Z = torch.empty(k, nz, dtype=values.dtype, device=dev)
    else:
        J, Z = out
    o = _opts(nb)
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_decompose_csr(rowptr.data_ptr(), colind.data_ptr(), values.data_ptr(), _DTYPES[values.dtype], m,
                                    n, values.numel(), k, ctypes.byref(o), J.data_ptr(), Z.data_ptr(), Z.stride(0),
                                    workspace.buf.data_ptr(), workspace.buf.numel(),
                                    ctypes.byref(info) if sync else None, _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_decompose_csr")
    return J, Z, (info.as_dict() if sync else None)


def two_sided_workspace(dtype: torch.dtype, m: int, n: int, k: int, *, nb: int = 0, device=None) -> Workspace:
    o = _opts(nb)
    nbytes = int(lib().id_two_sided_workspace_size(_DTYPES[dtype], m, n, k, ctypes.byref(o)))
    if nbytes == 0:
        raise IdError(ID_EINVAL, "id_two_sided_workspace_size")
    return Workspace(torch.empty(nbytes, dtype=torch.uint8, device=device))


def id_decompose_two_sided(A: torch.Tensor, k: int, *, nb: int = 0, workspace: Workspace | None = None,
                           out: tuple | None = None, sync: bool = True):
    """Rank-k two-sided ID A ~= X.T @ A[I][:, J] @ Z (the variant the paper's
    Sec. 1.2 footnote names): a column ID then a row ID of its skeleton (the
    roles swap for m > n). Returns (I, J, X, Z, infos) with X (k, m), Z (k, n)
    and infos a pair of dicts (stage 1, stage 2) when sync."""
    _check_cuda_matrix(A, "A")
    m, n = A.shape
    dev = A.device
    if workspace is None:
        workspace = two_sided_workspace(A.dtype, m, n, k, nb=nb, device=dev)
    if out is None:
        I = torch.empty(k, dtype=torch.int32, device=dev)
        J = torch.empty(k, dtype=torch.int32, device=dev)
        X = torch.empty(k, m, dtype=A.dtype, device=dev)
        Z = torch.empty(k, n, dtype=A.dtype, device=dev)
    else:
        I, J, X, Z = out
    o = _opts(nb)
    infos = (IdInfo * 2)()
    with torch.cuda.device(dev):
        rc = lib().id_decompose_two_sided(A.data_ptr(), _DTYPES[A.dtype], m, n, A.stride(0), k, ctypes.byref(o),
                                          I.data_ptr(), J.data_ptr(), X.data_ptr(), X.stride(0), Z.data_ptr(),
                                          Z.stride(0), workspace.buf.data_ptr(), workspace.buf.numel(),
                                          infos if sync else None, _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_decompose_two_sided")
    return I, J, X, Z, ((infos[0].as_dict(), infos[1].as_dict()) if sync else None)


def reconstruct_workspace(dtype: torch.dtype, m: int, n: int, k: int, *, transposed: bool = False,
                          device=None) -> Workspace:
    nbytes = int(lib().id_reconstruct_workspace_size(_DTYPES[dtype], m, n, k, 1 if transposed else 0))
    if nbytes == 0:
        raise IdError(ID_EINVAL, "id_reconstruct_workspace_size")
    return Workspace(torch.empty(nbytes, dtype=torch.uint8, device=device))


def id_reconstruct(A: torch.Tensor, J: torch.Tensor, Z: torch.Tensor, *, transposed: bool = False,
                   out: torch.Tensor | None = None, workspace: Workspace | None = None, sync: bool = True):
    """The ID's approximation of A: A[:, J] @ Z (column ID), or Z.T @ A[J, :]
    (row ID of an m > n matrix, transposed=True). Returns (approx, info)."""
    _check_cuda_matrix(A, "A")
    _check_cuda_matrix(Z, "Z")
    m, n = A.shape
    k = J.numel()
    dev = A.device
    dt = _DTYPES[A.dtype]
    if workspace is None:
        workspace = reconstruct_workspace(A.dtype, m, n, k, transposed=transposed, device=dev)
    Out = torch.empty(m, n, dtype=A.dtype, device=dev) if out is None else out
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_reconstruct(A.data_ptr(), dt, m, n, A.stride(0), k, J.data_ptr(), Z.data_ptr(), Z.stride(0),
                                  1 if transposed else 0, Out.data_ptr(), Out.stride(0), workspace.buf.data_ptr(),
                                  workspace.buf.numel(), ctypes.byref(info) if sync else None, _stream(dev))
    if rc in _CALL_ERRORS or (sync and info.status == ID_EINVAL):
        raise IdError(ID_EINVAL if rc == 0 else rc, "id_reconstruct")
    return Out, (info.as_dict() if sync else None)


def gemm(A: torch.Tensor, B: torch.Tensor, *, ta: bool = False, tb: bool = False, alpha: float = 1.0,
         beta: float = 0.0, out: torch.Tensor | None = None, sync: bool = True):
    """out = alpha op(A) op(B) + beta out for row-major CUDA matrices of one dtype, op(X) = X or X.T:
    FP64 on the FP64 pipe, FP32 as FP32-accurate 3xTF32 products on the tensor cores. Returns (out, info)."""
    _check_cuda_matrix(A, "A")
    _check_cuda_matrix(B, "B")
    if A.dtype != B.dtype:
        raise ValueError("A and B must have one dtype")
    M, K = (A.shape[1], A.shape[0]) if ta else (A.shape[0], A.shape[1])
    K2, N = (B.shape[1], B.shape[0]) if tb else (B.shape[0], B.shape[1])
    if K != K2:
        raise ValueError("inner dimensions differ")
    dev = A.device
    dt = _DTYPES[A.dtype]
    if out is None:
        out = torch.zeros(M, N, dtype=A.dtype, device=dev)
    _check_cuda_matrix(out, "out")
    nbytes = int(lib().id_gemm_workspace_size(dt, M, N, K))
    if nbytes == 0:
        raise IdError(ID_EINVAL, "id_gemm_workspace_size")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_gemm(dt, 1 if ta else 0, 1 if tb else 0, M, N, K, float(alpha), A.data_ptr(), A.stride(0),
                           B.data_ptr(), B.stride(0), float(beta), out.data_ptr(), out.stride(0), ws.data_ptr(),
                           ws.numel(), ctypes.byref(info) if sync else None, _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_gemm")
    return out, (info.as_dict() if sync else None)


def id_refine(A: torch.Tensor, J: torch.Tensor, Z: torch.Tensor, *, workspace: Workspace | None = None,
              sync: bool = True):
    """One least-squares refinement of Z (k x n FP32, in place) against the FP32 CUDA matrix A
    (m x n, m <= n) for the skeleton J: Z <- Z + (C^T C)^{-1} C^T (A - C Z), C = A[:, J]."""
    _check_cuda_matrix(A, "A")
    if A.dtype != torch.float32 or Z.dtype != torch.float32 or not Z.is_cuda or Z.stride(1) != 1:
        raise ValueError("A and Z must be row-major float32 CUDA matrices")
    if J.dtype != torch.int32 or not J.is_cuda:
        raise ValueError("J must be an int32 CUDA vector")
    m, n = A.shape
    k = J.numel()
    dev = A.device
    if workspace is None:
        nbytes = int(lib().id_refine_workspace_size(ID_F32, m, n, k))
        if nbytes == 0:
            raise IdError(ID_EINVAL, "id_refine_workspace_size")
        workspace = Workspace(torch.empty(nbytes, dtype=torch.uint8, device=dev))
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_refine(A.data_ptr(), ID_F32, m, n, A.stride(0), k, J.data_ptr(), Z.data_ptr(), Z.stride(0),
                             workspace.buf.data_ptr(), workspace.buf.numel(), ctypes.byref(info) if sync else None,
                             _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_refine")
    return Z, (info.as_dict() if sync else None)


def id_backward(A: torch.Tensor, J: torch.Tensor, Z: torch.Tensor, dZ: torch.Tensor, *,
                workspace: Workspace | None = None, out: torch.Tensor | None = None, sync: bool = True):
    """dL/dA through the ID with the skeleton J frozen, given dL/dZ (FP32 CUDA, A m x n with m <= n)."""
    _check_cuda_matrix(A, "A")
    for name, X in (("Z", Z), ("dZ", dZ)):
        if X.dtype != torch.float32 or not X.is_cuda or X.dim() != 2 or X.stride(1) != 1:
            raise ValueError(f"{name} must be a row-major float32 CUDA matrix")
    if A.dtype != torch.float32 or J.dtype != torch.int32 or not J.is_cuda:
        raise ValueError("A must be float32 and J an int32 CUDA vector")
    m, n = A.shape
    k = J.numel()
    dev = A.device
    if workspace is None:
        nbytes = int(lib().id_backward_workspace_size(ID_F32, m, n, k))
        if nbytes == 0:
            raise IdError(ID_EINVAL, "id_backward_workspace_size")
        workspace = Workspace(torch.empty(nbytes, dtype=torch.uint8, device=dev))
    dA = out if out is not None else torch.empty(m, n, dtype=torch.float32, device=dev)
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_backward(A.data_ptr(), ID_F32, m, n, A.stride(0), k, J.data_ptr(), Z.data_ptr(), Z.stride(0),
                               dZ.data_ptr(), dZ.stride(0), dA.data_ptr(), dA.stride(0), workspace.buf.data_ptr(),
                               workspace.buf.numel(), ctypes.byref(info) if sync else None, _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_backward")
    return dA, (info.as_dict() if sync else None)


class BackwardPlan:
    """dL/dA for many IDs of one size (FP32, m <= n), spread over ``streams``
    CUDA streams so that the problems' small kernels overlap; each stream has
    its own workspace. ``run`` forks from the current stream and joins back
    into it, so it can be captured in a CUDA graph and replayed."""

    def __init__(self, m: int, n: int, k: int, *, streams: int = 16, device="cuda"):
        nbytes = int(lib().id_backward_workspace_size(ID_F32, m, n, k))
        if nbytes == 0:
            raise IdError(ID_EINVAL, "id_backward_workspace_size")
        self.shape = (m, n, k)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(max(1, int(streams)))]
        self.workspaces = [Workspace(torch.empty(nbytes, dtype=torch.uint8, device=device)) for _ in self.streams]

    def run(self, As, Js, Zs, dZs, dAs):
        cur = torch.cuda.current_stream()
        for st in self.streams:
            st.wait_stream(cur)
        for b, (A, J, Z, dZ, dA) in enumerate(zip(As, Js, Zs, dZs, dAs)):
            q = b % len(self.streams)
            with torch.cuda.stream(self.streams[q]):
                id_backward(A, J, Z, dZ, workspace=self.workspaces[q], out=dA, sync=False)
        for st in self.streams:
            cur.wait_stream(st)
        return dAs


class IdFunction(torch.autograd.Function):
    """Z = ID(A) with the skeleton frozen after the forward pass (FP32 CUDA, m <= n):
    forward runs id_decompose, backward id_backward."""

    @staticmethod
    def forward(ctx, A, k):
        J, Z, _ = id_decompose(A.contiguous(), k, sync=False)
        ctx.save_for_backward(A, J, Z)
        ctx.mark_non_differentiable(J)
        return J, Z

    @staticmethod
    def backward(ctx, dJ, dZ):
        A, J, Z = ctx.saved_tensors
        dA, _ = id_backward(A.contiguous(), J, Z, dZ.contiguous(), sync=False)
        return dA, None


def read_info(workspace: Workspace) -> dict:
    info = IdInfo()
    dev = workspace.buf.device
    with torch.cuda.device(dev):
        rc = lib().id_info_read(workspace.buf.data_ptr(), ctypes.byref(info), _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_info_read")
    return info.as_dict()


class RandomizedPipeline:
    """Randomized IDs of a stream of HOST matrices of one size (id_rid_pipe): each
    submit enqueues one ID and returns at once; the host-to-device copy of the next
    ID's inputs and the copy-back of the previous ID's J and Z overlap the current
    ID on the device. Each ID equals id_decompose_randomized on the same inputs.

    Inputs: A (m x n float32, CPU, row-major), omega (l x m bfloat16, CPU); outputs:
    J (k int32), Z (k x n float32), CPU tensors. Pinned host tensors keep the
    copies asynchronous. Inputs must not change, nor outputs be read, until
    synchronize() returns."""

    def __init__(self, m: int, n: int, l: int, k: int, *, nb: int = 0, refine: bool = True, device="cuda"):
        self.m, self.n, self.l, self.k = m, n, l, k
        self._opts = _opts(nb, refine)
        nbytes = int(lib().id_rid_pipe_workspace_size(m, n, l, k, ctypes.byref(self._opts)))
        if nbytes == 0:
            raise IdError(ID_EINVAL, "id_rid_pipe_workspace_size")
        self.device = torch.device(device)
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._pipe = ctypes.c_void_p()
        self._infos = []   # pinned status records the device writes into (kept alive until synchronize)
        self._keep = []    # host tensors referenced by enqueued copies
        # pinned chunks of 64 status records, allocated ahead of the submits
        self._pools = [torch.zeros(64, ctypes.sizeof(IdInfo), dtype=torch.uint8, pin_memory=True)]
        with torch.cuda.device(self.device):
            rc = lib().id_rid_pipe_create(ctypes.byref(self._pipe), m, n, l, k, ctypes.byref(self._opts),
                                          self.buf.data_ptr(), nbytes)
        if rc != ID_OK:
            raise IdError(rc, "id_rid_pipe_create")

    def submit(self, A: torch.Tensor, omega: torch.Tensor, J: torch.Tensor, Z: torch.Tensor) -> int:
        """Enqueue one ID on the current stream; returns its index (for results())."""
        for t, name, dt, shape in ((A, "A", torch.float32, (self.m, self.n)),
                                   (omega, "omega", torch.bfloat16, (self.l, self.m)),
                                   (J, "J", torch.int32, (self.k,)), (Z, "Z", torch.float32, (self.k, self.n))):
            if t.is_cuda or t.dtype != dt or tuple(t.shape) != shape or t.stride(-1) != 1:
                raise ValueError(f"{name} must be a CPU {dt} tensor of shape {shape} with unit last stride")
        # the status lands in pinned memory (a copy into pageable memory would wait for the ID); the
        # records come from chunks allocated ahead, since pinning memory between submits can
        # wait for the device
        i = len(self._infos)
        if i == 64 * len(self._pools):
            self._pools.append(torch.zeros(64, ctypes.sizeof(IdInfo), dtype=torch.uint8, pin_memory=True))
        info = self._pools[i // 64][i % 64]
        with torch.cuda.device(self.device):
            rc = lib().id_rid_pipe_submit(self._pipe, A.data_ptr(), A.stride(0), omega.data_ptr(), omega.stride(0),
                                          J.data_ptr(), Z.data_ptr(), Z.stride(0), info.data_ptr(),
                                          _stream(self.device))
        if rc != ID_OK:
            raise IdError(rc, "id_rid_pipe_submit")
        self._infos.append(info)
        self._keep.append((A, omega, J, Z))
        return len(self._infos) - 1

    def synchronize(self) -> list:
        """Wait until every submitted ID's outputs are on the host; returns their info dicts."""
        rc = lib().id_rid_pipe_sync(self._pipe)
        if rc != ID_OK:
            raise IdError(rc, "id_rid_pipe_sync")
        out = [IdInfo.from_address(i.data_ptr()).as_dict() for i in self._infos]
        self._infos, self._keep = [], []
        del self._pools[1:]   # the first chunk serves the next round of submits
        return out

    def close(self):
        if self._pipe:
            lib().id_rid_pipe_destroy(self._pipe)
            self._pipe = ctypes.c_void_p()
            self._infos, self._keep, self._pools = [], [], []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def id_decompose_host(A: torch.Tensor, k: int, *, nb: int = 0, engine: int = ENGINE_AUTO,
                      workspace: Workspace | None = None,
                      out: tuple | None = None, device="cuda"):
    """The same ID for a HOST matrix (ideally pinned): copies in, decomposes, copies J, Z back, waits."""
    if A.is_cuda or A.dtype not in _DTYPES or A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a 2-D row-major float32/float64 CPU tensor")
    m, n = A.shape
    nz = max(m, n)
    if workspace is None:
        workspace = Workspace.for_problem(A.dtype, m, n, k, nb, device, host_io=True)
    if out is None:
        pin = A.is_pinned()
        J = torch.empty(k, dtype=torch.int32, pin_memory=pin)
        Z = torch.empty(k, nz, dtype=A.dtype, pin_memory=pin)
    else:
        J, Z = out
    o = _opts(nb, engine=engine)
    info = IdInfo()
    dev = workspace.buf.device
    with torch.cuda.device(dev):
        rc = lib().id_decompose_host(A.data_ptr(), _DTYPES[A.dtype], m, n, A.stride(0), k, ctypes.byref(o),
                                     J.data_ptr(), Z.data_ptr(), Z.stride(0), workspace.buf.data_ptr(),
                                     workspace.buf.numel(), ctypes.byref(info), _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_decompose_host")
    return J, Z, info.as_dict()


def id_cpqr(Xcm: torch.Tensor, m: int, k: int, *, nb: int = 0, workspace: torch.Tensor | None = None,
            residual_norms: bool = False):
    """k-step CPQR in place of a column-major m x n matrix.

    ``Xcm`` is a CUDA tensor of shape (n, ldx): row l holds column l of X (so
    X = Xcm[:, :m].T), ldx >= m a multiple of 8. Returns (perm, tau, info), and
    with residual_norms=True also the n residual column norms (FP64, by position)."""
    if not Xcm.is_cuda or Xcm.dtype not in _DTYPES or Xcm.dim() != 2 or Xcm.stride(1) != 1:
        raise ValueError("Xcm must be a 2-D contiguous CUDA float32/float64 tensor")
    n, ldx = Xcm.shape[0], Xcm.stride(0)
    dev = Xcm.device
    o = _opts(nb)
    if workspace is None:
        nbytes = int(lib().id_cpqr_workspace_size(_DTYPES[Xcm.dtype], m, n, ldx, k, ctypes.byref(o)))
        if nbytes == 0:
            raise IdError(ID_EINVAL, "id_cpqr_workspace_size")
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    tau = torch.empty(k, dtype=torch.float64, device=dev)
    info = IdInfo()
    with torch.cuda.device(dev):
        rc = lib().id_cpqr(Xcm.data_ptr(), _DTYPES[Xcm.dtype], m, n, ldx, k, ctypes.byref(o), perm.data_ptr(),
                           tau.data_ptr(), workspace.data_ptr(), workspace.numel(), ctypes.byref(info),
                           _stream(dev))
    if rc in _CALL_ERRORS:
        raise IdError(rc, "id_cpqr")
    if not residual_norms:
        return perm, tau, info.as_dict()
    nu = torch.empty(n, dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        rc = lib().id_cpqr_residual_norms(workspace.data_ptr(), _DTYPES[Xcm.dtype], m, n, ldx, k, ctypes.byref(o),
                                          nu.data_ptr(), _stream(dev))
    if rc != ID_OK:
        raise IdError(rc, "id_cpqr_residual_norms")
    return perm, tau, info.as_dict(), nu


def id_solve(Xcm: torch.Tensor, k: int) -> torch.Tensor:
    """T = R11^{-1} R12 (FP64, k x (n-k)) from a matrix factored by ``id_cpqr``."""
    if not Xcm.is_cuda or Xcm.dtype not in _DTYPES or Xcm.dim() != 2 or Xcm.stride(1) != 1:
        raise ValueError("Xcm must be a 2-D contiguous CUDA float32/float64 tensor")
    n, ldx = Xcm.shape[0], Xcm.stride(0)
    dev = Xcm.device
    T = torch.empty(k, max(n - k, 1), dtype=torch.float64, device=dev)
    with torch.cuda.device(dev):
        rc = lib().id_solve(Xcm.data_ptr(), _DTYPES[Xcm.dtype], n, ldx, k, T.data_ptr(), T.stride(0), _stream(dev))
    if rc < 0:
        raise IdError(rc, "id_solve")
    return T[:, : n - k]


SELFTEST_WORK_BYTES = 4096    # ID_SELFTEST_WORK_BYTES


def selftest_bounded_wait(device=None) -> int:
    """Run the library's bounded device wait on a counter nothing increments
    (id_selftest_bounded_wait). Returns ID_ETIMEOUT when the wait gave up as
    designed; waits for the device (a few seconds)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    work = torch.empty(SELFTEST_WORK_BYTES, dtype=torch.uint8, device=dev)
    status = ctypes.c_int(1)
    with torch.cuda.device(dev):
        rc = lib().id_selftest_bounded_wait(work.data_ptr(), work.numel(), ctypes.byref(status), _stream(dev))
    if rc != ID_OK:
        raise IdError(rc, "id_selftest_bounded_wait")
    return int(status.value)


def launch_count(dtype: torch.dtype, m: int, n: int, k: int, nb: int = 0, engine: int = ENGINE_AUTO) -> int:
    """Kernel launches one id_decompose call enqueues (as the library counts them; -1 if the
    engine cannot take the problem)."""
    o = _opts(nb, engine=engine)
    return int(lib().id_launch_count(_DTYPES[dtype], m, n, k, ctypes.byref(o)))


def rid_launch_count(m: int, n: int, l: int, k: int, nb: int = 0, refine: bool = True) -> int:
    """Kernel launches one id_decompose_randomized call enqueues (as the library counts them)."""
    o = _opts(nb, refine)
    return int(lib().id_rid_launch_count(m, n, l, k, ctypes.byref(o)))


def cpqr_timeline(buf: torch.Tensor | None) -> None:
    """Stamp the CPQR kernel's phase boundaries of each pivot step into buf (CUDA int64,
    8 entries per step; None switches the diagnostic off). See id_cpqr_timeline."""
    if buf is None:
        rc = lib().id_cpqr_timeline(None, 0)
    else:
        if not buf.is_cuda or buf.dtype != torch.int64 or not buf.is_contiguous():
            raise ValueError("buf must be a contiguous CUDA int64 tensor")
        rc = lib().id_cpqr_timeline(buf.data_ptr(), buf.numel() // 8)
    if rc != ID_OK:
        raise IdError(rc, "id_cpqr_timeline")


def trace_enable(capacity: int = 4096) -> None:
    if lib().id_trace_enable(int(capacity)) != ID_OK:
        raise IdError(ID_ECUDA, "id_trace_enable")


def trace_read() -> dict:
    """{kind: (total_ms, launches)} for the launches traced since the last read."""
    nk = len(TRACE_KINDS)
    ms = (ctypes.c_double * nk)()
    cnt = (ctypes.c_int64 * nk)()
    if lib().id_trace_read(ms, cnt, nk) < 0:
        raise IdError(ID_ECUDA, "id_trace_read")
    return {name: (ms[i], cnt[i]) for i, name in enumerate(TRACE_KINDS)}


def version() -> str:
    return lib().id_version().decode()


# ------------------------------------------------------------------ batched --
BATCHED_MAX_K = 64            # ID_BATCHED_MAX_K in gbid.h
BATCHED_MAX_MIN_DIM = 1024    # ID_BATCHED_MAX_MIN_DIM
BATCHED_WORK_BYTES = 256      # ID_BATCHED_WORK_BYTES


class IdProblem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("k", ctypes.c_int64), ("J", ctypes.c_void_p), ("Z", ctypes.c_void_p), ("ldz", ctypes.c_int64),
                ("work", ctypes.c_void_p)]


class IdBatchedConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("cols_per_warp", ctypes.c_int32), ("rows_per_lane", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def batched_configs(dtype=torch.float32) -> list:
    """The batched kernel's instances (tile shapes) for dtype, index 0 the default."""
    dt = _DTYPES[dtype]
    out = []
    for i in range(int(lib().id_batched_config_count(dt))):
        c = IdBatchedConfig()
        rc = lib().id_batched_config_get(dt, i, ctypes.byref(c))
        if rc != ID_OK:
            raise IdError(rc, "id_batched_config_get")
        out.append(c.as_dict())
    return out


def _shape_signature(dtype, device, mats, ks) -> tuple:
    """Key of the tuner's choice: dtype, device and the multiset of (m, n, k)."""
    return (str(dtype), str(device), tuple(sorted((int(A.shape[0]), int(A.shape[1]), int(k)) for A, k in zip(mats, ks))))


_TUNED: dict = {}

# The tuner's choices can also persist across processes: set GBID_TUNE_CACHE
# to a JSON file path. Entries are keyed by the element type, the GPU's name,
# the library's instance table and a digest of the batch's shapes, so a
# rebuilt library with other instances, or another GPU model, never reuses a
# stale choice. Without the variable nothing is read or written.
TUNE_CACHE_ENV = "GBID_TUNE_CACHE"


def tune_cache_key(dtype_name: str, device_name: str, configs: list, shapes: list) -> str:
    """Key of a persisted tuning: dtype, GPU name, instance table, shape multiset."""
    import hashlib
    import json

    body = json.dumps({"configs": configs, "shapes": sorted([int(a), int(b), int(c)] for a, b, c in shapes)},
                      sort_keys=True)
    return f"{dtype_name}|{device_name}|{hashlib.sha256(body.encode()).hexdigest()[:32]}"


def tune_cache_get(path: str, key: str):
    """(config index, ms per instance) stored under key in the JSON file, or None
    (missing or unreadable file, missing key, malformed entry)."""
    import json

    try:
        with open(path) as f:
            entry = json.load(f).get(key)
        if entry is None:
            return None
        return int(entry["config"]), [float(x) for x in entry["ms"]]
    except (OSError, ValueError, TypeError, KeyError, AttributeError):
        return None


def tune_cache_put(path: str, key: str, config: int, ms: list) -> None:
    """Store one tuning in the JSON file (read, update, write to a temporary file
    and rename, so a reader never sees a half-written file)."""
    import json
    import tempfile

    data = {}
    try:
        with open(path) as f:
            loaded = json.load(f)
        if isinstance(loaded, dict):
            data = loaded
    except (OSError, ValueError):
        pass
    data[key] = {"config": int(config), "ms": [float(x) for x in ms]}
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".gbid_tune_", suffix=".json")
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def _persisted_key(plan) -> str:
    shapes = [(A.shape[0], A.shape[1], k) for A, k in zip(plan.mats, plan.ks)]
    return tune_cache_key(str(plan.dtype), torch.cuda.get_device_name(plan.device), batched_configs(plan.dtype),
                          shapes)


class BatchedPlan:
    """Descriptors, outputs and scratch of id_decompose_batched for a fixed list
    of CUDA matrices (one dtype, one device). ``run()`` enqueues one memset and
    one kernel and never waits or allocates, so it can be captured in a CUDA
    graph and replayed. Problems are queued largest first (k m n descending) so
    that the persistent CTAs finish together; outputs keep the caller's order.

    ``config`` picks the kernel instance (an index into batched_configs());
    ``autotune=True`` instead times every instance on this batch
    (id_batched_autotune, which waits for the device) and keeps the fastest.
    The choice is remembered per (dtype, device, multiset of shapes), so a
    later plan over the same shapes reuses it without timing again, and, when
    GBID_TUNE_CACHE names a JSON file, across processes too. All instances
    give bit-identical results; ``tune_ms`` holds the timings.
    """

    def __init__(self, mats: list, ks: list, *, config: int | None = None, autotune: bool = False,
                 tune_reps: int = 3):
        if len(mats) != len(ks):
            raise ValueError("one k per matrix")
        if not mats:
            raise ValueError("empty batch")
        dt = mats[0].dtype
        dev = mats[0].device
        for A in mats:
            _check_cuda_matrix(A, "A")
            if A.dtype != dt or A.device != dev:
                raise ValueError("every matrix must share one dtype and device")
        self.dtype, self.device, self.mats, self.ks = dt, dev, list(mats), [int(k) for k in ks]
        sizes = []
        for A, k in zip(self.mats, self.ks):
            nbytes = int(lib().id_batched_problem_workspace_size(_DTYPES[dt], A.shape[0], A.shape[1], k))
            if nbytes == 0:
                raise IdError(ID_EINVAL, f"batched problem {tuple(A.shape)} k={k}")
            sizes.append(nbytes)
        offs, total = [], 0
        for nb in sizes:
            offs.append(total)
            total += (nb + 255) // 256 * 256
        self.work = torch.empty(total, dtype=torch.uint8, device=dev)
        self.J = [torch.empty(k, dtype=torch.int32, device=dev) for k in self.ks]
        self.Z = [torch.empty(k, max(A.shape), dtype=dt, device=dev) for A, k in zip(self.mats, self.ks)]
        order = sorted(range(len(self.mats)), key=lambda i: -self.ks[i] * self.mats[i].shape[0] * self.mats[i].shape[1])
        self.order = order
        arr = (IdProblem * len(order))()
        base = self.work.data_ptr()
        for slot, i in enumerate(order):
            A = self.mats[i]
            arr[slot] = IdProblem(A.data_ptr(), A.shape[0], A.shape[1], A.stride(0), self.ks[i],
                                  self.J[i].data_ptr(), self.Z[i].data_ptr(), self.Z[i].stride(0), base + offs[i])
        raw = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
        self.desc = raw.to(dev)
        self.infos = torch.zeros(len(order) * ctypes.sizeof(IdInfo), dtype=torch.uint8, device=dev)
        self.batch_work = torch.zeros(BATCHED_WORK_BYTES, dtype=torch.uint8, device=dev)
        self.tune_ms = None
        self.config = 0 if config is None else int(config)
        if config is None and autotune:
            cached = _TUNED.get(_shape_signature(dt, dev, self.mats, self.ks))
            path = os.environ.get(TUNE_CACHE_ENV)
            if cached is None and path:
                cached = tune_cache_get(path, _persisted_key(self))
                if cached is not None and not 0 <= cached[0] < len(cached[1]):
                    cached = None
                if cached is not None:
                    _TUNED[_shape_signature(dt, dev, self.mats, self.ks)] = cached
            if cached is not None:
                self.config, self.tune_ms = cached
            else:
                self.autotune(tune_reps)

    def autotune(self, reps: int = 3):
        """Time every kernel instance on this batch, make the fastest this plan's
        instance and remember it for these shapes; returns (best index, ms per
        instance). Waits for the device; leaves the batch's results in J, Z and
        the infos."""
        ncfg = int(lib().id_batched_config_count(_DTYPES[self.dtype]))
        ms = (ctypes.c_float * ncfg)()
        best = ctypes.c_int(-1)
        with torch.cuda.device(self.device):
            rc = lib().id_batched_autotune(self.desc.data_ptr(), len(self.order), _DTYPES[self.dtype],
                                           self.batch_work.data_ptr(), self.batch_work.numel(), self.infos.data_ptr(),
                                           int(reps), ms, ctypes.byref(best), _stream(self.device))
        if rc != ID_OK:
            raise IdError(rc, "id_batched_autotune")
        self.config, self.tune_ms = int(best.value), [float(x) for x in ms]
        _TUNED[_shape_signature(self.dtype, self.device, self.mats, self.ks)] = (self.config, self.tune_ms)
        path = os.environ.get(TUNE_CACHE_ENV)
        if path:
            tune_cache_put(path, _persisted_key(self), self.config, self.tune_ms)
        return self.config, self.tune_ms

    def __len__(self):
        return len(self.mats)

    def run(self):
        with torch.cuda.device(self.device):
            rc = lib().id_decompose_batched_with(self.desc.data_ptr(), len(self.order), _DTYPES[self.dtype],
                                                 self.batch_work.data_ptr(), self.batch_work.numel(),
                                                 self.infos.data_ptr(), self.config, _stream(self.device))
        if rc in _CALL_ERRORS:
            raise IdError(rc, "id_decompose_batched_with")

    def read_infos(self) -> list:
        """Per-problem info dicts in the caller's order (waits for the device)."""
        raw = self.infos.cpu().numpy().tobytes()
        sz = ctypes.sizeof(IdInfo)
        out = [None] * len(self.order)
        for slot, i in enumerate(self.order):
            out[i] = IdInfo.from_buffer_copy(raw[slot * sz:(slot + 1) * sz]).as_dict()
        return out


def id_decompose_batched(mats: list, ks: list, *, sync: bool = True, config: int | None = None,
                         autotune: bool = False):
    """Rank-k_i IDs of the CUDA matrices mats[i] in one launch. Returns (Js, Zs, infos, plan);
    infos is None when sync is False (read them later with plan.read_infos()). ``config`` and
    ``autotune`` choose the kernel instance as in BatchedPlan."""
    plan = BatchedPlan(mats, ks, config=config, autotune=autotune)
    plan.run()
    return plan.J, plan.Z, (plan.read_infos() if sync else None), plan

