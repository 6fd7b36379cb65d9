"""id_decompose_noalloc: the decomposition for callers that cannot allocate device memory.

Such callers (code running during a global-mode stream capture, plug-ins whose
host framework owns all device memory, real-time loops) use the library's
fixed scratch array instead of a workspace. This checks, through the C ABI,
that two calls in a row give the same J as the workspace entry point and a Z
within the FP64 parity tolerance of the other tests (1e-10 relative), with the
default options and with the normal-equation route (a non-NULL opts), and that
a problem too large for the fixed scratch is refused before any GPU work.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbid():
    import __graft_entry__ as g

    g.build()
    import paper_2105_07076_gb300 as m

    return m


def _noalloc(gbid, A, k, opts=None):
    m, n = A.shape
    J = torch.empty(k, dtype=torch.int32, device=A.device)
    Z = torch.empty(k, max(m, n), dtype=A.dtype, device=A.device)
    info = gbid.IdInfo()
    rc = gbid.lib().id_decompose_noalloc(ctypes.c_void_p(A.data_ptr()), gbid.ID_F64, m, n, A.stride(0), k,
                                         ctypes.byref(opts) if opts is not None else None,
                                         ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(Z.data_ptr()), Z.stride(0),
                                         ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, J, Z, info


def test_noalloc_matches_workspace_entry_point_twice(gbid):
    A = torch.as_tensor(synth.lowrank(300, 700, np.exp(-np.arange(300) / 25.0), 31).numpy()).cuda()
    k = 40
    J0, Z0, _ = gbid.id_decompose(A, k)
    for _ in range(2):
        rc, J, Z, info = _noalloc(gbid, A, k)
        torch.cuda.synchronize()
        assert rc == gbid.ID_OK and info.status == gbid.ID_OK
        assert torch.equal(J, J0)
        rel = (torch.linalg.norm(Z - Z0) / torch.linalg.norm(Z0)).item()
        assert rel <= 1e-10, rel


def test_noalloc_normal_equation_route_twice(gbid):
    """A non-NULL opts: Z from the paper's normal equations (zsolve = 1), whose
    products run in the library's own kernels, through the fixed scratch."""
    A = torch.as_tensor(synth.lowrank(300, 700, np.exp(-np.arange(300) / 25.0), 31).numpy()).cuda()
    k = 40
    J0, Z0, _ = gbid.id_decompose(A, k, normal_eq=True)
    for _ in range(2):
        rc, J, Z, info = _noalloc(gbid, A, k, gbid._opts(0, zsolve=1))
        torch.cuda.synchronize()
        assert rc == gbid.ID_OK and info.status == gbid.ID_OK
        assert torch.equal(J, J0)
        rel = (torch.linalg.norm(Z - Z0) / torch.linalg.norm(Z0)).item()
        assert rel <= 1e-10, rel


def test_noalloc_refuses_problems_beyond_its_scratch(gbid):
    m, n, k = 4096, 8192, 64          # 4096 x 8192 FP64 working copy alone is 256 MiB
    assert gbid.workspace_size(torch.float64, m, n, k) > gbid.NOALLOC_SCRATCH_BYTES
    fake = ctypes.c_void_p(256)
    rc = gbid.lib().id_decompose_noalloc(fake, gbid.ID_F64, m, n, n, k, None, fake, fake, n, None, None)
    assert rc == gbid.ID_ENOMEM
