"""Sparse (CSR) input: id_decompose_csr forms the working matrix directly and
runs the grid-engine CPQR, so on the same matrix it must return exactly what
the dense id_decompose (grid engine) returns; and its pivots must pass the
oracle's greedy replay on the oracle's densified matrix."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import id_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbid():
    import __graft_entry__ as g

    g.build()
    import paper_2105_07076_gb300 as m

    return m


def _dev(rowptr, colind, vals, dtype):
    return (torch.as_tensor(rowptr, device="cuda"), torch.as_tensor(colind, device="cuda"),
            torch.as_tensor(vals, dtype=dtype, device="cuda"))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,k,density", [(300, 700, 30, 0.03), (700, 300, 30, 0.03), (128, 2000, 64, 0.01),
                                           (1000, 1000, 50, 0.005)])
def test_csr_equals_dense(gbid, dtype, m, n, k, density):
    rowptr, colind, vals = synth.sparse_powerlaw_csr(m, n, density, m + n)
    Ad = orc.csr_to_dense(rowptr, colind, vals, m, n)
    J, Z, info = gbid.id_decompose_csr(*_dev(rowptr, colind, vals, dtype), (m, n), k)
    A = torch.as_tensor(Ad, dtype=dtype, device="cuda")
    J0, Z0, info0 = gbid.id_decompose(A, k, engine=gbid.ENGINE_GRID)
    assert info["status"] == info0["status"]
    assert torch.equal(J, J0) and torch.equal(Z, Z0)
    if info["status"] == gbid.ID_OK:
        tol = 1e-6 if dtype == torch.float64 else 64 * 2.0 ** -24 * math.sqrt(max(m, n))
        X = Ad if m <= n else Ad.T
        ok, worst = orc.verify_pivots(X, J.cpu().numpy().astype(np.int64), tol)
        assert ok, worst.max()


def test_csr_duplicates_and_empty_rows(gbid):
    # row 1 empty, (0, 3) given twice, an empty last row
    rowptr = np.array([0, 3, 3, 5, 7, 7], dtype=np.int64)
    colind = np.array([3, 0, 3, 1, 5, 2, 6], dtype=np.int32)
    vals = np.array([1.0, 2.0, 0.5, -1.0, 3.0, 4.0, 1.0])
    Ad = orc.csr_to_dense(rowptr, colind, vals, 5, 8)
    J, Z, info = gbid.id_decompose_csr(*_dev(rowptr, colind, vals, torch.float64), (5, 8), 3)
    J0, Z0, _ = gbid.id_decompose(torch.as_tensor(Ad, device="cuda"), 3, engine=gbid.ENGINE_GRID)
    assert torch.equal(J, J0) and torch.equal(Z, Z0)


@pytest.mark.parametrize("bad", ["column", "rowptr"])
def test_csr_malformed_is_reported(gbid, bad):
    rowptr = np.array([0, 2, 4, 6], dtype=np.int64)
    colind = np.array([0, 1, 2, 3, 4, 5], dtype=np.int32)
    vals = np.arange(1.0, 7.0)
    if bad == "column":
        colind[3] = 9
    else:
        rowptr[2] = 1
    with pytest.raises(gbid.IdError) as e:     # found on the device, reported as ID_EINVAL
        gbid.id_decompose_csr(*_dev(rowptr, colind, vals, torch.float64), (3, 8), 2)
    assert e.value.status == gbid.ID_EINVAL
