"""Two-sided ID X^T A[I, J] Z on the GPU against the oracle's two_sided_interp_decomp.

Each stage's pivots must pass the oracle's greedy replay (stage 1 on A, stage
2 on the skeleton, transposed for a row ID), X[:, I] and Z[:, J] must be
identities, X and Z must match the oracle's IDs with the GPU's pivots forced
(FP64 1e-9 relative; FP32 max(1e-4, 2 cond u_32)), and the two-sided error
must equal the first stage's (the second stage is exact in exact arithmetic).
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import id_oracle as orc

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def gbid():
    import __graft_entry__ as g

    g.build()
    import paper_2105_07076_gb300 as m

    return m


def _zbar(dtype, M, piv):
    if dtype == torch.float64:
        return 1e-9
    return max(1e-4, 2 * np.linalg.cond(M[:, piv]) * U32)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,k", [(300, 700, 40), (700, 300, 40), (64, 64, 20), (40, 100, 40), (100, 40, 40),
                                   (1000, 2000, 64)])
def test_two_sided_matches_oracle(gbid, dtype, m, n, k):
    A = synth.lowrank(m, n, synth.spectrum("exp64", min(m, n)), 17, dtype=dtype).cuda()
    I, J, X, Z, (i1, i2) = gbid.id_decompose_two_sided(A, k)
    assert i1["status"] == gbid.ID_OK and i2["status"] == gbid.ID_OK, (i1, i2)
    Ah = A.double().cpu().numpy()
    Ig = I.cpu().numpy().astype(np.int64)
    Jg = J.cpu().numpy().astype(np.int64)
    Xg = X.double().cpu().numpy()
    Zg = Z.double().cpu().numpy()
    assert np.array_equal(Xg[:, Ig], np.eye(k)) and np.array_equal(Zg[:, Jg], np.eye(k))
    tol = 1e-6 if dtype == torch.float64 else 64 * U32 * math.sqrt(max(m, n))
    if m <= n:
        ok, w = orc.verify_pivots(Ah, Jg, tol)                 # stage 1: column ID of A
        assert ok, w.max()
        C = Ah[:, Jg]
        if m > k:
            ok, w = orc.verify_pivots(C.T, Ig, tol)            # stage 2: row ID of C
            assert ok, w.max()
        _, Zo, _ = orc.interp_decomp(Ah, k, pivots=Jg)
        Xo = np.eye(k) if m == k else orc.interp_decomp(C, k, pivots=Ig)[1]
        e1 = orc.rel_error(Ah, Jg, Zg)
        assert np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo) <= _zbar(dtype, Ah, Jg)
        assert np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo) <= (1e-9 if dtype == torch.float64 else
                                                                max(1e-4, 2 * np.linalg.cond(C[Ig, :]) * U32))
    else:
        ok, w = orc.verify_pivots(Ah.T, Ig, tol)               # stage 1: row ID of A
        assert ok, w.max()
        R = Ah[Ig, :]
        if n > k:
            ok, w = orc.verify_pivots(R, Jg, tol)              # stage 2: column ID of R
            assert ok, w.max()
        _, Xo, _ = orc.interp_decomp(Ah, k, pivots=Ig)
        Zo = np.eye(k) if n == k else orc.interp_decomp(R, k, pivots=Jg)[1]
        e1 = orc.rel_error(Ah, Ig, Xg, transposed=True)
        assert np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo) <= _zbar(dtype, Ah.T, Ig)
        assert np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo) <= (1e-9 if dtype == torch.float64 else
                                                                max(1e-4, 2 * np.linalg.cond(R[:, Jg]) * U32))
    e2 = np.linalg.norm(Ah - orc.two_sided_reconstruct(Ah, Ig, Jg, Xg, Zg)) / np.linalg.norm(Ah)
    assert abs(e2 - e1) <= (1e-9 if dtype == torch.float64 else 1e-4) * max(e1, 1e-3)


def test_two_sided_exact_rank(gbid):
    s = np.where(np.arange(200) < 30, np.exp(-np.arange(200) / 10.0), 0.0)
    A = synth.lowrank(200, 500, s, 3).cuda()
    I, J, X, Z, _ = gbid.id_decompose_two_sided(A, 30)
    Ah = A.cpu().numpy()
    approx = orc.two_sided_reconstruct(Ah, I.cpu().numpy().astype(np.int64), J.cpu().numpy().astype(np.int64),
                                       X.cpu().numpy(), Z.cpu().numpy())
    assert np.linalg.norm(Ah - approx) / np.linalg.norm(Ah) <= 1e-11
