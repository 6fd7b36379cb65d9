"""Column-sampling Optim RID (Sec. 2.2) on the GPU vs the oracle's sampled_interp_decomp.

The same sample idx goes to both. The GPU's pivots on A_S must pass the
oracle's greedy replay on A_S (FP64 margin 1e-6, FP32 64 u_32 sqrt(m)); J must
equal idx[P_k]; Z must match the oracle's normal-equation Z for the GPU's J
within 1e-8 relative (FP64 normal equations carry cond(C)^2 eps) or, in FP32
data, within the least-squares sensitivity max(1e-6, 4 cond(C)^2 eps_64 + ...).
"""
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


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,n,k,spec", [(784, 1000, 190, "poly1.5"), (300, 700, 40, "exp64"), (1000, 600, 30, "poly2"),
                                        (64, 64, 20, "poly2")])
def test_sampled_rid_matches_oracle(gbid, dtype, m, n, k, spec):
    A = synth.lowrank(m, n, synth.spectrum(spec, min(m, n)), 11, dtype=dtype).cuda()
    p = min(n, k + int(0.2 * k))
    idx = np.random.default_rng(m + n + k).choice(n, size=p, replace=False).astype(np.int32)
    J, Z, info = gbid.id_decompose_sampled(A, idx, k)
    assert info["status"] == gbid.ID_OK, info
    Ah = A.double().cpu().numpy()
    Jg = J.cpu().numpy().astype(np.int64)
    assert set(Jg.tolist()) <= set(idx.tolist()) and len(set(Jg.tolist())) == k
    tol = 1e-6 if dtype == torch.float64 else 64 * 2.0 ** -24 * math.sqrt(m)
    AS = Ah[:, idx]
    pos = {int(c): i for i, c in enumerate(idx)}
    ok, worst = orc.verify_pivots(AS, np.array([pos[int(c)] for c in Jg]), tol)
    assert ok, worst.max()
    Zg = Z.double().cpu().numpy()
    assert np.array_equal(Zg[:, Jg], np.eye(k))
    C = Ah[:, Jg]
    R = np.linalg.qr(C, mode="r")
    Zo = orc.normal_equation_z(Ah, Jg, R)
    cond = np.linalg.cond(C)
    bar = max(1e-8, 16 * cond ** 2 * np.finfo(np.float64).eps)
    if dtype == torch.float32:
        bar = max(bar, 1e-6)
    rest = np.setdiff1d(np.arange(n), Jg)
    err = np.linalg.norm(Zg[:, rest] - Zo[:, rest]) / np.linalg.norm(Zo[:, rest])
    assert err <= bar, (err, bar, cond)
    # the oracle's own Optim RID with the same sample picks the same skeleton (up to near-ties)
    Jo, Zo2, oinfo = orc.sampled_interp_decomp(Ah, idx, k)
    near = np.flatnonzero(oinfo["gap"] < tol)
    first = int(near[0]) if near.size else k
    assert np.array_equal(Jg[:first], Jo[:first])


def test_sampled_rid_every_column_is_the_deterministic_skeleton(gbid):
    A = synth.lowrank(200, 400, synth.spectrum("pow2_half", 200), 1).cuda()
    idx = np.random.default_rng(3).permutation(400).astype(np.int32)
    J, Z, info = gbid.id_decompose_sampled(A, idx, 20)
    J0, Z0, _ = gbid.id_decompose(A, 20)
    assert info["status"] == gbid.ID_OK
    assert torch.equal(J, J0)
    # T = R11^-1 R12 against the normal equations' Z: equal up to cond(C)^2 eps
    cond = np.linalg.cond(A[:, J.long()].cpu().numpy())
    bar = max(1e-12, 16 * cond ** 2 * np.finfo(np.float64).eps)
    assert (torch.linalg.norm(Z - Z0) / torch.linalg.norm(Z0)).item() <= bar


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sampled_rid_reports_rank_deficiency(gbid, dtype):
    """A of exact rank 10 asked for k = 15: the CPQR of the sample finds it."""
    s = np.where(np.arange(120) < 10, 1.0, 0.0)
    A = synth.lowrank(120, 300, s, 2, dtype=dtype).cuda()
    idx = np.random.default_rng(5).choice(300, size=40, replace=False).astype(np.int32)
    J, Z, info = gbid.id_decompose_sampled(A, idx, 15)
    assert info["status"] == gbid.ID_RANK_DEFICIENT
    assert info["rank"] == 10
    J10, Z10, info10 = gbid.id_decompose_sampled(A, idx, 10)
    assert info10["status"] == gbid.ID_OK
    Ah = A.double().cpu().numpy()
    err = orc.rel_error(Ah, J10.cpu().numpy().astype(np.int64), Z10.double().cpu().numpy())
    assert err <= (1e-10 if dtype == torch.float64 else 1e-5)


def test_sampled_rid_rejects_a_bad_sample(gbid):
    A = torch.randn(50, 80, dtype=torch.float64, device="cuda")
    for bad in ([1, 1, 2, 3], [0, 5, 80, 2], [-1, 2, 3, 4]):
        with pytest.raises(gbid.IdError):
            gbid.id_decompose_sampled(A, bad, 3)
