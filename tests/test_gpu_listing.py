"""The outputs of the paper's listings (Sec. 2.1): Z from the normal equations
R_k^T R_k Z = C^T A (Eq. final_eq), and the approximation approx = C @ Z.

id_decompose(normal_eq=True) runs the same CPQR as the default route, so J is
identical; its Z must match the oracle's normal-equation Z for that J within
the normal equations' own sensitivity, 16 cond(C)^2 eps_64 (FP32 data: at
least 1e-6, the FP32 rounding of the output). id_reconstruct is one GEMM on
the gathered skeleton: FP64 within 1e-12 of the oracle's C @ Z, FP32 within
1e-5 (FP32-accurate products over k terms).
"""
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
@pytest.mark.parametrize("m,n,k,spec", [(300, 700, 40, "poly1.5"), (512, 2048, 100, "exp64"), (64, 64, 20, "poly2"),
                                        (200, 400, 20, "pow2_half")])
def test_normal_equation_z(gbid, dtype, m, n, k, spec):
    A = synth.lowrank(m, n, synth.spectrum(spec, min(m, n)), 13, dtype=dtype).cuda()
    J, Z, info = gbid.id_decompose(A, k, normal_eq=True)
    J0, Z0, _ = gbid.id_decompose(A, k, engine=gbid.ENGINE_GRID)
    assert info["status"] == gbid.ID_OK, info
    assert torch.equal(J, J0)
    Ah = A.double().cpu().numpy()
    Jg = J.cpu().numpy().astype(np.int64)
    Zg = Z.double().cpu().numpy()
    assert np.array_equal(Zg[:, Jg], np.eye(k))
    C = Ah[:, Jg]
    Zo = orc.normal_equation_z(Ah, Jg, np.linalg.qr(C, mode="r"))
    bar = max(1e-8, 16 * np.linalg.cond(C) ** 2 * np.finfo(np.float64).eps)
    if dtype == torch.float32:
        bar = max(bar, 1e-6)
    assert np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo) <= bar
    assert info["n_gt2"] == int(np.count_nonzero(np.abs(Zg) > 2.0))
    assert info["max_abs_z"] == pytest.approx(np.abs(Zg).max(), rel=1e-12)


def test_normal_equation_z_rank_deficient(gbid):
    s = np.where(np.arange(150) < 12, 1.0, 0.0)
    A = synth.lowrank(150, 400, s, 4).cuda()
    _, _, info = gbid.id_decompose(A, 20, normal_eq=True)
    assert info["status"] == gbid.ID_RANK_DEFICIENT and info["rank"] == 12


def test_normal_equation_z_needs_a_column_id(gbid):
    A = torch.randn(300, 100, dtype=torch.float64, device="cuda")
    with pytest.raises(gbid.IdError):
        gbid.id_decompose(A, 10, normal_eq=True)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("m,n,k", [(300, 700, 40), (700, 300, 40), (129, 1000, 64), (1000, 129, 33)])
def test_reconstruct(gbid, dtype, tol, m, n, k):
    A = synth.lowrank(m, n, synth.spectrum("poly1.5", min(m, n)), 21, dtype=dtype).cuda()
    J, Z, info = gbid.id_decompose(A, k)
    tr = m > n
    Zv = Z if not tr else Z[:, :m]
    approx, rinfo = gbid.id_reconstruct(A, J, Zv, transposed=tr)
    assert rinfo["status"] == gbid.ID_OK
    Ah = A.double().cpu().numpy()
    want = orc.reconstruct(Ah, J.cpu().numpy().astype(np.int64), Zv.double().cpu().numpy(), transposed=tr)
    got = approx.double().cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= tol
    # the error it implies is the ID's error
    err = np.linalg.norm(Ah - got) / np.linalg.norm(Ah)
    assert err == pytest.approx(orc.rel_error(Ah, J.cpu().numpy().astype(np.int64), Zv.double().cpu().numpy(),
                                              transposed=tr), rel=1e-8 if dtype == torch.float64 else 1e-3)


def test_reconstruct_bad_index(gbid):
    A = torch.randn(50, 80, dtype=torch.float64, device="cuda")
    J = torch.tensor([1, 2, 80], dtype=torch.int32, device="cuda")
    Z = torch.zeros(3, 80, dtype=torch.float64, device="cuda")
    with pytest.raises(gbid.IdError):
        gbid.id_reconstruct(A, J, Z)
