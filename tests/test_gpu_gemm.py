"""The library's matrix product (id_gemm) against an FP64 reference on the host.

FP32 data runs the 3xTF32 tensor-core kernel (tcgen05, TMA); FP64 data the
SIMT FP64 kernel. Shapes cover single elements, ragged tiles in every
dimension, K below and above one 16-wide block, both transpose flags, and the
alpha/beta update. The bound is per entry: FP32 products within 2^-18 of
sum_k |a_ik||b_kj| (the split's own error is about 2^-21 of it) plus the
rounding of beta C; FP64 within 4 K 2^-53 of the same sum.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbid():
    import __graft_entry__ as g

    g.build()
    import paper_2105_07076_gb300 as m

    return m


SHAPES = [(1, 1, 1), (130, 70, 33), (257, 300, 100), (128, 256, 16), (500, 40, 1000), (64, 600, 7), (300, 513, 48)]


def _ref(A, B, C, ta, tb, alpha, beta):
    a = A.T if ta else A
    b = B.T if tb else B
    return alpha * (a @ b) + beta * C, np.abs(a) @ np.abs(b)


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_gemm_matches_fp64(gbid, M, N, K, ta, tb, dtype):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K + 11 * ta + 5 * tb)
    A = torch.randn((K, M) if ta else (M, K), generator=g, dtype=torch.float64)
    B = torch.randn((N, K) if tb else (K, N), generator=g, dtype=torch.float64)
    C = torch.randn(M, N, generator=g, dtype=torch.float64)
    alpha, beta = -1.5, (0.0 if (M + N) % 2 else 0.75)
    Ad, Bd, Cd = (X.to(dtype) for X in (A, B, C))
    out = Cd.clone().cuda()
    got, info = gbid.gemm(Ad.cuda(), Bd.cuda(), ta=bool(ta), tb=bool(tb), alpha=alpha, beta=beta, out=out)
    assert info["status"] == gbid.ID_OK, info
    ref, mag = _ref(Ad.double().numpy(), Bd.double().numpy(), Cd.double().numpy(), ta, tb, alpha, beta)
    err = np.abs(got.cpu().double().numpy() - ref)
    if dtype == torch.float32:
        bound = 2.0 ** -18 * abs(alpha) * mag + 2.0 ** -23 * np.abs(ref) + 1e-30
    else:
        bound = 4 * K * 2.0 ** -53 * abs(alpha) * mag + 2.0 ** -52 * np.abs(ref) + 1e-300
    assert np.all(err <= bound), float((err / bound).max())


def test_gemm_fp32_beats_plain_tf32(gbid):
    # the split keeps FP32-level accuracy: a single TF32 product would err by ~2^-11
    g = torch.Generator().manual_seed(5)
    A = torch.randn(256, 512, generator=g, dtype=torch.float64).float()
    B = torch.randn(512, 384, generator=g, dtype=torch.float64).float()
    got, _ = gbid.gemm(A.cuda(), B.cuda())
    ref = A.double().numpy() @ B.double().numpy()
    mag = np.abs(A.double().numpy()) @ np.abs(B.double().numpy())
    rel = float((np.abs(got.cpu().double().numpy() - ref) / mag).max())
    assert rel < 2.0 ** -19, rel


def test_gemm_argument_errors(gbid):
    A = torch.zeros(4, 4, device="cuda")
    with pytest.raises(ValueError):
        gbid.gemm(A, torch.zeros(5, 4, device="cuda"))
