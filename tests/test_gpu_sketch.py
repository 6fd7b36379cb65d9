"""Sketch Y = Omega A on the tensor cores vs the FP64 oracle, element by element.

The kernel rounds A to BF16 (nearest even) and accumulates in FP32. The oracle
is given the same BF16-rounded A, so the only difference is FP32 accumulation:
each entry must satisfy |Y - Y_ref| <= K u_32 (|Omega| |A_bf16|)_ij (the
worst-case bound of a K-term FP32 sum; K = m).
"""
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


def _padded(t, mult):
    """Copy of a 2-D tensor whose row stride is a multiple of `mult` elements (TMA needs 16-byte strides)."""
    r, c = t.shape
    big = torch.zeros(r, (c + mult - 1) // mult * mult, dtype=t.dtype, device=t.device)
    big[:, :c] = t
    return big[:, :c]


def _check(Y, omega, A):
    Om = omega.double().cpu().numpy()
    Ab = A.to(torch.bfloat16).double().cpu().numpy()
    ref = orc.sketch(Om, Ab)
    bound = A.shape[0] * U32 * (np.abs(Om) @ np.abs(Ab)) + 1e-37
    err = np.abs(Y.double().cpu().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())
    return float(np.linalg.norm(err) / max(np.linalg.norm(ref), 1e-300))


@pytest.mark.parametrize("l,m,n", [
    (16, 64, 96), (128, 32, 96), (130, 100, 200), (200, 333, 517), (1, 40, 50), (640, 256, 300),
    (522, 1000, 1000), (64, 4096, 130),
])
def test_sketch_matches_oracle(gbid, l, m, n):
    g = torch.Generator().manual_seed(l * 1000003 + m * 1009 + n)
    A = _padded(torch.randn(m, n, generator=g).cuda(), 4)
    omega = _padded(synth.gaussian_sketch_bf16(l, m, seed=7 + l).cuda(), 8)
    Y, info = gbid.id_sketch(A, omega)
    torch.cuda.synchronize()
    assert info["status"] == gbid.ID_OK, info
    _check(Y, omega, A)


def test_sketch_leading_dimensions(gbid):
    m, n, l = 200, 300, 70
    Abig = torch.randn(m, n + 12).cuda()      # lda = 312, ldo = 224
    A = Abig[:, :n]
    Obig = synth.gaussian_sketch_bf16(l, m + 24, seed=3).cuda()
    omega = Obig[:, :m]
    Y = torch.full((l, n + 5), float("nan"), device="cuda")
    gbid.id_sketch(A, omega, out=Y[:, :n])
    _check(Y[:, :n], omega, A)
    assert torch.isnan(Y[:, n:]).all()            # nothing written beyond n columns


def test_sketch_argument_errors(gbid):
    A = torch.randn(64, 100).cuda()
    om = synth.gaussian_sketch_bf16(700, 64, seed=1).cuda()
    with pytest.raises(gbid.IdError):
        gbid.id_sketch(A, om)                      # l > 640
    A2 = torch.randn(64, 102).cuda()[:, :101]      # lda = 102 not a multiple of 4
    with pytest.raises(gbid.IdError):
        gbid.id_sketch(A2, synth.gaussian_sketch_bf16(8, 64, seed=1).cuda())


def test_sketch_full_size_sampled(gbid):
    """Randomized-ID workload: A 16384 x 32768 FP32, Omega (512+10) x 16384; 96 sampled entries."""
    m, n, l = 16384, 32768, 522
    A = synth.lowrank(m, n, synth.spectrum("poly1.5", m), 3, device="cuda", dtype=torch.float32,
                      gen_dtype=torch.float32)
    omega = synth.gaussian_sketch_bf16(l, m, seed=33, device="cuda")
    Y, info = gbid.id_sketch(A, omega)
    torch.cuda.synchronize()
    assert info["status"] == gbid.ID_OK
    rng = np.random.default_rng(5)
    rows = rng.integers(0, l, 96)
    cols = rng.integers(0, n, 96)
    Om = omega.double().cpu().numpy()
    Yh = Y.double().cpu().numpy()
    for i, j in zip(rows, cols):
        a = A[:, j].to(torch.bfloat16).double().cpu().numpy()
        ref = float(Om[i] @ a)
        bound = m * U32 * float(np.abs(Om[i]) @ np.abs(a))
        assert abs(Yh[i, j] - ref) <= bound, (i, j, Yh[i, j], ref)
