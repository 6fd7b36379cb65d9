"""The seeded synthetic inputs match the recipe they are documented with.

The generators feed both the oracle and the CUDA path (they hold none of the
method's arithmetic); these checks pin the spectra, the Haar factors, the
uneven batch and the sketch to their stated definitions, so a workload cannot
drift from the one the measurements describe.
"""
import math

import numpy as np
import pytest
import torch

import synth


def test_spectra_closed_forms():
    assert synth.spectrum("pow2_half", 5)[2] == pytest.approx(0.5, rel=1e-15)
    assert synth.spectrum("exp64", 200)[64] == pytest.approx(math.exp(-1.0), rel=1e-15)
    p = synth.spectrum("poly1.5", 10)
    assert p[0] == 1.0 and p[3] == pytest.approx(0.125, rel=1e-15)
    assert synth.spectrum("poly2", 10)[4] == pytest.approx(1 / 25, rel=1e-15)
    e = synth.spectrum("exp8m", 30, m=8)
    assert e[1] == pytest.approx(math.exp(-1.0), rel=1e-15)
    r = synth.spectrum("exp64", 300, rank=256)
    assert np.count_nonzero(r) == 256 and r[255] > 0
    with pytest.raises(ValueError):
        synth.spectrum("nope", 3)


def test_haar_factor_is_orthonormal_and_seeded():
    Q = synth.haar(90, 40, 11).numpy()
    assert np.abs(Q.T @ Q - np.eye(40)).max() < 1e-13
    assert np.array_equal(Q, synth.haar(90, 40, 11).numpy())
    assert not np.allclose(Q, synth.haar(90, 40, 12).numpy())


@pytest.mark.parametrize("m,n", [(40, 70), (70, 40)])
def test_lowrank_has_the_stated_singular_values(m, n):
    s = synth.spectrum("exp64", min(m, n))
    A = synth.lowrank(m, n, s, 5).numpy()
    assert A.shape == (m, n)
    assert np.allclose(np.linalg.svd(A, compute_uv=False), s, rtol=0, atol=1e-13)
    assert np.array_equal(A, synth.lowrank(m, n, s, 5).numpy())


def test_uneven_batch_recipe():
    """m ~ U[32, 256], n ~ U[m, 4m], k ~ U[8, min(64, m)], about 10% sparse
    non-negative matrices of density 5%, the rest with s_i = exp(-8 i / m)."""
    probs = synth.batched_uneven(300, 4, dtype=torch.float32)
    assert len(probs) == 300
    nsparse = 0
    nnz = total = 0
    for p in probs:
        m, n, k, A = p["m"], p["n"], p["k"], p["A"]
        assert 32 <= m <= 256 and m <= n <= 4 * m and 8 <= k <= min(64, m)
        assert A.shape == (m, n) and A.dtype == torch.float32 and A.is_contiguous()
        if p["kind"] == "sparse":
            nsparse += 1
            assert (A >= 0).all() and (A < 1).all()
            nnz += int(torch.count_nonzero(A))
            total += m * n
    assert 15 <= nsparse <= 45
    assert 0.045 <= nnz / total <= 0.055
    for p in [q for q in probs if q["kind"] == "lowrank"][:4]:
        m, n = p["m"], p["n"]
        s = synth.spectrum("exp8m", min(m, n), m=m)
        sv = np.linalg.svd(p["A"].double().numpy(), compute_uv=False)
        assert np.abs(sv - s).max() <= 1e-5          # FP32 storage of the FP64 product
    again = synth.batched_uneven(300, 4, dtype=torch.float32)
    assert all(torch.equal(a["A"], b["A"]) for a, b in zip(probs[:20], again[:20]))


def test_gaussian_sketch_is_bf16_standard_normal():
    om = synth.gaussian_sketch_bf16(64, 4096, 3)
    assert om.dtype == torch.bfloat16 and om.shape == (64, 4096)
    x = om.double()
    assert abs(x.mean().item()) < 0.01 and abs(x.std().item() - 1.0) < 0.01
    assert torch.equal(om, synth.gaussian_sketch_bf16(64, 4096, 3))


def test_paper_datasets_distributions():
    b = synth.paper_dataset("boolean", 1, 50, 60)
    assert set(np.unique(b).tolist()) == {0.0, 1.0}
    u = synth.paper_dataset("uniform", 1, 50, 60)
    assert u.min() >= 0.0 and u.max() < 1.0
    g = synth.paper_dataset("gaussian", 1, 200, 300)
    assert abs(g.mean()) < 0.02 and abs(g.std() - 1.0) < 0.02
