"""id_refine: one least-squares refinement of Z against A for a fixed skeleton J.

The least-squares problem is linear, so one exact Newton step from any Z lands
on the LS solution Z* = argmin ||A - A[:, J] Z||_F (the oracle's ``ls_interp``,
solved by an orthogonal factorisation, never through C^T C). The GPU forms
C^T C in FP64 and the residual in FP32, so the bar is relative to the
conditioning: ||Z - Z*|| / ||Z*|| <= max(1e-4, 2 sqrt(k) cond(C) u_32).
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


def _bar(Ah, J, Z0h=None):
    """Error bound of one seminormal-equation step in FP32 data and FP32 products:
    2 sqrt(k) cond(C) u_32 from the rounding of the residual, plus
    4 cond(C)^2 u_32 ||A - C Z0|| / (||C||_2 ||Z_ls||) from the normal equations'
    squared conditioning acting on the starting residual."""
    k = len(J)
    C = Ah[:, J]
    cond = np.linalg.cond(C)
    bar = 2 * math.sqrt(k) * cond * U32
    if Z0h is not None:
        Zls = orc.ls_interp(Ah, J)
        eta = np.linalg.norm(Ah - C @ Z0h) / (np.linalg.norm(C, 2) * np.linalg.norm(Zls))
        bar += 4 * cond ** 2 * U32 * eta
    return max(1e-4, bar)


@pytest.mark.parametrize("m,n,k,spec", [(300, 700, 40, "poly1.5"), (512, 2048, 100, "exp64"), (64, 64, 20, "poly2"),
                                        (200, 5000, 33, "poly1.5")])
def test_refine_lands_on_least_squares(gbid, m, n, k, spec):
    """Start from the randomized ID's unrefined Z (the sketch's T), as the
    randomized path does; one step must land on the least-squares Z."""
    A = synth.lowrank(m, n, synth.spectrum(spec, m), 7, dtype=torch.float32).cuda()
    l = min(k + 10, m)
    om = synth.gaussian_sketch_bf16(l, m, seed=k, device="cuda")
    big = torch.zeros(l, (m + 7) // 8 * 8, dtype=om.dtype, device="cuda")   # 16-byte row stride (TMA)
    big[:, :m] = om
    omega = big[:, :m]
    J, Z0, _ = gbid.id_decompose_randomized(A, omega, k, refine=False)
    Ah = A.double().cpu().numpy()
    Jg = J.cpu().numpy().astype(np.int64)
    Z0h = Z0.double().cpu().numpy()
    Z1, info = gbid.id_refine(A, J, Z0.clone())
    assert info["status"] == gbid.ID_OK and info["refined"]
    Z1h = Z1.double().cpu().numpy()
    assert np.array_equal(Z1h[:, Jg], np.eye(k))
    Zls = orc.ls_interp(Ah, Jg)
    assert np.linalg.norm(Z1h - Zls) / np.linalg.norm(Zls) <= _bar(Ah, Jg, Z0h)
    # the reconstruction error reaches the least-squares optimum for this skeleton
    e_ls = orc.rel_error(Ah, Jg, Zls)
    assert orc.rel_error(Ah, Jg, Z1h) <= e_ls * (1 + 1e-3)
    assert orc.rel_error(Ah, Jg, Z0h) >= e_ls
    assert info["max_abs_z"] == pytest.approx(np.abs(Z1h).max(), rel=1e-12)
    assert info["n_gt2"] == int(np.count_nonzero(np.abs(Z1h) > 2.0))


def test_refine_from_a_perturbed_z(gbid):
    """A start far from the optimum (every entry of T perturbed by 5%): the
    step still lands within the bound, which grows with the starting residual."""
    A = synth.lowrank(300, 700, synth.spectrum("poly1.5", 300), 7, dtype=torch.float32).cuda()
    k = 40
    J, Z0, _ = gbid.id_decompose(A, k)
    g = torch.Generator(device="cuda").manual_seed(3)
    Zs = Z0 + 0.05 * torch.randn(Z0.shape, generator=g, device="cuda")
    Zs[:, J.long()] = torch.eye(k, device="cuda")
    Ah = A.double().cpu().numpy()
    Jg = J.cpu().numpy().astype(np.int64)
    bar = _bar(Ah, Jg, Zs.double().cpu().numpy())
    Z1, info = gbid.id_refine(A, J, Zs.clone())
    Zls = orc.ls_interp(Ah, Jg)
    Z1h = Z1.double().cpu().numpy()
    assert np.linalg.norm(Z1h - Zls) / np.linalg.norm(Zls) <= bar
    # a second step starts from a residual at the optimum's level
    Z2, _ = gbid.id_refine(A, J, Z1.clone())
    Z2h = Z2.double().cpu().numpy()
    assert np.linalg.norm(Z2h - Zls) <= np.linalg.norm(Z1h - Zls)


def test_refine_keeps_the_deterministic_z(gbid):
    """The deterministic ID's T = R11^{-1} R12 already solves the LS problem:
    refining it moves Z by no more than the bar."""
    A = synth.lowrank(400, 900, synth.spectrum("exp64", 400), 5, dtype=torch.float32).cuda()
    k = 50
    J, Z0, _ = gbid.id_decompose(A, k)
    Z1, info = gbid.id_refine(A, J, Z0.clone())
    Ah = A.double().cpu().numpy()
    Jg = J.cpu().numpy().astype(np.int64)
    d = (torch.linalg.norm(Z1.double() - Z0.double()) / torch.linalg.norm(Z0.double())).item()
    assert d <= _bar(Ah, Jg)


def test_refine_rank_deficient_skeleton_leaves_z(gbid):
    """C with two equal columns: C^T C is singular, Z is left unchanged."""
    A = torch.randn(120, 300, dtype=torch.float32, generator=torch.Generator().manual_seed(1))
    A[:, 7] = A[:, 3]
    A = A.cuda()
    J = torch.tensor([3, 7, 11, 20], dtype=torch.int32, device="cuda")
    Z = torch.randn(4, 300, device="cuda")
    Z[:, J.long()] = torch.eye(4, device="cuda")
    Zc = Z.clone()
    _, info = gbid.id_refine(A, J, Z)
    assert not info["refined"]
    assert torch.equal(Z, Zc)


def test_refine_bad_skeleton_index(gbid):
    A = torch.randn(50, 80, device="cuda")
    J = torch.tensor([1, 2, 80], dtype=torch.int32, device="cuda")
    Z = torch.zeros(3, 80, device="cuda")
    with pytest.raises(gbid.IdError) as e:     # found on the device, reported as ID_EINVAL
        gbid.id_refine(A, J, Z)
    assert e.value.status == gbid.ID_EINVAL
    assert torch.count_nonzero(Z).item() == 0
