"""Randomized ID (Gaussian sketch -> CPQR of Y -> T from Y's R) vs the FP64 oracle.

Stage-wise (refinement off): the oracle replays the GPU's pivots on the GPU's own sketch Y
(FP32 tolerance 64 u_32 sqrt(l) on near-ties) and recomputes Z for those
pivots (1e-4 relative Frobenius, the FP32 bar, widened to 2 cond(Y_J) u_32
where the conditioning of the skeleton puts 1e-4 out of FP32's reach). End to end: the reconstruction
error on A is at most 1.05x that of the oracle's randomized ID on the exact
FP64 sketch Omega A (same algorithm, FP64 throughout).
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


def _tol(l):
    return 64 * 2.0 ** -24 * math.sqrt(l)


@pytest.mark.parametrize("m,n,k,p,seed", [(600, 1200, 60, 10, 1), (256, 700, 40, 8, 2), (512, 2048, 100, 10, 3)])
def test_randomized_stagewise_and_end_to_end(gbid, m, n, k, p, seed):
    l = k + p
    A = synth.lowrank(m, n, synth.spectrum("poly1.5", m), 10 + seed, dtype=torch.float32).cuda()
    omega = synth.gaussian_sketch_bf16(l, m, seed=20 + seed).cuda()
    if m % 8:
        pytest.skip("sketch needs ldo % 8 == 0")
    J, Z, info = gbid.id_decompose_randomized(A, omega, k, refine=False)
    assert info["status"] == gbid.ID_OK, info
    assert not info["refined"]
    Y, _ = gbid.id_sketch(A, omega)                      # the same (deterministic) sketch
    Yh = Y.double().cpu().numpy()
    Jg = J.cpu().numpy().astype(np.int64)
    Zg = Z.double().cpu().numpy()
    ok, worst = orc.verify_pivots(Yh, Jg, _tol(l))
    assert ok, worst.max()
    Zo = orc.interp_decomp(Yh, k, pivots=Jg)[1]
    assert np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo) <= 1e-4
    assert np.array_equal(Zg[:, Jg], np.eye(k))
    Ah = A.double().cpu().numpy()
    err_g = orc.rel_error(Ah, Jg, Zg)
    Jo, Zy, Zr, _ = orc.randomized_interp_decomp(Ah, omega.double().cpu().numpy(), k)
    err_o = orc.rel_error(Ah, Jo, Zy)
    assert err_g <= 1.05 * err_o, (err_g, err_o, orc.rel_error(Ah, Jo, Zr))
    # with the refinement: the least-squares Z for the GPU's skeleton, and an
    # error at most 1.05x that of the oracle's refined randomized ID
    J2, Z2, info2 = gbid.id_decompose_randomized(A, omega, k)
    assert info2["status"] == gbid.ID_OK and info2["refined"]
    assert torch.equal(J2, J)
    Z2h = Z2.double().cpu().numpy()
    assert np.array_equal(Z2h[:, Jg], np.eye(k))
    Zls = orc.ls_interp(Ah, Jg)
    cond = np.linalg.cond(Ah[:, Jg])
    assert np.linalg.norm(Z2h - Zls) / np.linalg.norm(Zls) <= max(1e-4, 2 * math.sqrt(k) * cond * 2.0 ** -24)
    err_r = orc.rel_error(Ah, Jg, Z2h)
    assert err_r <= 1.05 * orc.rel_error(Ah, Jo, Zr), (err_r, orc.rel_error(Ah, Jo, Zr))


def test_randomized_full_size(gbid):
    """16384 x 32768 FP32, s_i = (1+i)^-1.5, k = 512, Omega 522 x 16384 BF16.

    Every one of the 512 CPQR steps is replayed by the oracle on the GPU's own
    sketch Y, with Z against the oracle's Z for the GPU's pivots (one forced-pivot
    pass, in a worker process); the refined Z against the oracle's least-squares
    Z for the GPU's skeleton on all of A (in this process, meanwhile)."""
    from oracle_jobs import cores, forced_id, oracle_pool

    m, n, k, l = 16384, 32768, 512, 522
    A = synth.lowrank(m, n, synth.spectrum("poly1.5", m), 3, device="cuda", dtype=torch.float32,
                      gen_dtype=torch.float32)
    omega = synth.gaussian_sketch_bf16(l, m, seed=33, device="cuda")
    J, Z, info = gbid.id_decompose_randomized(A, omega, k, refine=False)
    assert info["status"] == gbid.ID_OK, info
    Jg = J.cpu().numpy().astype(np.int64)
    assert len(set(Jg.tolist())) == k
    Y, _ = gbid.id_sketch(A, omega)
    Yh = Y.double().cpu().numpy()
    Jr, Zr, info_r = gbid.id_decompose_randomized(A, omega, k)
    assert info_r["status"] == gbid.ID_OK and info_r["refined"] and torch.equal(Jr, J)
    Zg = Z.double().cpu().numpy()
    Zrh = Zr.double().cpu().numpy()
    with oracle_pool(1, max(1, cores() // 2)) as ex:
        fut = ex.submit(forced_id, Yh, k, Jg)
        Ah = A.double().cpu().numpy()
        Zls = orc.ls_interp(Ah, Jg)
        cond_c = np.linalg.cond(Ah[:, Jg])
        o = fut.result()
    # every step of the sketch's CPQR: the greedy rule within the FP32 margin
    assert o["rank"] == k
    assert np.all(o["short"] <= _tol(l)), (int(np.argmax(o["short"])), float(o["short"].max()))
    # Z against the oracle's T for the GPU's pivots on the GPU's sketch. An FP32
    # factorisation perturbs R by O(u_32) relative, which T = R11^{-1} R12
    # amplifies by cond(R11) = cond(Y_J) (about 1e4 here): the bar is
    # max(1e-4, 2 cond(Y_J) u_32).
    assert np.linalg.norm(Zg - o["Z"]) / np.linalg.norm(o["Z"]) <= max(1e-4, 2 * o["cond"] * 2.0 ** -24), o["cond"]
    # reconstruction error on A, between the Eckart-Young floor and a small multiple
    err = orc.rel_error(Ah, Jg, Zg)
    tail = synth.tail_bound(synth.spectrum("poly1.5", m), k)
    assert tail * (1 - 1e-6) <= err <= 10 * tail, (err, tail)
    # one refinement lands on the oracle's least-squares Z for J (the bar of the
    # small cases: max(1e-4, 2 sqrt(k) cond(C) u_32)) and on its error
    rel_ls = np.linalg.norm(Zrh - Zls) / np.linalg.norm(Zls)
    assert rel_ls <= max(1e-4, 2 * math.sqrt(k) * cond_c * 2.0 ** -24), (rel_ls, cond_c)
    err_ls = orc.rel_error(Ah, Jg, Zls)
    err_r = orc.rel_error(Ah, Jg, Zrh)
    assert err_r <= 1.01 * err_ls, (err_r, err_ls, err)
    assert err_r < err
