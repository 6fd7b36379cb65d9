"""id_rid_pipe: randomized IDs of host matrices with overlapped copies.

Each pipelined ID must be exactly id_decompose_randomized on the same inputs
(J, Z and status bit for bit): the pipe only moves data and orders streams.
Five submits cycle both device slots more than once, so the waits that guard a
slot's reuse (its inputs, its outputs) are exercised; the inputs differ per ID,
so a slot read before its copy landed, or outputs copied before the compute
finished, would not match.
"""
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


def _inputs(m, n, l, seed):
    A = synth.lowrank(m, n, synth.spectrum("poly1.5", m), seed, dtype=torch.float32)
    om = synth.gaussian_sketch_bf16(l, m, seed=seed + 100)
    return A.contiguous().pin_memory(), om.contiguous().pin_memory()


@pytest.mark.parametrize("refine", [True, False])
def test_pipeline_equals_single_calls(gbid, refine):
    m, n, l, k = 256, 1024, 74, 64
    ins = [_inputs(m, n, l, s) for s in range(5)]
    pipe = gbid.RandomizedPipeline(m, n, l, k, refine=refine)
    outs = []
    for A, om in ins:
        J = torch.empty(k, dtype=torch.int32, pin_memory=True)
        Z = torch.empty(k, n, dtype=torch.float32, pin_memory=True)
        pipe.submit(A, om, J, Z)
        outs.append((J, Z))
    infos = pipe.synchronize()
    pipe.close()
    assert len(infos) == 5
    for (A, om), (J, Z), info in zip(ins, outs, infos):
        Ad = A.cuda()
        big = torch.zeros(l, (m + 7) // 8 * 8, dtype=torch.bfloat16, device="cuda")   # 16-byte rows
        big[:, :m] = om.cuda()
        Jr, Zr, ir = gbid.id_decompose_randomized(Ad, big[:, :m], k, refine=refine)
        assert torch.equal(J, Jr.cpu())
        assert torch.equal(Z, Zr.cpu())
        assert info["status"] == ir["status"] == gbid.ID_OK
        assert info["refined"] == ir["refined"] == refine
        assert info["n_gt2"] == ir["n_gt2"] and info["max_abs_z"] == ir["max_abs_z"]


def test_pipeline_with_padded_host_rows(gbid):
    """Host rows with padding (lda > n, ldo > m, ldz > n): the copies take the pitches."""
    m, n, l, k = 200, 600, 40, 32
    A, om = _inputs(m, n, l, 7)
    Ap = torch.zeros(m, n + 5, dtype=torch.float32).pin_memory()
    Ap[:, :n] = A
    Op = torch.zeros(l, m + 3, dtype=torch.bfloat16).pin_memory()
    Op[:, :m] = om
    Zp = torch.full((k, n + 9), -7.0, dtype=torch.float32).pin_memory()
    J = torch.empty(k, dtype=torch.int32, pin_memory=True)
    pipe = gbid.RandomizedPipeline(m, n, l, k)
    pipe.submit(Ap[:, :n], Op[:, :m], J, Zp[:, :n])
    (info,) = pipe.synchronize()
    pipe.close()
    big = torch.zeros(l, (m + 7) // 8 * 8, dtype=torch.bfloat16, device="cuda")
    big[:, :m] = om.cuda()
    Jr, Zr, _ = gbid.id_decompose_randomized(A.cuda(), big[:, :m], k)
    assert info["status"] == gbid.ID_OK
    assert torch.equal(J, Jr.cpu()) and torch.equal(Zp[:, :n], Zr.cpu())
    assert torch.all(Zp[:, n:] == -7.0)   # the padding of Z's rows is not written
