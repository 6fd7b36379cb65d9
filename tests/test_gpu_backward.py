"""id_backward (gradient through the ID with the skeleton frozen) vs the oracle.

The oracle's ``id_grad`` (pinned by central differences on the CPU) is the
reference. The gradient contains (C^T C)^{-1}, so it carries cond(C)^2: the GPU
forms W in FP64 and the products with C, A - C Z and Z in FP32, and the bar is
max(1e-4, 8 sqrt(n) cond(C) u_32) relative (Frobenius).
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


@pytest.mark.parametrize("m,n,k,spec", [(120, 300, 16, "poly2"), (512, 1024, 64, "poly2"), (64, 64, 10, "exp64"),
                                        (96, 5000, 24, "poly1.5")])
def test_backward_matches_oracle(gbid, m, n, k, spec):
    A = synth.lowrank(m, n, synth.spectrum(spec, m), 5, dtype=torch.float32).cuda()
    J, Z, info = gbid.id_decompose(A, k)
    assert info["status"] == gbid.ID_OK
    g = torch.Generator(device="cuda").manual_seed(m + n + k)
    dZ = torch.randn(k, n, generator=g, device="cuda")
    dA, binfo = gbid.id_backward(A, J, Z, dZ)
    assert binfo["status"] == gbid.ID_OK
    Ah = A.double().cpu().numpy()
    Jg = J.cpu().numpy().astype(np.int64)
    rest = np.setdiff1d(np.arange(n), Jg)
    perm = np.concatenate([Jg, rest])
    ref = orc.id_grad(Ah, Jg, perm, dZ.double().cpu().numpy())
    cond = np.linalg.cond(Ah[:, Jg])
    bar = max(1e-4, 8 * math.sqrt(n) * cond * U32)
    err = np.linalg.norm(dA.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= bar, (err, bar, cond)


def test_backward_ignores_dz_on_the_skeleton(gbid):
    A = synth.lowrank(100, 250, synth.spectrum("poly2", 100), 6, dtype=torch.float32).cuda()
    k = 12
    J, Z, _ = gbid.id_decompose(A, k)
    dZ = torch.randn(k, 250, device="cuda")
    dA1, _ = gbid.id_backward(A, J, Z, dZ)
    dZ2 = dZ.clone()
    dZ2[:, J.long()] = 1e3
    dA2, _ = gbid.id_backward(A, J, Z, dZ2)
    assert torch.equal(dA1, dA2)


def test_autograd_function(gbid):
    """torch.autograd through IdFunction agrees with id_backward for L = <G, Z>."""
    A = synth.lowrank(80, 200, synth.spectrum("poly2", 80), 8, dtype=torch.float32).cuda().requires_grad_(True)
    k = 10
    J, Z = gbid.IdFunction.apply(A, k)
    G = torch.randn_like(Z)
    (G * Z).sum().backward()
    dA, _ = gbid.id_backward(A.detach(), J, Z.detach(), G)
    assert torch.equal(A.grad, dA)


def test_backward_rank_deficient(gbid):
    A = torch.randn(60, 150, device="cuda")
    A[:, 5] = A[:, 2]
    J = torch.tensor([2, 5, 9], dtype=torch.int32, device="cuda")
    Z = torch.zeros(3, 150, device="cuda")
    dA, info = gbid.id_backward(A, J, Z, torch.randn(3, 150, device="cuda"))
    assert info["status"] == gbid.ID_RANK_DEFICIENT


def test_backward_plan_matches_single_calls(gbid):
    """Many problems over several streams (each with its own workspace), also
    replayed from a CUDA graph: the same gradients as one call at a time."""
    m, n, k, nb = 128, 300, 16, 12
    mats = [synth.lowrank(m, n, synth.spectrum("poly2", m), 300 + b, dtype=torch.float32).cuda() for b in range(nb)]
    g = torch.Generator(device="cuda").manual_seed(2)
    outs = [gbid.id_decompose(A, k) for A in mats]
    Gs = [torch.randn(k, n, generator=g, device="cuda") for _ in range(nb)]
    ref = [gbid.id_backward(A, J, Z, G)[0] for A, (J, Z, _), G in zip(mats, outs, Gs)]
    plan = gbid.BackwardPlan(m, n, k, streams=4)
    dAs = [torch.empty(m, n, device="cuda") for _ in range(nb)]
    Js = [o[0] for o in outs]
    Zs = [o[1] for o in outs]
    plan.run(mats, Js, Zs, Gs, dAs)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(dAs, ref))
    for d in dAs:
        d.zero_()
    graph = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cs):
        with torch.cuda.graph(graph, stream=cs):
            plan.run(mats, Js, Zs, Gs, dAs)
    torch.cuda.current_stream().wait_stream(cs)
    graph.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(dAs, ref))


def test_backward_matches_central_differences_512x1024(gbid):
    """The differentiable workload's shape (512 x 1024, s_i = (1+i)^-2, k = 64,
    L = <G, Z> with G ~ N(0,1)): the GPU gradient against FP64 central
    differences with step 1e-6 of L(A) = <G, Z(A)>, Z(A) the oracle's
    least-squares Z for the frozen skeleton (Sec. 2.1), on 64 sampled entries,
    half of them in skeleton columns. The bar is the Frobenius test's,
    max(1e-4, 8 sqrt(n) cond(C) u_32), relative to the sample's largest entry;
    the differences' own error (h^2 truncation and eps/h rounding) is far below it."""
    m, n, k = 512, 1024, 64
    A = synth.lowrank(m, n, synth.spectrum("poly2", m), 5, dtype=torch.float32).cuda()
    J, Z, info = gbid.id_decompose(A, k)
    assert info["status"] == gbid.ID_OK
    g = torch.Generator(device="cuda").manual_seed(5)
    G = torch.randn(k, n, generator=g, device="cuda")
    dA, binfo = gbid.id_backward(A, J, Z, G)
    assert binfo["status"] == gbid.ID_OK
    Ah = A.double().cpu().numpy()
    Jg = J.cpu().numpy().astype(np.int64)
    Gh = G.double().cpu().numpy()
    rest = np.setdiff1d(np.arange(n), Jg)
    rng = np.random.default_rng(11)
    cols = np.concatenate([rng.choice(Jg, 32), rng.choice(rest, 32)])
    rows = rng.integers(0, m, 64)
    h = 1e-6

    def loss(X):
        return float(np.sum(Gh * orc.ls_interp(X, Jg)))

    fd = np.empty(64)
    for s, (i, j) in enumerate(zip(rows, cols)):
        Xp = Ah.copy()
        Xp[i, j] += h
        Xm = Ah.copy()
        Xm[i, j] -= h
        fd[s] = (loss(Xp) - loss(Xm)) / (2 * h)
    got = dA.double().cpu().numpy()[rows, cols]
    cond = np.linalg.cond(Ah[:, Jg])
    bar = max(1e-4, 8 * math.sqrt(n) * cond * U32)
    assert np.max(np.abs(got - fd)) <= bar * np.max(np.abs(fd)), (np.max(np.abs(got - fd)) / np.max(np.abs(fd)), bar)
