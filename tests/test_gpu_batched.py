"""Batched ID (one persistent launch over many uneven matrices) vs the FP64 oracle.

Each problem is checked as the single-matrix ID is: the GPU's pivots must pass
the oracle's greedy replay (FP64: margin 1e-6; FP32: 64 u_32 sqrt(m), the
FP32 rounding level of a residual norm) up to the numerical rank, Z must match
the oracle's Z for the GPU's pivots (FP64 1e-10; FP32 max(1e-4, 2 cond(X_J)
u_32)), and Z[:, J] = I exactly.
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


def _check_problem(A, k, J, Z, info, dtype, check_pivots=True):
    Ah = A.double().cpu().numpy()
    m, n = Ah.shape
    trans = m > n
    X = Ah.T if trans else Ah
    Jg = J.cpu().numpy().astype(np.int64)
    Zg = Z.double().cpu().numpy()
    assert info["transposed"] == trans
    Jo, Zo_free, io = orc.interp_decomp(Ah, k)
    rank = io["rank"]
    if dtype == torch.float64:
        assert info["rank"] == rank, (info, rank)
    r = min(rank, info["rank"])
    assert len(set(Jg.tolist())) == k
    assert np.array_equal(Zg[np.arange(k), Jg], np.ones(k))
    assert np.count_nonzero(Zg[:, Jg]) == k
    if check_pivots and r > 0:
        tol = 1e-6 if dtype == torch.float64 else 64 * U32 * math.sqrt(X.shape[0])
        ok, worst = orc.verify_pivots(X, Jg[:r], tol)
        assert ok, (worst.max(), np.argmax(worst))
    if rank == k and info["status"] == 0:
        Zo = orc.interp_decomp(Ah, k, pivots=Jg)[1]
        cond = np.linalg.cond(X[:, Jg])
        bar = 1e-10 if dtype == torch.float64 else max(1e-4, 2 * cond * U32)
        assert np.linalg.norm(Zg - Zo) / np.linalg.norm(Zo) <= bar, cond
        assert info["max_abs_z"] == pytest.approx(np.abs(Zg).max(), rel=1e-12)
        assert info["n_gt2"] == int(np.count_nonzero(np.abs(Zg) > 2.0))


def _mixed_batch(dtype, count, seed):
    probs = synth.batched_uneven(count, seed, m_range=(8, 96), k_range=(1, 40), dtype=dtype)
    mats = [p["A"].cuda() for p in probs]
    ks = [p["k"] for p in probs]
    # the m > n route and a ragged leading dimension
    g = torch.Generator().manual_seed(seed)
    T = synth.lowrank(90, 40, synth.spectrum("exp8m", 40, m=40), seed + 1).to(dtype)
    mats.append(T.cuda())
    ks.append(12)
    big = torch.randn(50, 77, generator=g, dtype=torch.float64).to(dtype)
    mats.append(big.cuda()[:, :70])
    ks.append(20)
    return mats, ks


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batched_mixed_shapes(gbid, dtype):
    mats, ks = _mixed_batch(dtype, 40, 4)
    Js, Zs, infos, plan = gbid.id_decompose_batched(mats, ks)
    for A, k, J, Z, info in zip(mats, ks, Js, Zs, infos):
        assert info["status"] in (gbid.ID_OK, gbid.ID_RANK_DEFICIENT), info
        _check_problem(A, k, J, Z, info, dtype)


def test_batched_matches_single_id(gbid):
    """FP64: the batched kernel and id_decompose agree on pivots; Z to 1e-12."""
    mats, ks = _mixed_batch(torch.float64, 16, 9)
    Js, Zs, infos, _ = gbid.id_decompose_batched(mats, ks)
    for A, k, J, Z, info in zip(mats, ks, Js, Zs, infos):
        if info["status"] != gbid.ID_OK:
            continue
        J1, Z1, i1 = gbid.id_decompose(A.contiguous(), k)
        assert torch.equal(J.cpu(), J1.cpu())
        assert (torch.linalg.norm(Z - Z1) / torch.linalg.norm(Z1)).item() < 1e-12


def test_batched_bad_descriptor_is_isolated(gbid):
    """A problem whose k breaks the rules gets ID_EINVAL; the rest still run."""
    mats, ks = _mixed_batch(torch.float32, 6, 11)
    plan = gbid.BatchedPlan(mats, ks)
    # corrupt one descriptor on the device: k = min(m, n) + 1
    import ctypes

    victim = plan.order.index(2)
    off = victim * ctypes.sizeof(gbid.IdProblem) + gbid.IdProblem.k.offset
    A = mats[2]
    bad = torch.tensor([min(A.shape) + 1], dtype=torch.int64).view(torch.uint8).cuda()
    plan.desc[off:off + 8] = bad
    plan.run()
    infos = plan.read_infos()
    assert infos[2]["status"] == gbid.ID_EINVAL
    for i, info in enumerate(infos):
        if i != 2:
            assert info["status"] in (gbid.ID_OK, gbid.ID_RANK_DEFICIENT)
            _check_problem(mats[i], ks[i], plan.J[i], plan.Z[i], info, torch.float32, check_pivots=False)


def test_batched_graph_capture_replay(gbid):
    mats, ks = _mixed_batch(torch.float32, 24, 13)
    plan = gbid.BatchedPlan(mats, ks)
    plan.run()
    torch.cuda.synchronize()
    ref = [z.clone() for z in plan.Z]
    for z in plan.Z:
        z.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, plan.Z):
        assert torch.equal(a, b)


def test_batched_nonfinite_and_zero_matrix(gbid):
    A = torch.randn(20, 30, dtype=torch.float64)
    A[3, 7] = float("nan")
    Zm = torch.zeros(16, 24, dtype=torch.float64)
    Js, Zs, infos, _ = gbid.id_decompose_batched([A.cuda(), Zm.cuda()], [5, 4])
    assert infos[0]["status"] == gbid.ID_ENONFINITE
    assert infos[1]["status"] == gbid.ID_RANK_DEFICIENT and infos[1]["rank"] == 0
    # all-zero columns tie at norm 0: the smallest original indices win
    assert Js[1].cpu().tolist() == [0, 1, 2, 3]


def test_batched_full_workload_4096(gbid):
    """4096 FP32 problems, m ~ U[32, 256], n ~ U[m, 4m], k ~ U[8, 64], 10% sparse,
    every problem checked against the oracle (a forced-pivot oracle ID each, in
    a pool of worker processes): status, identity block, the greedy replay up
    to the numerical rank, Z against the oracle's Z for the GPU's pivots, the Z
    statistics, and the reconstruction error of every low-rank problem above
    its Eckart-Young floor."""
    from oracle_jobs import cores, forced_id, oracle_pool

    probs = synth.batched_uneven(4096, 4, dtype=torch.float32, device="cuda")
    mats = [p["A"] for p in probs]
    ks = [p["k"] for p in probs]
    Js, Zs, infos, plan = gbid.id_decompose_batched(mats, ks)
    host = []
    for i, (p, J, Z, info) in enumerate(zip(probs, Js, Zs, infos)):
        assert info["status"] in (gbid.ID_OK, gbid.ID_RANK_DEFICIENT), (i, info)
        k = p["k"]
        assert torch.equal(Z[torch.arange(k, device=Z.device), J.long()], torch.ones(k, device=Z.device))
        if p["kind"] == "lowrank":
            A64 = p["A"].double().cuda()
            err = (torch.linalg.norm(A64 - A64[:, J.long()] @ Z.double()) / torch.linalg.norm(A64)).item()
            s = synth.spectrum("exp8m", min(p["m"], p["n"]), m=p["m"])
            # the floor of the FP64 matrix, less the FP32 rounding of the input
            assert err >= synth.tail_bound(s, k) * (1 - 1e-4) - 1e-6, (i, err)
        host.append((p["A"].double().cpu().numpy(), k, J.cpu().numpy().astype(np.int64), Z.double().cpu().numpy()))
    with oracle_pool(cores(), 1) as ex:
        res = list(ex.map(forced_id, [h[0] for h in host], [h[1] for h in host], [h[2] for h in host], chunksize=32))
    n_z = 0
    for i, ((Ah, k, Jg, Zg), o, info) in enumerate(zip(host, res, infos)):
        m, n = Ah.shape
        assert info["transposed"] == (m > n)
        assert len(set(Jg.tolist())) == k
        assert np.count_nonzero(Zg[:, Jg]) == k
        r = min(o["rank"], info["rank"])
        tol = 64 * U32 * math.sqrt(min(m, n))
        assert np.all(o["short"][:r] <= tol), (i, float(o["short"][:r].max()))
        if o["rank"] == k and info["status"] == gbid.ID_OK:
            bar = max(1e-4, 2 * o["cond"] * U32)
            assert np.linalg.norm(Zg - o["Z"]) / np.linalg.norm(o["Z"]) <= bar, (i, o["cond"])
            assert info["max_abs_z"] == pytest.approx(np.abs(Zg).max(), rel=1e-12)
            assert info["n_gt2"] == int(np.count_nonzero(np.abs(Zg) > 2.0))
            n_z += 1
    assert n_z >= 4000, n_z   # the rank-deficient (sparse) problems are the only ones without a Z check


def _path_batch(dtype, seed):
    """Shapes whose column segments take every path of every kernel instance
    (a segment of up to 32 R rows in registers, up to 64 R with half the
    columns, longer in two passes, for R = 4 and 8), both routes (m > n takes
    the transpose), k up to the maximum, and an all-zero matrix."""
    shapes = [(20, 50, 7), (100, 260, 30), (130, 131, 64), (200, 700, 40), (256, 300, 64), (300, 620, 33),
              (520, 600, 64), (700, 900, 50), (1024, 1100, 16), (900, 300, 25), (640, 129, 64), (33, 1000, 8)]
    mats, ks = [], []
    for i, (m, n, k) in enumerate(shapes):
        d = min(m, n)
        A = synth.lowrank(m, n, synth.spectrum("exp8m", d, m=d), seed + i).to(dtype)
        mats.append(A.cuda())
        ks.append(k)
    mats.append(torch.zeros(40, 90, dtype=dtype, device="cuda"))
    ks.append(10)
    return mats, ks


def _same(a, b):
    """Equal values, NaN where the other has NaN (Z past the numerical rank of a
    rank-deficient problem is 0/0)."""
    return torch.equal(a.isnan(), b.isnan()) and torch.equal(a.nan_to_num(0.0), b.nan_to_num(0.0))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_every_instance_gives_identical_results(gbid, dtype):
    """The kernel's instances (tile shapes the tuner picks from) perform the
    same operations in the same order: J, Z and id_info agree exactly with the
    default instance, which itself passes the oracle checks."""
    mats, ks = _path_batch(dtype, 21)
    cfgs = gbid.batched_configs(dtype)
    assert len(cfgs) >= 2
    base = gbid.BatchedPlan(mats, ks, config=0)
    base.run()
    infos0 = base.read_infos()
    for A, k, J, Z, info in zip(mats, ks, base.J, base.Z, infos0):
        assert info["status"] in (gbid.ID_OK, gbid.ID_RANK_DEFICIENT), info
        if torch.count_nonzero(A).item():
            _check_problem(A, k, J, Z, info, dtype)
    assert infos0[-1]["status"] == gbid.ID_RANK_DEFICIENT and infos0[-1]["rank"] == 0
    for c in range(1, len(cfgs)):
        plan = gbid.BatchedPlan(mats, ks, config=c)
        plan.run()
        infos = plan.read_infos()
        for i in range(len(mats)):
            assert torch.equal(plan.J[i], base.J[i]), (cfgs[c], i)
            assert _same(plan.Z[i], base.Z[i]), (cfgs[c], i)
            assert infos[i] == infos0[i], (cfgs[c], i)


def test_autotune_picks_the_fastest_instance(gbid):
    """id_batched_autotune times every instance on the batch, returns the
    fastest and leaves the batch's results; a later plan over the same shapes
    reuses the choice."""
    mats, ks = _mixed_batch(torch.float32, 64, 17)
    ref = gbid.BatchedPlan(mats, ks, config=0)
    ref.run()
    plan = gbid.BatchedPlan(mats, ks, autotune=True, tune_reps=2)
    ms = plan.tune_ms
    assert len(ms) == len(gbid.batched_configs(torch.float32)) and min(ms) > 0
    assert plan.config == int(np.argmin(ms))
    torch.cuda.synchronize()
    for i in range(len(mats)):
        assert torch.equal(plan.J[i], ref.J[i]) and _same(plan.Z[i], ref.Z[i])
    again = gbid.BatchedPlan(mats, ks, autotune=True)
    assert again.config == plan.config and again.tune_ms is plan.tune_ms
    again.run()
    torch.cuda.synchronize()
    for i in range(len(mats)):
        assert _same(again.Z[i], ref.Z[i])
