"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or the mathematics fixes:
closed forms, brute force on tiny inputs, an independent library routine, the
paper's printed statistics, or invariances. A plausible bug in the oracle (a
dropped term, a wrong sign or index, a transposed operand, a wrong tie rule)
fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import id_oracle as orc
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lowrank_np(m, n, s, seed):
    return synth.lowrank(m, n, s, seed).numpy()


# ---------------------------------------------------------------- reflector ---
@pytest.mark.parametrize("x", [
    np.array([3.0, 4.0]),
    np.array([-3.0, 4.0, 12.0]),
    np.array([0.0, 1.0, -2.0]),
    np.array([5.0]),
    np.array([-2.0, 0.0, 0.0]),
])
def test_householder_maps_to_beta_e0(x):
    v, tau, beta = orc.householder(x)
    H = np.eye(len(x)) - tau * np.outer(v, v)
    # orthogonal and maps x to beta e_0 with |beta| = ||x|| and sign opposite to x_0
    assert np.allclose(H @ H.T, np.eye(len(x)), atol=1e-15)
    e0 = np.zeros(len(x)); e0[0] = 1.0
    assert np.allclose(H @ x, beta * e0, atol=1e-14)
    assert abs(abs(beta) - np.linalg.norm(x)) < 1e-14
    assert beta <= 0.0 if x[0] >= 0.0 else beta > 0.0
    assert v[0] == 1.0


def test_householder_zero_vector_is_identity():
    v, tau, beta = orc.householder(np.zeros(4))
    assert tau == 0.0 and beta == 0.0


# -------------------------------------------------------- brute-force greedy ---
def _greedy_by_projection(A, k):
    """Greedy max-residual column selection, by a different route than the oracle:

    residuals are (I - P_S) a_l with P_S built by modified Gram-Schmidt applied
    twice, in extended precision. Ties go to the smallest index (strict '>').
    Also returns the relative gap between the best and second-best residual.
    """
    A = np.asarray(A, dtype=np.longdouble)
    m, n = A.shape
    chosen, basis, gaps = [], [], []

    def resid(col):
        r = A[:, col].copy()
        for _ in range(2):
            for q in basis:
                r = r - (q @ r) * q
        return r

    for _ in range(k):
        norms = [(float(np.sqrt(resid(l) @ resid(l))), l) for l in range(n) if l not in chosen]
        best = norms[0]
        for nrm, l in norms[1:]:
            if nrm > best[0]:
                best = (nrm, l)
        others = sorted((nv for nv, l in norms if l != best[1]), reverse=True)
        gaps.append((best[0] - others[0]) / best[0] if others else 1.0)
        chosen.append(best[1])
        r = resid(best[1])
        basis.append(r / np.sqrt(r @ r))
    return chosen, gaps


@pytest.mark.parametrize("seed", range(12))
def test_pivots_equal_bruteforce_greedy_small(seed):
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(3, 9))
    n = int(rng.integers(m, 13))
    A = rng.standard_normal((m, n)) * rng.uniform(0.2, 3.0, size=n)
    k = int(rng.integers(1, m + 1))
    ref, gaps = _greedy_by_projection(A, k)
    if min(gaps) < 1e-9:
        pytest.skip("near-tie in this draw")
    J, Z, info = orc.interp_decomp(A, k)
    assert list(J) == ref
    # the winning residual norms are |R_jj|
    assert np.allclose(info["nu"], np.abs(np.diag(info["R"][:, :k])), rtol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_error_not_below_best_subset(seed):
    """Any k-column ID is at least as bad as the best k-subset projection (n <= 10)."""
    rng = np.random.default_rng(200 + seed)
    m, n, k = 5, 9, 3
    A = rng.standard_normal((m, n))
    J, Z, info = orc.interp_decomp(A, k)
    err = orc.rel_error(A, J, Z)
    best = min(
        np.linalg.norm(A - A[:, list(S)] @ np.linalg.lstsq(A[:, list(S)], A, rcond=None)[0])
        for S in itertools.combinations(range(n), k)
    ) / np.linalg.norm(A)
    assert err >= best - 1e-12


def test_tie_goes_to_smallest_original_index():
    # columns 2 and 5 have equal norms and are orthogonal to everything else
    A = np.zeros((4, 6))
    A[0, 2] = 3.0
    A[1, 5] = -3.0
    A[2, 0] = 1.0
    A[3, 1] = 0.5
    A[2, 3] = 0.25
    A[3, 4] = 0.125
    J, Z, info = orc.interp_decomp(A, 2)
    assert list(J) == [2, 5]
    # reversed column order: the same two columns, again smallest index first
    Jr, _, _ = orc.interp_decomp(A[:, ::-1], 2)
    assert list(Jr) == [0, 3]


# --------------------------------------------------------------- closed forms ---
def test_tail_bound_closed_form_pow2():
    s = synth.spectrum("pow2_half", 200)
    # sum_{i>=20} 2^-i / sum_{i>=0} 2^-i = 2^-20 (1 - 2^-180) / (1 - 2^-200)
    assert synth.tail_bound(s, 20) == pytest.approx(2.0 ** -10, rel=1e-12)


def test_tail_bounds_of_the_workloads():
    assert synth.tail_bound(synth.spectrum("exp64", 4096), 256) == pytest.approx(
        math.exp(-4.0) * math.sqrt((1 - math.exp(-2 * 3840 / 64)) / (1 - math.exp(-2 * 4096 / 64))), rel=1e-12)
    assert synth.tail_bound(synth.spectrum("exp64", 4096, rank=256), 256) == 0.0


def test_error_above_eckart_young_and_near_it():
    s = synth.spectrum("pow2_half", 200)
    A = _lowrank_np(200, 400, s, 1)
    J, Z, info = orc.interp_decomp(A, 20)
    err = orc.rel_error(A, J, Z)
    tail = synth.tail_bound(s, 20)
    assert err >= tail * (1 - 1e-9)
    assert err <= 10.0 * tail
    assert np.all(np.abs(Z[:, J] - np.eye(20)) == 0.0)


def test_exact_rank_reconstruction():
    s = synth.spectrum("exp64", 240, rank=40)
    A = _lowrank_np(240, 480, s, 7)
    J, Z, info = orc.interp_decomp(A, 40)
    assert orc.rel_error(A, J, Z) <= 1e-12


def test_full_rank_k_equals_m_is_exact():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 50))
    J, Z, info = orc.interp_decomp(A, 30)
    assert orc.rel_error(A, J, Z) <= 1e-13


def test_identity_columns_exact():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((40, 90))
    J, Z, _ = orc.interp_decomp(A, 17)
    assert np.array_equal(Z[:, J], np.eye(17))


def test_numerical_rank_detected():
    s = synth.spectrum("exp64", 60, rank=9)
    A = _lowrank_np(60, 100, s, 8)
    _, _, info = orc.interp_decomp(A, 15)
    assert info["rank"] == 9


# ------------------------------------------------------------ library check ---
@pytest.mark.parametrize("shape,k,seed", [((60, 120), 25, 0), ((200, 400), 20, 1), ((64, 64), 64, 2)])
def test_pivots_match_lapack_geqp3(shape, k, seed):
    rng = np.random.default_rng(300 + seed)
    A = rng.standard_normal(shape) * np.exp(-np.arange(shape[1]) / 50.0)[rng.permutation(shape[1])]
    J, Z, info = orc.interp_decomp(A, k)
    _, R, P = scipy.linalg.qr(A, pivoting=True, mode="economic")
    gap_ok = info["gap"] > 1e-6
    # LAPACK downdates norms, so compare only up to the first near-tie
    first_tie = int(np.argmin(gap_ok)) if not gap_ok.all() else k
    assert list(P[:first_tie]) == list(J[:first_tie])
    assert np.allclose(np.abs(np.diag(R))[:first_tie], info["nu"][:first_tie], rtol=1e-10)


# --------------------------------------------------- equivalent formulations ---
def test_back_substitution_equals_normal_equations_and_lstsq():
    s = synth.spectrum("pow2_half", 200)
    A = _lowrank_np(200, 400, s, 1)
    k = 20
    J, Z, info = orc.interp_decomp(A, k)
    R11 = info["R"][:, :k]
    Zn = orc.normal_equation_z(A, J, R11)
    Zl = orc.ls_interp(A, J)
    cond = np.linalg.cond(R11)
    scale = np.linalg.norm(Z)
    assert np.linalg.norm(Zn - Z) / scale <= 50 * cond ** 2 * orc.EPS64
    assert np.linalg.norm(Zl - Z) / scale <= 50 * cond * orc.EPS64 * 1e3


def test_tall_matrix_takes_the_transpose_route():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((90, 40)) @ np.diag(np.exp(-np.arange(40) / 5.0))
    A = A @ rng.standard_normal((40, 40))
    J, Z, info = orc.interp_decomp(A, 12)
    assert info["transposed"] and Z.shape == (12, 90)
    Jt, Zt, _ = orc.interp_decomp(A.T.copy(), 12)
    assert np.array_equal(J, Jt) and np.allclose(Z, Zt, rtol=0, atol=1e-13)
    # row ID: A ~= Z^T A[J, :]
    err = np.linalg.norm(A - Z.T @ A[J, :]) / np.linalg.norm(A)
    assert err == pytest.approx(orc.rel_error(A, J, Z, transposed=True), rel=1e-12)


# --------------------------------------------------------------- invariances ---
def test_left_orthogonal_transform_keeps_J_and_Z():
    s = synth.spectrum("pow2_half", 80)
    A = _lowrank_np(80, 160, s, 11)
    Q = synth.haar(80, 80, 99).numpy()
    k = 12
    J, Z, info = orc.interp_decomp(A, k)
    J2, Z2, _ = orc.interp_decomp(Q @ A, k)
    assert np.all(info["gap"] > 1e-8)
    assert np.array_equal(J, J2)
    assert np.linalg.norm(Z - Z2) / np.linalg.norm(Z) < 1e-10


def test_power_of_two_scaling_is_exact():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((50, 70))
    J, Z, _ = orc.interp_decomp(A, 9)
    J2, Z2, _ = orc.interp_decomp(A * 2.0 ** -7, 9)
    assert np.array_equal(J, J2) and np.array_equal(Z, Z2)


def test_column_permutation_permutes_J():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((40, 60)) * np.linspace(1.0, 2.0, 60)
    pi = rng.permutation(60)
    J, Z, info = orc.interp_decomp(A, 10)
    J2, Z2, _ = orc.interp_decomp(A[:, pi], 10)
    assert np.all(info["gap"] > 1e-8)
    assert np.array_equal(pi[J2], J)
    assert np.allclose(Z2, Z[:, pi], atol=1e-12)


# ------------------------------------------------------------ verify_pivots ---
def test_verify_pivots_accepts_own_and_rejects_planted_swap():
    s = synth.spectrum("pow2_half", 100)
    A = _lowrank_np(100, 200, s, 12)
    J, Z, info = orc.interp_decomp(A, 15)
    ok, worst = orc.verify_pivots(A, J, 1e-12)
    assert ok and worst.max() <= 1e-12
    bad = J.copy()
    bad[[3, 4]] = bad[[4, 3]]
    ok2, worst2 = orc.verify_pivots(A, bad, 1e-6)
    assert not ok2 and worst2[3] > 1e-6


def test_forced_pivot_shortfall_equals_the_replay():
    """cpqr's largest residual norm per step: equal to the winner's on a free
    run, and with forced pivots 1 - nu / top is the replay's shortfall (the
    planted swap shows from the swapped step on; an independent replay computes it)."""
    s = synth.spectrum("pow2_half", 100)
    A = _lowrank_np(100, 200, s, 12)
    J, _, info = orc.interp_decomp(A, 15)
    assert np.array_equal(info["top"], info["nu"])
    bad = J.copy()
    bad[[3, 4]] = bad[[4, 3]]
    _, _, ib = orc.interp_decomp(A, 15, pivots=bad)
    _, worst = orc.verify_pivots(A, bad, 1e-6)
    assert np.allclose(1.0 - ib["nu"] / ib["top"], worst, rtol=0, atol=1e-13)
    assert worst[3] > 1e-6 and np.all(worst[:3] <= 1e-12)


def test_forced_pivots_reproduce_free_run():
    rng = np.random.default_rng(13)
    A = rng.standard_normal((30, 45))
    J, Z, info = orc.interp_decomp(A, 10)
    J2, Z2, info2 = orc.interp_decomp(A, 10, pivots=J)
    assert np.array_equal(J, J2) and np.array_equal(Z, Z2)


# ------------------------------------------------------------- randomized ID ---
def test_randomized_with_identity_sketch_is_deterministic_id():
    rng = np.random.default_rng(14)
    A = rng.standard_normal((25, 60)) * np.exp(-np.arange(60) / 20.0)
    J, Z, _ = orc.interp_decomp(A, 8)
    Jr, Zy, Zr, info = orc.randomized_interp_decomp(A, np.eye(25), 8)
    assert np.array_equal(J, Jr)
    assert np.allclose(Zy, Z, atol=1e-12)
    assert np.allclose(Zr, orc.ls_interp(A, Jr), atol=1e-10)


def test_refined_z_solves_the_least_squares_problem():
    s = synth.spectrum("poly1.5", 120)
    A = _lowrank_np(120, 300, s, 15)
    omega = synth.gaussian_sketch_bf16(30, 120, 16).double().numpy()
    J, Zy, Zr, info = orc.randomized_interp_decomp(A, omega, 20)
    Zl = orc.ls_interp(A, J)
    assert np.linalg.norm(Zr - Zl) / np.linalg.norm(Zl) < 1e-10
    # the refined Z is never worse than the sketch's Z on A
    assert orc.rel_error(A, J, Zr) <= orc.rel_error(A, J, Zy) + 1e-15


# ------------------------------------------------------ column-sampling RID ---
def test_sampled_rid_with_every_column_is_the_deterministic_id():
    """p = n (every column sampled, in any order): the same skeleton as the
    deterministic ID (up to ties) and the same Z (normal equations against back
    substitution, equal in exact arithmetic)."""
    A = synth.lowrank(60, 140, np.exp(-np.arange(60) / 8.0), 3).numpy()
    k = 12
    idx = np.random.default_rng(4).permutation(140)
    J, Z, info = orc.sampled_interp_decomp(A, idx, k)
    Jd, Zd, _ = orc.interp_decomp(A, k)
    assert np.array_equal(J, Jd)
    assert np.linalg.norm(Z - Zd) / np.linalg.norm(Zd) < 1e-9


def test_sampled_rid_properties():
    A = synth.lowrank(80, 300, synth.spectrum("poly2", 80), 5).numpy()
    k = 20
    p = k + int(0.2 * k)
    idx = np.random.default_rng(9).choice(300, size=p, replace=False)
    J, Z, info = orc.sampled_interp_decomp(A, idx, k)
    assert set(J.tolist()) <= set(idx.tolist()) and len(set(J.tolist())) == k
    # C Z reproduces C (Z[:, J] = I in exact arithmetic)
    assert np.allclose(Z[:, J], np.eye(k), atol=1e-8)
    # the normal-equation Z is the least-squares Z for that skeleton
    Zl = orc.ls_interp(A, J)
    assert np.linalg.norm(Z - Zl) / np.linalg.norm(Zl) < 1e-8
    # never below the Eckart-Young floor
    tail = synth.tail_bound(synth.spectrum("poly2", 80), k)
    assert orc.rel_error(A, J, Z) >= tail * (1 - 1e-9)
    # sampling without replacement is required
    with pytest.raises(ValueError):
        orc.sampled_interp_decomp(A, np.array([1, 1, 2]), 2)


# ------------------------------------------------------------- sparse input ---
def test_csr_to_dense_matches_the_library_routine():
    """The oracle's CSR densification against scipy.sparse (duplicates summed)."""
    sp = pytest.importorskip("scipy.sparse")
    rowptr, colind, vals = synth.sparse_powerlaw_csr(40, 90, 0.08, 3)
    # plant a duplicate entry in row 5 and an empty row 7
    A = orc.csr_to_dense(rowptr, colind, vals, 40, 90)
    B = sp.csr_matrix((vals, colind, rowptr), shape=(40, 90)).toarray()
    assert np.array_equal(A, B)
    r = np.array([0, 2, 2, 3], dtype=np.int64)
    c = np.array([4, 4, 1], dtype=np.int32)
    v = np.array([1.5, 2.0, -1.0])
    D = orc.csr_to_dense(r, c, v, 3, 6)
    assert D[0, 4] == 3.5 and D[2, 1] == -1.0 and np.count_nonzero(D) == 2
    assert np.array_equal(D, sp.csr_matrix((v, c, r), shape=(3, 6)).toarray())


def test_sparse_generator_shape():
    rowptr, colind, vals = synth.sparse_powerlaw_csr(300, 800, 0.02, 5)
    assert rowptr[0] == 0 and rowptr[-1] == colind.size == vals.size
    assert np.all(np.diff(rowptr) >= 0) and colind.min() >= 0 and colind.max() < 800
    assert 0.6 * 0.02 * 300 * 800 <= colind.size <= 0.02 * 300 * 800    # the heaviest columns are capped at m
    deg = np.bincount(colind, minlength=800)
    assert deg.max() > 10 * max(1, np.median(deg))          # heavy-tailed column degrees


# ---------------------------------------------------------------- two-sided ---
@pytest.mark.parametrize("m,n", [(60, 140), (140, 60), (80, 80)])
def test_two_sided_exact_rank(m, n):
    """Rank k exactly: X^T A[I, J] Z reproduces A."""
    k = 12
    s = np.where(np.arange(min(m, n)) < k, np.exp(-np.arange(min(m, n)) / 4.0), 0.0)
    A = synth.lowrank(m, n, s, 8).numpy()
    I, J, X, Z = orc.two_sided_interp_decomp(A, k)
    assert X.shape == (k, m) and Z.shape == (k, n)
    err = np.linalg.norm(A - orc.two_sided_reconstruct(A, I, J, X, Z)) / np.linalg.norm(A)
    assert err <= 1e-12


@pytest.mark.parametrize("m,n", [(60, 140), (140, 60)])
def test_two_sided_error_is_the_one_sided_error(m, n):
    """The second stage is exact in exact arithmetic, so the two-sided error
    equals the first stage's ID error; X[:, I] and Z[:, J] are identities."""
    k = 15
    A = synth.lowrank(m, n, np.exp(-np.arange(min(m, n)) / 6.0), 9).numpy()
    I, J, X, Z = orc.two_sided_interp_decomp(A, k)
    assert np.array_equal(X[:, I], np.eye(k)) and np.array_equal(Z[:, J], np.eye(k))
    e2 = np.linalg.norm(A - orc.two_sided_reconstruct(A, I, J, X, Z)) / np.linalg.norm(A)
    if m <= n:
        e1 = orc.rel_error(A, J, Z)
    else:
        e1 = orc.rel_error(A, I, X, transposed=True)
    assert abs(e2 - e1) <= 1e-10 * e1
    # never below the Eckart-Young floor
    assert e2 >= np.sqrt(np.sum(np.exp(-np.arange(k, min(m, n)) / 3.0)) / np.sum(np.exp(-np.arange(min(m, n)) / 3.0))) * (1 - 1e-9)


def test_two_sided_transpose_symmetry():
    """The two-sided ID of A^T is that of A with the roles of (I, X) and (J, Z) swapped."""
    k = 10
    A = synth.lowrank(50, 120, np.exp(-np.arange(50) / 5.0), 10).numpy()
    I, J, X, Z = orc.two_sided_interp_decomp(A, k)
    It, Jt, Xt, Zt = orc.two_sided_interp_decomp(A.T.copy(), k)
    assert np.array_equal(It, J) and np.array_equal(Jt, I)
    assert np.allclose(Xt, Z, atol=1e-12) and np.allclose(Zt, X, atol=1e-12)


# ----------------------------------------------------------------- gradient ---
def test_gradient_matches_central_differences():
    rng = np.random.default_rng(17)
    m, n, k = 12, 20, 4
    A = rng.standard_normal((m, n)) * np.exp(-np.arange(n) / 6.0)
    G = rng.standard_normal((k, n))
    J, Z, info = orc.interp_decomp(A, k)
    perm = info["perm"]
    dA = orc.id_grad(A, J, perm, G)

    def loss(Ap):
        Zp = orc.ls_interp(Ap, J)           # J frozen
        return float(np.sum(G * Zp))

    h = 1e-6
    for (i, j) in [(0, 0), (3, int(J[1])), (5, int(perm[k + 2])), (11, int(perm[-1])), (7, int(J[-1]))]:
        Ap = A.copy(); Ap[i, j] += h
        Am = A.copy(); Am[i, j] -= h
        fd = (loss(Ap) - loss(Am)) / (2 * h)
        assert fd == pytest.approx(dA[i, j], rel=1e-5, abs=1e-7)


# ------------------------------------------------------ paper's statistics ---
def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "paper_tables_synthetic.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, m, n, k, e_id, e_svd, zmax, e_rid, zmax_rid = line.split()
            rows.append((name, int(m), int(n), int(k), float(e_id), float(e_svd), float(zmax), float(e_rid),
                         float(zmax_rid)))
    return rows


@pytest.mark.slow
@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_paper_table_statistics(row):
    name, m, n, k, e_id, e_svd, zmax, e_rid, zmax_rid = row
    A = synth.paper_dataset(name, seed=2021)
    J, Z, info = orc.interp_decomp(A, k)
    err = orc.rel_error(A, J, Z)
    assert err == pytest.approx(e_id, abs=0.005)
    assert info["max_abs_z"] <= zmax + 1e-9
    sv = np.linalg.svd(A, compute_uv=False)
    assert synth.tail_bound(sv, k) == pytest.approx(e_svd, abs=0.005)
    # the column-sampling Optim RID (Sec. 2.2) with the paper's oversampling p = k + floor(0.2 k)
    p = k + int(0.2 * k)
    idx = np.random.default_rng(2021).choice(n, size=p, replace=False)
    Jr, Zr = orc.sampled_interp_decomp(A, idx, k)[:2]
    assert orc.rel_error(A, np.asarray(Jr), Zr) == pytest.approx(e_rid, abs=0.005)
    assert np.abs(Zr).max() <= zmax_rid + 1e-9
