"""FP64 CPU oracle of the interpolative decomposition (ID) hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
this module. The product path (the CUDA library and its Python binding) never
calls it, shares no code with it, and fails loudly when its extension is
missing instead of falling back here.

What it computes (Advani & O'Hagan, "Efficient Algorithms for Constructing an
Interpolative Decomposition", arXiv 2105.07076):

* Definition 1 (Sec. 1.2): A ~= C Z with C = k columns of A, a k x k identity
  inside Z, |Z_ij| <= 2.
* Sec. 2 footnote: if m > n the method is applied to A^T and the result is
  transposed (a row ID).
* Sec. 2.1: column-pivoted QR  A P = Q R, skeleton columns = the first k pivots,
  C = A P_k, and Z solves min ||A - C Z||_F. With C = Q_k R_k the normal
  equations (Eq. normal_eq) reduce to R_k^T R_k Z = C^T A (Eq. final_eq). Since
  Q_k^T A P = [R_11 R_12], that system is solved exactly by Z P = [I  T] with
  T = R_11^{-1} R_12, which is what ``interp_decomp`` computes (back
  substitution). ``normal_equation_z`` keeps the paper's own route as a
  cross-check.
* Sec. 2.1 / Sec. 4.1: the QR is stopped after k pivots; the first k greedy
  pivots and R_11, R_12 do not depend on later steps.
* Sec. 2.2: the least-squares target min ||A - C Z||_F for a fixed skeleton set,
  used by the randomized variant (``ls_interp``) and by the refinement of T.
* Sec. 1.2 footnote: the two-sided ID X^T A[I, J] Z, built from a column ID and
  a row ID of its skeleton (``two_sided_interp_decomp``).
* Sec. 3 (sparse test matrices): a CSR input is the dense matrix of its
  entries, duplicates summed (``csr_to_dense``); its ID is interp_decomp's.

Readings where the paper is silent:
* pivot = column of largest residual 2-norm over the not-yet-chosen columns;
  exact ties go to the smallest ORIGINAL column index;
* Householder sign: beta = -sign(x_0) ||x|| with sign(0) = +1, reflector
  H = I - tau v v^T with v_0 = 1 and tau = (beta - x_0) / beta (tau = 0 for a
  zero column);
* residual norms are recomputed from scratch at every step (the plain greedy
  definition; no downdating);
* numerical rank: the first j with |R_jj| <= sqrt(max(m, n)) * eps * |R_00|
  (0 if R_00 = 0), eps of the arithmetic's precision (sqrt(max(m, n)) eps is
  the typical size of the rounding noise left in a residual column); J, Z are
  then meaningful for the first ``rank`` rows only.
"""
from __future__ import annotations

import numpy as np

EPS64 = np.finfo(np.float64).eps


def householder(x: np.ndarray):
    """Reflector H = I - tau v v^T with H x = beta e_0 (Sec. 2.1, AP = QR).

    Returns (v, tau, beta) with v[0] = 1, beta = -sign(x_0) ||x||, sign(0) = +1.
    A zero vector gives tau = 0, beta = 0 (H = I).
    """
    x = np.asarray(x, dtype=np.float64)
    alpha = float(np.sqrt(np.dot(x, x)))
    if alpha == 0.0:
        v = np.zeros_like(x)
        v[0] = 1.0
        return v, 0.0, 0.0
    x0 = float(x[0])
    beta = -alpha if x0 >= 0.0 else alpha
    v = x / (x0 - beta)
    v[0] = 1.0
    tau = (beta - x0) / beta
    return v, tau, beta


def cpqr(X: np.ndarray, k: int, pivots=None):
    """k steps of Businger-Golub column-pivoted Householder QR of X (m x n).

    Sec. 2.1: X P = Q R, stopped after k pivots (Sec. 4.1). Every step
    recomputes the residual column norms ||X(j:m, l)||_2 of the unchosen
    columns from scratch, takes the largest (ties: smallest original index),
    swaps it into position j and applies one reflector to the trailing columns.
    With ``pivots`` (k original column indices) the pivot order is forced
    instead of chosen; everything else is unchanged.

    Returns a dict with
      F      m x n FP64: R in the upper triangle of the first k rows (R_11 in
             columns 0..k-1, R_12 in columns k..n-1), reflector tails below the
             diagonal of the first k columns (v_0 = 1 implicit);
      perm   n int64: perm[i] = original index of the column now at position i;
      tau    k FP64 reflector scalars;
      nu     k FP64: the winning residual norm at each step (= |R_jj|);
      top    k FP64: the largest residual norm at each step (= nu unless the
             pivots are forced; 1 - nu / top is then the forced choice's
             shortfall against the greedy rule, as verify_pivots reports it);
      gap    k FP64: relative gap (nu_max - nu_second) / nu_max at each step;
      rank   numerical rank found within the k steps (k if none is small).
    """
    F = np.array(X, dtype=np.float64, copy=True)
    m, n = F.shape
    if not (1 <= k <= min(m, n)):
        raise ValueError("need 1 <= k <= min(m, n)")
    perm = np.arange(n, dtype=np.int64)
    tau = np.zeros(k)
    nu_win = np.zeros(k)
    nu_top = np.zeros(k)
    gap = np.full(k, np.inf)
    for j in range(k):
        B = F[j:, j:]
        nu = np.sqrt(np.einsum("ij,ij->j", B, B))
        top = nu.max()
        if pivots is None:
            ties = np.flatnonzero(nu == top)
            p = j + int(ties[np.argmin(perm[j + ties])])
        else:
            p = j + int(np.flatnonzero(perm[j:] == int(pivots[j]))[0])
        if nu.size > 1:
            rest = np.delete(nu, p - j)
            second = rest.max()
            gap[j] = (top - second) / top if top > 0 else 0.0
        nu_win[j] = nu[p - j]
        nu_top[j] = top
        if p != j:
            F[:, [j, p]] = F[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        v, t, beta = householder(F[j:, j])
        tau[j] = t
        if j + 1 < n:
            w = v @ F[j:, j + 1:]
            F[j:, j + 1:] -= t * np.outer(v, w)
        F[j, j] = beta
        F[j + 1:, j] = v[1:]
    d = np.abs(np.diag(F[:k, :k]))
    rank = k
    thresh = np.sqrt(max(m, n)) * EPS64 * d[0]
    for j in range(k):
        if d[0] == 0.0 or d[j] <= thresh:
            rank = j
            break
    return {"F": F, "perm": perm, "tau": tau, "nu": nu_win, "top": nu_top, "gap": gap, "rank": rank}


def back_substitute(R11: np.ndarray, R12: np.ndarray) -> np.ndarray:
    """T = R_11^{-1} R_12 by back substitution, row k-1 first (Sec. 2.1)."""
    k = R11.shape[0]
    T = np.zeros_like(R12, dtype=np.float64)
    for i in range(k - 1, -1, -1):
        T[i] = (R12[i] - R11[i, i + 1:] @ T[i + 1:]) / R11[i, i]
    return T


def assemble_z(perm: np.ndarray, T: np.ndarray, k: int) -> np.ndarray:
    """Z (k x n) with Z[:, perm[i]] = e_i for i < k and Z[:, perm[k:]] = T (Def. 1)."""
    n = perm.shape[0]
    Z = np.zeros((k, n))
    Z[np.arange(k), perm[:k]] = 1.0
    Z[:, perm[k:]] = T
    return Z


def interp_decomp(A: np.ndarray, k: int, pivots=None):
    """Deterministic rank-k ID of A (Sec. 2.1), with the m > n route (Sec. 2 footnote).

    Returns (J, Z, info). For m <= n: A ~= A[:, J] @ Z, Z is k x n.
    For m > n the method runs on A^T: A^T ~= A^T[:, J] @ Z, i.e.
    A ~= Z^T @ A[J, :] (a row ID), Z is k x m, and info["transposed"] is True.
    """
    A = np.asarray(A, dtype=np.float64)
    transposed = A.shape[0] > A.shape[1]
    X = A.T if transposed else A
    f = cpqr(X, k, pivots)
    R = np.triu(f["F"][:k, :])
    T = back_substitute(R[:, :k], R[:, k:])
    Z = assemble_z(f["perm"], T, k)
    J = f["perm"][:k].copy()
    info = {
        "transposed": transposed,
        "perm": f["perm"],
        "T": T,
        "R": R,
        "tau": f["tau"],
        "nu": f["nu"],
        "top": f["top"],
        "gap": f["gap"],
        "rank": f["rank"],
        "n_gt2": int(np.count_nonzero(np.abs(Z) > 2.0)),
        "max_abs_z": float(np.abs(Z).max()),
    }
    return J, Z, info


def reconstruct(A: np.ndarray, J: np.ndarray, Z: np.ndarray, transposed: bool = False) -> np.ndarray:
    """C Z with C = A[:, J] (or Z^T A[J, :] for a row ID)."""
    A = np.asarray(A, dtype=np.float64)
    if transposed:
        return Z.T @ A[J, :]
    return A[:, J] @ Z


def rel_error(A: np.ndarray, J: np.ndarray, Z: np.ndarray, transposed: bool = False) -> float:
    """||A - C Z||_F / ||A||_F (Sec. 3.2, the error measure of Table 2)."""
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm(A - reconstruct(A, J, Z, transposed)) / np.linalg.norm(A))


def normal_equation_z(A: np.ndarray, J: np.ndarray, R11: np.ndarray) -> np.ndarray:
    """The paper's own route to Z: solve R_k^T R_k Z = C^T A (Eq. final_eq).

    Forward substitution with R_k^T, then back substitution with R_k.
    """
    A = np.asarray(A, dtype=np.float64)
    C = A[:, J]
    rhs = C.T @ A
    k = R11.shape[0]
    Y = np.zeros_like(rhs)
    L = R11.T
    for i in range(k):
        Y[i] = (rhs[i] - L[i, :i] @ Y[:i]) / L[i, i]
    Zt = np.zeros_like(rhs)
    for i in range(k - 1, -1, -1):
        Zt[i] = (Y[i] - R11[i, i + 1:] @ Zt[i + 1:]) / R11[i, i]
    return Zt


def ls_interp(A: np.ndarray, J: np.ndarray) -> np.ndarray:
    """Z minimising ||A - A[:, J] Z||_F for a fixed skeleton set J (Sec. 2.1-2.2).

    Solved with an orthogonal factorisation of C = A[:, J] (numpy lstsq), never
    through C^T C.
    """
    A = np.asarray(A, dtype=np.float64)
    C = A[:, J]
    Z, *_ = np.linalg.lstsq(C, A, rcond=None)
    return Z


def verify_pivots(X: np.ndarray, J: np.ndarray, tol: float):
    """Replay a candidate pivot sequence J on X with the exact greedy residual norms.

    At step j the residual norms of all unchosen columns are recomputed from
    scratch (as in ``cpqr``) and the candidate's norm must be at least
    (1 - tol) * max. The replay then continues with the candidate's choice, so
    one legitimate near-tie does not make every later step disagree.

    Returns (ok, worst) where worst[j] = 1 - nu[J[j]] / max nu at step j.
    """
    F = np.array(X, dtype=np.float64, copy=True)
    m, n = F.shape
    k = len(J)
    cols = list(range(n))      # position -> original index
    worst = np.zeros(k)
    for j in range(k):
        B = F[j:, j:]
        nu = np.sqrt(np.einsum("ij,ij->j", B, B))
        top = nu.max()
        try:
            p = j + cols[j:].index(int(J[j]))
        except ValueError:
            return False, worst
        worst[j] = 1.0 - nu[p - j] / top if top > 0 else 0.0
        if p != j:
            F[:, [j, p]] = F[:, [p, j]]
            cols[j], cols[p] = cols[p], cols[j]
        v, t, beta = householder(F[j:, j])
        if j + 1 < n:
            F[j:, j + 1:] -= t * np.outer(v, v @ F[j:, j + 1:])
        F[j, j] = beta
        F[j + 1:, j] = 0.0
    return bool(np.all(worst <= tol)), worst


def sketch(omega: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Y = Omega A in FP64 (Gaussian row sketch; Omega's BF16 values taken exactly)."""
    return np.asarray(omega, dtype=np.float64) @ np.asarray(A, dtype=np.float64)


def sampled_interp_decomp(A: np.ndarray, idx: np.ndarray, k: int):
    """Optim RID (Sec. 2.2, the randomized algorithm built on column sampling).

    The p sampled column indices ``idx`` (drawn without replacement; the paper
    takes p = k + floor(0.2 k)) are an input. CPQR of A_S = A[:, idx] selects
    the skeleton J = idx[P_k]; with C = A[:, J] and R_k the leading k x k block
    of that CPQR's R, Z solves the normal equations R_k^T R_k Z = C^T A
    (Eq. final_eq) by a forward and a back substitution with R_k. (The paper
    uses a symmetric-indefinite solve because C may be rank deficient; the two
    substitutions give the same Z whenever R_k is nonsingular, and ``rank``
    reports when it is not.) Returns (J, Z, info).
    """
    A = np.asarray(A, dtype=np.float64)
    idx = np.asarray(idx, dtype=np.int64)
    if len(np.unique(idx)) != len(idx) or idx.min() < 0 or idx.max() >= A.shape[1]:
        raise ValueError("idx must hold distinct column indices")
    f = cpqr(A[:, idx], k)
    J = idx[f["perm"][:k]]
    R = np.triu(f["F"][:k, :k])
    Z = normal_equation_z(A, J, R)
    return J, Z, {"perm": f["perm"], "R": R, "rank": f["rank"], "gap": f["gap"]}


def csr_to_dense(rowptr: np.ndarray, colind: np.ndarray, values: np.ndarray, m: int, n: int) -> np.ndarray:
    """The dense m x n matrix of a CSR triple (row i holds colind/values[rowptr[i]:rowptr[i+1]]);
    duplicate entries are summed. The sparse-input ID is interp_decomp of this matrix."""
    A = np.zeros((m, n), dtype=np.float64)
    for i in range(m):
        for q in range(int(rowptr[i]), int(rowptr[i + 1])):
            A[i, int(colind[q])] += float(values[q])
    return A


def two_sided_interp_decomp(A: np.ndarray, k: int):
    """Two-sided ID A ~= X^T A[I, J] Z, the variant of Cheng et al. that the
    footnote of Sec. 1.2 names.

    m <= n: the column ID (J, Z) of A (Sec. 2.1), then a row ID (I, X) of the
    skeleton C = A[:, J] (the Sec. 2 footnote's m > n route on an m x k
    matrix). m > n: the roles swap, a row ID (I, X) of A, then the column ID
    (J, Z) of R = A[I, :]. A rank-k m x k (k x n) skeleton has an exact k-row
    (k-column) ID, so in exact arithmetic the second stage adds no error:
    X^T C[I, :] = C. A stage whose matrix is already k x k keeps every row
    (column): the identity. Returns (I, J, X, Z); X is k x m, Z is k x n.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if not (1 <= k <= min(m, n)):
        raise ValueError("need 1 <= k <= min(m, n)")
    if m <= n:
        J, Z, _ = interp_decomp(A, k)
        C = A[:, J]
        if m == k:
            I, X = np.arange(k), np.eye(k)
        else:
            I, X, _ = interp_decomp(C, k)          # m > k: a row ID of C
    else:
        I, X, _ = interp_decomp(A, k)              # m > n: a row ID of A
        R = A[I, :]
        if n == k:
            J, Z = np.arange(k), np.eye(k)
        else:
            J, Z, _ = interp_decomp(R, k)          # k < n: a column ID of R
    return I, J, X, Z


def two_sided_reconstruct(A: np.ndarray, I: np.ndarray, J: np.ndarray, X: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """X^T A[I, J] Z."""
    A = np.asarray(A, dtype=np.float64)
    return X.T @ A[np.ix_(I, J)] @ Z


def randomized_interp_decomp(A: np.ndarray, omega: np.ndarray, k: int):
    """Randomized ID: skeleton from CPQR of Y = Omega A, Z refined against A.

    The skeleton set comes from k CPQR steps on the sketch Y. T is first taken
    from Y's R (T_Y = R_11^{-1} R_12), then one refinement step
    T <- T + argmin ||A_J dT - (A_rest - A_J T)||_F, which in exact arithmetic
    lands on the least-squares Z of Sec. 2.2 (min ||A - C Z||_F) for that J.
    Returns (J, Z_sketch, Z_refined, info).
    """
    A = np.asarray(A, dtype=np.float64)
    Y = sketch(omega, A)
    J, Zy, info = interp_decomp(Y, k)
    perm = info["perm"]
    C = A[:, J]
    rest = perm[k:]
    resid = A[:, rest] - C @ info["T"]
    dT, *_ = np.linalg.lstsq(C, resid, rcond=None)
    T = info["T"] + dT
    Zr = assemble_z(perm, T, k)
    info = dict(info, T_refined=T)
    return J, Zy, Zr, info


def id_grad(A: np.ndarray, J: np.ndarray, perm: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Gradient of L = <G, Z> w.r.t. A with the skeleton set frozen.

    Z[:, J] = I is constant; Z[:, rest] = T = C^+ B with C = A[:, J] and
    B = A[:, rest] (the least-squares solution of Sec. 2.1). With Gb = G[:, rest]
    and W = (C^T C)^{-1} Gb:
        dB = C W,   dC = (B - C T) W^T - C W T^T.
    Returns dA (m x n) with dA[:, J] = dC and dA[:, rest] = dB.
    """
    A = np.asarray(A, dtype=np.float64)
    k = len(J)
    rest = perm[k:]
    C = A[:, J]
    B = A[:, rest]
    Qc, Rc = np.linalg.qr(C)
    T = np.linalg.solve(Rc, Qc.T @ B)
    Gb = np.asarray(G, dtype=np.float64)[:, rest]
    W = np.linalg.solve(Rc, np.linalg.solve(Rc.T, Gb))
    dA = np.zeros_like(A)
    dA[:, rest] = C @ W
    dA[:, J] = (B - C @ T) @ W.T - C @ W @ T.T
    return dA
