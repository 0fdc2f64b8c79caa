"""Plain FP64 CPU oracle for the block orthogonalization of Dreier & Engwer,
"A Hardware-aware and Stable Orthogonalization Framework" (arXiv 2204.13393).

TEST INFRASTRUCTURE ONLY.  This module is a slow, obviously-correct restatement
of what the method computes.  It exists to check the CUDA path, never to run
in its place: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
/ reference arm of ``bench.py`` may import it.  It shares no code, headers,
tables or helpers with the CUDA library (``paper_2204_13393_gb300``) and
imports nothing from it.  Inputs come from the separate seeded generators.

Everything is float64 numpy.  Library primitives used as single steps: matrix
products (``@``), ``np.sqrt``, ``np.dot``.  No blocking, fusion or reordering
beyond what the cited definition or algorithm states.

Contents (paper section / equation / algorithm each function follows):

* ``cholesky_upper``       textbook Cholesky, N^T N = M (Sec. 3, CholQR); an
                           exactly zero component gives a zero row.
* ``solve_upper_right``    Y N^{-1} by column-wise substitution.
* ``householder_qr``       column-wise Householder QR (Sec. 2.2, eq. (hh),
                           Alg. 6 with an empty prior basis).
* ``pqr_householder``      the project-and-normalize (PQR) problem, eq. (pqr),
                           solved by its plain definition: the thin QR of [Q X]
                           with a positive diagonal.  Oracle A.
* ``pqr_mgs2``             PQR by modified Gram-Schmidt applied twice
                           (Alg. 4 reiterated as in Alg. 5).  Oracle B.
* ``pqr_mgs2_deflate``     the deflated PQR of Sec. 3 (t < s; kept as t = s
                           with zero rows of N and zero columns of U): oracle
                           B with a column dropped when what remains of it
                           is at most delta ||X||_F.
* ``bcgs_pip``             Alg. 7 (BCGS-PIP).
* ``bcgs_pip2``            Alg. 8 (BCGS-PIP+), with the combination step read
                           as P = P1 + P2 N1, N = N2 N1 (the printed formula is
                           not consistent with eq. (pqr); see the test that pins it).
* ``LocallyOrthogonalBasis`` the locally orthogonal representation
                           Q = diag(Q_1..Q_p) [T_1; ..; T_p] of Sec. 4.1, with
                           ``orthogonalize`` = Alg. 9 (TreeTSPQR): local PQR per
                           chunk, reduction PQR of the stacked factors, then the
                           assembly of U (Sec. 4.1, block-wise products).
* ``block_qr``             Alg. 2 (block-column QR by successive PQR solves).
* ``block_arnoldi``        Alg. 1 (block Arnoldi), operator given as a callable.
* ``e_perp``, ``residual`` eq. (ortho_error) and ||A - QR||_F / ||A||_F.

Every function here is pinned by ``tests/test_oracle_pins.py`` against things
other than itself (LAPACK, 50-digit arithmetic, closed forms, invariants and
the values printed in the paper's stability table).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "Breakdown",
    "cholesky_upper",
    "solve_upper_right",
    "householder_qr",
    "sign_normalize",
    "pqr_householder",
    "pqr_mgs2",
    "pqr_mgs2_deflate",
    "bcgs_pip",
    "bcgs_pip2",
    "pqr",
    "chunk_bounds",
    "LocallyOrthogonalBasis",
    "block_qr",
    "block_arnoldi",
    "e_perp",
    "residual",
    "SUBALGORITHMS",
]


class Breakdown(ArithmeticError):
    """A Cholesky pivot was not positive and the block was not exactly zero
    there: a rank deficiency while deflation (Sec. 3, t < s) is off."""


def _sgn(x: float) -> float:
    """sgn with sgn(0) = +1 (the sign choice of Alg. 6)."""
    return 1.0 if x >= 0.0 else -1.0


def cholesky_upper(M: np.ndarray, deflate: float = 0.0) -> np.ndarray:
    """Upper-triangular N with N^T N = M (textbook Cholesky, row by row).

    This is the factorization CholQR and BCGS-PIP use (Sec. 3): for the PQR
    Gram matrix it is applied to G - P^T P.  A pivot that is exactly zero
    while the rest of its row is exactly zero too (the block has an exactly
    zero component there, e.g. a column that vanishes on one chunk) gives a
    zero row of N: Sec. 3 allows keeping t = s and carrying the rank
    deficiency in N, and with exact zeros no tolerance is involved.  Any other
    non-positive or non-finite pivot raises ``Breakdown``.

    With ``deflate`` > 0 a finite pivot d <= deflate is deflated as well (the
    deflation case of Sec. 3: the column is, to that tolerance, in the span of
    what came before it): row i of N is zero, and the later rows do not see
    it.  The pivot is the squared distance of column i to the span of the
    earlier columns, so ``deflate`` is a squared norm.
    """
    M = np.asarray(M, dtype=np.float64)
    s = M.shape[0]
    N = np.zeros((s, s))
    for i in range(s):
        d = M[i, i] - sum(N[l, i] * N[l, i] for l in range(i))
        rest = [M[i, j] - sum(N[l, i] * N[l, j] for l in range(i)) for j in range(i + 1, s)]
        if d == 0.0 and all(r == 0.0 for r in rest):
            continue  # exactly zero component: zero row
        if deflate > 0.0 and np.isfinite(d) and d <= deflate:
            continue  # deflated: zero row
        if not (d > 0.0) or not np.isfinite(d):
            raise Breakdown(f"Cholesky pivot {i} = {d!r}")
        N[i, i] = np.sqrt(d)
        for j in range(i + 1, s):
            N[i, j] = rest[j - i - 1] / N[i, i]
    return N


def solve_upper_right(Y: np.ndarray, N: np.ndarray) -> np.ndarray:
    """Return Y N^{-1} for upper-triangular N, by substitution over columns
    (column j of the result solves sum_{l<=j} X[:, l] N[l, j] = Y[:, j]).

    For a zero row j of N (an exactly zero component, see ``cholesky_upper``)
    column j of the result is zero: X N = Y then holds for every Y whose
    columns lie in the row space of N."""
    Y = np.asarray(Y, dtype=np.float64)
    s = N.shape[0]
    X = np.zeros_like(Y)
    for j in range(s):
        if N[j, j] == 0.0:
            continue
        acc = Y[:, j].copy()
        for l in range(j):
            acc -= X[:, l] * N[l, j]
        X[:, j] = acc / N[j, j]
    return X


def householder_qr(A: np.ndarray):
    """Thin QR of A (n x m, n >= m) by column-wise Householder reflections.

    Follows Sec. 2.2: reflector H_j = I - 2 v_j v_j^T with ||v_j|| = 1; for
    column j the lower part u = A[j:, j] gives lambda = ||u||,
    sigma = -sgn(u[0]) (sgn(0) = +1), R[j, j] = sigma * lambda and
    v_j = (u - sigma*lambda e_1) / ||u - sigma*lambda e_1||.  The explicit Q is
    obtained by applying H_0 ... H_{m-1} to the first m unit vectors (eq. (hh)
    and the line after it).  R is returned with the reflections' signs; use
    ``sign_normalize`` for the positive-diagonal convention.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    n, m = A.shape
    if n < m:
        raise ValueError("householder_qr needs n >= m")
    vs = []
    for j in range(m):
        u = A[j:, j]
        lam = np.sqrt(np.dot(u, u))
        sigma = -_sgn(u[0])
        v = u.copy()
        v[0] -= sigma * lam
        nv = np.sqrt(np.dot(v, v))
        if nv == 0.0:  # u == 0: no reflection needed (rank-deficient column)
            vs.append(None)
            continue
        v /= nv
        # apply H_j = I - 2 v v^T to the trailing columns
        A[j:, j:] -= 2.0 * np.outer(v, v @ A[j:, j:])
        A[j + 1:, j] = 0.0
        vs.append(v)
    R = np.triu(A[:m, :m])
    Q = np.zeros((n, m))
    Q[:m, :m] = np.eye(m)
    for j in reversed(range(m)):
        v = vs[j]
        if v is None:
            continue
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    return Q, R


def sign_normalize(Q: np.ndarray, R: np.ndarray):
    """Q D, D R with D = diag(sgn(R_jj)), sgn(0) = +1, so that diag(R) >= 0
    (the normalization that makes the thin QR, hence the PQR solution, unique)."""
    d = np.array([_sgn(x) for x in np.diag(R)])
    return Q * d[None, :], R * d[:, None]


def pqr_householder(Q: np.ndarray, X: np.ndarray):
    """Oracle A: the PQR problem, eq. (pqr), by its plain definition.

    For orthonormal Q (n x k) and X (n x s) with [Q X] of full rank the unique
    U (n x s, orthonormal, Q^T U = 0), P (k x s) and upper-triangular N (s x s,
    positive diagonal) with [Q X] = [Q U] [[I, P], [0, N]] are read off the
    sign-normalized thin QR of [Q X]: U = Qhat[:, k:], P = Rhat[:k, k:],
    N = Rhat[k:, k:].  Returns (U, P, N).  ``Rhat[:k, :k]`` equals I to
    rounding because Q is orthonormal; this is checked by the tests.
    """
    Q = np.asarray(Q, dtype=np.float64).reshape(X.shape[0], -1)
    k = Q.shape[1]
    Qh, Rh = sign_normalize(*householder_qr(np.hstack([Q, X])))
    return Qh[:, k:], Rh[:k, k:], Rh[k:, k:]


def pqr_mgs2(Q: np.ndarray, X: np.ndarray):
    """Oracle B: PQR by modified Gram-Schmidt with one reorthogonalization.

    Column j of X is projected against every column of Q and every new column
    u_0..u_{j-1}, one at a time (Alg. 4), and the whole projection is done a
    second time (the reiteration of Alg. 5); the coefficients of both sweeps
    are summed.  N[j, j] is the norm of what remains, u_j the normalized rest.
    """
    Q = np.asarray(Q, dtype=np.float64).reshape(X.shape[0], -1)
    n, k = Q.shape
    s = X.shape[1]
    U = np.zeros((n, s))
    P = np.zeros((k, s))
    N = np.zeros((s, s))
    for j in range(s):
        v = X[:, j].astype(np.float64).copy()
        for _sweep in range(2):
            for c in range(k):
                coef = np.dot(Q[:, c], v)
                v -= coef * Q[:, c]
                P[c, j] += coef
            for c in range(j):
                coef = np.dot(U[:, c], v)
                v -= coef * U[:, c]
                N[c, j] += coef
        nrm = np.sqrt(np.dot(v, v))
        if not (nrm > 0.0):
            raise Breakdown(f"column {j} is linearly dependent")
        N[j, j] = nrm
        U[:, j] = v / nrm
    return U, P, N


def pqr_mgs2_deflate(Q: np.ndarray, X: np.ndarray, delta: float):
    """The deflated PQR problem (Sec. 3, t < s) by its plain definition.

    Column j of X is treated as in ``pqr_mgs2`` (two sweeps of projections
    against Q and the kept new columns, coefficients summed into P and N); if
    the norm of what remains is at most delta ||X||_F, the column is in the
    span of Q and the earlier columns to that tolerance: it is deflated,
    U[:, j] = 0 and row j of N is zero (t = s is kept, the rank deficiency is
    carried in N, as Sec. 3 allows), otherwise N[j, j] is that norm and
    U[:, j] the normalized rest.  X = Q P + U N holds to the deflation
    tolerance; the nonzero columns of U are orthonormal and orthogonal to Q.
    """
    Q = np.asarray(Q, dtype=np.float64).reshape(X.shape[0], -1)
    n, k = Q.shape
    s = X.shape[1]
    thr = float(delta) * float(np.sqrt(np.sum(np.asarray(X, dtype=np.float64) ** 2)))
    U = np.zeros((n, s))
    P = np.zeros((k, s))
    N = np.zeros((s, s))
    for j in range(s):
        v = X[:, j].astype(np.float64).copy()
        for _pass in range(2):
            for c in range(k):
                coef = np.dot(Q[:, c], v)
                v -= coef * Q[:, c]
                P[c, j] += coef
            for c in range(j):
                if N[c, c] == 0.0:
                    continue  # a deflated column of U is zero: nothing to project on
                coef = np.dot(U[:, c], v)
                v -= coef * U[:, c]
                N[c, j] += coef
        nrm = np.sqrt(np.dot(v, v))
        if nrm <= thr:
            continue  # deflated
        N[j, j] = nrm
        U[:, j] = v / nrm
    return U, P, N


def bcgs_pip(Q: np.ndarray, X: np.ndarray, deflate: float = 0.0):
    """Alg. 7 (BCGS-PIP): P = Q^T X and G = X^T X, N = chol(G - P^T P),
    U = X N^{-1} - Q P N^{-1} (= (X - Q P) N^{-1}).  ``deflate``: the squared
    norm below which a Cholesky pivot is deflated (see ``cholesky_upper``)."""
    Q = np.asarray(Q, dtype=np.float64).reshape(X.shape[0], -1)
    P = Q.T @ X
    G = X.T @ X
    N = cholesky_upper(G - P.T @ P, deflate)
    U = solve_upper_right(X - Q @ P, N)
    return U, P, N


def bcgs_pip2(Q: np.ndarray, X: np.ndarray, deflate: float = 0.0):
    """Alg. 8 (BCGS-PIP+): Alg. 7 applied to X, then to its output U1.

    From X = Q P1 + U1 N1 and U1 = Q P2 + U N2 it follows that
    X = Q (P1 + P2 N1) + U (N2 N1); hence P = P1 + P2 N1 and N = N2 N1.
    Deflation (``deflate`` > 0) is decided in the first pass; the second
    sees the deflated columns as exact zeros.
    """
    U1, P1, N1 = bcgs_pip(Q, X, deflate)
    U, P2, N2 = bcgs_pip(Q, U1)
    return U, P1 + P2 @ N1, N2 @ N1


SUBALGORITHMS = {
    "hh": pqr_householder,
    "mgs2": pqr_mgs2,
    "pip": bcgs_pip,
    "pip2": bcgs_pip2,
}


def pqr(Q, X, alg: str = "hh", deflate: float = 0.0):
    """Solve eq. (pqr) with the named sub-algorithm ('hh', 'mgs2', 'pip', 'pip2');
    ``deflate`` (a squared norm) only for the Cholesky-based 'pip' and 'pip2'."""
    if deflate > 0.0:
        if alg not in ("pip", "pip2"):
            raise ValueError("deflation needs a Cholesky-based sub-algorithm")
        return SUBALGORITHMS[alg](Q, X, deflate)
    return SUBALGORITHMS[alg](Q, X)


def chunk_bounds(n: int, chunk_rows: int):
    """Row ranges of the local blocks: p = max(1, n // chunk_rows) chunks of
    chunk_rows rows, the remainder joining the last chunk (the paper assumes
    p * chunk_rows = n, Sec. 5.1.3; this is the reading for other n)."""
    p = max(1, n // chunk_rows)
    starts = [i * chunk_rows for i in range(p)]
    ends = starts[1:] + [n]
    return list(zip(starts, ends))


class LocallyOrthogonalBasis:
    """The locally orthogonal representation of Sec. 4.1.

    Q = diag(Q_1, .., Q_p) [T_1; ..; T_p] where Q_i (n_i x k) has orthonormal
    columns and the stacked T_i (k x k each, upper triangular) are orthonormal,
    sum_i T_i^T T_i = I.  ``orthogonalize`` runs Alg. 9 (TreeTSPQR).

    With a Cholesky-based local solver ('pip', 'pip2') a block that is
    exactly zero in some column of a chunk gives that chunk a zero column in
    Q_i (Q_i^T Q_i is then diagonal with entries 0 and 1) and a zero row in
    T_i, so Q itself stays orthonormal; the Householder solver completes Q_i
    with unit directions instead.
    """

    def __init__(self, n: int, s: int, chunk_rows: int):
        self.n, self.s = int(n), int(s)
        self.bounds = chunk_bounds(self.n, int(chunk_rows))
        self.Qloc = [np.zeros((e - b, 0)) for b, e in self.bounds]
        self.T = [np.zeros((0, 0)) for _ in self.bounds]

    @property
    def k(self) -> int:
        return self.T[0].shape[0]

    @property
    def num_blocks(self) -> int:
        return self.k // self.s

    def orthogonalize(self, X: np.ndarray, local: str = "hh", reduction: str = "hh", deflation: float = 0.0):
        """One PQR step, Alg. 9.  Returns (U, P, N) with P = H (k x s) and
        N = R (s x s).  The representation gains the new column block.

        ``deflation`` = delta > 0: the deflated PQR (Sec. 3, t < s, kept as
        t = s with zero rows of N): in the local first pass and in the
        reduction a Cholesky pivot at most tau = max(delta^2, 64 s eps)
        ||X||_F^2 (a column whose distance to the span of the earlier ones is
        at most delta ||X||_F, ||X||_F the norm of the whole block) is
        deflated.  The floor 64 s eps: a pivot of the Gram matrix G - P^T P
        carries rounding noise of order eps ||X||_F^2 from the cancellation,
        so distances below about sqrt(eps) ||X||_F cannot be told from zero.

        1. Local PQR per chunk: [Q_i X_i] = [Q_i U_i] [[I, P_i], [0, N_i]].
        2. Reduction PQR of the stacked factors:
           [[T_i, P_i], [0, N_i]]_i = [[T_i, Pt_i], [0, Nt_i]]_i [[I, P], [0, N]].
        3. Assembly: rows of chunk i of U are [Q_i U_i] [Pt_i; Nt_i].
        4. Representation update: Q_i <- [Q_i U_i], T_i <- [[T_i, Pt_i], [0, Nt_i]].
        """
        X = np.asarray(X, dtype=np.float64)
        s, k = self.s, self.k
        assert X.shape == (self.n, s)
        eps = np.finfo(np.float64).eps
        tau = max(float(deflation) ** 2, 64.0 * s * eps) * float(np.sum(X * X)) if deflation > 0.0 else 0.0
        loc = []
        for (b, e), Qi in zip(self.bounds, self.Qloc):
            loc.append(pqr(Qi, X[b:e], local, tau if local in ("pip", "pip2") else 0.0))
        # stacked reduction problem: "Q" rows are [T_i; 0], "X" rows are [P_i; N_i]
        Qs = np.vstack([np.vstack([Ti, np.zeros((s, k))]) for Ti in self.T])
        Xs = np.vstack([np.vstack([Pi, Ni]) for (_, Pi, Ni) in loc])
        Us, P, N = pqr(Qs, Xs, reduction, tau)
        if tau == 0.0 and np.any(np.diag(N) == 0.0):
            # the block has an exactly zero component on every chunk: a global
            # rank deficiency (the deflation case of Sec. 3, not handled)
            raise Breakdown("the block is rank deficient against the basis")
        U = np.zeros((self.n, s))
        for i, ((b, e), (Ui, _, _)) in enumerate(zip(self.bounds, loc)):
            blk = Us[i * (k + s):(i + 1) * (k + s)]
            Pt, Nt = blk[:k], blk[k:]
            U[b:e] = self.Qloc[i] @ Pt + Ui @ Nt
            self.Qloc[i] = np.hstack([self.Qloc[i], Ui])
            Tn = np.zeros((k + s, k + s))
            Tn[:k, :k] = self.T[i]
            Tn[:k, k:] = Pt
            Tn[k:, k:] = Nt
            self.T[i] = Tn
        return U, P, N

    def explicit(self) -> np.ndarray:
        """The explicit basis Q = diag(Q_i) [T_i] (n x k)."""
        return np.vstack([Qi @ Ti for Qi, Ti in zip(self.Qloc, self.T)])

    def apply_Q(self, C: np.ndarray) -> np.ndarray:
        """Q C computed chunk-wise as Q_i (T_i C) (the product QC of Sec. 5.1)."""
        C = np.asarray(C, dtype=np.float64)
        return np.vstack([Qi @ (Ti @ C) for Qi, Ti in zip(self.Qloc, self.T)])

    def tree_gram(self) -> np.ndarray:
        """sum_i T_i^T T_i, which equals I for a valid representation (Sec. 4.1)."""
        return sum(Ti.T @ Ti for Ti in self.T)


def block_qr(A: np.ndarray, s: int, solver):
    """Alg. 2: QR of A (n x m) by successive PQR solves on its s-column blocks.

    ``solver(Qprev, Ablock) -> (U, P, N)`` may be a plain PQR function (the
    explicit basis is kept) or ``LocallyOrthogonalBasis.orthogonalize`` wrapped
    to ignore Qprev.  Returns the explicit Q (n x m) and R (m x m)."""
    A = np.asarray(A, dtype=np.float64)
    n, m = A.shape
    assert m % s == 0
    Qcols = np.zeros((n, 0))
    R = np.zeros((m, m))
    for b in range(m // s):
        U, P, N = solver(Qcols, A[:, b * s:(b + 1) * s])
        k = Qcols.shape[1]
        R[:k, k:k + s] = P
        R[k:k + s, k:k + s] = N
        Qcols = np.hstack([Qcols, U])
    return Qcols, R


def block_arnoldi(apply_A, R0: np.ndarray, m: int, solver):
    """Alg. 1: V_0 H_0 = R0 (a PQR with empty basis), then for i = 0..m-1:
    X = A V_i, [V X] = [V V_{i+1}] [[I, P], [0, N]], H gains the column
    block [P; N].  Returns (V (n x (m+1)s), H ((m+1)s x m s), H_0 (s x s))."""
    n, s = R0.shape
    V = np.zeros((n, 0))
    U0, _, H0 = solver(V, R0)
    V = U0
    H = np.zeros(((m + 1) * s, m * s))
    for i in range(m):
        X = apply_A(V[:, i * s:(i + 1) * s])
        U, P, N = solver(V, X)
        k = V.shape[1]
        H[:k, i * s:(i + 1) * s] = P
        H[k:k + s, i * s:(i + 1) * s] = N
        V = np.hstack([V, U])
    return V, H, H0


def e_perp(Q: np.ndarray) -> float:
    """Orthogonality error ||I - Q^T Q||_F, eq. (ortho_error)."""
    Q = np.asarray(Q, dtype=np.float64)
    return float(np.linalg.norm(np.eye(Q.shape[1]) - Q.T @ Q))


def residual(A: np.ndarray, Q: np.ndarray, R: np.ndarray) -> float:
    """Relative factorization residual ||A - Q R||_F / ||A||_F."""
    return float(np.linalg.norm(A - Q @ R) / np.linalg.norm(A))
