"""Pins of the CPU oracle against things other than itself (CPU only).

Each test pins a part of ``oracle/lo_oracle.py`` to LAPACK, to 50-digit
arithmetic, to a closed form, to an invariant the paper states, or to the
values printed in the paper's stability table, so that a dropped term, a wrong
sign or index, or a transposed operand anywhere in the oracle fails one of them.
"""

import os

import numpy as np
import pytest

from paper_2204_13393_gb300 import inputs as I

if os.environ.get("LO_ORACLE_MUTANT"):
    # test_oracle_mutations.py runs these pins against a copy of the oracle
    # with one planted mistake
    import importlib.util

    _spec = importlib.util.spec_from_file_location("lo_oracle_mutant", os.environ["LO_ORACLE_MUTANT"])
    O = importlib.util.module_from_spec(_spec)
    _spec.loader.exec_module(O)
else:
    from oracle import lo_oracle as O

ALGS = ["hh", "mgs2", "pip", "pip2"]
HERE = os.path.dirname(os.path.abspath(__file__))


def _orthonormal(n, k, seed):
    return I.haar(n, k, seed) if k else np.zeros((n, 0))


def _lapack_qr(A):
    q, r = np.linalg.qr(A)
    d = np.where(np.diag(r) >= 0, 1.0, -1.0)
    return q * d[None, :], r * d[:, None]


# ---------------------------------------------------------------- primitives

def test_cholesky_matches_lapack():
    """cholesky_upper vs LAPACK potrf (numpy.linalg.cholesky gives L = N^T)."""
    A = I.gaussian(50, 7, 1)
    M = A.T @ A
    N = O.cholesky_upper(M)
    L = np.linalg.cholesky(M)
    np.testing.assert_allclose(N, L.T, rtol=0, atol=1e-13 * np.abs(L).max())
    assert np.all(np.tril(N, -1) == 0)


def test_cholesky_breakdown():
    M = np.array([[1.0, 2.0], [2.0, 1.0]])  # indefinite
    with pytest.raises(O.Breakdown):
        O.cholesky_upper(M)
    with pytest.raises(O.Breakdown):
        O.cholesky_upper(np.array([[np.nan]]))


def test_solve_upper_right():
    """X N^{-1} against a direct check X == Y @ N."""
    Y = I.gaussian(40, 5, 2)
    N = np.triu(I.gaussian(5, 5, 3)) + 4 * np.eye(5)
    X = O.solve_upper_right(Y, N)
    np.testing.assert_allclose(X @ N, Y, atol=1e-13)


@pytest.mark.parametrize("shape", [(200, 7), (33, 33), (64, 1), (1000, 16)])
def test_householder_matches_lapack(shape):
    """Textbook HH QR vs LAPACK geqrf/orgqr after sign normalization."""
    A = I.gaussian(*shape, seed=11 + shape[1])
    Q, R = O.sign_normalize(*O.householder_qr(A))
    Ql, Rl = _lapack_qr(A)
    np.testing.assert_allclose(Q, Ql, atol=1e-13)
    np.testing.assert_allclose(R, Rl, atol=1e-12 * np.abs(Rl).max())
    assert np.all(np.diag(R) >= 0)
    assert np.all(np.tril(R, -1) == 0)


def test_householder_sign_choice_on_zero_pivot():
    """sgn(0) = +1: a column whose pivot entry is exactly 0 still gives a
    reflection with R_jj = -lambda before normalization (Alg. 6 sign rule)."""
    A = np.array([[0.0, 1.0], [3.0, 0.0], [4.0, 2.0]])
    Q, R = O.householder_qr(A)
    assert R[0, 0] == pytest.approx(-5.0)
    np.testing.assert_allclose(Q @ R, A, atol=1e-14)


# ------------------------------------------------------- 50-digit brute force

def _mp_pqr(Q, X, dps=50):
    """PQR by classical Gram-Schmidt in 50-digit arithmetic (mpmath)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = dps
    n, k = Q.shape
    s = X.shape[1]
    cols = [[mp.mpf(float(Q[r, c])) for r in range(n)] for c in range(k)]
    # Q as given is orthonormal only to double precision: orthonormalize it
    # exactly first (this changes it by ~1e-16, below the tolerances used).
    basis = []
    for v in cols:
        w = list(v)
        for b in basis:
            c = mp.fsum(bi * wi for bi, wi in zip(b, w))
            w = [wi - c * bi for wi, bi in zip(w, b)]
        nr = mp.sqrt(mp.fsum(wi * wi for wi in w))
        basis.append([wi / nr for wi in w])
    P = np.zeros((k, s))
    N = np.zeros((s, s))
    U = np.zeros((n, s))
    newb = []
    for j in range(s):
        w = [mp.mpf(float(X[r, j])) for r in range(n)]
        for c, b in enumerate(basis):
            co = mp.fsum(bi * wi for bi, wi in zip(b, w))
            P[c, j] = float(co)
            w = [wi - co * bi for wi, bi in zip(w, b)]
        for c, b in enumerate(newb):
            co = mp.fsum(bi * wi for bi, wi in zip(b, w))
            N[c, j] = float(co)
            w = [wi - co * bi for wi, bi in zip(w, b)]
        nr = mp.sqrt(mp.fsum(wi * wi for wi in w))
        N[j, j] = float(nr)
        b = [wi / nr for wi in w]
        newb.append(b)
        U[:, j] = [float(x) for x in b]
    return U, P, N


@pytest.mark.parametrize("n,k,s", [(9, 3, 2), (12, 0, 3), (7, 4, 3), (10, 6, 1)])
@pytest.mark.parametrize("alg", ALGS)
def test_pqr_vs_50_digit_gram_schmidt(n, k, s, alg):
    Q = _orthonormal(n, k, 100 + n)
    X = I.gaussian(n, s, 200 + n + s)
    Ue, Pe, Ne = _mp_pqr(Q, X)
    U, P, N = O.pqr(Q, X, alg)
    np.testing.assert_allclose(U, Ue, atol=1e-14)
    np.testing.assert_allclose(P, Pe, atol=1e-14)
    np.testing.assert_allclose(N, Ne, atol=1e-14)


@pytest.mark.parametrize("alg", ALGS)
def test_tree_vs_50_digit(alg):
    """TreeTSPQR with 3 local blocks (10, 10, 13 rows) on a tiny two-step
    problem equals the 50-digit PQR of the explicit basis."""
    n, s = 33, 2
    B = O.LocallyOrthogonalBasis(n, s, 10)
    assert [e - b for b, e in B.bounds] == [10, 10, 13]
    X0 = I.gaussian(n, s, 5)
    X1 = I.gaussian(n, s, 6)
    B.orthogonalize(X0, alg, alg)
    Qexp = B.explicit()
    Ue, Pe, Ne = _mp_pqr(Qexp, X1)
    U, P, N = B.orthogonalize(X1, alg, alg)
    np.testing.assert_allclose(U, Ue, atol=1e-14)
    np.testing.assert_allclose(P, Pe, atol=1e-14)
    np.testing.assert_allclose(N, Ne, atol=1e-14)


# -------------------------------------------------------------- closed forms

@pytest.mark.parametrize("alg", ALGS)
def test_single_column_empty_basis(alg):
    """s = 1, k = 0: U = w/||w||, N = ||w|| (sum of squares written out)."""
    w = I.gaussian(300, 1, 7)
    nrm = np.sqrt(sum(float(x) ** 2 for x in w[:, 0]))
    U, P, N = O.pqr(np.zeros((300, 0)), w, alg)
    assert P.shape == (0, 1)
    assert N[0, 0] == pytest.approx(nrm, rel=1e-14)
    np.testing.assert_allclose(U[:, 0], w[:, 0] / nrm, atol=1e-15)


@pytest.mark.parametrize("alg", ALGS)
def test_unit_vector_basis(alg):
    """Q = I[:, :k]: P = X[:k], N = R-factor (LAPACK) of X[k:]."""
    n, k, s = 80, 6, 4
    Q = np.eye(n)[:, :k]
    X = I.gaussian(n, s, 8)
    U, P, N = O.pqr(Q, X, alg)
    np.testing.assert_allclose(P, X[:k], atol=1e-14)
    Ql, Rl = _lapack_qr(X[k:])
    np.testing.assert_allclose(N, Rl, atol=1e-13)
    np.testing.assert_allclose(U[:k], 0, atol=1e-14)
    np.testing.assert_allclose(U[k:], Ql, atol=1e-13)


@pytest.mark.parametrize("alg", ALGS)
def test_known_decomposition(alg):
    """X = Q M + Z S with Z orthonormal, Z ⟂ Q, S upper with positive
    diagonal: the unique solution is P = M, N = S, U = Z.  A transposed P, a
    wrong sign or a dropped term in any sub-algorithm breaks this."""
    n, k, s = 200, 12, 5
    QZ = I.haar(n, k + s, 9)
    Q, Z = QZ[:, :k], QZ[:, k:]
    M = I.gaussian(k, s, 10)
    S = np.triu(I.gaussian(s, s, 11)) + np.diag(np.arange(1.0, s + 1) + 2.0)
    S = S * np.where(np.diag(S) > 0, 1.0, -1.0)[:, None]
    X = Q @ M + Z @ S
    U, P, N = O.pqr(Q, X, alg)
    np.testing.assert_allclose(P, M, atol=1e-12)
    np.testing.assert_allclose(N, S, atol=1e-12)
    np.testing.assert_allclose(U, Z, atol=1e-12)


@pytest.mark.parametrize("alg", ALGS)
def test_already_orthogonal_block(alg):
    """X ⟂ span(Q), orthonormal: P = 0, N = I, U = X."""
    QZ = I.haar(150, 10, 12)
    Q, Z = QZ[:, :6], QZ[:, 6:]
    U, P, N = O.pqr(Q, Z, alg)
    np.testing.assert_allclose(P, 0, atol=1e-14)
    np.testing.assert_allclose(N, np.eye(4), atol=1e-14)
    np.testing.assert_allclose(U, Z, atol=1e-14)


def test_cholqr_identity():
    """k = 0: N^T N = X^T X and N = chol(X^T X)^T (LAPACK), the CholQR
    identity of Sec. 3."""
    X = I.gaussian(500, 6, 13)
    for alg in ALGS:
        _, _, N = O.pqr(np.zeros((500, 0)), X, alg)
        L = np.linalg.cholesky(X.T @ X)
        np.testing.assert_allclose(N, L.T, atol=1e-12 * np.abs(L).max())


def test_pip2_combination_formula():
    """The reiteration combine: X = Q P + U N must hold with
    P = P1 + P2 N1 and N = N2 N1; the printed variant P1 N2 + P2, N2 + N1 N2
    violates it (this pins the reading of Alg. 5 / Alg. 8)."""
    n, k, s = 300, 8, 4
    Q = I.haar(n, k, 14)
    X = I.stewart(n, s, 1e3, 15) + Q @ I.gaussian(k, s, 16)
    U1, P1, N1 = O.bcgs_pip(Q, X)
    U, P2, N2 = O.bcgs_pip(Q, U1)
    _, P, N = O.bcgs_pip2(Q, X)
    np.testing.assert_allclose(Q @ P + U @ N, X, atol=1e-12)
    printed_P, printed_N = P1 @ N2 + P2, N2 + N1 @ N2
    assert np.linalg.norm(Q @ printed_P + U @ printed_N - X) > 1e-3


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("local,reduction", [("hh", "hh"), ("pip2", "pip2"), ("pip", "pip2"),
                                             ("mgs2", "hh"), ("pip2", "hh")])
@pytest.mark.parametrize("n,chunk", [(1000, 128), (777, 100), (300, 1000)])
def test_tree_tspqr_equals_direct(local, reduction, n, chunk):
    """Alg. 9 over several steps gives the same U, P, N as the direct PQR of
    the explicit basis (the solution is unique), keeps every local Q_i
    orthonormal, keeps sum T_i^T T_i = I, and its explicit basis is the
    Q-factor of the direct QR of all blocks (Alg. 2 with LAPACK)."""
    s, steps = 4, 5
    B = O.LocallyOrthogonalBasis(n, s, chunk)
    Xs = [I.gaussian(n, s, 300 + j) for j in range(steps)]
    Rfull = np.zeros((s * steps, s * steps))
    for j, X in enumerate(Xs):
        Qexp = B.explicit()
        Ud, Pd, Nd = O.pqr_householder(Qexp, X)
        U, P, N = B.orthogonalize(X, local, reduction)
        np.testing.assert_allclose(U, Ud, atol=1e-13)
        np.testing.assert_allclose(P, Pd, atol=1e-13)
        np.testing.assert_allclose(N, Nd, atol=1e-12)
        Rfull[:j * s, j * s:(j + 1) * s] = P
        Rfull[j * s:(j + 1) * s, j * s:(j + 1) * s] = N
        for Qi in B.Qloc:
            assert O.e_perp(Qi) < 1e-13
        np.testing.assert_allclose(B.tree_gram(), np.eye(B.k), atol=1e-13)
        for Ti in B.T:
            np.testing.assert_allclose(np.tril(Ti, -1), 0, atol=1e-14)
    A = np.hstack(Xs)
    Ql, Rl = _lapack_qr(A)
    np.testing.assert_allclose(B.explicit(), Ql, atol=1e-12)
    np.testing.assert_allclose(Rfull, Rl, atol=1e-11 * np.abs(Rl).max())


def test_single_chunk_tree_is_the_leaf():
    """p = 1: the reduction acts on [[T_1, P_1], [0, N_1]] with T_1 = I-like,
    so TreeTSPQR returns the leaf's own P and N."""
    n, s = 256, 4
    B = O.LocallyOrthogonalBasis(n, s, 1024)
    assert len(B.bounds) == 1
    X0, X1 = I.gaussian(n, s, 20), I.gaussian(n, s, 21)
    B.orthogonalize(X0, "pip2", "pip2")
    Q = B.Qloc[0] @ B.T[0]
    Ul, Pl, Nl = O.bcgs_pip2(Q, X1)
    U, P, N = B.orthogonalize(X1, "pip2", "pip2")
    np.testing.assert_allclose(P, Pl, atol=1e-13)
    np.testing.assert_allclose(N, Nl, atol=1e-13)
    np.testing.assert_allclose(U, Ul, atol=1e-13)


def test_apply_Q_matches_explicit():
    n, s = 640, 3
    B = O.LocallyOrthogonalBasis(n, s, 64)
    for j in range(4):
        B.orthogonalize(I.gaussian(n, s, 40 + j), "hh", "hh")
    C = I.gaussian(B.k, 5, 50)
    np.testing.assert_allclose(B.apply_Q(C), B.explicit() @ C, atol=1e-13)
    A = np.hstack([I.gaussian(n, s, 40 + j) for j in range(4)])
    Ql, _ = _lapack_qr(A)
    np.testing.assert_allclose(B.apply_Q(np.eye(B.k)), Ql, atol=1e-12)


def test_block_arnoldi_relation():
    """Alg. 1: A V_m = V_{m+1} H (block Arnoldi relation) and V orthonormal,
    with the operator a 1D Laplacian."""
    n, s, m = 400, 2, 6

    def lap(V):
        out = 2 * V
        out[1:] -= V[:-1]
        out[:-1] -= V[1:]
        return out

    R0 = I.uniform(n, s, 60)
    B = O.LocallyOrthogonalBasis(n, s, 64)
    V, H, H0 = O.block_arnoldi(lap, R0, m, lambda Q, X: B.orthogonalize(X, "pip2", "pip2"))
    assert O.e_perp(V) < 1e-13
    np.testing.assert_allclose(lap(V[:, :m * s]), V @ H, atol=1e-12)
    np.testing.assert_allclose(V[:, :s] @ H0, R0, atol=1e-13)


# ---------------------------------------------- values printed in the paper

def _golden():
    rows = {}
    with open(os.path.join(HERE, "golden", "tspqr_stability_kappa1e4.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            q, alg, lo, hi = line.split()
            rows[(q, alg)] = (float(lo), float(hi))
    return rows


@pytest.mark.slow
@pytest.mark.parametrize("alg", ["pip", "pip2", "hh"])
def test_paper_stability_table(alg):
    """Sec. 6.1 table, kappa = 1e4, n = 2^16, 32 columns, s = 4, 256-row local
    problems: our Stewart matrix is another random draw, so the oracle must land
    within a factor 10 of the printed range (e_perp) and below 10x its top
    (residual).  The PIP case (~1e-9) pins the eps*kappa^2 loss of Alg. 7."""
    g = _golden()
    n, m, s = 2 ** 16, 32, 4
    A = I.stewart(n, m, 1e4, 77)
    B = O.LocallyOrthogonalBasis(n, s, 256)
    Q, R = O.block_qr(A, s, lambda Qp, X: B.orthogonalize(X, alg, alg))
    ep, res = O.e_perp(Q), O.residual(A, Q, R)
    lo, hi = g[("e_perp", alg)]
    assert lo / 10 <= ep <= hi * 10, (alg, ep)
    assert res <= g[("residual", alg)][1] * 10, (alg, res)


@pytest.mark.parametrize("alg,slope", [("pip", 2.0), ("pip2", 0.0), ("hh", 0.0), ("mgs2", 0.0)])
def test_error_law_slopes(alg, slope):
    """Sec. 3 / Sec. 6.1: e_perp = O(eps kappa^2) for PIP, O(eps) for PIP+
    (while eps kappa^2 <= 1/2) and for HH; O(eps) for Gram-Schmidt with one
    reorthogonalization (Sec. 2, Alg. 5; a single sweep loses orthogonality
    in proportion to kappa).  Fit log e_perp over kappa = 1e2..1e6."""
    n, m, s = 4096, 16, 4
    ks = [1e2, 1e3, 1e4, 1e5, 1e6] if alg != "pip" else [1e2, 1e3, 1e4, 1e5]
    errs = []
    for kappa in ks:
        A = I.stewart(n, m, kappa, 90)
        B = O.LocallyOrthogonalBasis(n, s, 256)
        Q, R = O.block_qr(A, s, lambda Qp, X: B.orthogonalize(X, alg, alg))
        errs.append(O.e_perp(Q))
    fit = np.polyfit(np.log10(ks), np.log10(errs), 1)[0]
    assert abs(fit - slope) < 0.6, (alg, fit, errs)


# ------------------------------------------------ exactly zero components

def test_cholesky_zero_rows_match_lapack_on_the_rest():
    """An exactly zero column of the factored block gives a zero row of N;
    the other rows are LAPACK's Cholesky of the matrix without that index."""
    B = I.gaussian(60, 6, 5)
    B[:, [1, 4]] = 0.0
    M = B.T @ B
    N = O.cholesky_upper(M)
    J = [0, 2, 3, 5]
    assert np.all(N[[1, 4]] == 0.0) and np.all(N[:, [1, 4]] == 0.0)
    L = np.linalg.cholesky(M[np.ix_(J, J)])
    np.testing.assert_allclose(N[np.ix_(J, J)], L.T, rtol=0, atol=1e-13 * np.abs(L).max())
    np.testing.assert_allclose(N.T @ N, M, rtol=0, atol=1e-12 * np.abs(M).max())
    assert np.all(O.cholesky_upper(np.zeros((3, 3))) == 0.0)
    # a zero pivot whose row is not zero (indefinite) still breaks down
    with pytest.raises(O.Breakdown):
        O.cholesky_upper(np.array([[0.0, 1.0], [1.0, 1.0]]))


def test_solve_upper_right_zero_rows():
    """Columns of the result at zero rows of N are zero, and X N = Y for Y in
    the row space of N (checked against a least-squares solve)."""
    N = np.triu(I.gaussian(5, 5, 6)) + 4 * np.eye(5)
    N[2] = 0.0
    Y = I.gaussian(30, 5, 7) @ N
    X = O.solve_upper_right(Y, N)
    assert np.all(X[:, 2] == 0.0)
    np.testing.assert_allclose(X @ N, Y, atol=1e-12 * np.abs(Y).max())
    Xl = np.linalg.lstsq(np.delete(N, 2, axis=0).T, Y.T, rcond=None)[0].T
    np.testing.assert_allclose(np.delete(X, 2, axis=1), Xl, atol=1e-12)


@pytest.mark.parametrize("local,reduction", [("pip2", "pip2"), ("pip", "pip2"), ("pip2", "hh"),
                                             ("hh", "hh")])
@pytest.mark.parametrize("n,chunk", [(1000, 128), (777, 100)])
def test_tree_tspqr_blocks_vanishing_on_chunks(local, reduction, n, chunk):
    """Blocks that are exactly zero on whole chunks or on some columns of a
    chunk (globally of full rank): Alg. 9 still gives the unique U, P, N of
    the direct PQR and LAPACK's QR of all blocks; Q_i^T Q_i is diagonal with
    entries 0 and 1 for the Cholesky leaves and sum T_i^T T_i = I."""
    s, steps = 4, 4
    B = O.LocallyOrthogonalBasis(n, s, chunk)
    bounds = B.bounds
    p = len(bounds)
    Xs = []
    for j in range(steps):
        # column c lives on chunks c, c + s, ... (plus the first half of chunk
        # p - 1 for the odd steps); chunk 1 is empty for every column
        sup = [[bounds[i] for i in range(c, p, s) if i != 1] for c in range(s)]
        if j % 2:
            b, e = bounds[p - 1]
            sup = [r + [(b, (b + e) // 2)] for r in sup]
        Xs.append(I.localized(n, s, 700 + j, sup))
    Rfull = np.zeros((s * steps, s * steps))
    for j, X in enumerate(Xs):
        Ud, Pd, Nd = O.pqr_householder(B.explicit(), X)
        U, P, N = B.orthogonalize(X, local, reduction)
        np.testing.assert_allclose(U, Ud, atol=1e-13)
        np.testing.assert_allclose(P, Pd, atol=1e-13)
        np.testing.assert_allclose(N, Nd, atol=1e-12)
        Rfull[:j * s, j * s:(j + 1) * s] = P
        Rfull[j * s:(j + 1) * s, j * s:(j + 1) * s] = N
        np.testing.assert_allclose(B.tree_gram(), np.eye(B.k), atol=1e-13)
        if local != "hh":
            G1 = B.Qloc[1].T @ B.Qloc[1]
            assert np.all(G1 == 0.0)  # chunk 1 never saw a nonzero value
            for Qi in B.Qloc:
                G = Qi.T @ Qi
                d = np.diag(G)
                assert np.all((np.abs(d - 1) < 1e-13) | (d == 0.0))
                np.testing.assert_allclose(G - np.diag(d), 0, atol=1e-13)
    A = np.hstack(Xs)
    Ql, Rl = _lapack_qr(A)
    np.testing.assert_allclose(B.explicit(), Ql, atol=1e-12)
    np.testing.assert_allclose(Rfull, Rl, atol=1e-11 * np.abs(Rl).max())
    assert O.e_perp(B.explicit()) < 1e-13


def test_block_vanishing_everywhere_in_one_column_breaks_down():
    """A column that is zero on every chunk is a global rank deficiency (the
    deflation case), which the Cholesky reduction reports."""
    n, s = 512, 3
    B = O.LocallyOrthogonalBasis(n, s, 128)
    X = I.localized(n, s, 9, [[(0, 512)], [], [(100, 300)]])
    with pytest.raises(O.Breakdown):
        B.orthogonalize(X, "pip2", "pip2")


@pytest.mark.parametrize("local,reduction", [("hh", "hh"), ("pip2", "pip2")])
def test_power_of_two_scaling_commutes(local, reduction):
    """The PQR of 2^j X is (U, 2^j P, 2^j N) (eq. (pqr) is homogeneous in X);
    products, sums, quotients and square roots commute with power-of-two
    scaling, so the oracle's results scale bit for bit."""
    n, s, cr = 600, 3, 128
    Xs = [I.gaussian(n, s, 4400 + j) for j in range(3)]
    runs = {}
    for j in (0, 300, -300):
        B = O.LocallyOrthogonalBasis(n, s, cr)
        runs[j] = [B.orthogonalize(np.ldexp(X, j), local, reduction) for X in Xs]
    for j in (300, -300):
        for (U, P, N), (U0, P0, N0) in zip(runs[j], runs[0]):
            assert np.array_equal(U, U0)
            assert np.array_equal(P, np.ldexp(P0, j))
            assert np.array_equal(N, np.ldexp(N0, j))


# ------------------------------------------------ definitions in closed form

def test_chunk_bounds_reading():
    """p = max(1, floor(n / chunk_rows)) chunks of chunk_rows rows, the
    remainder joining the last (the reading of Sec. 5.1.3 for other n)."""
    assert O.chunk_bounds(777, 100) == [(0, 100), (100, 200), (200, 300), (300, 400), (400, 500),
                                        (500, 600), (600, 777)]
    assert O.chunk_bounds(800, 100)[-1] == (700, 800) and len(O.chunk_bounds(800, 100)) == 8
    assert O.chunk_bounds(99, 100) == [(0, 99)]


def test_error_measures_closed_form():
    """e_perp = ||I - Q^T Q||_F (eq. (ortho_error)) and the residual is
    ||A - QR||_F / ||A||_F: values where the Frobenius and spectral norms, and
    the relative and absolute residuals, differ."""
    Q = 2.0 * np.eye(3)[:, :2]                  # I - Q^T Q = -3 I_2
    assert O.e_perp(Q) == pytest.approx(3.0 * np.sqrt(2.0), rel=1e-15)
    A = 2.0 * np.eye(2)
    assert O.residual(A, np.eye(2), np.eye(2)) == pytest.approx(0.5, rel=1e-15)
    Qw = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    R = np.array([[1.0, 2.0], [0.0, 3.0]])
    Aw = Qw @ R
    Aw[2, 1] = 4.0                              # A - QR = 4 e_3 e_2^T
    assert O.residual(Aw, Qw, R) == pytest.approx(4.0 / np.sqrt(1 + 4 + 9 + 16), rel=1e-15)


# --- deflation (Sec. 3: t < s, kept as t = s with zero rows of N) ----------

def _deficient_block(n, k, seed):
    """Q (n x k orthonormal) and X (n x 6) whose column 2 = col 0 + 2 col 1,
    column 4 lies in span(Q) and column 5 = col 3 - col 0 + Q c: rank 3
    against Q, the dependent columns at 2, 4 and 5."""
    Q = _orthonormal(n, k, seed)
    G = I.gaussian(n, 6, seed + 1)
    X = G.copy()
    X[:, 2] = G[:, 0] + 2.0 * G[:, 1]
    X[:, 4] = Q @ I.gaussian(k, 1, seed + 2)[:, 0]
    X[:, 5] = G[:, 3] - G[:, 0] + Q @ I.gaussian(k, 1, seed + 3)[:, 0]
    return Q, X


def test_deflate_full_rank_is_mgs2():
    Q = _orthonormal(300, 5, 901)
    X = I.gaussian(300, 4, 902)
    for a, b in zip(O.pqr_mgs2_deflate(Q, X, 1e-8), O.pqr_mgs2(Q, X)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("k", [0, 7])
def test_deflate_exact_dependencies(k):
    """Exactly dependent columns: the kept count equals LAPACK's numerical
    rank of (I - Q Q^T) X (an SVD), the dropped ones are the dependent
    positions, kept columns of U are orthonormal and orthogonal to Q, dropped
    ones and their rows of N are zero, and X = Q P + U N."""
    n = 400
    Q, X = _deficient_block(n, k, 903 + k)
    if k == 0:
        X[:, 4] = 0.5 * X[:, 1]
        X[:, 5] = X[:, 3] - X[:, 0]
    U, P, N = O.pqr_mgs2_deflate(Q, X, 1e-8)
    Xp = X - Q @ (Q.T @ X) if k else X
    rank = np.linalg.matrix_rank(Xp, tol=1e-8 * np.linalg.norm(X))
    kept = np.flatnonzero(np.diag(N) != 0.0)
    assert len(kept) == rank == 3
    assert list(np.flatnonzero(np.diag(N) == 0.0)) == [2, 4, 5]
    for j in (2, 4, 5):
        assert np.all(U[:, j] == 0.0) and np.all(N[j, :] == 0.0)
    assert np.allclose(np.triu(N), N, atol=0.0)
    Uk = U[:, kept]
    assert np.linalg.norm(Uk.T @ Uk - np.eye(len(kept))) < 1e-14
    if k:
        assert np.linalg.norm(Q.T @ U) < 1e-14
    assert np.linalg.norm(X - Q @ P - U @ N) <= 1e-14 * np.linalg.norm(X)


def test_deflate_spans_the_svd_truncated_normalizer():
    """Sec. 3's deflation: the eigendecomposition G - P^T P = V S V^T with the
    small values dropped gives U' = (X - Q P) V_t S_t^{-1/2}; the deflated
    Gram-Schmidt spans the same space (projectors agree)."""
    Q, X = _deficient_block(500, 6, 910)
    U, P, N = O.pqr_mgs2_deflate(Q, X, 1e-8)
    P0 = Q.T @ X
    lam, V = np.linalg.eigh(X.T @ X - P0.T @ P0)
    keep = lam > 1e-12 * lam.max()
    Us = (X - Q @ P0) @ V[:, keep] / np.sqrt(lam[keep])[None, :]
    Uk = U[:, np.diag(N) != 0.0]
    assert Us.shape[1] == Uk.shape[1] == 3
    assert np.linalg.norm(Uk @ Uk.T - Us @ Us.T) < 1e-12


def test_deflate_threshold_closed_form():
    """A column at distance eta from the span of the others is dropped iff
    eta <= delta ||X||_F."""
    n, delta = 256, 1e-6
    X = I.gaussian(n, 3, 920)
    e = I.gaussian(n, 1, 921)[:, 0]
    B = X[:, :2]
    e -= B @ np.linalg.lstsq(B, e, rcond=None)[0]
    e /= np.linalg.norm(e)
    for factor, dropped in ((0.5, True), (2.0, False)):
        Y = X.copy()
        Y[:, 2] = X[:, 0] - X[:, 1]
        nrm = np.linalg.norm(Y)  # ||X||_F barely moves with eta this small
        Y[:, 2] += factor * delta * nrm * e
        _, _, N = O.pqr_mgs2_deflate(np.zeros((n, 0)), Y, delta)
        assert (N[2, 2] == 0.0) == dropped, factor


def test_cholesky_deflation_rows():
    """cholesky_upper with a deflation threshold: the Gram of a block with a
    dependent column gets a zero row exactly there, and N^T N reproduces the
    Gram to rounding on the rest."""
    X = I.gaussian(200, 4, 930)
    X[:, 1] = 3.0 * X[:, 0]
    G = X.T @ X
    N = O.cholesky_upper(G, 1e-20 * np.trace(G) + 1e-12 * np.trace(G))
    assert np.all(N[1] == 0.0) and np.all(np.diag(N)[[0, 2, 3]] > 0)
    assert np.linalg.norm(N.T @ N - G) <= 1e-12 * np.linalg.norm(G)
    N0 = O.cholesky_upper(G)           # without deflation: a rounding-level pivot, kept
    assert N0[1, 1] ** 2 <= 1e-12 * np.trace(G)


@pytest.mark.parametrize("chunk", [64, 150, 1000])
def test_tree_tspqr_with_deflation_equals_the_definition(chunk):
    """TreeTSPQR (Alg. 9) with deflating BCGS-PIP+ sub-algorithms (delta =
    1e-6: the Gram pivots resolve distances down to about sqrt(eps) ||X||)
    on a basis of two blocks, then the deficient block: U, P, N equal the
    plain definition (pqr_mgs2_deflate on the explicit basis); the next
    full-rank block still works and the representation stays orthonormal on
    the kept columns."""
    n, s = 1000, 6
    ora = O.LocallyOrthogonalBasis(n, s, chunk)
    for j in range(2):
        ora.orthogonalize(I.gaussian(n, s, 940 + j), "pip2", "pip2")
    Qx = ora.explicit()
    _, X = _deficient_block(n, 12, 950)
    X[:, 4] = Qx @ I.gaussian(12, 1, 951)[:, 0]
    X[:, 5] = X[:, 3] - X[:, 0] + Qx @ I.gaussian(12, 1, 952)[:, 0]
    Uo, Po, No = O.pqr_mgs2_deflate(Qx, X, 1e-8)
    U, P, N = ora.orthogonalize(X, "pip2", "pip2", deflation=1e-6)
    assert list(np.flatnonzero(np.diag(N) == 0.0)) == [2, 4, 5]
    assert np.linalg.norm(U - Uo) <= 1e-12 and np.linalg.norm(P - Po) <= 1e-12 * np.linalg.norm(Po)
    assert np.linalg.norm(N - No) <= 1e-12 * np.linalg.norm(No)
    U2, _, N2 = ora.orthogonalize(I.gaussian(n, s, 953), "pip2", "pip2", deflation=1e-6)
    assert np.all(np.diag(N2) > 0)
    Q = ora.explicit()
    kept = np.linalg.norm(Q, axis=0) > 0.5
    assert kept.sum() == 4 * s - 3
    assert np.linalg.norm(Q[:, kept].T @ Q[:, kept] - np.eye(kept.sum())) < 1e-13
