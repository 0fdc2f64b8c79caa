"""Deflation (Sec. 3: t < s, kept as t = s with zero rows of R) against the
oracle.

A block with exactly dependent columns -- one a combination of earlier
columns, one in the span of the basis, one both -- is orthogonalized with
deflation on: the dropped columns of U and rows of R are exactly zero, the
kept part matches the plain definition (Gram-Schmidt twice with the drop
rule, on the oracle's explicit basis) and the oracle's TreeTSPQR with
deflating BCGS-PIP+ solvers element by element, and the basis goes on
working.
"""

import numpy as np
import pytest

from oracle import lo_oracle as O
from paper_2204_13393_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_REL = 1e-10
TOL_PERP = 1e-12
DELTA = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_13393_gb300 import lo

    lo.library()
    torch.cuda.set_device(0)


def lo():
    from paper_2204_13393_gb300 import lo as L

    return L


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(x):
    torch.cuda.synchronize()
    return x.detach().cpu().numpy()


def errs(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    mb = np.abs(b).max()
    return (np.linalg.norm(a - b) / (nb if nb > 0 else 1.0), np.abs(a - b).max() / (mb if mb > 0 else 1.0))


def close(a, b, tol=TOL_REL):
    f, e = errs(a, b)
    return f <= tol and e <= tol


def deficient(Qx, n, s, seed):
    """Columns 2 = col 0 + 2 col 1, 4 in span(Q), 5 = col 3 - col 0 + Q c."""
    X = I.gaussian(n, s, seed)
    k = Qx.shape[1]
    X[:, 2] = X[:, 0] + 2.0 * X[:, 1]
    if k:
        X[:, 4] = Qx @ I.gaussian(k, 1, seed + 1)[:, 0]
        X[:, 5] = X[:, 3] - X[:, 0] + Qx @ I.gaussian(k, 1, seed + 2)[:, 0]
    else:
        X[:, 4] = 0.25 * X[:, 1]
        X[:, 5] = X[:, 3] - X[:, 0]
    return X


@pytest.mark.parametrize("precision,leaf,cr", [
    ("fp64", "pip2", 1000), ("fp64_tc", "pip2", 1000), ("fp64_tc", "pip2", 4096), ("fp64", "auto", 700),
])
def test_deflated_block_matches_oracle(precision, leaf, cr):
    n, s, M = 12000, 8, 5
    L = lo()
    b = L.Basis(n, s, M, cr, precision=precision, leaf=leaf, deflation_tol=DELTA)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    for j in range(2):
        W = I.gaussian(n, s, I.seed_for(11, j))
        U, H, R = b.orthogonalize(dev(W))
        Uo, Po, No = ora.orthogonalize(W, "pip2", "pip2", deflation=DELTA)
        assert close(host(U), Uo) and close(host(R), No)
        assert b.last_rank() == s
    Qx = ora.explicit()
    X = deficient(Qx, n, s, I.seed_for(11, 10))
    U, H, R = b.orthogonalize(dev(X))
    Ug, Hg, Rg = host(U), host(H), host(R)
    assert b.last_rank() == 5
    assert list(np.flatnonzero(np.diag(Rg) == 0.0)) == [2, 4, 5]
    for j in (2, 4, 5):
        assert np.all(Ug[:, j] == 0.0) and np.all(Rg[j, :] == 0.0)
    Ud, Pd, Nd = O.pqr_mgs2_deflate(Qx, X, DELTA)
    assert close(Ug, Ud) and close(Hg, Pd) and close(Rg, Nd), (errs(Ug, Ud), errs(Hg, Pd), errs(Rg, Nd))
    Uo, Po, No = ora.orthogonalize(X, "pip2", "pip2", deflation=DELTA)
    assert close(Ug, Uo) and close(Hg, Po) and close(Rg, No)
    # the next full-rank block
    W = I.gaussian(n, s, I.seed_for(11, 20))
    U, H, R = b.orthogonalize(dev(W))
    Uo, Po, No = ora.orthogonalize(W, "pip2", "pip2", deflation=DELTA)
    assert close(host(U), Uo) and close(host(H), Po) and close(host(R), No)
    Q = host(b.apply_Q(dev(np.eye(b.k))))
    kept = np.linalg.norm(Q, axis=0) > 0.5
    assert kept.sum() == b.k - 3
    assert np.all(Q[:, ~kept] == 0.0)
    assert O.e_perp(Q[:, kept]) <= TOL_PERP
    assert close(Q, ora.explicit())


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_block_entirely_in_the_span_deflates_to_rank_zero(precision):
    """W = Q C: every column is dropped, U = 0, R = 0 and H = C."""
    n, s, cr = 8000, 8, 1000
    L = lo()
    b = L.Basis(n, s, 3, cr, precision=precision, deflation_tol=DELTA)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    W = I.gaussian(n, s, I.seed_for(11, 30))
    b.orthogonalize(dev(W))
    ora.orthogonalize(W, "pip2", "pip2")
    C = I.gaussian(s, s, I.seed_for(11, 31))
    X = ora.explicit() @ C
    U, H, R = b.orthogonalize(dev(X))
    assert b.last_rank() == 0
    assert np.all(host(U) == 0.0) and np.all(host(R) == 0.0)
    assert close(host(H), C)


@pytest.mark.parametrize("leaf", ["pip2", "hh"])
def test_first_block_deficient(leaf):
    """k = 0 with dependent columns (the Householder leaf keeps every local
    column; the reduction drops the dependent ones)."""
    s, cr = 8, 2048
    n = 9 * cr + 1000          # the Householder tile of the last chunk fits
    X = deficient(np.zeros((n, 0)), n, s, I.seed_for(11, 40))
    b = lo().Basis(n, s, 2, cr, leaf=leaf, deflation_tol=DELTA)
    U, _, R = b.orthogonalize(dev(X))
    Ug, Rg = host(U), host(R)
    assert b.last_rank() == 5
    assert list(np.flatnonzero(np.diag(Rg) == 0.0)) == [2, 4, 5]
    Ud, _, Nd = O.pqr_mgs2_deflate(np.zeros((n, 0)), X, DELTA)
    assert close(Ug, Ud) and close(Rg, Nd), (errs(Ug, Ud), errs(Rg, Nd))
    assert np.linalg.norm(X - Ug @ Rg) <= 1e-13 * np.linalg.norm(X)


def test_without_deflation_the_same_block_breaks_down():
    n, s, cr = 8000, 8, 1000
    L = lo()
    b = L.Basis(n, s, 2, cr)
    X = deficient(np.zeros((n, 0)), n, s, I.seed_for(11, 50))
    with pytest.raises(L.LoError) as e:
        b.orthogonalize(dev(X))
    assert e.value.name == "LO_ERR_BREAKDOWN"
    assert b.num_blocks == 0
