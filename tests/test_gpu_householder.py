"""The Householder leaf (LO_LEAF_HH: Alg. 6 per chunk, on chip) against the
oracle.

At k = 0 each chunk's QR is the unique thin QR with a positive diagonal, so
the local factors Q_i, the tree factors T_i and the outputs U, R are compared
with the oracle's TreeTSPQR with Householder local solvers element by
element; the tall-skinny sweep's condition numbers up to 1e10 are covered
without the shifted retry the Gram-based leaves need there.
"""

import numpy as np
import pytest

from oracle import lo_oracle as O
from paper_2204_13393_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_REL = 1e-10
TOL_PERP = 1e-12
TOL_RES = 1e-13
EPS = np.finfo(float).eps


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


def hh_chunk_rows(s):
    """The largest power-of-two chunk whose tile (with a remainder of up to
    half a chunk) fits the 200 KiB tile."""
    cr = 2048
    while int(1.5 * cr) * s * 8 > 200 * 1024:
        cr //= 2
    return cr


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e10])
@pytest.mark.parametrize("s", [1, 2, 3, 4, 8, 16, 32])
def test_householder_leaf_tsqr(s, kappa, precision):
    """k = 0 with the Householder leaf: U, R and the local representation
    against the oracle's Householder TreeTSPQR, U^T U = I and A = U R to
    float64 accuracy, one local pass."""
    if precision == "fp64_tc" and s == 3:
        pytest.skip("s = 3 has no tensor-core form")
    cr = hh_chunk_rows(s)
    n = 9 * cr + cr // 2 + 3   # ragged last chunk
    A = I.stewart(n, s, kappa, I.seed_for(8, 10 * s + int(np.log10(kappa))))
    b = lo().Basis(n, s, 1, cr, precision=precision, leaf="hh")
    U, _, R = b.orthogonalize(dev(A))
    Ug, Rg = host(U), host(R)
    assert O.e_perp(Ug) <= TOL_PERP
    assert O.residual(A, Ug, Rg) <= TOL_RES
    assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)
    assert b.last_step_info()[0] == 1
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    Uo, _, No = ora.orthogonalize(A, "hh", "hh")
    tol = max(TOL_REL, 100 * kappa * EPS)
    assert close(Ug, Uo, tol), errs(Ug, Uo)
    assert close(Rg, No, tol), errs(Rg, No)
    for c in (0, 4, b.num_chunks - 1):
        Qi, Ti = b.export_chunk(c)
        assert close(Qi, ora.Qloc[c], tol), (c, errs(Qi, ora.Qloc[c]))
        assert O.e_perp(Qi) <= TOL_PERP
        assert close(Ti, np.triu(ora.T[c]), tol), (c, errs(Ti, np.triu(ora.T[c])))


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_householder_leaf_then_pip2(precision):
    """A multi-block basis with the Householder leaf: the first block by
    Householder, the next ones by BCGS-PIP+ (with digit planes of the
    Householder panel in the tensor-core form); every output, the explicit
    basis and the representation against the oracle."""
    s, M = 8, 5
    cr = hh_chunk_rows(s)
    n = 9 * cr + 1000          # the last chunk (with the remainder) still fits the tile
    L = lo()
    b = L.Basis(n, s, M, cr, precision=precision, leaf="hh")
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    for j in range(M):
        W = I.gaussian(n, s, I.seed_for(8, 500 + j))
        U, H, R = b.orthogonalize(dev(W))
        Uo, Po, No = ora.orthogonalize(W, "hh", "hh")
        assert close(host(U), Uo), (j, errs(host(U), Uo))
        assert close(host(R), No), (j, errs(host(R), No))
        if j:
            assert close(host(H), Po), (j, errs(host(H), Po))
    Q = host(b.apply_Q(dev(np.eye(b.k))))
    assert O.e_perp(Q) <= TOL_PERP
    assert close(Q, ora.explicit())
    for c in (0, b.num_chunks - 1):
        Qi, Ti = b.export_chunk(c)
        assert close(Qi, ora.Qloc[c]) and close(Ti, np.triu(ora.T[c])), c


def test_householder_leaf_vanishing_chunks():
    """Columns that are exactly zero on whole chunks: the Householder leaf
    keeps the unit direction there (no reflection, R_jj = 0), as the oracle's
    Householder solver does; U and R are the unique solution."""
    s = 8
    cr = hh_chunk_rows(s)
    n = 11 * cr + 700
    bounds = O.chunk_bounds(n, cr)
    sup = [[bounds[(2 * c) % len(bounds)], bounds[(2 * c + 5) % len(bounds)]] for c in range(s)]
    W = I.localized(n, s, I.seed_for(8, 600), sup)
    b = lo().Basis(n, s, 1, cr, leaf="hh")
    U, _, R = b.orthogonalize(dev(W))
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    Uo, _, No = ora.orthogonalize(W, "hh", "hh")
    assert close(host(U), Uo) and close(host(R), No)
    for c in range(b.num_chunks):
        Qi, Ti = b.export_chunk(c)
        assert close(Qi, ora.Qloc[c]) and close(Ti, np.triu(ora.T[c])), c
        assert O.e_perp(Qi) <= TOL_PERP


def test_householder_leaf_nonfinite_and_tuner():
    """A NaN in the block is reported with the basis unchanged; the chunk-size
    tuner only proposes chunks whose tiles fit, and the tuned basis is
    orthonormal."""
    L = lo()
    s = 8
    cr = hh_chunk_rows(s)
    n = 24 * cr + 333
    b = L.Basis(n, s, 2, cr, leaf="hh")
    W = I.gaussian(n, s, I.seed_for(8, 700))
    W[1234, 3] = np.nan
    with pytest.raises(L.LoError) as e:
        b.orthogonalize(dev(W))
    assert e.value.name == "LO_ERR_NONFINITE"
    assert b.num_blocks == 0
    crt = L.tune_chunk_rows(n, s, 1, precision="fp64", leaf="hh")
    assert crt * s * 8 <= 200 * 1024
    bt = L.Basis(n, s, 1, crt, leaf="hh")
    U, _, R = bt.orthogonalize(dev(I.gaussian(n, s, I.seed_for(8, 701))))
    assert O.e_perp(host(U)) <= TOL_PERP


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
@pytest.mark.parametrize("kappa", [1e2, 1e10])
@pytest.mark.parametrize("s,cr", [(1, 65536), (3, 30000), (8, 16384), (16, 6000), (32, 4096)])
def test_householder_flat_chunks(s, cr, kappa, precision):
    """Chunks larger than one shared-memory tile: the Householder leaf walks
    them as sub-tiles in FlatTSPQR order (each factored under the previous R,
    the local factor formed backwards).  The chunk's QR is unique, so Q_i,
    T_i, U and R match the oracle's Householder QR of the whole chunk."""
    if precision == "fp64_tc" and s == 3:
        pytest.skip("s = 3 has no tensor-core form")
    n = 3 * cr + cr // 3 + 5
    A = I.stewart(n, s, kappa, I.seed_for(8, 800 + s + int(np.log10(kappa))))
    b = lo().Basis(n, s, 2, cr, precision=precision, leaf="hh")
    U, _, R = b.orthogonalize(dev(A))
    Ug, Rg = host(U), host(R)
    assert b.last_step_info()[0] == 1
    assert O.e_perp(Ug) <= TOL_PERP
    assert O.residual(A, Ug, Rg) <= TOL_RES
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    Uo, _, No = ora.orthogonalize(A, "hh", "hh")
    tol = max(TOL_REL, 100 * kappa * EPS)
    # R is well determined (element by element); U and Q_i element by element
    # only where their forward-error bound kappa eps is small, else in norm
    # (their backward errors, e_perp and the residual, are checked above)
    assert close(Rg, No), errs(Rg, No)
    cmp = close if kappa * EPS <= 1e-10 else (lambda x, y, t: errs(x, y)[0] <= t)
    assert cmp(Ug, Uo, tol), errs(Ug, Uo)
    for c in range(b.num_chunks):
        Qi, Ti = b.export_chunk(c)
        assert cmp(Qi, ora.Qloc[c], tol), (c, errs(Qi, ora.Qloc[c]))
        assert O.e_perp(Qi) <= TOL_PERP
        assert cmp(Ti, np.triu(ora.T[c]), tol), c
    # the basis goes on past the flat leaf (BCGS-PIP+ with the flat panel as prior block)
    W = I.gaussian(n, s, I.seed_for(8, 900 + s))
    U2, H2, R2 = b.orthogonalize(dev(W))
    Uo2, Po2, No2 = ora.orthogonalize(W, "hh", "hh")
    assert cmp(host(U2), Uo2, tol) and cmp(host(H2), Po2, tol) and cmp(host(R2), No2, tol)


@pytest.mark.parametrize("M", [1, 4])
def test_leaf_tuner(M):
    """lo_tune_leaf returns one of the two leaves with a chunk size the basis
    accepts; the tuned basis orthogonalizes to float64 accuracy."""
    L = lo()
    n, s = 300000, 8
    leaf, cr = L.tune_leaf(n, s, M, precision="fp64_tc")
    assert leaf in ("pip2", "hh") and cr >= 256
    b = L.Basis(n, s, M, cr, precision="fp64_tc", leaf=leaf)
    U, _, R = b.orthogonalize(dev(I.gaussian(n, s, I.seed_for(8, 950))))
    assert O.e_perp(host(U)) <= TOL_PERP
