"""Parity with the oracle at the depths the benchmark runs.

The block-GMRes workload orthogonalizes 31 blocks (k up to 240 columns at
s = 8); the mixed-precision workload steps at k = 480 with s = 16.  These
tests run the same depths at reduced n (16k-20k rows, several chunks, so the
tensor-core kernels run their column groups, output flushes and digit planes
at full depth) and compare every output of every step with the CPU oracle,
element by element and in relative Frobenius norm.

Inputs never come from the CUDA path: the Krylov-like sequences are the
oracle's own block Arnoldi (Alg. 1) with a 2D 5-point Laplacian, i.e. block
j + 1 is the operator applied to the oracle's block j; both sides
orthogonalize the same blocks.  The oracle steps use BCGS-PIP+ local solvers
(cheap at depth) and a Householder reduction; at chosen steps the outputs are
also checked against the plain definition of the PQR step (oracle A: the
sign-normalized Householder QR of [Q X] with the oracle's explicit basis Q).
"""

import copy
import functools

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
    """(relative Frobenius error, largest element error relative to max|b|)."""
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    mb = np.abs(b).max()
    return (np.linalg.norm(a - b) / (nb if nb > 0 else 1.0),
            np.abs(a - b).max() / (mb if mb > 0 else 1.0))


def close(a, b, tol=TOL_REL):
    f, e = errs(a, b)
    return f <= tol and e <= tol


def lap2d(V, nx, ny):
    """y = L v for the 2D 5-point Dirichlet Laplacian, columns of V (n x s, n = nx ny)."""
    G = V.reshape(ny, nx, -1)
    out = 4 * G
    out[:, 1:] -= G[:, :-1]
    out[:, :-1] -= G[:, 1:]
    out[1:] -= G[:-1]
    out[:-1] -= G[1:]
    return out.reshape(nx * ny, -1)


@pytest.mark.parametrize("s,nx,ny,cr,check_at,reduction", [
    (8, 160, 128, 4096, (15, 30), "hh"),    # k up to 240: two Gram column groups, 31 panels
    (16, 128, 128, 2048, (30,), "pip2"),    # k up to 480 (the mixed workload's depth)
])
def test_arnoldi_depth_every_step(s, nx, ny, cr, check_at, reduction):
    """31 blocks of block Arnoldi (Alg. 1) on the tensor-core form with digit
    planes: every step's U, H, R against the oracle TreeTSPQR (element by
    element), selected steps against oracle A, and at the end the local
    representation (Q_i, T_i), ||Q^T Q - I|| and ||A - QR|| / ||A||."""
    n, m = nx * ny, 31
    L = lo()
    b = L.Basis(n, s, m, cr, precision="fp64_tc")
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    W = I.uniform(n, s, I.seed_for(2, 50 + s))
    A = []
    Rfull = np.zeros((m * s, m * s))
    for j in range(m):
        A.append(W)
        if j in check_at:
            Qx = ora.explicit()
        U, H, R = b.orthogonalize(dev(W))
        Uo, Po, No = ora.orthogonalize(W, "pip2", reduction)
        Ug, Rg = host(U), host(R)
        assert close(Ug, Uo), (j, errs(Ug, Uo))
        assert close(Rg, No), (j, errs(Rg, No))
        assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0), j
        if j:
            Hg = host(H)
            assert close(Hg, Po), (j, errs(Hg, Po))
            Rfull[:j * s, j * s:(j + 1) * s] = Hg
        Rfull[j * s:(j + 1) * s, j * s:(j + 1) * s] = Rg
        if j in check_at:
            Ua, Pa, Na = O.pqr_householder(Qx, W)
            assert close(Ug, Ua), (j, errs(Ug, Ua))
            assert close(Rg, Na), (j, errs(Rg, Na))
            assert close(host(H), Pa), (j, errs(host(H), Pa))
        W = lap2d(Uo, nx, ny)      # the oracle's next Krylov block
    Q = host(b.apply_Q(dev(np.eye(m * s))))
    assert O.e_perp(Q) <= TOL_PERP
    assert O.residual(np.hstack(A), Q, Rfull) <= TOL_RES
    assert close(Q, ora.explicit())
    for c in range(b.num_chunks):
        Qi, Ti = b.export_chunk(c)
        assert close(Qi, ora.Qloc[c]), (c, errs(Qi, ora.Qloc[c]))
        assert close(Ti, np.triu(ora.T[c])), (c, errs(Ti, np.triu(ora.T[c])))


# --- the mixed workload's shape: s = 16, 30 prior blocks (k = 480) ---------

MIX_N, MIX_S, MIX_KB, MIX_CR = 8192, 16, 30, 1024


@functools.lru_cache(maxsize=None)
def _mixed_prior():
    """The 30 prior Gaussian blocks and the oracle basis built from them."""
    blocks = [I.gaussian(MIX_N, MIX_S, I.seed_for(4, j)) for j in range(MIX_KB)]
    ora = O.LocallyOrthogonalBasis(MIX_N, MIX_S, MIX_CR)
    outs = [ora.orthogonalize(W, "pip2", "pip2") for W in blocks]
    return blocks, ora, outs


@functools.lru_cache(maxsize=None)
def _mixed_block(kappa):
    """A Stewart block U diag(sigma) V^T with condition kappa plus a component
    along the last prior block (a Krylov-like block), and the oracle's step on
    it with Householder local and reduction solvers (Alg. 9 with Alg. 6)."""
    blocks, ora, _ = _mixed_prior()
    W = I.stewart(MIX_N, MIX_S, kappa, I.seed_for(4, 100 + int(np.log10(kappa))))
    W = W + 0.5 * blocks[-1] / np.sqrt(MIX_N)
    o = copy.deepcopy(ora)
    Uo, Po, No = o.orthogonalize(W, "hh", "hh")
    return W, Uo, Po, No, o.explicit()


@pytest.mark.parametrize("precision", ["fp64_tc", "mixed_tc", "mixed_fp32"])
def test_mixed_workload_shape_vs_oracle(precision):
    """n = 8192, s = 16, 30 prior blocks (k = 480), 1024-row chunks: the prior
    steps against the oracle element by element, then a Stewart block with
    kappa in {1e2, 1e4, 1e6} (each from the same 30-block basis): U, H, R
    within max(1e-10, 100 kappa eps) of the oracle's Householder step (their
    forward error grows with kappa), ||Q^T Q - I|| <= 1e-12 and
    ||[Q W] - [Q U][[I, H], [0, R]]|| <= 1e-13 ||[Q W]|| for the new basis."""
    blocks, _, outs = _mixed_prior()
    L = lo()
    b = L.Basis(MIX_N, MIX_S, MIX_KB + 1, MIX_CR, precision=precision)
    for j, (W, (Uo, Po, No)) in enumerate(zip(blocks, outs)):
        U, H, R = b.orthogonalize(dev(W))
        assert close(host(U), Uo), (j, errs(host(U), Uo))
        assert close(host(R), No), (j, errs(host(R), No))
        if j:
            assert close(host(H), Po), (j, errs(host(H), Po))
    report = {}
    for kappa in (1e2, 1e4, 1e6):
        W, Uo, Po, No, Qo = _mixed_block(kappa)
        b.truncate(MIX_KB)
        U, H, R = b.orthogonalize(dev(W))
        Ug, Hg, Rg = host(U), host(H), host(R)
        tol = max(TOL_REL, 100 * kappa * EPS)
        report[kappa] = (errs(Ug, Uo), errs(Hg, Po), errs(Rg, No))
        assert close(Ug, Uo, tol), (kappa, report[kappa])
        assert close(Hg, Po, tol), (kappa, report[kappa])
        assert close(Rg, No, tol), (kappa, report[kappa])
        assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)
        Q = host(b.apply_Q(dev(np.eye(b.k))))
        assert O.e_perp(Q) <= TOL_PERP, (kappa, O.e_perp(Q))
        assert close(Q, Qo, tol), (kappa, errs(Q, Qo))
        k = MIX_KB * MIX_S
        Rf = np.eye(k + MIX_S)
        Rf[:k, k:] = Hg
        Rf[k:, k:] = Rg
        QW = np.hstack([Q[:, :k], W])
        assert np.linalg.norm(QW - Q @ Rf) <= TOL_RES * np.linalg.norm(QW), kappa
    print(f"{precision}: (U, H, R) errors vs the oracle per kappa: {report}")


# --- values spread over 30 decades inside one column of one chunk ----------

def graded_blocks(n, s, cr, count, seed0):
    """Gaussian blocks in which one column, on the rows of chunk 1, is scaled
    by 10^(-30 u) with u uniform in [0, 1) (seeded): magnitudes from 1 down to
    1e-30 inside one column of one chunk, where the digit forms align every
    value to the column's largest exponent on that chunk."""
    b, e = O.chunk_bounds(n, cr)[1]
    out = []
    for j in range(count):
        W = I.gaussian(n, s, seed0 + j)
        u = (I.uniform(e - b, 1, seed0 + 50 + j)[:, 0] + 1.0) / 2.0
        W[b:e, j % s] *= 10.0 ** (-30.0 * u)
        out.append(W)
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc", "mixed_tc"])
@pytest.mark.parametrize("s", [8, 16])
def test_graded_magnitudes_inside_a_column(precision, s):
    """Every block (k = 0 and with prior blocks, so both the k = 0 kernels and
    the digit planes of the prior panels see graded columns) against the
    oracle's Householder TreeTSPQR, element by element, plus the local
    representation.  Entries far below a column's largest one on a chunk
    contribute below float64 rounding of the products they enter, so the
    float64 tolerance holds."""
    n, cr, M = 20000, 4096, 4
    blocks = graded_blocks(n, s, cr, M, I.seed_for(6, s))
    L = lo()
    b = L.Basis(n, s, M, cr, precision=precision)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    for j, W in enumerate(blocks):
        U, H, R = b.orthogonalize(dev(W))
        Uo, Po, No = ora.orthogonalize(W, "hh", "hh")
        assert close(host(U), Uo), (j, errs(host(U), Uo))
        assert close(host(R), No), (j, errs(host(R), No))
        if j:
            assert close(host(H), Po), (j, errs(host(H), Po))
    Q = host(b.apply_Q(dev(np.eye(b.k))))
    assert O.e_perp(Q) <= TOL_PERP
    assert close(Q, ora.explicit())
    if precision != "mixed_tc":
        for c in range(b.num_chunks):
            Qi, Ti = b.export_chunk(c)
            assert close(Qi, ora.Qloc[c]), (c, errs(Qi, ora.Qloc[c]))
            assert close(Ti, np.triu(ora.T[c])), (c, errs(Ti, np.triu(ora.T[c])))
