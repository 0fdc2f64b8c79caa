"""The block-Arnoldi step with the 5-point Laplacian fused into the first Gram
pass (lo_orthogonalize_laplace5) against lo_laplace5_apply followed by
lo_orthogonalize (bit for bit) and against the oracle's block Arnoldi
(Alg. 1) with the same operator, element by element.

Both GPU runs take as V the oracle's previous Krylov block, so every input
comes from the oracle; the oracle's operator subtracts the four neighbours in
the same order as the library's, so L V is the same on both sides.
"""

import numpy as np
import pytest

from oracle import lo_oracle as O
from paper_2204_13393_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_REL = 1e-10


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
    nb = np.linalg.norm(b)
    mb = np.abs(b).max()
    return (np.linalg.norm(a - b) / (nb if nb > 0 else 1.0), np.abs(a - b).max() / (mb if mb > 0 else 1.0))


def close(a, b, tol=TOL_REL):
    f, e = errs(a, b)
    return f <= tol and e <= tol


def lap2d(V, nx, ny):
    G = V.reshape(ny, nx, -1)
    out = 4 * G
    out[:, 1:] -= G[:, :-1]
    out[:, :-1] -= G[:, 1:]
    out[1:] -= G[:-1]
    out[:-1] -= G[1:]
    return out.reshape(nx * ny, -1)


@pytest.mark.parametrize("precision,s", [
    ("fp64", 8), ("fp64", 3), ("fp64", 16),          # float64 Grams: the stencil inside k_gram1 / k_gram
    ("fp64_tc", 8), ("fp64_tc", 16), ("fp64_tc", 32),  # tcgen05 Gram over digit planes: inside its producers
    ("fp64_tc", 4), ("mixed_tc", 8),                 # no on-the-fly form: the operator kernel first
])
def test_fused_operator_step(precision, s):
    nx, ny, m, cr = 96, 80, 6, 1024
    n = nx * ny
    L = lo()
    bf = L.Basis(n, s, m + 1, cr, precision=precision)
    bu = L.Basis(n, s, m + 1, cr, precision=precision)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    R0 = I.uniform(n, s, I.seed_for(13, s))
    bf.orthogonalize(dev(R0))
    bu.orthogonalize(dev(R0))
    Uo, _, _ = ora.orthogonalize(R0, "pip2", "pip2")
    tol = TOL_REL if precision != "mixed_tc" else 1e-9
    for j in range(m):
        V = dev(Uo)
        Uf = torch.empty(n, s, dtype=torch.float64, device="cuda")
        U1, H1, R1 = bf.orthogonalize_laplace5(nx, ny, V, U=Uf)
        X = L.laplace5_apply(nx, ny, V, torch.empty(n, s, dtype=torch.float64, device="cuda"))
        U2, H2, R2 = bu.orthogonalize(X)
        for x, y in ((U1, U2), (H1, H2), (R1, R2)):
            assert np.array_equal(host(x), host(y)), j
        W = lap2d(Uo, nx, ny)
        assert np.array_equal(host(X), W)
        Uo, Po, No = ora.orthogonalize(W, "pip2", "pip2")
        assert close(host(U1), Uo, tol) and close(host(H1), Po, tol) and close(host(R1), No, tol), \
            (j, errs(host(U1), Uo), errs(host(R1), No))
    Q = host(bf.apply_Q(dev(np.eye(bf.k))))
    assert O.e_perp(Q) <= 1e-12


def test_fused_operator_arguments():
    L = lo()
    nx, ny, s = 40, 30, 4
    b = L.Basis(nx * ny, s, 3, 400)
    V = dev(I.uniform(nx * ny, s, 1))
    b.orthogonalize(V)
    with pytest.raises(L.LoError):
        b.orthogonalize_laplace5(nx + 1, ny, V)            # n != nx ny
    with pytest.raises(L.LoError):
        b.orthogonalize_laplace5(nx, ny, V, U=V)           # U overlaps V
    assert b.num_blocks == 1
