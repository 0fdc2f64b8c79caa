"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison uses the same seeded float64 inputs on both sides.  The PQR
solution (U, P, N with diag(N) > 0) and the locally orthogonal representation
(local Q_i and tree factors T_i) are unique, so they are compared element by
element with the oracle's Householder-based TreeTSPQR.

Tolerances (float64 path): relative Frobenius error of U, H, R, Q_i, T_i
<= 1e-10; ||Q^T Q - I||_F <= 1e-12; ||A - QR||_F / ||A||_F <= 1e-13.
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


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def close(a, b, tol=TOL_REL):
    """Relative Frobenius error <= tol and, element by element,
    |a - b| <= tol * max|b| (so no single entry hides in a small norm)."""
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.abs(b).max() if b.size else 0.0
    ew = np.abs(a - b).max() / (scale if scale > 0 else 1.0) if b.size else 0.0
    return rel(a, b) <= tol and ew <= tol


def errs(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    scale = np.abs(b).max() if b.size else 1.0
    return rel(a, b), (np.abs(a - b).max() / (scale if scale > 0 else 1.0) if b.size else 0.0)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(x):
    torch.cuda.synchronize()
    return x.detach().cpu().numpy()


def run_and_compare(n, s, M, cr, blocks, oracle_local="hh", oracle_reduction="hh", check_local=True,
                    **opts):
    """Orthogonalize `blocks` one after another on the GPU and in the oracle;
    compare every output and the representation.  Returns the GPU basis."""
    b = lo().Basis(n, s, M, cr, **opts)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    assert b.num_chunks == len(ora.bounds)
    A = np.hstack(blocks)
    Rfull = np.zeros((A.shape[1], A.shape[1]))
    for j, Wh in enumerate(blocks):
        U, H, R = b.orthogonalize(dev(Wh))
        Uo, Po, No = ora.orthogonalize(Wh, oracle_local, oracle_reduction)
        assert close(host(U), Uo), (j, errs(host(U), Uo))
        assert close(host(R), No), (j, errs(host(R), No))
        if j > 0:
            assert close(host(H), Po), (j, errs(host(H), Po))
            Rfull[:j * s, j * s:(j + 1) * s] = host(H)
        Rfull[j * s:(j + 1) * s, j * s:(j + 1) * s] = host(R)
        assert np.all(np.diag(host(R)) > 0)
        assert np.all(np.tril(host(R), -1) == 0)
    assert b.num_blocks == len(blocks)
    Q = host(b.apply_Q(dev(np.eye(b.k))))
    assert O.e_perp(Q) <= TOL_PERP
    assert O.residual(A, Q, Rfull) <= TOL_RES
    assert close(Q, ora.explicit())
    if check_local:
        Tg = 0
        for c in range(b.num_chunks):
            Qi, Ti = b.export_chunk(c)
            assert close(Qi, ora.Qloc[c]), c
            assert close(Ti, np.triu(ora.T[c])), c
            assert O.e_perp(Qi) <= TOL_PERP
            Tg = Tg + Ti.T @ Ti
        assert np.abs(Tg - np.eye(b.k)).max() <= TOL_PERP
    return b


def gaussian_blocks(n, s, count, seed0):
    return [I.gaussian(n, s, seed0 + j) for j in range(count)]


PRECISIONS = ["fp64", "fp64_tc"]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_arnoldi_step_small_workload(precision):
    """n = 4096, s = 4, chunk_rows = 512: 8 prior blocks from seeded N(0,1)
    blocks, then the new block; outputs H (32 x 4) and R (4 x 4)."""
    n, s = 4096, 4
    b = run_and_compare(n, s, 9, 512, gaussian_blocks(n, s, 9, I.seed_for(1)), precision=precision)
    assert b.k == 36


@pytest.mark.parametrize("n,s,cr,M", [
    (5000, 4, 512, 6),      # ragged last chunk (904 rows), ragged slabs
    (777, 2, 100, 5),       # small chunks, 7 chunks, last 177 rows
    (300, 8, 1000, 4),      # one chunk (n < chunk_rows)
    (2048, 1, 256, 8),      # s = 1
    (4099, 16, 1024, 4),    # s = 16, ragged
    (3000, 32, 1000, 3),    # s = 32 (maximum width)
    (65573, 8, 4096, 6),    # many slabs per chunk, ragged
])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_shapes_and_ragged(n, s, cr, M, precision):
    run_and_compare(n, s, M, cr, gaussian_blocks(n, s, M, 1000 + n + s), precision=precision)


@pytest.mark.parametrize("leaf", ["pip", "pip2", "auto"])
@pytest.mark.parametrize("reduction", ["pip", "pip2", "auto"])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_leaf_and_reduction_modes(leaf, reduction, precision):
    n, s = 6000, 4
    run_and_compare(n, s, 5, 700, gaussian_blocks(n, s, 5, 2000), leaf=leaf, reduction=reduction,
                    check_local=False, precision=precision)


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6, 1e8, 1e10])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_stewart_block_qr(kappa, precision):
    """Alg. 2 on a Stewart matrix (32 columns, s = 4) with the automatic
    reiteration: orthogonality and residual at float64 level; H and R are
    compared with the oracle where their forward error kappa*eps allows."""
    n, m, s = 16384, 32, 4
    A = I.stewart(n, m, kappa, 500 + int(np.log10(kappa)))
    blocks = [A[:, j * s:(j + 1) * s].copy() for j in range(m // s)]
    b = lo().Basis(n, s, m // s, 1024, precision=precision)
    ora = O.LocallyOrthogonalBasis(n, s, 1024)
    Rg = np.zeros((m, m))
    Ro = np.zeros((m, m))
    for j, Wh in enumerate(blocks):
        U, H, R = b.orthogonalize(dev(Wh))
        Uo, Po, No = ora.orthogonalize(Wh, "hh", "hh")
        if j:
            Rg[:j * s, j * s:(j + 1) * s] = host(H)
            Ro[:j * s, j * s:(j + 1) * s] = Po
        Rg[j * s:(j + 1) * s, j * s:(j + 1) * s] = host(R)
        Ro[j * s:(j + 1) * s, j * s:(j + 1) * s] = No
    Q = host(b.apply_Q(dev(np.eye(m))))
    assert O.e_perp(Q) <= TOL_PERP
    assert O.residual(A, Q, Rg) <= TOL_RES
    bound = 100 * kappa * np.finfo(float).eps
    assert rel(Rg, Ro) <= max(TOL_REL, bound)


@pytest.mark.parametrize("s", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e10])
@pytest.mark.parametrize("precision", PRECISIONS)
def test_tall_skinny_qr_sweep(s, kappa, precision):
    """The tall-skinny QR sweep's structure at reduced n (2^18 rows): k = 0,
    A = U diag(sigma) V^T with log-spaced sigma; orthogonality and residual at
    float64 level for every width and condition number; R compared with the
    oracle (Householder TreeTSPQR) within its forward-error bound."""
    n, cr = 2 ** 18, 4096
    A = I.stewart(n, s, kappa, 700 + s + int(np.log10(kappa)))
    b = lo().Basis(n, s, 1, cr, precision=precision)
    U, _, R = b.orthogonalize(dev(A))
    Uh, Rh = host(U), host(R)
    assert O.e_perp(Uh) <= TOL_PERP
    assert O.residual(A, Uh, Rh) <= TOL_RES
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    _, _, Ro = ora.orthogonalize(A, "hh", "hh")
    assert rel(Rh, Ro) <= max(TOL_REL, 100 * kappa * np.finfo(float).eps)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_apply_Q_parity(precision):
    n, s = 9000, 4
    b = lo().Basis(n, s, 6, 1000, precision=precision)
    ora = O.LocallyOrthogonalBasis(n, s, 1000)
    for j in range(6):
        Wh = I.gaussian(n, s, 3000 + j)
        b.orthogonalize(dev(Wh))
        ora.orthogonalize(Wh, "hh", "hh")
    for m in (1, 5, 64):
        C = I.gaussian(b.k, m, 3100 + m)
        Y = host(b.apply_Q(dev(C)))
        assert rel(Y, ora.apply_Q(C)) <= TOL_REL
        # host C and host Y through the same entry point
        Yh = b.apply_Q(C)
        assert np.array_equal(Yh, Y)


def test_host_buffers_match_device_bitwise():
    n, s = 5000, 8
    W = [I.gaussian(n, s, 3200 + j) for j in range(3)]
    bd = lo().Basis(n, s, 3, 512)
    bh = lo().Basis(n, s, 3, 512)
    for Wh in W:
        Ud, Hd, Rd = bd.orthogonalize(dev(Wh))
        Uh, Hh, Rh = bh.orthogonalize(Wh)        # numpy in, numpy out
        assert isinstance(Uh, np.ndarray)
        assert np.array_equal(host(Ud), Uh)
        assert np.array_equal(host(Rd), Rh)
        if Hd is not None:
            assert np.array_equal(host(Hd), Hh)


def test_strided_and_aliased_buffers():
    """W with a row stride > s, and U written over W in place."""
    n, s = 4000, 4
    big = I.gaussian(n, 7, 3300)
    Wh = big[:, 1:1 + s]
    b1 = lo().Basis(n, s, 2, 500)
    b2 = lo().Basis(n, s, 2, 500)
    b1.orthogonalize(dev(I.gaussian(n, s, 3301)))
    b2.orthogonalize(dev(I.gaussian(n, s, 3301)))
    Wd = torch.from_numpy(big).cuda()[:, 1:1 + s]
    assert Wd.stride(0) == 7
    U1, _, R1 = b1.orthogonalize(Wd)
    Wc = dev(Wh)
    U2, _, R2 = b2.orthogonalize(Wc, U=Wc)
    assert np.array_equal(host(U1), host(Wc))
    assert np.array_equal(host(R1), host(R2))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_bitwise_determinism(precision):
    n, s = 20000, 8
    blocks = gaussian_blocks(n, s, 4, 3400)
    outs = []
    for _ in range(2):
        b = lo().Basis(n, s, 4, 2048, precision=precision)
        res = [tuple(host(x) for x in b.orthogonalize(dev(Wh)) if x is not None) for Wh in blocks]
        outs.append(res)
    for r1, r2 in zip(*outs):
        for x, y in zip(r1, r2):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_error_paths_leave_basis_unchanged(precision):
    L = lo()
    n, s = 3000, 4
    b = L.Basis(n, s, 3, 600, precision=precision)
    b.orthogonalize(dev(I.gaussian(n, s, 3500)))
    # a block inside the span of the basis: breakdown, block count unchanged
    Q = host(b.apply_Q(dev(np.eye(s))))
    with pytest.raises(L.LoError) as e:
        b.orthogonalize(dev(Q @ I.gaussian(s, s, 3501)))
    assert e.value.name == "LO_ERR_BREAKDOWN"
    assert b.num_blocks == 1
    # NaN in the block
    Wn = I.gaussian(n, s, 3502)
    Wn[17, 2] = np.nan
    with pytest.raises(L.LoError) as e:
        b.orthogonalize(dev(Wn))
    assert e.value.name in ("LO_ERR_NONFINITE", "LO_ERR_BREAKDOWN")
    assert b.num_blocks == 1
    # the basis still works and agrees with the oracle
    ora = O.LocallyOrthogonalBasis(n, s, 600)
    ora.orthogonalize(I.gaussian(n, s, 3500), "hh", "hh")
    Wg = I.gaussian(n, s, 3503)
    U, H, R = b.orthogonalize(dev(Wg))
    Uo, Po, No = ora.orthogonalize(Wg, "hh", "hh")
    assert rel(host(U), Uo) <= TOL_REL
    b.orthogonalize(dev(I.gaussian(n, s, 3504)))
    with pytest.raises(L.LoError) as e:
        b.orthogonalize(dev(I.gaussian(n, s, 3505)))
    assert e.value.name == "LO_ERR_CAPACITY"
    assert b.num_blocks == 3


@pytest.mark.parametrize("precision", ["mixed_fp32", "mixed_tc"])
def test_mixed_precision_form(precision):
    """First Gram pass in float32, shifted Cholesky, float64 refinement: the
    results meet the float64 tolerances for Gaussian blocks."""
    n, s = 32768, 16
    blocks = gaussian_blocks(n, s, 4, 3600)
    run_and_compare(n, s, 4, 2048, blocks, precision=precision, check_local=False)


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
@pytest.mark.parametrize("precision", ["mixed_fp32", "mixed_tc"])
def test_mixed_precision_stewart(kappa, precision):
    n, m, s = 32768, 32, 16
    A = I.stewart(n, m, kappa, 600 + int(np.log10(kappa)))
    b = lo().Basis(n, s, 2, 4096, precision=precision)
    U0, _, R0 = b.orthogonalize(dev(A[:, :s].copy()))
    U1, H1, R1 = b.orthogonalize(dev(A[:, s:].copy()))
    Q = host(b.apply_Q(dev(np.eye(m))))
    R = np.zeros((m, m))
    R[:s, :s] = host(R0)
    R[:s, s:] = host(H1)
    R[s:, s:] = host(R1)
    assert O.e_perp(Q) <= TOL_PERP
    assert O.residual(A, Q, R) <= TOL_RES


def test_batched_uneven():
    L = lo()
    specs = [(5000, 4, 3), (12000, 8, 2), (3001, 16, 2), (9000, 4, 5)]
    bases, oras, Ws, Us, Hs, Rs, want = [], [], [], [], [], [], []
    for i, (n, s, kb) in enumerate(specs):
        cr = max(512, (kb + 1) * s)
        b = L.Basis(n, s, kb + 1, cr)
        o = O.LocallyOrthogonalBasis(n, s, cr)
        for j in range(kb):
            Wh = I.gaussian(n, s, 3700 + 10 * i + j)
            b.orthogonalize(dev(Wh))
            o.orthogonalize(Wh, "hh", "hh")
        Wh = I.gaussian(n, s, 3790 + i)
        want.append(o.orthogonalize(Wh, "hh", "hh"))
        bases.append(b)
        Ws.append(dev(Wh))
        Us.append(torch.empty(n, s, dtype=torch.float64, device="cuda"))
        Hs.append(torch.empty(kb * s, s, dtype=torch.float64, device="cuda"))
        Rs.append(torch.empty(s, s, dtype=torch.float64, device="cuda"))
    L.orthogonalize_batched(bases, Ws, Us, Hs, Rs)
    for b, (Uo, Po, No), U, H, R in zip(bases, want, Us, Hs, Rs):
        assert rel(host(U), Uo) <= TOL_REL
        assert rel(host(H), Po) <= TOL_REL
        assert rel(host(R), No) <= TOL_REL
        assert b.num_blocks == len(Po) // b.s + 1


def test_batched_graph_reuse_and_truncate():
    """A repeat batched call with the same arguments replays the cached graph:
    truncating the bases back and re-running gives bit-identical results, equal
    to sequential calls; truncate drops blocks exactly."""
    L = lo()
    specs = [(6000, 8, 2), (20000, 4, 3), (3001, 16, 1)]
    bases, Ws, Us, Hs, Rs, seq = [], [], [], [], [], []
    for i, (n, s, kb) in enumerate(specs):
        b = L.Basis(n, s, kb + 2, 1000)
        b2 = L.Basis(n, s, kb + 2, 1000)
        for j in range(kb):
            Wj = dev(I.gaussian(n, s, 4000 + 10 * i + j))
            b.orthogonalize(Wj)
            b2.orthogonalize(Wj)
        Wn = dev(I.gaussian(n, s, 4090 + i))
        seq.append(tuple(host(x) for x in b2.orthogonalize(Wn)))
        bases.append(b)
        Ws.append(Wn)
        Us.append(torch.empty(n, s, dtype=torch.float64, device="cuda"))
        Hs.append(torch.empty(kb * s, s, dtype=torch.float64, device="cuda"))
        Rs.append(torch.empty(s, s, dtype=torch.float64, device="cuda"))
    outs = []
    for rep in range(3):
        for b, (n, s, kb) in zip(bases, specs):
            b.truncate(kb)
        L.orthogonalize_batched(bases, Ws, Us, Hs, Rs)
        outs.append([(host(U), host(H), host(R)) for U, H, R in zip(Us, Hs, Rs)])
    for rep in range(1, 3):
        for a, c in zip(outs[0], outs[rep]):
            for x, y in zip(a, c):
                assert np.array_equal(x, y)
    for (U, H, R), (Us_, Hs_, Rs_) in zip(outs[0], seq):
        assert np.array_equal(U, Us_) and np.array_equal(H, Hs_) and np.array_equal(R, Rs_)
    with pytest.raises(L.LoError):
        bases[0].truncate(bases[0].num_blocks + 1)


def test_batched_cache_evicts_destroyed_bases():
    """Cached batched graphs name their bases by process-unique ids: destroying
    a basis evicts every graph that names it, and bases created afterwards
    (their handles may reuse freed addresses) get new ids and new graphs whose
    results match the oracle."""
    L = lo()

    def make(n, s, kb, seed):
        b = L.Basis(n, s, kb + 1, 1000)
        o = O.LocallyOrthogonalBasis(n, s, 1000)
        for j in range(kb):
            Wh = I.gaussian(n, s, seed + j)
            b.orthogonalize(dev(Wh))
            o.orthogonalize(Wh, "hh", "hh")
        return b, o

    seen = set()
    for rnd, specs in enumerate([[(6000, 8, 2), (9000, 4, 3)], [(7000, 16, 1), (5000, 8, 3)],
                                 [(6000, 8, 2), (9000, 4, 3)]]):
        pairs = [make(n, s, kb, 8000 + 100 * rnd + 10 * i) for i, (n, s, kb) in enumerate(specs)]
        bases = [b for b, _ in pairs]
        ids = [b.id for b in bases]
        assert not (set(ids) & seen)          # ids are never reused
        seen |= set(ids)
        Ws, Us, Hs, Rs, want = [], [], [], [], []
        for i, ((b, o), (n, s, kb)) in enumerate(zip(pairs, specs)):
            Wh = I.gaussian(n, s, 8090 + 100 * rnd + i)
            want.append(o.orthogonalize(Wh, "hh", "hh"))
            Ws.append(dev(Wh))
            Us.append(torch.empty(n, s, dtype=torch.float64, device="cuda"))
            Hs.append(torch.empty(kb * s, s, dtype=torch.float64, device="cuda"))
            Rs.append(torch.empty(s, s, dtype=torch.float64, device="cuda"))
        L.orthogonalize_batched(bases, Ws, Us, Hs, Rs)
        for (Uo, Po, No), U, H, R in zip(want, Us, Hs, Rs):
            assert rel(host(U), Uo) <= TOL_REL and rel(host(H), Po) <= TOL_REL and rel(host(R), No) <= TOL_REL
        assert all(L.batched_cache_entries(i) == 1 for i in ids)
        for b in bases:
            b.close()
        assert all(L.batched_cache_entries(i) == 0 for i in ids)


def test_batched_host_buffers():
    """Host W, U, H, R in the batched call: staged like lo_orthogonalize, with
    the same results bit for bit as device buffers in a twin set of bases."""
    L = lo()
    specs = [(5000, 4, 2), (7000, 8, 1), (3001, 16, 2)]
    bd, bh, Wd, Ud, Hd, Rd, Wh_, Uh_, Hh_, Rh_ = [], [], [], [], [], [], [], [], [], []
    for i, (n, s, kb) in enumerate(specs):
        b1, b2 = L.Basis(n, s, kb + 1, 1000), L.Basis(n, s, kb + 1, 1000)
        for j in range(kb):
            Wj = dev(I.gaussian(n, s, 8200 + 10 * i + j))
            b1.orthogonalize(Wj)
            b2.orthogonalize(Wj)
        bd.append(b1)
        bh.append(b2)
        Wn = I.gaussian(n, s, 8290 + i)
        Wd.append(dev(Wn))
        Wh_.append(Wn)
        Ud.append(torch.empty(n, s, dtype=torch.float64, device="cuda"))
        Hd.append(torch.empty(kb * s, s, dtype=torch.float64, device="cuda"))
        Rd.append(torch.empty(s, s, dtype=torch.float64, device="cuda"))
        Uh_.append(np.zeros((n, s)))
        Hh_.append(np.zeros((kb * s, s)))
        Rh_.append(np.zeros((s, s)))
    L.orthogonalize_batched(bd, Wd, Ud, Hd, Rd)
    L.orthogonalize_batched(bh, Wh_, Uh_, Hh_, Rh_)
    for U, H, R, Uh, Hh, Rh in zip(Ud, Hd, Rd, Uh_, Hh_, Rh_):
        assert np.array_equal(host(U), Uh) and np.array_equal(host(H), Hh) and np.array_equal(host(R), Rh)
    assert [b.num_blocks for b in bh] == [kb + 1 for (_, _, kb) in specs]


def test_chunk_rows_tuner():
    L = lo()
    cr = L.tune_chunk_rows(200000, 8, 6)
    assert cr >= 256 and cr <= 200000 and (cr & (cr - 1)) == 0
    assert L.tune_chunk_rows(200000, 8, 6) == cr    # memoized
    b = L.Basis(200000, 8, 6, cr)
    U, _, R = b.orthogonalize(dev(I.gaussian(200000, 8, 4100)))
    assert O.e_perp(host(U)) <= TOL_PERP


def test_laplace5_operator():
    nx, ny, s = 37, 23, 3
    X = I.uniform(nx * ny, s, 3800)
    Y = host(lo().laplace5_apply(nx, ny, dev(X), torch.empty(nx * ny, s, dtype=torch.float64, device="cuda")))
    G = X.reshape(ny, nx, s)
    ref = 4 * G
    ref[:, 1:] -= G[:, :-1]
    ref[:, :-1] -= G[:, 1:]
    ref[1:] -= G[:-1]
    ref[:-1] -= G[1:]
    assert np.abs(Y - ref.reshape(-1, s)).max() <= 1e-14


@pytest.mark.parametrize("precision", PRECISIONS)
def test_full_size_sampled_rows(precision):
    """The block-GMRes workload's sizes (n = 2^20, s = 8, 4096-row chunks):
    three independent Gaussian blocks; every output compared with the oracle
    (BCGS-PIP+ sub-algorithms) on 4096 sampled rows and in full for H, R."""
    n, s, cr = 2 ** 20, 8, 4096
    blocks = gaussian_blocks(n, s, 3, 3900)
    b = lo().Basis(n, s, 31, cr, precision=precision)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    rows = np.sort(I.rng(3999).choice(n, 4096, replace=False))
    for j, Wh in enumerate(blocks):
        U, H, R = b.orthogonalize(dev(Wh))
        Uo, Po, No = ora.orthogonalize(Wh, "pip2", "pip2")
        assert rel(host(U)[rows], Uo[rows]) <= TOL_REL
        assert rel(host(R), No) <= TOL_REL
        if j:
            assert rel(host(H), Po) <= TOL_REL
    Q = b.apply_Q(dev(np.eye(b.k)))
    G = (Q.T @ Q).cpu().numpy()
    assert np.linalg.norm(G - np.eye(b.k)) <= TOL_PERP


# --- digit planes of the tensor-core forms -----------------------------------

@pytest.mark.parametrize("precision", ["fp64_tc", "mixed_tc"])
@pytest.mark.parametrize("n,s,cr,M", [
    (10001, 8, 1111, 40),   # odd chunk starts: 8-byte plane rows; 3 Gram column groups
    (8191, 16, 700, 20),    # assembly over more than 256 columns (flush inside a row tile)
    (6000, 32, 1500, 8),    # 512-row slabs; 8 Gram column groups
    (65536, 16, 2048, 5),   # more CTAs than SMs: stage 2 reads the last iterate from the new panel
    (65536, 32, 4096, 6),   # the same with four output groups per row tile
])
def test_digit_planes_bitwise(n, s, cr, M, precision):
    """Panels kept as digit planes give the products of re-splitting the
    float64 panels in every pass: bit for bit at the first step (no prior
    panels) and, at s = 8, for H and R of the second (the Gram and the
    8-output iterate are exact), within the float64 parity tolerance
    elsewhere, every output of
    every step with the reiteration passes included, and the final basis
    against the oracle.  Past the first step the two differ only where the
    tensor-core assembly with 16 outputs per group sums the digit pairs of
    each of its three lowest classes in one float32 accumulator (an error of
    the size of a float64 dot product's, test_merged_classes_cpu.py) instead
    of exactly; the ill-conditioned blocks of this test magnify that
    to about 1e-12.  The mixed form's first pass
    differs on purpose (with planes: the leading digits on the tensor cores;
    without: float32 on the CUDA cores), so there both bases must agree within
    the float64 tolerances instead."""
    L = lo()
    on = L.Basis(n, s, M, cr, precision=precision)
    off = L.Basis(n, s, M, cr, precision=precision, digit_planes=False)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    bitwise = precision == "fp64_tc"
    A = []
    for j in range(M):
        Wh = I.gaussian(n, s, 5000 + j)
        if j % 3 == 2:  # a block close to the span of the first forces a third pass
            Wh = Wh + 1e3 * A[0] @ I.gaussian(s, s, 5100 + j)
        A.append(Wh)
        W = dev(Wh)
        r1 = [host(x) for x in on.orthogonalize(W) if x is not None]
        r2 = [host(x) for x in off.orthogonalize(W) if x is not None]
        Uo, Po, No = ora.orthogonalize(Wh, "pip2", "pip2")
        for i, (x, y) in enumerate(zip(r1, r2)):
            # at s = 8 the second step's H and R come from exact digit products
            # only (the k = 0 panel, the 8-output iterate, the Gram): bit for bit
            exact_hr = s == 8 and j == 1 and i >= 1
            if bitwise and (j == 0 or exact_hr):
                assert np.array_equal(x, y), (j, i)
            elif bitwise:
                assert close(x, y), (j, errs(x, y))
            else:
                assert rel(x, y) <= TOL_REL, j
        # the planes-on outputs against the oracle: U, R (and H past the first block)
        assert close(r1[0], Uo), (j, errs(r1[0], Uo))
        assert close(r1[-1], No), (j, errs(r1[-1], No))
        if j:
            assert close(r1[1], Po), (j, errs(r1[1], Po))
    Q = host(on.apply_Q(dev(np.eye(on.k))))
    assert O.e_perp(Q) <= TOL_PERP
    assert close(Q, ora.explicit()), errs(Q, ora.explicit())
    for c in (0, on.num_chunks - 1):
        Qa, Ta = on.export_chunk(c)
        Qb, Tb = off.export_chunk(c)
        assert close(Qa, Qb), errs(Qa, Qb)
        assert close(np.triu(Ta), np.triu(Tb)), errs(np.triu(Ta), np.triu(Tb))


@pytest.mark.parametrize("planes", [True, False])
def test_saturated_digits_long_slab(planes):
    """Columns of equal magnitude 1.99 make every leading digit 254; over a
    512-row slab (s = 32) the leading digit products sum past 2^24 and must be
    flushed before float32 rounds them.  One local pass (BCGS-PIP), so R is the
    first Gram's Cholesky factor and shows any rounding there."""
    n, s = 4096, 32
    X = 1.99 * np.where(I.uniform(n, s, 5200) < 0.0, -1.0, 1.0)
    b = lo().Basis(n, s, 1, n, precision="fp64_tc", leaf="pip", reduction="pip", digit_planes=planes)
    U, _, R = b.orthogonalize(dev(X))
    ora = O.LocallyOrthogonalBasis(n, s, n)
    _, _, Ro = ora.orthogonalize(X, "hh", "hh")
    assert rel(host(R), Ro) <= TOL_REL
    assert O.e_perp(host(U)) <= TOL_PERP


@pytest.mark.parametrize("s", [8, 16])
@pytest.mark.parametrize("kappa", [1e2, 1e8])
def test_single_block_tensor_core_tsqr(s, kappa):
    """A basis of one block (no digit planes) as a fresh process would build
    it first: the k = 0 tensor-core kernels on their own, against the oracle."""
    n, cr = 40000, 4096
    A = I.stewart(n, s, kappa, 5300 + s + int(np.log10(kappa)))
    b = lo().Basis(n, s, 1, cr, precision="fp64_tc")
    U, _, R = b.orthogonalize(dev(A))
    Uh, Rh = host(U), host(R)
    assert O.e_perp(Uh) <= TOL_PERP
    assert O.residual(A, Uh, Rh) <= TOL_RES
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    _, _, Ro = ora.orthogonalize(A, "hh", "hh")
    assert rel(Rh, Ro) <= max(TOL_REL, 100 * kappa * np.finfo(float).eps)


@pytest.mark.parametrize("s", [3, 4])
def test_narrow_one_block_basis_runs_native(s):
    """A one-block tensor-core basis of at most 4 columns runs the native
    float64 kernels (any s <= 4, s = 3 included): its QR matches the oracle and
    is bit for bit the native form's; with prior blocks the tensor-core form
    keeps its own width rule (s = 3 is unsupported there)."""
    n, cr = 50000, 4096
    A = I.stewart(n, s, 1e6, 7100 + s)
    outs = {}
    for prec in ("fp64", "fp64_tc"):
        b = lo().Basis(n, s, 1, cr, precision=prec)
        U, _, R = b.orthogonalize(dev(A))
        outs[prec] = (host(U), host(R))
    (Uf, Rf), (Ut, Rt) = outs["fp64"], outs["fp64_tc"]
    assert np.array_equal(Uf, Ut) and np.array_equal(Rf, Rt)
    assert O.e_perp(Ut) <= TOL_PERP
    assert O.residual(A, Ut, Rt) <= TOL_RES
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    _, _, Ro = ora.orthogonalize(A, "hh", "hh")
    assert rel(Rt, Ro) <= max(TOL_REL, 100 * 1e6 * np.finfo(float).eps)
    if s == 3:
        with pytest.raises(lo().LoError) as e:
            lo().Basis(n, s, 2, cr, precision="fp64_tc")
        assert "UNSUPPORTED" in str(e.value)


def _orthonormal_columns(X):
    """Q of X = QR by CholeskyQR2 (the s x s Cholesky on the host), for
    device-side test inputs of full size."""
    for _ in range(2):
        G = (X.T @ X).cpu().numpy()
        Linv_t = np.linalg.inv(np.linalg.cholesky(G)).T
        X = X @ torch.from_numpy(np.ascontiguousarray(Linv_t)).to(X.device)
    return X


def test_full_cycle_every_step_properties():
    """The block-GMRes workload in the benchmark's launch configuration
    (n = 2^20, s = 8, 31 blocks, 4096-row chunks, float64 on the tensor cores):
    every step k = 0 .. 240 satisfies W = Q H + U R to float64 accuracy, and
    the final 248-column basis is orthonormal.  Properties that hold at any
    size; the oracle at these sizes is the CPU baseline's minutes."""
    n, s, m, cr = 2 ** 20, 8, 31, 4096
    L = lo()
    b = L.Basis(n, s, m, cr, precision="fp64_tc")
    g = torch.Generator(device="cuda")
    g.manual_seed(2204133930 + 2000)
    worst = 0.0
    for j in range(m):
        W = torch.randn(n, s, dtype=torch.float64, device="cuda", generator=g)
        if j:  # a Krylov-like block: a component along the basis
            W = W + b.apply_Q(torch.randn(b.k, s, dtype=torch.float64, device="cuda", generator=g))
        k = b.k
        U, H, R = b.orthogonalize(W)
        recon = U @ R
        if k:
            C = torch.zeros(b.k, s, dtype=torch.float64, device="cuda")
            C[:k] = H
            recon = recon + b.apply_Q(C)
        res = float(torch.linalg.norm(W - recon) / torch.linalg.norm(W))
        worst = max(worst, res)
        assert res <= TOL_RES, (j, res)
    Q = b.apply_Q(torch.eye(b.k, dtype=torch.float64, device="cuda"))
    G = Q.T @ Q
    eperp = float(torch.linalg.norm(G - torch.eye(b.k, dtype=torch.float64, device="cuda")))
    assert eperp <= TOL_PERP, eperp


@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e10])
def test_tsqr_target_size_properties(kappa):
    """The tall-skinny QR at the target size (n = 2^24, s = 8, one block,
    chunk rows from the tuner, float64 on the tensor cores), A = U diag(sigma)
    V^T with orthonormal U, V and sigma log-spaced to 1/kappa: U^T U = I and
    A = U R to float64 accuracy, R upper triangular with a positive diagonal."""
    n, s = 2 ** 24, 8
    L = lo()
    g = torch.Generator(device="cuda")
    g.manual_seed(2204133930 + 3000 + int(np.log10(kappa)))
    Uh = _orthonormal_columns(torch.randn(n, s, dtype=torch.float64, device="cuda", generator=g))
    Vh = _orthonormal_columns(torch.randn(s, s, dtype=torch.float64, device="cuda", generator=g))
    sig = torch.tensor([kappa ** (-j / (s - 1.0)) for j in range(s)], dtype=torch.float64, device="cuda")
    A = (Uh * sig) @ Vh.T
    del Uh
    cr = L.tune_chunk_rows(n, s, 1, precision="fp64_tc")
    b = L.Basis(n, s, 1, cr, precision="fp64_tc")
    U, _, R = b.orthogonalize(A)
    eye = torch.eye(s, dtype=torch.float64, device="cuda")
    assert float(torch.linalg.norm(U.T @ U - eye)) <= TOL_PERP
    assert float(torch.linalg.norm(A - U @ R) / torch.linalg.norm(A)) <= TOL_RES
    Rh = host(R)
    assert np.allclose(np.tril(Rh, -1), 0.0) and np.all(np.diag(Rh) > 0)


def test_bounded_wait_expires_cleanly():
    """The timeout path of the tcgen05 kernels without a fault: with the test
    hook the k > 0 Gram's issuer issues nothing, so its producers' and
    drainers' bounded waits expire.  The step reports LO_ERR_TIMEOUT, the basis
    keeps its blocks, and the context stays usable: the same basis without the
    hook's effect (a fresh one) and this one's next step on k = 0 work."""
    n, s, cr = 65536, 8, 4096
    L = lo()
    W0, W1 = (dev(I.gaussian(n, s, 7200 + j)) for j in range(2))
    b = L.Basis(n, s, 3, cr, precision="fp64_tc", test_stall=True)
    b.orthogonalize(W0)                       # k = 0: the k = 0 kernels, no hook
    with pytest.raises(L.LoError) as e:
        b.orthogonalize(W1)                   # k = 8: the Gram's issuer withholds its work
    assert e.value.name == "LO_ERR_TIMEOUT"
    assert b.num_blocks == 1
    b.truncate(0)                             # the status word was read and cleared
    U, _, R = b.orthogonalize(W0)
    assert O.e_perp(host(U)) <= TOL_PERP
    ok = L.Basis(n, s, 3, cr, precision="fp64_tc")
    for W in (W0, W1):
        ok.orthogonalize(W)
    Q = host(ok.apply_Q(dev(np.eye(ok.k))))
    assert O.e_perp(Q) <= TOL_PERP


def test_bounded_wait_expires_with_work_in_flight():
    """The timeout path with loads and MMAs in flight, without a fault: with
    test hook 2 the Gram's drainers never release a drained accumulator
    buffer, so the issuer's bounded wait for it expires after it has issued
    the loads and MMAs of the first intervals; it waits for those to finish,
    and the step returns LO_ERR_TIMEOUT with the basis unchanged.  The
    context stays usable: the same basis runs a k = 0 step, and a fresh basis
    the same two steps, matching the oracle.  2^18 rows: 1024 slab items over
    the persistent CTAs, so each CTA reaches a third accumulation interval and
    waits for a released buffer."""
    n, s, cr = 2 ** 18, 8, 4096
    L = lo()
    W0h, W1h = (I.gaussian(n, s, 7300 + j) for j in range(2))
    W0, W1 = dev(W0h), dev(W1h)
    b = L.Basis(n, s, 3, cr, precision="fp64_tc", test_stall=2)
    b.orthogonalize(W0)
    with pytest.raises(L.LoError) as e:
        b.orthogonalize(W1)
    assert e.value.name == "LO_ERR_TIMEOUT"
    assert b.num_blocks == 1
    b.truncate(0)
    U, _, R = b.orthogonalize(W0)
    assert O.e_perp(host(U)) <= TOL_PERP
    ok = L.Basis(n, s, 3, cr, precision="fp64_tc")
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    for Wd, Wh in ((W0, W0h), (W1, W1h)):
        U, H, R = ok.orthogonalize(Wd)
        Uo, Po, No = ora.orthogonalize(Wh, "hh", "hh")
        assert close(host(U), Uo) and close(host(R), No)


def vanishing_blocks(n, s, cr, count, seed0):
    """Blocks that are exactly zero on whole chunks: column c lives on two
    chunks, chunk 1 is empty for every column, and odd blocks add the first
    half of the last chunk (so its local panel mixes zero and full columns)."""
    bounds = O.chunk_bounds(n, cr)
    p = len(bounds)
    out = []
    for j in range(count):
        sup = []
        for c in range(s):
            chunks = {(2 + c + j) % p, (2 + c + j + p // 2) % p} - {1}
            sup.append([bounds[i] for i in sorted(chunks)])
        if j % 2:
            b, e = bounds[p - 1]
            sup = [r + [(b, (b + e) // 2)] for r in sup]
        out.append(I.localized(n, s, seed0 + j, sup))
    return out


@pytest.mark.parametrize("n,s,cr,M,precision", [
    (40000, 8, 4096, 4, "fp64"),
    (40000, 8, 4096, 4, "fp64_tc"),
    (20000, 4, 2048, 4, "fp64"),
    (20000, 4, 2048, 4, "fp64_tc"),
    (20000, 4, 2048, 1, "fp64"),      # one-block basis: the narrow k = 0 kernels
    (70000, 16, 8192, 3, "fp64_tc"),
    (70000, 16, 8192, 3, "mixed_tc"),
    (40000, 8, 4096, 3, "mixed_fp32"),
])
def test_blocks_vanishing_on_chunks(n, s, cr, M, precision):
    """Exactly zero components of a block on some chunks (globally of full
    rank) give zero normalizer rows locally and zero columns in the local
    panels; U, H, R match the unique solution of the oracle, the local
    representation matches the oracle's Cholesky leaf, and Q is orthonormal."""
    blocks = vanishing_blocks(n, s, cr, M, 4100 + s)
    b = lo().Basis(n, s, M, cr, precision=precision)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    ora_loc = O.LocallyOrthogonalBasis(n, s, cr)
    A = np.hstack(blocks)
    Rfull = np.zeros((A.shape[1], A.shape[1]))
    for j, Wh in enumerate(blocks):
        U, H, R = b.orthogonalize(dev(Wh))
        Uo, Po, No = ora.orthogonalize(Wh, "hh", "hh")
        ora_loc.orthogonalize(Wh, "pip2", "hh")
        assert rel(host(U), Uo) <= TOL_REL, (j, rel(host(U), Uo))
        assert rel(host(R), No) <= TOL_REL, (j, rel(host(R), No))
        if j > 0:
            assert rel(host(H), Po) <= TOL_REL, (j, rel(host(H), Po))
            Rfull[:j * s, j * s:(j + 1) * s] = host(H)
        Rfull[j * s:(j + 1) * s, j * s:(j + 1) * s] = host(R)
    Q = host(b.apply_Q(dev(np.eye(b.k))))
    assert O.e_perp(Q) <= TOL_PERP
    assert O.residual(A, Q, Rfull) <= TOL_RES
    if precision in ("fp64", "fp64_tc"):
        for c in range(b.num_chunks):
            Qi, Ti = b.export_chunk(c)
            assert rel(Qi, ora_loc.Qloc[c]) <= TOL_REL, c
            assert rel(Ti, np.triu(ora_loc.T[c])) <= TOL_REL, c
            G = Qi.T @ Qi
            d = np.diag(G)
            assert np.all((np.abs(d - 1) <= TOL_PERP) | (d == 0.0)), c
            assert np.abs(G - np.diag(d)).max() <= TOL_PERP, c
        Qi, _ = b.export_chunk(1)
        assert np.all(Qi == 0.0)  # chunk 1 never saw a nonzero value


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_component_vanishing_everywhere_is_a_breakdown(precision):
    """A column that is zero on every chunk is a global rank deficiency (the
    unsupported deflation case): LO_ERR_BREAKDOWN, basis unchanged."""
    L = lo()
    n, s, cr = 16384, 8, 2048
    b = L.Basis(n, s, 3, cr, precision=precision)
    b.orthogonalize(dev(I.gaussian(n, s, 4200)))
    Wz = I.gaussian(n, s, 4201)
    Wz[:, 5] = 0.0
    with pytest.raises(L.LoError) as e:
        b.orthogonalize(dev(Wz))
    assert e.value.name == "LO_ERR_BREAKDOWN"
    assert b.num_blocks == 1
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    ora.orthogonalize(I.gaussian(n, s, 4200), "hh", "hh")
    Wg = I.gaussian(n, s, 4202)
    U, H, R = b.orthogonalize(dev(Wg))
    Uo, Po, No = ora.orthogonalize(Wg, "hh", "hh")
    assert rel(host(U), Uo) <= TOL_REL and rel(host(H), Po) <= TOL_REL and rel(host(R), No) <= TOL_REL


@pytest.mark.parametrize("n,s,cr,M,precision", [
    (40000, 8, 4096, 3, "fp64"),
    (40000, 8, 4096, 3, "fp64_tc"),
    (20000, 4, 2048, 3, "fp64"),
    (20000, 4, 2048, 1, "fp64_tc"),
    (70000, 16, 8192, 3, "fp64_tc"),
    (70000, 16, 8192, 3, "mixed_tc"),
    (40000, 8, 4096, 3, "mixed_fp32"),
    (30000, 3, 4096, 3, "mixed_fp32"),
])
def test_power_of_two_scaling_is_exact(n, s, cr, M, precision):
    """The PQR of 2^j W is (U, 2^j H, 2^j R).  Every form scales by exponent
    (float64 arithmetic, the digit splits against column exponents, the
    float32 pass's per-slab column scaling), so blocks scaled by 2^300 and
    2^-300 -- whose products overflow or underflow float32 -- give the same
    U and Q bit for bit and H, R scaled bit for bit; the unscaled run
    matches the oracle."""
    blocks = gaussian_blocks(n, s, M, 4300 + s)
    runs = {}
    for j in (0, 300, -300):
        b = lo().Basis(n, s, M, cr, precision=precision)
        res = []
        for Wh in blocks:
            U, H, R = b.orthogonalize(dev(np.ldexp(Wh, j)))
            res.append((host(U), np.zeros((0, s)) if H is None else host(H), host(R)))
        runs[j] = (res, host(b.apply_Q(dev(np.eye(b.k)))))
        b.close()
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    for (U, H, R), Wh in zip(runs[0][0], blocks):
        Uo, Po, No = ora.orthogonalize(Wh, "hh", "hh")
        assert rel(U, Uo) <= TOL_REL and rel(R, No) <= TOL_REL
        if Po.size:
            assert rel(H, Po) <= TOL_REL
    assert O.e_perp(runs[0][1]) <= TOL_PERP
    for j in (300, -300):
        res, Q = runs[j]
        assert np.array_equal(Q, runs[0][1]), j
        for i, ((U, H, R), (U0, H0, R0)) in enumerate(zip(res, runs[0][0])):
            assert np.array_equal(U, U0), (j, i, rel(U, U0))
            assert np.array_equal(H, np.ldexp(H0, j)), (j, i)
            assert np.array_equal(R, np.ldexp(R0, j)), (j, i, rel(R, np.ldexp(R0, j)))


@pytest.mark.parametrize("n,s,cr,M,nb,precision", [
    (40000, 8, 4096, 5, 5, "fp64_tc"),      # full basis: the last panel has no digit planes
    (40000, 8, 4096, 5, 3, "fp64_tc"),      # the last panel has planes but is split all the same
    (70001, 16, 8192, 4, 4, "fp64_tc"),     # ragged slabs and last chunk
    (50000, 32, 8192, 3, 3, "fp64_tc"),     # two output groups per assembly
    (40000, 8, 4096, 4, 4, "mixed_tc"),
])
def test_apply_Q_tensor_cores(n, s, cr, M, nb, precision):
    """apply_Q of a basis with digit planes runs the tensor-core assembly:
    Y = Q C matches the float64 product of the basis's own representation
    (sum over chunks of Q_i (T_i C), evaluated on the host) to float64
    accuracy and the oracle's basis within the parity tolerance, for m below,
    equal to and above s, host and device buffers, and a strided Y."""
    L = lo()
    b = L.Basis(n, s, M, cr, precision=precision)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    for j in range(nb):
        Wh = I.gaussian(n, s, 4500 + j)
        b.orthogonalize(dev(Wh))
        ora.orthogonalize(Wh, "hh", "hh")
    rep = O.LocallyOrthogonalBasis(n, s, cr)  # the GPU basis's own representation
    for c in range(b.num_chunks):
        rep.Qloc[c], rep.T[c] = b.export_chunk(c)
    before = L.launch_count()
    for m in (1, s - 3, s, s + 5, 2 * s + 1):
        C = I.gaussian(b.k, m, 4600 + m)
        Y = host(b.apply_Q(dev(C)))
        want = rep.apply_Q(C)
        assert rel(Y, want) <= 1e-14, (m, rel(Y, want))
        assert rel(Y, ora.apply_Q(C)) <= TOL_REL, m
        Yh = b.apply_Q(C)
        assert np.array_equal(Yh, Y), m
        Ys = torch.full((n, m + 3), 7.0, dtype=torch.float64, device="cuda")
        b.apply_Q(dev(C), Ys[:, :m])
        Ys = host(Ys)
        assert np.array_equal(Ys[:, :m], Y) and np.all(Ys[:, m:] == 7.0), m
    # one coefficient kernel and one assembly per s columns of C
    groups = sum(3 * ((m + s - 1) // s) for m in (1, s - 3, s, s + 5, 2 * s + 1))
    assert L.launch_count() - before == 2 * groups


@pytest.mark.parametrize("s,precision", [(8, "fp64_tc"), (16, "fp64_tc"), (32, "fp64_tc"), (8, "mixed_tc"),
                                         (8, "mixed_fp32"), (4, "fp64_tc")])
def test_strided_and_aliased_tensor_cores(s, precision):
    """The tensor-core and mixed forms, at k = 0 and with digit planes at
    k > 0 (two output groups at s = 32): W as a strided view whose rows start
    off 16-byte alignment gives the same results bit for bit as a contiguous
    copy orthogonalized in place (U written over W)."""
    n, cr, M = 20000, 2048, 4
    b1 = lo().Basis(n, s, M, cr, precision=precision)
    b2 = lo().Basis(n, s, M, cr, precision=precision)
    for j in range(3):
        big = I.gaussian(n, s + 3, 4700 + j)
        Wd = torch.from_numpy(big).cuda()[:, 1:1 + s]
        assert Wd.stride(0) == s + 3
        Wc = dev(big[:, 1:1 + s])
        U1, H1, R1 = b1.orthogonalize(Wd)
        U2, H2, R2 = b2.orthogonalize(Wc, U=Wc)
        assert np.array_equal(host(U1), host(Wc)), j
        assert np.array_equal(host(R1), host(R2)), j
        if j > 0:
            assert np.array_equal(host(H1), host(H2)), j
    Q = host(b1.apply_Q(dev(np.eye(b1.k))))
    assert O.e_perp(Q) <= TOL_PERP


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc", "mixed_fp32", "mixed_tc"])
def test_gram_overflow_is_nonfinite(precision):
    """A block whose Gram matrix leaves the float64 range (entries 2^520, the
    Gram 2^1040) is reported as LO_ERR_NONFINITE with the basis unchanged,
    and the basis goes on working; 2^500 (Gram 2^1000) is in range and
    matches the oracle."""
    L = lo()
    n, s, cr = 16384, 8, 2048
    b = L.Basis(n, s, 3, cr, precision=precision)
    ora = O.LocallyOrthogonalBasis(n, s, cr)
    W0 = I.gaussian(n, s, 4800)
    b.orthogonalize(dev(W0))
    ora.orthogonalize(W0, "hh", "hh")
    with pytest.raises(L.LoError) as e:
        b.orthogonalize(dev(np.ldexp(I.gaussian(n, s, 4801), 520)))
    assert e.value.name == "LO_ERR_NONFINITE"
    assert b.num_blocks == 1
    W1 = np.ldexp(I.gaussian(n, s, 4802), 500)
    U, H, R = b.orthogonalize(dev(W1))
    Uo, Po, No = ora.orthogonalize(W1, "hh", "hh")
    assert rel(host(U), Uo) <= TOL_REL and rel(host(H), Po) <= TOL_REL and rel(host(R), No) <= TOL_REL
