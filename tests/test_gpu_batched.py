"""The persistent batched launch (lo_set_batched_route, lo_orthogonalize_batched)
against sequential calls and the oracle.

Route 'persistent' puts every instance the persistent kernel can run into one
launch: a work list of (instance, slab) and (instance, chunk) items with
ticketed leaf and reduction factorizations.  For float64 bases past their
first block it runs the same kernels' arithmetic in the same order as the
sequential launches, so the outputs are compared bit for bit; every instance
is also compared with the oracle, and the bases go on working afterwards
(their representation, and for tensor-core bases the new panel's exponents
and digit planes, are current).
"""

import numpy as np
import pytest

from oracle import lo_oracle as O
from paper_2204_13393_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_REL = 1e-10
TOL_PERP = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_13393_gb300 import lo

    lo.library()
    torch.cuda.set_device(0)
    yield
    lo.set_batched_route("auto")


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


def build(specs, precision, seed0, twins=False):
    """Bases with kb prior Gaussian blocks each (and identical twins), the
    oracle bases, and the new blocks with output buffers."""
    L = lo()
    out = []
    for i, (n, s, kb, cr) in enumerate(specs):
        b = L.Basis(n, s, kb + 2, cr, precision=precision)
        t = L.Basis(n, s, kb + 2, cr, precision=precision) if twins else None
        o = O.LocallyOrthogonalBasis(n, s, cr)
        for j in range(kb):
            W = I.gaussian(n, s, seed0 + 100 * i + j)
            b.orthogonalize(dev(W))
            if t is not None:
                t.orthogonalize(dev(W))
            o.orthogonalize(W, "pip2", "pip2")
        Wn = I.gaussian(n, s, seed0 + 100 * i + 99)
        bufs = (torch.empty(n, s, dtype=torch.float64, device="cuda"),
                torch.empty(max(kb, 1) * s, s, dtype=torch.float64, device="cuda"),
                torch.empty(s, s, dtype=torch.float64, device="cuda"))
        out.append(dict(b=b, t=t, o=o, W=Wn, Wd=dev(Wn), bufs=bufs, kb=kb, s=s, n=n))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_persistent_route_matches_sequential_and_oracle(precision):
    specs = [(4096, 4, 8, 512), (6000, 8, 3, 1000), (3001, 16, 2, 1000), (9000, 4, 5, 700),
             (20000, 8, 12, 2048), (5000, 32, 2, 1024), (7000, 2, 6, 900), (12000, 16, 4, 2048),
             (4096, 8, 0, 512), (10000, 4, 0, 1000)]
    L = lo()
    inst = build(specs, precision, I.seed_for(12, 0), twins=True)
    L.set_batched_route("persistent")
    L.orthogonalize_batched([d["b"] for d in inst], [d["Wd"] for d in inst], [d["bufs"][0] for d in inst],
                            [d["bufs"][1] if d["kb"] else None for d in inst], [d["bufs"][2] for d in inst])
    assert L.batched_persistent_count() == len(specs)
    for d in inst:
        U, H, R = (host(x) for x in d["bufs"])
        Ut, Ht, Rt = (host(x) if x is not None else None for x in d["t"].orthogonalize(d["Wd"]))
        Uo, Po, No = d["o"].orthogonalize(d["W"], "pip2", "pip2")
        assert d["b"].num_blocks == d["kb"] + 1
        assert close(U, Uo) and close(R, No), (d["n"], d["s"], d["kb"], errs(U, Uo), errs(R, No))
        if d["kb"]:
            assert close(H, Po), (d["n"], d["s"], errs(H, Po))
        if precision == "fp64" and d["kb"]:
            # the same kernels' arithmetic in the same order: bit for bit
            assert np.array_equal(U, Ut) and np.array_equal(R, Rt) and np.array_equal(H, Ht)
        # the basis goes on: a further step on the regular path matches the oracle
        W2 = I.gaussian(d["n"], d["s"], 77 + d["n"])
        U2, H2, R2 = d["b"].orthogonalize(dev(W2))
        Uo2, Po2, No2 = d["o"].orthogonalize(W2, "pip2", "pip2")
        assert close(host(U2), Uo2) and close(host(H2), Po2) and close(host(R2), No2)
        Q = host(d["b"].apply_Q(dev(np.eye(d["b"].k))))
        assert O.e_perp(Q) <= TOL_PERP and close(Q, d["o"].explicit())


@pytest.mark.parametrize("precision", ["fp64", "fp64_tc"])
def test_sixty_four_uneven_instances_vs_oracle(precision):
    """64 instances with n log-uniform, s from {4, 8, 16}, 1 .. 30 prior blocks
    (the batched workload's recipe at reduced n), auto route (float64 bases:
    the small ones in the persistent launch; tensor-core bases: their own
    branches): every output against the oracle; replaying the cached graph
    gives the same bits."""
    L = lo()
    L.set_batched_route("auto")
    raw = I.batch_instances(64, I.seed_for(12, 1000), n_lo=3e3, n_hi=4e4)
    specs = []
    for n, s, kb in raw:
        cr = 1024
        while cr < (kb + 2) * s:
            cr *= 2
        n = max(n, cr)
        specs.append((n, s, kb, cr))
    inst = build(specs, precision, I.seed_for(12, 2000))
    bases = [d["b"] for d in inst]
    args = ([d["Wd"] for d in inst], [d["bufs"][0] for d in inst], [d["bufs"][1] for d in inst],
            [d["bufs"][2] for d in inst])
    L.orthogonalize_batched(bases, *args)
    first = [tuple(host(x) for x in d["bufs"]) for d in inst]
    n_persistent = L.batched_persistent_count()
    if precision == "fp64":
        assert 0 < n_persistent < 64
    else:
        assert n_persistent == 0
    for d, (U, H, R) in zip(inst, first):
        Uo, Po, No = d["o"].orthogonalize(d["W"], "pip2", "pip2")
        assert close(U, Uo) and close(H, Po) and close(R, No), (d["n"], d["s"], d["kb"])
    for b, d in zip(bases, inst):
        b.truncate(d["kb"])
    L.orthogonalize_batched(bases, *args)
    for d, (U, H, R) in zip(inst, first):
        assert np.array_equal(host(d["bufs"][0]), U) and np.array_equal(host(d["bufs"][2]), R)


def test_persistent_route_falls_back_for_the_shifted_retry():
    """An instance whose block lies in the span of its basis to 1e-10 breaks
    the first Cholesky down: the shifted retry forces more passes than the
    persistent launch runs, so the call redoes that instance on the regular
    path -- bit for bit a sequential call on a twin basis -- while its
    neighbour in the launch keeps the persistent result."""
    L = lo()
    L.set_batched_route("persistent")
    specs = [(8000, 8, 3, 1000), (8000, 8, 3, 1000)]
    inst = build(specs, "fp64", I.seed_for(12, 3000), twins=True)
    d = inst[1]
    Qx = d["o"].explicit()
    W = Qx @ I.gaussian(Qx.shape[1], 8, 5) + 1e-10 * d["W"]
    d["W"], d["Wd"] = W, dev(W)
    L.orthogonalize_batched([x["b"] for x in inst], [x["Wd"] for x in inst], [x["bufs"][0] for x in inst],
                            [x["bufs"][1] for x in inst], [x["bufs"][2] for x in inst])
    assert inst[1]["b"].last_step_info()[0] == 3           # the regular path's shifted-retry passes
    for x in inst:
        U, H, R = (host(y) for y in x["bufs"])
        Ut, Ht, Rt = (host(y) for y in x["t"].orthogonalize(x["Wd"]))
        assert np.array_equal(U, Ut) and np.array_equal(H, Ht) and np.array_equal(R, Rt)
        assert x["b"].num_blocks == 4
        assert O.e_perp(host(x["b"].apply_Q(dev(np.eye(x["b"].k))))) <= TOL_PERP
    Uo, Po, No = inst[0]["o"].orthogonalize(inst[0]["W"], "pip2", "pip2")
    assert close(host(inst[0]["bufs"][0]), Uo) and close(host(inst[0]["bufs"][2]), No)
