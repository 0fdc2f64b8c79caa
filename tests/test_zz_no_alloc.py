"""The allocation-free entry point lo_tsqr_noalloc, checked against the
allocating path (lo_basis_create + lo_orthogonalize on an empty basis).

Some callers cannot allocate device memory: applications whose device memory
is owned by their own pool and fixed at start-up, or host threads that may not
call cudaMalloc/cudaFree (which synchronize the device).  lo_tsqr_noalloc
serves them with a fixed scratch array inside the library.  This file is
collected last so that a stop-at-first-failure run has run every other test
before it; it also passes when run alone in a fresh process.
"""

import ctypes

import numpy as np
import pytest

from paper_2204_13393_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_REL = 1e-10   # the float64 parity tolerance used by the other GPU tests


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_13393_gb300 import lo

    torch.cuda.set_device(0)
    return lo


def _reference(L, W, cr):
    n, s = W.shape
    b = L.Basis(n, s, 1, cr)
    U, _, R = b.orthogonalize(W)
    torch.cuda.synchronize()
    out = U.cpu().numpy(), R.cpu().numpy()
    b.close()
    return out


def _noalloc(L, W, cr, inplace=False):
    """Call lo_tsqr_noalloc through the C ABI (ctypes), device buffers only."""
    n, s = W.shape
    lib = L.library()
    U = W if inplace else torch.empty(n, s, dtype=torch.float64, device="cuda")
    R = torch.empty(s, s, dtype=torch.float64, device="cuda")
    code = lib.lo_tsqr_noalloc(n, s, cr, ctypes.c_void_p(W.data_ptr()), W.stride(0),
                               ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 0, L.STATUS.get(code, code)
    torch.cuda.synchronize()
    return U.cpu().numpy(), R.cpu().numpy()


def test_noalloc_matches_allocating_path_twice(L):
    """Two calls in a row (different sizes, so the shared scratch holds the
    first call's contents when the second starts), each equal to the
    allocating entry point within the float64 tolerance."""
    for n, s, cr, seed in [(100000, 8, 4096, 11), (37001, 4, 2048, 12)]:
        Wh = I.gaussian(n, s, I.seed_for(7, seed))
        W = torch.from_numpy(Wh).cuda()
        U0, R0 = _reference(L, W, cr)
        U1, R1 = _noalloc(L, W, cr)
        assert _rel(U1, U0) <= TOL_REL
        assert _rel(R1, R0) <= TOL_REL
        assert np.linalg.norm(U1.T @ U1 - np.eye(s)) <= 1e-12
        assert np.allclose(np.tril(R1, -1), 0) and np.all(np.diag(R1) > 0)


def test_noalloc_in_place_and_repeat(L):
    n, s, cr = 50000, 16, 4096
    Wh = I.stewart(n, s, 1e4, I.seed_for(7, 20))
    W = torch.from_numpy(Wh).cuda()
    U0, R0 = _reference(L, W, cr)
    for _ in range(2):
        Wc = W.clone()
        U1, R1 = _noalloc(L, Wc, cr, inplace=True)
        assert _rel(U1, U0) <= TOL_REL
        assert _rel(R1, R0) <= max(TOL_REL, 100 * 1e4 * np.finfo(float).eps)


def test_noalloc_rejects_oversized_problem(L):
    """A problem whose scratch exceeds the fixed array is rejected before any
    device work, with real buffers: 2048 chunks of a 32-column block need far
    more than the array holds (the host-only size query says so too).  The
    output buffers are left untouched."""
    n, s, cr = 65536, 32, 32
    st, need, cap = L.tsqr_noalloc_scratch(n, s, cr)
    assert st == "LO_ERR_CAPACITY" and need > cap
    W = torch.from_numpy(I.gaussian(n, s, I.seed_for(7, 30))).cuda()
    U = torch.full((n, s), 3.0, dtype=torch.float64, device="cuda")
    R = torch.full((s, s), 5.0, dtype=torch.float64, device="cuda")
    lib = L.library()
    code = lib.lo_tsqr_noalloc(n, s, cr, ctypes.c_void_p(W.data_ptr()), s, ctypes.c_void_p(U.data_ptr()),
                               ctypes.c_void_p(R.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 2  # LO_ERR_CAPACITY
    torch.cuda.synchronize()
    assert bool((U == 3.0).all()) and bool((R == 5.0).all())


def test_noalloc_ill_conditioned(L):
    """kappa = 1e8 (the top of the float64 tolerance range): the reiterated
    leaf keeps U^T U = I to 1e-12, and U, R agree with the allocating path."""
    n, s, cr = 60000, 8, 4096
    Wh = I.stewart(n, s, 1e8, I.seed_for(7, 40))
    W = torch.from_numpy(Wh).cuda()
    U0, R0 = _reference(L, W, cr)
    U1, R1 = _noalloc(L, W, cr)
    assert np.linalg.norm(U1.T @ U1 - np.eye(s)) <= 1e-12
    assert np.linalg.norm(Wh - U1 @ R1) / np.linalg.norm(Wh) <= 1e-13
    assert _rel(U1, U0) <= max(TOL_REL, 100 * 1e8 * np.finfo(float).eps)
    assert _rel(R1, R0) <= max(TOL_REL, 100 * 1e8 * np.finfo(float).eps)
