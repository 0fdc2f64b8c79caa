"""Host-side checks that need no GPU: the library builds, loads, exports every
symbol include/lo.h declares, and rejects bad arguments before any device work."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_13393_gb300 import build, lo

    if not os.path.exists(lo.LIB_PATH):
        build.build()
    return lo.library()


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(lo_[a-zA-Z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ["lo_basis_create", "lo_orthogonalize", "lo_apply_Q", "lo_basis_destroy",
                 "lo_orthogonalize_batched"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_exports(lib):
    from paper_2204_13393_gb300 import lo

    assert set(lo.EXPORTED) <= set(declared_symbols())


def test_status_strings(lib):
    for code in range(10):
        assert lib.lo_status_string(code)
    assert lib.lo_status_string(4).decode().startswith("Cholesky")


def test_create_rejects_bad_arguments_without_device(lib):
    """Validation happens before any CUDA call, so it runs on a CPU-only host."""
    from paper_2204_13393_gb300 import lo

    h = ctypes.c_void_p()
    cases = [
        ((0, 4, 8, 512), 1),           # n < 1
        ((4096, 0, 8, 512), 1),        # s < 1
        ((4096, 33, 8, 512), 1),       # s > 32
        ((4096, 4, 0, 512), 1),        # max_blocks < 1
        ((4096, 32, 64, 4096), 1),     # max_blocks*s > 1024 ... and k*s too large
        ((4096, 4, 8, 16), 3),         # chunk_rows < max_blocks*s
        ((20, 4, 8, 512), 3),          # single chunk with n < max_blocks*s
    ]
    for (n, s, M, cr), want in cases:
        code = lib.lo_basis_create(n, s, M, cr, None, None, ctypes.byref(h))
        assert code == want, ((n, s, M, cr), code)
        assert h.value is None
    bad = lo.Options()
    lib.lo_options_default(ctypes.byref(bad))
    bad.leaf = 7
    assert lib.lo_basis_create(4096, 4, 8, 512, ctypes.byref(bad), None, ctypes.byref(h)) == 1
    lib.lo_options_default(ctypes.byref(bad))
    bad.digit_planes = 2
    assert lib.lo_basis_create(4096, 4, 8, 512, ctypes.byref(bad), None, ctypes.byref(h)) == 1
    lib.lo_options_default(ctypes.byref(bad))
    bad.test_stall = 3
    assert lib.lo_basis_create(4096, 4, 8, 512, ctypes.byref(bad), None, ctypes.byref(h)) == 1


def test_null_handles_are_rejected(lib):
    assert lib.lo_orthogonalize(None, None, 4, None, 4, None, None) == 1
    assert lib.lo_apply_Q(None, None, 1, 1, None, 1) == 1
    assert lib.lo_basis_num_blocks(None) == -1
    lib.lo_basis_destroy(None)


def test_options_default(lib):
    from paper_2204_13393_gb300 import lo

    o = lo.Options()
    lib.lo_options_default(ctypes.byref(o))
    assert (o.precision, o.leaf, o.reduction, o.sync) == (0, 2, 0, 1)
    assert o.refine_tol == pytest.approx(1e-13)
    assert (o.digit_planes, o.test_stall) == (0, 0)
    assert o.deflation_tol == 0.0
    assert ctypes.sizeof(o) == 40


def test_tuner_and_noalloc_reject_bad_arguments_without_device(lib):
    """lo_tune_chunk_rows and lo_tsqr_noalloc validate before any CUDA call."""
    import numpy as np

    out = ctypes.c_int32(-1)
    assert lib.lo_tune_chunk_rows(4096, 4, 8, None, None, None) == 1                  # no output
    for n, s, M, want in ((0, 4, 8, 1), (4096, 0, 8, 1), (4096, 33, 8, 1), (4096, 4, 0, 1),
                          (4096, 32, 64, 3), (20, 4, 8, 3)):
        assert lib.lo_tune_chunk_rows(n, s, M, None, None, ctypes.byref(out)) == want, (n, s, M)
    W = np.zeros((64, 8))
    U = np.zeros((64, 8))
    R = np.zeros((8, 8))
    w, u, r = W.ctypes.data, U.ctypes.data, R.ctypes.data
    cases = [
        ((0, 8, 16, w, 8, u, r), 1),           # n < 1
        ((64, 0, 16, w, 8, u, r), 1),          # s < 1
        ((64, 33, 16, w, 33, u, r), 1),        # s > 32
        ((64, 8, 0, w, 8, u, r), 1),           # chunk_rows < 1
        ((64, 8, 16, None, 8, u, r), 1),       # no W
        ((64, 8, 16, w, 8, None, r), 1),       # no U
        ((64, 8, 16, w, 8, u, None), 1),       # no R
        ((64, 8, 16, w, 7, u, r), 1),          # ldw < s
        ((32, 8, 16, w, 16, w, r), 1),         # in place with a strided block
        ((64, 8, 16, w, 8, w + 8, r), 1),      # distinct but overlapping buffers
        ((64, 8, 4, w, 8, u, r), 3),           # chunks shorter than s
        ((4, 8, 16, w, 8, u, r), 3),           # one chunk shorter than s
    ]
    for args, want in cases:
        assert lib.lo_tsqr_noalloc(*args, None) == want, args


def test_noalloc_scratch_query_without_device(lib):
    """lo_tsqr_noalloc_scratch sizes the fixed scratch on the host alone: small
    problems fit, tiny chunks of a wide block do not, and bad sizes give the
    entry point's own argument errors."""
    from paper_2204_13393_gb300 import lo

    st, need, cap = lo.tsqr_noalloc_scratch(100000, 8, 4096)
    assert st == "LO_OK" and 0 < need <= cap and cap == 16 << 20
    st2, need2, _ = lo.tsqr_noalloc_scratch(200000, 8, 4096)
    assert st2 == "LO_OK" and need2 > need            # more chunks and slabs, more scratch
    st, need, cap = lo.tsqr_noalloc_scratch(65536, 32, 32)   # 2048 chunks of 32 x 32 factors
    assert st == "LO_ERR_CAPACITY" and need > cap
    st, need, cap = lo.tsqr_noalloc_scratch(2 ** 26, 32, 512)
    assert st == "LO_ERR_CAPACITY" and need > cap
    assert lo.tsqr_noalloc_scratch(0, 8, 16)[0] == "LO_ERR_INVALID_ARG"
    assert lo.tsqr_noalloc_scratch(64, 33, 16)[0] == "LO_ERR_INVALID_ARG"
    assert lo.tsqr_noalloc_scratch(64, 8, 4)[0] == "LO_ERR_CHUNK_TOO_SMALL"
    assert lib.lo_tsqr_noalloc_scratch(64, 8, 16, None, None) == 0


def test_batched_cache_hooks_without_device(lib):
    """The cache inspection hooks are host-only: no basis, no entries."""
    assert lib.lo_basis_id(None) == 0
    assert lib.lo_batched_cache_entries(0) == 0
    assert lib.lo_batched_cache_entries(12345) == 0


def test_householder_leaf_option_without_device(lib):
    """LO_LEAF_HH passes validation for any chunk size (chunks larger than one
    tile are walked as sub-tiles), so on a CPU-only host create gets as far as
    the device allocation; leaf values past LO_LEAF_HH are rejected."""
    from paper_2204_13393_gb300 import lo

    h = ctypes.c_void_p()
    o = lo.Options()
    lib.lo_options_default(ctypes.byref(o))
    o.leaf = lo.LEAF["hh"]
    for n, s, cr in ((2 ** 20, 8, 4096), (100000, 32, 1024), (6000, 8, 512)):
        assert lib.lo_basis_create(n, s, 1, cr, ctypes.byref(o), None, ctypes.byref(h)) not in (1, 3, 9), (n, s, cr)
        assert h.value is None
    o.leaf = 4
    assert lib.lo_basis_create(4096, 4, 1, 512, ctypes.byref(o), None, ctypes.byref(h)) == 1


def test_deflation_option_checks_without_device(lib):
    """deflation_tol must be finite and >= 0, and is for the float64 forms
    only (the mixed forms' first pass cannot resolve the distances)."""
    from paper_2204_13393_gb300 import lo

    h = ctypes.c_void_p()
    o = lo.Options()
    for prec, tol, want in (("fp64", -1.0, 1), ("fp64", float("nan"), 1), ("fp64", float("inf"), 1),
                            ("mixed_fp32", 1e-6, 9), ("mixed_tc", 1e-6, 9)):
        lib.lo_options_default(ctypes.byref(o))
        o.precision = lo.PRECISION[prec]
        o.deflation_tol = tol
        assert lib.lo_basis_create(4096, 8, 4, 512, ctypes.byref(o), None, ctypes.byref(h)) == want, (prec, tol)
        assert h.value is None


def test_tune_leaf_rejects_bad_arguments_without_device(lib):
    out1, out2 = ctypes.c_int32(-1), ctypes.c_int32(-1)
    assert lib.lo_tune_leaf(4096, 4, 8, None, None, None, ctypes.byref(out2)) == 1
    assert lib.lo_tune_leaf(4096, 4, 8, None, None, ctypes.byref(out1), None) == 1
    assert lib.lo_tune_leaf(0, 4, 8, None, None, ctypes.byref(out1), ctypes.byref(out2)) == 1
