"""Thin Python binding of the C ABI in include/lo.h (argument marshalling only).

Every step of the orthogonalization runs in the CUDA library ``liblo.so``;
this module only converts tensors/arrays to pointers and strides and status
codes to exceptions.  If the library has not been built it raises: there is no
Python or CPU fallback.

Matrices are float64 and row-major with unit column stride: torch tensors
(CUDA or CPU) or numpy arrays.  The row stride is passed as ``ld``.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int32, c_int64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblo.so")

STATUS = {
    0: "LO_OK",
    1: "LO_ERR_INVALID_ARG",
    2: "LO_ERR_CAPACITY",
    3: "LO_ERR_CHUNK_TOO_SMALL",
    4: "LO_ERR_BREAKDOWN",
    5: "LO_ERR_NONFINITE",
    6: "LO_ERR_TIMEOUT",
    7: "LO_ERR_CUDA",
    8: "LO_ERR_OOM",
    9: "LO_ERR_UNSUPPORTED",
}
PRECISION = {"fp64": 0, "mixed_fp32": 1, "fp64_tc": 2, "mixed_tc": 3}
LEAF = {"auto": 0, "pip": 1, "pip2": 2, "hh": 3}
REDUCTION = {"auto": 0, "pip": 1, "pip2": 2}

EXPORTED = [
    "lo_options_default", "lo_status_string", "lo_basis_create", "lo_basis_destroy",
    "lo_basis_reset", "lo_basis_num_blocks", "lo_basis_num_chunks", "lo_basis_sync",
    "lo_orthogonalize", "lo_orthogonalize_batched", "lo_apply_Q", "lo_basis_export_chunk",
    "lo_laplace5_apply", "lo_launch_count", "lo_basis_set_profiling", "lo_basis_profile_read",
    "lo_basis_last_step_info", "lo_tsqr_noalloc", "lo_tsqr_noalloc_scratch", "lo_basis_truncate",
    "lo_tune_chunk_rows", "lo_basis_id", "lo_batched_cache_entries", "lo_basis_last_rank",
    "lo_set_batched_route", "lo_batched_persistent_count", "lo_orthogonalize_laplace5", "lo_tune_leaf",
]
KERNEL_GROUPS = ["gram", "leaf", "tree", "update", "apply_q", "refine"]


class LoError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = int(code)
        self.name = STATUS.get(self.code, str(code))
        super().__init__(f"{where}: {self.name} ({_lib().lo_status_string(self.code).decode()})")


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("leaf", c_int32), ("reduction", c_int32),
                ("sync", c_int32), ("refine_tol", c_double), ("digit_planes", c_int32),
                ("test_stall", c_int32), ("deflation_tol", c_double)]


_L = None


def _lib():
    global _L
    if _L is not None:
        return _L
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(LIB_PATH)
    L.lo_options_default.argtypes = [POINTER(Options)]
    L.lo_options_default.restype = None
    L.lo_status_string.argtypes = [c_int32]
    L.lo_status_string.restype = c_char_p
    L.lo_basis_create.argtypes = [c_int64, c_int32, c_int32, c_int32, POINTER(Options), c_void_p,
                                  POINTER(c_void_p)]
    L.lo_basis_create.restype = c_int32
    L.lo_basis_destroy.argtypes = [c_void_p]
    L.lo_basis_destroy.restype = None
    L.lo_basis_reset.argtypes = [c_void_p]
    L.lo_basis_reset.restype = c_int32
    L.lo_basis_num_blocks.argtypes = [c_void_p]
    L.lo_basis_num_blocks.restype = c_int32
    L.lo_basis_num_chunks.argtypes = [c_void_p]
    L.lo_basis_num_chunks.restype = c_int32
    L.lo_basis_sync.argtypes = [c_void_p]
    L.lo_basis_sync.restype = c_int32
    L.lo_orthogonalize.argtypes = [c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_void_p]
    L.lo_orthogonalize.restype = c_int32
    L.lo_orthogonalize_batched.argtypes = [POINTER(c_void_p), c_int32, POINTER(c_void_p), POINTER(c_int64),
                                           POINTER(c_void_p), POINTER(c_int64), POINTER(c_void_p),
                                           POINTER(c_void_p)]
    L.lo_orthogonalize_batched.restype = c_int32
    L.lo_apply_Q.argtypes = [c_void_p, c_void_p, c_int32, c_int64, c_void_p, c_int64]
    L.lo_apply_Q.restype = c_int32
    L.lo_basis_export_chunk.argtypes = [c_void_p, c_int32, c_void_p, c_void_p, POINTER(c_int64)]
    L.lo_basis_export_chunk.restype = c_int32
    L.lo_laplace5_apply.argtypes = [c_int32, c_int32, c_int32, c_void_p, c_int64, c_void_p, c_int64, c_void_p]
    L.lo_laplace5_apply.restype = c_int32
    L.lo_launch_count.argtypes = []
    L.lo_launch_count.restype = ctypes.c_longlong
    L.lo_basis_set_profiling.argtypes = [c_void_p, c_int32]
    L.lo_basis_set_profiling.restype = c_int32
    L.lo_basis_profile_read.argtypes = [c_void_p, POINTER(c_double), POINTER(c_int64), c_int32]
    L.lo_basis_profile_read.restype = c_int32
    L.lo_basis_last_step_info.argtypes = [c_void_p, POINTER(c_int32), POINTER(c_int32)]
    L.lo_basis_last_step_info.restype = c_int32
    L.lo_orthogonalize_laplace5.argtypes = [c_void_p, c_int32, c_int32, c_void_p, c_int64, c_void_p, c_int64,
                                            c_void_p, c_void_p]
    L.lo_orthogonalize_laplace5.restype = c_int32
    L.lo_tune_leaf.argtypes = [c_int64, c_int32, c_int32, POINTER(Options), c_void_p, POINTER(c_int32),
                               POINTER(c_int32)]
    L.lo_tune_leaf.restype = c_int32
    L.lo_set_batched_route.argtypes = [c_int32]
    L.lo_set_batched_route.restype = c_int32
    L.lo_batched_persistent_count.argtypes = []
    L.lo_batched_persistent_count.restype = c_int32
    L.lo_basis_last_rank.argtypes = [c_void_p, POINTER(c_int32)]
    L.lo_basis_last_rank.restype = c_int32
    L.lo_tsqr_noalloc.argtypes = [c_int64, c_int32, c_int32, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]
    L.lo_tsqr_noalloc.restype = c_int32
    L.lo_tsqr_noalloc_scratch.argtypes = [c_int64, c_int32, c_int32, POINTER(ctypes.c_uint64),
                                          POINTER(ctypes.c_uint64)]
    L.lo_tsqr_noalloc_scratch.restype = c_int32
    L.lo_basis_id.argtypes = [c_void_p]
    L.lo_basis_id.restype = ctypes.c_uint64
    L.lo_batched_cache_entries.argtypes = [ctypes.c_uint64]
    L.lo_batched_cache_entries.restype = c_int32
    L.lo_basis_truncate.argtypes = [c_void_p, c_int32]
    L.lo_basis_truncate.restype = c_int32
    L.lo_tune_chunk_rows.argtypes = [c_int64, c_int32, c_int32, POINTER(Options), c_void_p, POINTER(c_int32)]
    L.lo_tune_chunk_rows.restype = c_int32
    _L = L
    return L


def library():
    """The loaded ctypes library (loads it on first use)."""
    return _lib()


def _check(code: int, where: str):
    if code != 0:
        raise LoError(code, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return x.data_ptr()
    return x.ctypes.data


def _ld(x, cols: int) -> int:
    """Row stride (elements) of a row-major float64 matrix with unit column stride."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float64:
            raise TypeError("float64 required")
        if x.dim() != 2 or (x.shape[1] > 1 and x.stride(1) != 1):
            raise ValueError("2D row-major tensor with unit column stride required")
        return int(x.stride(0)) if x.shape[0] > 1 else max(cols, int(x.stride(0)))
    if x.dtype != np.float64 or x.ndim != 2 or (x.shape[1] > 1 and x.strides[1] != 8):
        raise ValueError("2D float64 row-major array with unit column stride required")
    return int(x.strides[0] // 8) if x.shape[0] > 1 else cols


def _stream_handle(stream) -> int:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _empty_like_kind(ref, shape):
    if _is_torch(ref):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=ref.device)
    return np.empty(shape, dtype=np.float64)


class Basis:
    """A locally orthogonal basis (lo_basis) on the current CUDA device."""

    def __init__(self, n: int, s: int, max_blocks: int, chunk_rows: int, precision: str = "fp64",
                 leaf: str = "pip2", reduction: str = "auto", sync: bool = True,
                 refine_tol: float = 0.0, stream=None, digit_planes: bool = True, test_stall: bool = False,
                 deflation_tol: float = 0.0):
        L = _lib()
        o = Options()
        L.lo_options_default(ctypes.byref(o))
        o.precision = PRECISION[precision]
        o.leaf = LEAF[leaf]
        o.reduction = REDUCTION[reduction]
        o.sync = 1 if sync else 0
        if refine_tol > 0:
            o.refine_tol = refine_tol
        o.digit_planes = 0 if digit_planes else 1
        o.test_stall = int(test_stall)
        o.deflation_tol = float(deflation_tol)
        h = c_void_p()
        self._h = None
        _check(L.lo_basis_create(int(n), int(s), int(max_blocks), int(chunk_rows), ctypes.byref(o),
                                 c_void_p(_stream_handle(stream)), ctypes.byref(h)), "lo_basis_create")
        self._h = h
        self.n, self.s, self.max_blocks, self.chunk_rows = int(n), int(s), int(max_blocks), int(chunk_rows)

    def close(self):
        if self._h is not None:
            _lib().lo_basis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def id(self) -> int:
        """Process-unique id of the basis (never reused)."""
        return int(_lib().lo_basis_id(self._h))

    @property
    def num_blocks(self) -> int:
        return _lib().lo_basis_num_blocks(self._h)

    @property
    def num_chunks(self) -> int:
        return _lib().lo_basis_num_chunks(self._h)

    @property
    def k(self) -> int:
        return self.num_blocks * self.s

    def reset(self):
        _check(_lib().lo_basis_reset(self._h), "lo_basis_reset")

    def sync(self):
        _check(_lib().lo_basis_sync(self._h), "lo_basis_sync")

    def orthogonalize(self, W, U=None, H=None, R=None, want_h=True):
        """One PQR step.  Returns (U, H, R); outputs default to W's kind."""
        k = self.k
        if U is None:
            U = _empty_like_kind(W, (self.n, self.s))
        if want_h and H is None and k > 0:
            H = _empty_like_kind(W, (k, self.s))
        if R is None:
            R = _empty_like_kind(W, (self.s, self.s))
        _check(_lib().lo_orthogonalize(self._h, _ptr(W), _ld(W, self.s), _ptr(U), _ld(U, self.s),
                                       _ptr(H) if k > 0 else None, _ptr(R)), "lo_orthogonalize")
        return U, H, R

    def orthogonalize_laplace5(self, nx: int, ny: int, V, U=None, H=None, R=None):
        """One block-Arnoldi step with the 5-point Laplacian fused in: the PQR
        step of W = L V (device tensors; U must not overlap V)."""
        k = self.k
        if U is None:
            U = _empty_like_kind(V, (self.n, self.s))
        if H is None and k > 0:
            H = _empty_like_kind(V, (k, self.s))
        if R is None:
            R = _empty_like_kind(V, (self.s, self.s))
        _check(_lib().lo_orthogonalize_laplace5(self._h, int(nx), int(ny), _ptr(V), _ld(V, self.s), _ptr(U),
                                                _ld(U, self.s), _ptr(H) if k > 0 else None, _ptr(R)),
               "lo_orthogonalize_laplace5")
        return U, H, R

    def apply_Q(self, C, Y=None):
        """Y = Q C (C is k x m)."""
        m = int(C.shape[1])
        if Y is None:
            Y = _empty_like_kind(C, (self.n, m))
        _check(_lib().lo_apply_Q(self._h, _ptr(C), m, _ld(C, m), _ptr(Y), _ld(Y, m)), "lo_apply_Q")
        return Y

    def truncate(self, num_blocks: int):
        _check(_lib().lo_basis_truncate(self._h, int(num_blocks)), "lo_basis_truncate")

    def last_rank(self) -> int:
        """Rank of the last step's normalizer R (< s only with deflation)."""
        t = c_int32()
        _check(_lib().lo_basis_last_rank(self._h, ctypes.byref(t)), "lo_basis_last_rank")
        return t.value

    def last_step_info(self):
        """(local Gram passes, reduction iterations) of the last step."""
        a, t = c_int32(), c_int32()
        _check(_lib().lo_basis_last_step_info(self._h, ctypes.byref(a), ctypes.byref(t)),
               "lo_basis_last_step_info")
        return a.value, t.value

    def set_profiling(self, enable: bool = True):
        _check(_lib().lo_basis_set_profiling(self._h, 1 if enable else 0), "lo_basis_set_profiling")

    def profile_read(self):
        """{group: (milliseconds, intervals)} since the last read."""
        ms = (c_double * 8)()
        cnt = (c_int64 * 8)()
        _check(_lib().lo_basis_profile_read(self._h, ms, cnt, 8), "lo_basis_profile_read")
        return {g: (ms[i], cnt[i]) for i, g in enumerate(KERNEL_GROUPS)}

    def export_chunk(self, chunk: int):
        """(Q_i, T_i) of one chunk as numpy arrays (host copies)."""
        k = self.k
        rows = c_int64()
        _check(_lib().lo_basis_export_chunk(self._h, int(chunk), None, None, ctypes.byref(rows)),
               "lo_basis_export_chunk")
        Qi = np.zeros((rows.value, k))
        Ti = np.zeros((k, k))
        _check(_lib().lo_basis_export_chunk(self._h, int(chunk), Qi.ctypes.data if k else None,
                                            Ti.ctypes.data if k else None, ctypes.byref(rows)),
               "lo_basis_export_chunk")
        return Qi, Ti


def orthogonalize_batched(bases, Ws, Us, Hs=None, Rs=None):
    """lo_orthogonalize_batched: torch tensors (device or host) or numpy arrays."""
    cnt = len(bases)
    arr = lambda vals, t: (t * cnt)(*vals)
    hb = arr([b.handle.value for b in bases], c_void_p)
    pw = arr([_ptr(w) for w in Ws], c_void_p)
    pu = arr([_ptr(u) for u in Us], c_void_p)
    lw = arr([_ld(w, b.s) for w, b in zip(Ws, bases)], c_int64)
    lu = arr([_ld(u, b.s) for u, b in zip(Us, bases)], c_int64)
    ph = arr([_ptr(h) for h in Hs], c_void_p) if Hs is not None else None
    pr = arr([_ptr(r) for r in Rs], c_void_p) if Rs is not None else None
    _check(_lib().lo_orthogonalize_batched(hb, cnt, pw, lw, pu, lu, ph, pr), "lo_orthogonalize_batched")


def tsqr_noalloc_scratch(n: int, s: int, chunk_rows: int):
    """(status name, bytes needed, bytes available) of lo_tsqr_noalloc's scratch
    for this problem (host-only)."""
    need, cap = ctypes.c_uint64(), ctypes.c_uint64()
    code = _lib().lo_tsqr_noalloc_scratch(int(n), int(s), int(chunk_rows), ctypes.byref(need), ctypes.byref(cap))
    return STATUS.get(code, str(code)), int(need.value), int(cap.value)


BATCH_ROUTE = {"auto": 0, "persistent": 1, "graph": 2}


def set_batched_route(mode: str = "auto"):
    """Route of lo_orthogonalize_batched's instances: 'auto', 'persistent'
    (the persistent launch wherever it can run) or 'graph'."""
    _check(_lib().lo_set_batched_route(BATCH_ROUTE[mode]), "lo_set_batched_route")


def batched_persistent_count() -> int:
    """Instances the last batched graph runs in the persistent launch."""
    return int(_lib().lo_batched_persistent_count())


def batched_cache_entries(basis_id: int = 0) -> int:
    """Cached batched graphs that name the basis with this id (0: all)."""
    return int(_lib().lo_batched_cache_entries(int(basis_id)))


def tsqr_noalloc(W, U, R, chunk_rows: int, stream=None):
    """lo_tsqr_noalloc: W = U R without any device allocation (device tensors;
    U contiguous n x s, R s x s)."""
    n, s = int(W.shape[0]), int(W.shape[1])
    _check(_lib().lo_tsqr_noalloc(n, s, int(chunk_rows), _ptr(W), _ld(W, s), _ptr(U), _ptr(R),
                                  c_void_p(_stream_handle(stream))), "lo_tsqr_noalloc")
    return U, R


def tune_chunk_rows(n: int, s: int, max_blocks: int, precision: str = "fp64", leaf: str = "pip2",
                    stream=None) -> int:
    """lo_tune_chunk_rows: the fastest chunk size for this shape (measured)."""
    L = _lib()
    o = Options()
    L.lo_options_default(ctypes.byref(o))
    o.precision = PRECISION[precision]
    o.leaf = LEAF[leaf]
    out = c_int32()
    _check(L.lo_tune_chunk_rows(int(n), int(s), int(max_blocks), ctypes.byref(o),
                                c_void_p(_stream_handle(stream)), ctypes.byref(out)), "lo_tune_chunk_rows")
    return out.value


def tune_leaf(n: int, s: int, max_blocks: int, precision: str = "fp64", stream=None):
    """lo_tune_leaf: (leaf name, chunk rows) of the faster leaf for this shape (measured)."""
    L = _lib()
    o = Options()
    L.lo_options_default(ctypes.byref(o))
    o.precision = PRECISION[precision]
    leaf, cr = c_int32(), c_int32()
    _check(L.lo_tune_leaf(int(n), int(s), int(max_blocks), ctypes.byref(o), c_void_p(_stream_handle(stream)),
                          ctypes.byref(leaf), ctypes.byref(cr)), "lo_tune_leaf")
    return {v: k for k, v in LEAF.items()}[leaf.value], cr.value


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(_lib().lo_launch_count())


def laplace5_apply(nx: int, ny: int, X, Y, stream=None):
    s = int(X.shape[1])
    _check(_lib().lo_laplace5_apply(int(nx), int(ny), s, _ptr(X), _ld(X, s), _ptr(Y), _ld(Y, s),
                                    c_void_p(_stream_handle(stream))), "lo_laplace5_apply")
    return Y
