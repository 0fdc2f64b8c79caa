"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and builds test matrices; it contains
none of the orthogonalization arithmetic.  Both the CUDA path's tests/bench
and the CPU oracle take their inputs from here, so both sides see bit-identical
float64 data.

* Gaussian blocks (the Krylov blocks of a block Arnoldi run, Alg. 1).
* Stewart matrices X = U diag(sigma) V^T with singular values spaced
  exponentially between 1/kappa and 1 (Sec. 6.1, after Stewart 2008).
* Haar-distributed orthonormal factors: the sign-fixed QR of a Gaussian matrix
  (Mezzadri 2007), computed with LAPACK through numpy (input generation only).
* The uneven batch of the batched workload: n log-uniform, s from {4, 8, 16},
  prior blocks uniform in [1, 30].
* Localized blocks: Gaussian columns that are exactly zero outside given row
  ranges (the degenerate case of a block that vanishes on whole chunks).
"""

from __future__ import annotations

import numpy as np

SEED_BASE = 2204133930


def seed_for(workload: int, instance: int = 0) -> int:
    """Deterministic seed of one input of one workload."""
    return SEED_BASE + 1000 * int(workload) + int(instance)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def gaussian(n: int, s: int, seed: int) -> np.ndarray:
    """n x s block with i.i.d. N(0, 1) entries (C-contiguous, row-major)."""
    return np.ascontiguousarray(rng(seed).standard_normal((n, s)))


def uniform(n: int, s: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n x s block with i.i.d. U(lo, hi) entries."""
    return np.ascontiguousarray(rng(seed).uniform(lo, hi, size=(n, s)))


def haar(n: int, m: int, seed: int) -> np.ndarray:
    """n x m matrix with Haar-distributed orthonormal columns (m <= n)."""
    g = rng(seed).standard_normal((n, m))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return np.ascontiguousarray(q * d[None, :])


def stewart(n: int, s: int, kappa: float, seed: int) -> np.ndarray:
    """Stewart matrix: U diag(sigma) V^T with U (n x s) and V (s x s) Haar and
    sigma_j = kappa^(-j/(s-1)), j = 0..s-1 (from 1 down to 1/kappa).  For
    s = 1 the condition number is 1 whatever kappa is."""
    U = haar(n, s, seed)
    V = haar(s, s, seed + 7919)
    if s == 1:
        sig = np.ones(1)
    else:
        sig = np.asarray(float(kappa)) ** (-np.arange(s) / (s - 1.0))
    return np.ascontiguousarray((U * sig[None, :]) @ V.T)


def localized(n: int, s: int, seed: int, supports) -> np.ndarray:
    """n x s block whose column j is N(0, 1) on the row ranges supports[j]
    (a list of (begin, end) pairs) and exactly zero elsewhere: a block of
    point-source-like right-hand sides, which vanishes on most row chunks."""
    X = gaussian(n, s, seed)
    keep = np.zeros((n, s), dtype=bool)
    for j, ranges in enumerate(supports):
        for b, e in ranges:
            keep[b:e, j] = True
    X[~keep] = 0.0
    return np.ascontiguousarray(X)


def batch_instances(count: int, seed: int, n_lo: float = 1e4, n_hi: float = 2.0 ** 20,
                    widths=(4, 8, 16), k_lo: int = 1, k_hi: int = 30):
    """(n, s, prior_blocks) for ``count`` uneven problems: n log-uniform in
    [n_lo, n_hi], s uniform over ``widths``, prior blocks uniform in [k_lo, k_hi]."""
    g = rng(seed)
    out = []
    for _ in range(count):
        n = int(round(np.exp(g.uniform(np.log(n_lo), np.log(n_hi)))))
        s = int(g.choice(np.asarray(widths)))
        kb = int(g.integers(k_lo, k_hi + 1))
        out.append((n, s, kb))
    return out
