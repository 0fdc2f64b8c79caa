"""The seeded input generators produce what their recipes state (CPU only):
the workloads' shapes, value distributions and structure, deterministically."""

import numpy as np
import pytest

from paper_2204_13393_gb300 import inputs as I


def test_deterministic_and_seed_dependent():
    assert np.array_equal(I.gaussian(100, 4, 7), I.gaussian(100, 4, 7))
    assert not np.array_equal(I.gaussian(100, 4, 7), I.gaussian(100, 4, 8))
    assert I.seed_for(2, 3) == 2204133930 + 2003
    X = I.gaussian(64, 8, 1)
    assert X.flags["C_CONTIGUOUS"] and X.dtype == np.float64 and X.shape == (64, 8)


def test_gaussian_and_uniform_moments():
    X = I.gaussian(200000, 2, 3)
    assert abs(X.mean()) < 0.01 and abs(X.std() - 1.0) < 0.01
    Y = I.uniform(200000, 2, 4)
    assert Y.min() >= -1.0 and Y.max() < 1.0 and abs(Y.mean()) < 0.01
    assert abs(Y.var() - 1.0 / 3.0) < 0.01


def test_haar_is_orthonormal():
    Q = I.haar(300, 12, 5)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-13)


@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e10])
def test_stewart_singular_values(kappa):
    """U diag(sigma) V^T with sigma_j = kappa^(-j/(m-1)) (Sec. 6.1)."""
    m = 8
    A = I.stewart(2000, m, kappa, 6)
    sv = np.linalg.svd(A, compute_uv=False)
    want = kappa ** (-np.arange(m) / (m - 1.0))
    np.testing.assert_allclose(sv, want, rtol=1e-6 if kappa > 1e8 else 1e-10)


def test_localized_support():
    n, s = 1000, 3
    X = I.localized(n, s, 8, [[(0, 100), (500, 600)], [], [(990, 1000)]])
    assert np.all(X[:, 1] == 0.0)
    assert np.all(X[100:500, 0] == 0.0) and np.all(X[600:, 0] == 0.0)
    assert np.all(X[:100, 0] != 0.0) and np.all(X[500:600, 0] != 0.0)
    assert np.all(X[:990, 2] == 0.0) and np.all(X[990:, 2] != 0.0)
    assert np.array_equal(X[:100, 0], I.gaussian(n, s, 8)[:100, 0])


def test_batch_instances_ranges():
    specs = I.batch_instances(64, 11)
    assert len(specs) == 64
    ns = np.array([n for n, _, _ in specs])
    assert ns.min() >= 1e4 and ns.max() <= 2 ** 20
    assert {s for _, s, _ in specs} <= {4, 8, 16} and len({s for _, s, _ in specs}) == 3
    assert all(1 <= kb <= 30 for _, _, kb in specs)
    # log-uniform: about half of the n lie below the geometric midpoint
    assert 20 <= int(np.sum(ns < np.sqrt(1e4 * 2 ** 20))) <= 44
