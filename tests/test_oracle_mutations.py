"""The oracle's pins catch plausible mistakes: each case plants one mistake in
a copy of the oracle (on the CPU, never in the committed file) -- a dropped
term, a wrong sign or index, a transposed operand, a skipped reiteration --
and runs the pin suite against the copy, which must fail.  A copy without a
planted mistake must pass, so a failure is the mistake's doing."""

import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ORACLE = os.path.join(ROOT, "oracle", "lo_oracle.py")

# (what is wrong, text in the oracle, replacement)
MUTATIONS = [
    ("Cholesky: row term with a wrong index",
     "N[i, j] = rest[j - i - 1] / N[i, i]", "N[i, j] = rest[j - i - 1] / N[j, j] if N[j, j] else 0.0"),
    ("Cholesky: pivot without the update",
     "d = M[i, i] - sum(N[l, i] * N[l, i] for l in range(i))", "d = M[i, i]"),
    ("substitution: wrong sign",
     "acc -= X[:, l] * N[l, j]", "acc += X[:, l] * N[l, j]"),
    ("Householder: reflector sign",
     "sigma = -_sgn(u[0])", "sigma = _sgn(u[0])"),
    ("sign normalization dropped on R",
     "return Q * d[None, :], R * d[:, None]", "return Q * d[None, :], R"),
    ("MGS2: one sweep instead of two",
     "for _sweep in range(2):", "for _sweep in range(1):"),
    ("PIP: projection left out of U",
     "U = solve_upper_right(X - Q @ P, N)", "U = solve_upper_right(X, N)"),
    ("PIP+: the printed combination (P1 N2 + P2)",
     "return U, P1 + P2 @ N1, N2 @ N1", "return U, P1 @ N2 + P2, N2 @ N1"),
    ("PIP+: normalizers multiplied in the wrong order",
     "return U, P1 + P2 @ N1, N2 @ N1", "return U, P1 + P2 @ N1, N1 @ N2"),
    ("tree: assembly without the prior-basis term",
     "U[b:e] = self.Qloc[i] @ Pt + Ui @ Nt", "U[b:e] = Ui @ Nt"),
    ("tree: T_i stacked transposed",
     "Qs = np.vstack([np.vstack([Ti, np.zeros((s, k))]) for Ti in self.T])",
     "Qs = np.vstack([np.vstack([Ti.T, np.zeros((s, k))]) for Ti in self.T])"),
    ("tree: remainder rows dropped from the last chunk",
     "ends = starts[1:] + [n]", "ends = starts[1:] + [p * chunk_rows]"),
    ("apply_Q: T_i C transposed",
     "return np.vstack([Qi @ (Ti @ C) for Qi, Ti in zip(self.Qloc, self.T)])",
     "return np.vstack([Qi @ (Ti.T @ C) for Qi, Ti in zip(self.Qloc, self.T)])"),
    ("block Arnoldi: H block in the wrong column",
     "H[k:k + s, i * s:(i + 1) * s] = N", "H[k:k + s, max(i - 1, 0) * s:max(i, 1) * s] = N"),
    ("e_perp: Q Q^T instead of Q^T Q",
     "np.eye(Q.shape[1]) - Q.T @ Q", "np.eye(Q.shape[1]) - (Q @ Q.T)[:Q.shape[1], :Q.shape[1]]"),
    ("chunks: remainder as a chunk of its own",
     "    p = max(1, n // chunk_rows)\n", "    p = max(1, -(-n // chunk_rows))\n"),
    ("e_perp: spectral instead of Frobenius norm",
     "return float(np.linalg.norm(np.eye(Q.shape[1]) - Q.T @ Q))",
     "return float(np.linalg.norm(np.eye(Q.shape[1]) - Q.T @ Q, 2))"),
    ("residual: absolute instead of relative",
     "return float(np.linalg.norm(A - Q @ R) / np.linalg.norm(A))", "return float(np.linalg.norm(A - Q @ R))"),
    ("tree: projection block of T_i dropped",
     "Tn[:k, k:] = Pt", "Tn[:k, k:] = 0.0"),
    ("deflation: threshold compared with the squared distance",
     "        if nrm <= thr:\n            continue  # deflated", "        if nrm * nrm <= thr:\n            continue  # deflated"),
    ("deflation: small Cholesky pivots kept",
     "        if deflate > 0.0 and np.isfinite(d) and d <= deflate:",
     "        if deflate > 0.0 and np.isfinite(d) and d < 0.0:"),
    ("deflation: left out of the local solvers",
     "loc.append(pqr(Qi, X[b:e], local, tau if local in (\"pip\", \"pip2\") else 0.0))",
     "loc.append(pqr(Qi, X[b:e], local, 0.0))"),
    ("exact zero component: zero row not kept",
     "        if d == 0.0 and all(r == 0.0 for r in rest):\n            continue",
     "        if d == 0.0 and all(r == 0.0 for r in rest):\n            d = 1.0"),
]


def run_pins(tmp_path, source, name):
    path = tmp_path / f"{name}.py"
    path.write_text(source)
    env = dict(os.environ, LO_ORACLE_MUTANT=str(path))
    cmd = [sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"), "-x", "-q",
           "-p", "no:cacheprovider", "-m", "not gpu"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes(tmp_path):
    r = run_pins(tmp_path, open(ORACLE).read(), "copy")
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, what, old, new):
    src = open(ORACLE).read()
    assert src.count(old) == 1, what
    r = run_pins(tmp_path, src.replace(old, new), "mutant")
    assert r.returncode != 0, f"the pins did not catch: {what}"
