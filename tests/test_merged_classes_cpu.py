"""The error of the merged digit classes of the 16-output tensor-core
assembly, in an exact model of its arithmetic (CPU, no GPU, no oracle).

The assembly splits each float64 operand into 7 digits of 8 bits aligned to
its column's largest exponent and multiplies the digit pairs (t, u), t + u <= 8,
with float32 accumulation over an interval of 256 terms.  Classes v = t + u <= 5
keep one exact accumulator per pair; the pairs of each class 6, 7, 8 share one
float32 accumulator that every step (16 terms) of every digit t adds to.  The
claim: the merged classes change an output by less than 2^-46 of
256 max|a| max|b| (in units of the column alignment), whether the float32
additions round to nearest or truncate.  Here the digit products and their
per-step partial sums are exact integers, the accumulator additions are
rounded (or truncated) to 24 significant bits, and the result is compared
with the all-exact class sums.
"""

import math
import random

import pytest

K = 256      # terms per accumulation interval
STEP = 16    # terms per MMA (K of one instruction)


def digits(m):
    """7 digits of 8 bits of a 56-bit aligned magnitude, most significant first."""
    return [(m >> (8 * (7 - t))) & 0xFF for t in range(1, 8)]


def to24(x, mode):
    """x (an integer) rounded to 24 significant bits: to nearest even, or toward zero."""
    if x == 0:
        return 0
    a = abs(x)
    sh = a.bit_length() - 24
    if sh <= 0:
        return x
    q, r = divmod(a, 1 << sh)
    if mode == "rn":
        half = 1 << (sh - 1)
        if r > half or (r == half and (q & 1)):
            q += 1
    return (q << sh) if x > 0 else -(q << sh)


def class_sums(da, sa, db, sb, mode):
    """Exact class sums S_v (v = 2..8) and the merged ones (classes 6..8 through a
    24-bit accumulator, steps of 16 terms, digits t = 1..7 in order)."""
    exact = {v: 0 for v in range(2, 9)}
    merged = {v: 0 for v in range(6, 9)}
    for k0 in range(0, K, STEP):
        for t in range(1, 8):
            for v in range(max(6, t + 1), 9):
                u = v - t
                part = sum(sa[k] * sb[k] * da[k][t - 1] * db[k][u - 1] for k in range(k0, k0 + STEP))
                merged[v] = to24(merged[v] + part, mode)
            for u in range(1, 9 - t):
                exact[t + u] += sum(sa[k] * sb[k] * da[k][t - 1] * db[k][u - 1] for k in range(k0, k0 + STEP))
    return exact, merged


def merged_error(exact, merged):
    """|change of the output| in units of the digit products of class 14 (2^(8 (14 - v))
    per unit of class v): the classes 6..8 weigh 2^64, 2^56, 2^48."""
    return sum(abs(merged[v] - exact[v]) * 2 ** (8 * (14 - v)) for v in range(6, 9))


BOUND = 2.0 ** -46 * K * 2 ** 112   # 256 max|a| max|b| in the same units (56-bit magnitudes)


def random_case(rng, kind):
    if kind == "full":      # every digit 255, equal signs: the largest class sums (exact: multiples of 16 255^2)
        da = [[255] * 7 for _ in range(K)]
        db = [[255] * 7 for _ in range(K)]
        sa = [1] * K
        sb = [1] * K
    elif kind == "mixed":   # random 56-bit magnitudes and signs
        da = [digits(rng.getrandbits(56)) for _ in range(K)]
        db = [digits(rng.getrandbits(56)) for _ in range(K)]
        sa = [rng.choice((-1, 1)) for _ in range(K)]
        sb = [rng.choice((-1, 1)) for _ in range(K)]
    else:                   # large leading digits, random low ones
        da = [[255] + [rng.randrange(256) for _ in range(6)] for _ in range(K)]
        db = [[255] + [rng.randrange(256) for _ in range(6)] for _ in range(K)]
        sa = [1] * K
        sb = [1] * K
    return da, sa, db, sb


@pytest.mark.parametrize("mode", ["rn", "rz"])
@pytest.mark.parametrize("kind", ["full", "mixed", "lead"])
def test_merged_class_error_below_bound(mode, kind):
    rng = random.Random(7100 + 10 * ["rn", "rz"].index(mode) + ["full", "mixed", "lead"].index(kind))
    da, sa, db, sb = random_case(rng, kind)
    exact, merged = class_sums(da, sa, db, sb, mode)
    err = merged_error(exact, merged)
    assert err < BOUND, (kind, mode, math.log2(err) if err else None)
    if kind == "lead":
        # full leading digits and random low ones: the accumulators pass 2^24
        # with odd low bits, so the merged sums do round
        assert any(merged[v] != exact[v] for v in range(6, 9))


def test_model_is_exact_below_24_bits():
    """With class sums below 2^24 the merged accumulators are exact (the model
    adds nothing of its own): a single term per interval."""
    da = [[255] * 7] + [[0] * 7 for _ in range(K - 1)]
    db = [[255] * 7] + [[0] * 7 for _ in range(K - 1)]
    exact, merged = class_sums(da, [1] * K, db, [1] * K, "rn")
    assert all(merged[v] == exact[v] for v in range(6, 9))
