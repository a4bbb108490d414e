"""Pins of oracle.division: the definitions against binary long division, the
defining inequalities of the reciprocal and of Barrett's quotient window, and
brute force on every small divisor."""
import random

import pytest

from oracle import division as D


def test_reciprocal_defining_inequality():
    rng = random.Random(5)
    for k in list(range(1, 70)) + [100, 127, 128, 129, 1000]:
        cands = {1 << (k - 1), (1 << k) - 1, (1 << (k - 1)) + 1,
                 rng.randrange(1 << (k - 1), 1 << k)}
        for m in (c for c in cands if (1 << (k - 1)) <= c < (1 << k)):
            R = D.reciprocal(m, k)
            assert m * R <= (1 << (2 * k)) - 1 < m * (R + 1)
            assert (1 << k) - 1 <= R < (1 << (k + 1))     # k + 1 bits


def test_reciprocal_brute_force_small():
    for k in range(1, 9):
        for m in range(1 << (k - 1), 1 << k):
            R = max(r for r in range(1 << (k + 2)) if m * r <= (1 << (2 * k)) - 1)
            assert D.reciprocal(m, k) == R


def test_reciprocal_rejects_wrong_width():
    with pytest.raises(ValueError):
        D.reciprocal(3, 4)
    with pytest.raises(ValueError):
        D.reciprocal(16, 4)


def test_divrem_matches_long_division():
    rng = random.Random(7)
    for _ in range(300):
        k = rng.randrange(1, 300)
        m = rng.randrange(1 << (k - 1), 1 << k)
        x = rng.randrange(0, 1 << (2 * k))
        assert D.divrem(x, m) == D.long_division(x, m)
    for x in range(64):
        for m in range(1, 20):
            q, r = D.divrem(x, m)
            assert q * m + r == x and 0 <= r < m
            assert (q, r) == D.long_division(x, m)


def test_barrett_quotient_window():
    """The window the library's corrections rely on: with x1 = floor(x / 2^(k-1))
    and R = reciprocal(m, k), every admissible high product w of x1 and R
    (n = k + 1 bits) satisfies q - 3 <= w <= q + 1."""
    rng = random.Random(11)
    for _ in range(2000):
        k = rng.randrange(1, 200)
        m = rng.choice([1 << (k - 1), (1 << k) - 1, rng.randrange(1 << (k - 1), 1 << k)])
        x = rng.choice([0, (1 << (2 * k)) - 1, rng.randrange(0, 1 << (2 * k))])
        q, _ = D.divrem(x, m)
        x1 = x >> (k - 1)
        R = D.reciprocal(m, k)
        prod = x1 * R
        lo = prod >> (k + 1)
        for w in (lo, lo + 1):
            if abs(prod - (w << (k + 1))) < (1 << (k + 1)):
                assert q - 3 <= w <= q + 1


def test_is_divrem_characterises_divrem():
    rng = random.Random(13)
    for _ in range(500):
        k = rng.randrange(1, 200)
        m = rng.randrange(1 << (k - 1), 1 << k)
        x = rng.randrange(0, 1 << (2 * k))
        q, r = D.divrem(x, m)
        assert D.is_divrem(x, m, q, r)
        # every neighbouring pair is rejected
        for dq, dr in ((1, 0), (-1, 0), (0, 1), (0, -1), (1, -m), (-1, m)):
            assert not D.is_divrem(x, m, q + dq, r + dr)
