"""The oracle's pins are sharp: a plausible mistake planted in the oracle (on
the CPU, through monkeypatching) makes the corresponding pin fail."""
import random

import numpy as np
import pytest

from oracle import series as S
from oracle import trace as T


def _lo_ok(n=12, b=4, N=3, trials=400):
    rnd = random.Random(0)
    for _ in range(trials):
        u, v = rnd.getrandbits(n), rnd.getrandbits(n)
        if T.trace("lo", u, v, n, b, N)["out"] != (u * v) % (1 << n):
            return False
    return True


def _hi_ok(n=12, b=4, N=4, trials=400):
    rnd = random.Random(0)
    for _ in range(trials):
        u, v = rnd.getrandbits(n), rnd.getrandbits(n)
        w = T.trace("hi", u, v, n, b, N)["out"]
        if not (0 <= w <= (1 << n) and abs(u * v - (w << n)) < (1 << n)):
            return False
    return True


def test_unmutated_pass():
    assert _lo_ok() and _hi_ok()


def test_dropped_term_in_low_coefficients(monkeypatch):
    def bad(w, N, b):
        w = np.asarray(w, dtype=np.int64)
        hi = np.zeros(N, dtype=np.int64); hi[: N - 1] = w[N:]
        return (w[:N] + hi) * (1 << b)                     # -w_(N+i-1) dropped
    monkeypatch.setattr(T, "low_coeffs", bad)
    assert not _lo_ok()


def test_wrong_sign_in_high_coefficients(monkeypatch):
    def bad(w, N, b):
        w = np.asarray(w, dtype=np.int64)
        low = np.zeros(N + 1, dtype=np.int64); low[:N] = w[:N]
        prev = np.zeros(N + 1, dtype=np.int64); prev[1:] = w[:N]
        return (low + w[N:]) * (1 << b) + prev             # sign flipped
    monkeypatch.setattr(T, "high_coeffs", bad)
    # the accept-set alone cannot see it (those terms move t by less than 1/2);
    # the long-division pin of Proposition 4.1 does
    from test_oracle_trace import test_coefficient_identities_against_polynomial_division as pin
    with pytest.raises(AssertionError):
        pin()


def test_off_by_one_split(monkeypatch):
    orig = T.balanced_digits

    def bad(x, count, b, balance_top):
        return orig(x << 1, count, b, balance_top)          # shifted by one bit
    monkeypatch.setattr(T, "balanced_digits", bad)
    assert not _lo_ok()


def test_wrong_alpha_coefficient_breaks_inversion(monkeypatch):
    from fractions import Fraction

    def bad(k, r, N, b):                                     # k/(k+r) factor dropped
        return Fraction(1) if r == 0 else S.gbinom(Fraction(k + r, N), r) * Fraction(-1, 1 << b) ** r
    monkeypatch.setattr(S, "alpha_coef", bad)
    from test_oracle_series import _compose
    comp = _compose(S.alpha_coef, S.beta_coef, 7, 4, 6)
    assert not (comp[0] == 1 and all(c == 0 for c in comp[1:]))
