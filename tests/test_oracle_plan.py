"""Pins for oracle.plan: every chosen plan satisfies the hypotheses of
Theorems 2.1-2.3, lambda is the least number of terms meeting its tail budget
(Lemmas 3.10, 3.11, 4.10, 4.11), b is maximal for its length, and the chosen
lengths are smooth (Section 5)."""
import pytest

from oracle import plan as P

NS = [1, 2, 7, 63, 64, 65, 100, 1000, 4095, 4096, 65536, 100000, 2**20, 10**6, 2**24, 2**28]


@pytest.mark.parametrize("n", NS)
def test_hypotheses(n):
    lo, hi, full = P.choose("lo", n), P.choose("hi", n), P.choose("full", n)
    for p in (lo, hi, full):
        assert P.B_MIN <= p["b"] <= P.B_MAX and P.is_valid_length(p["N"])
        assert p["e_max"] <= P.E_TARGET < 0.5
    assert lo["N"] >= 3 and lo["N"] * lo["b"] >= n                               # Thm 2.2
    assert hi["N"] >= 3 and (hi["N"] + 1) * hi["b"] >= n + P.ceil_log2(hi["N"]) + 2  # Thm 2.3
    nd = full["n_digits"]
    assert nd * full["b"] >= n + 1 and full["N"] >= 2 * nd - 1                   # Thm 2.1


@pytest.mark.parametrize("b", range(4, 25))
def test_lambda_minimal(b):
    u = P.U / 4
    la = P.lam_alpha(b)
    assert (16 / 15) * 2.0 ** (-la * b) <= u < (16 / 15) * 2.0 ** (-(la - 1) * b)
    q = (1 + 2.0 ** -b) * 2.0 ** -b
    lb = P.lam_beta(b)
    assert q ** lb / (1 - q) <= u < q ** (lb - 1) / (1 - q)
    for N in (4, 1000, 10**7):
        lg = P.lam_gamma(b, N)
        assert P.gamma_tail(lg, b, N) <= u < P.gamma_tail(lg - 1, b, N)


@pytest.mark.parametrize("n", [1000, 65536, 2**20])
def test_b_maximal(n):
    """At the chosen length, b + 1 either breaks a hypothesis or the bound."""
    lo = P.choose("lo", n)
    E, *_ = P.bound_lo(n, lo["b"] + 1, lo["N"])
    assert E > P.E_TARGET
    full = P.choose("full", n)
    b1 = full["b"] + 1
    if 2 * P.full_digits(n, b1) - 1 <= full["N"]:
        E, *_ = P.bound_full(n, b1, full["N"])
        assert E > P.E_TARGET


def test_smooth_lengths():
    assert P.smooth_at_least(5) == 6
    assert P.smooth_at_least(71000) == 71680          # 2^11 * 35, a Table 2 length
    assert P.is_valid_length(98304) and P.is_valid_length(18874368)
    assert not P.is_valid_length(22) and not P.is_valid_length(7)
    assert P.odd_prime_factor_count(2**11 * 35) == 2


def test_truncated_length_is_shorter():
    """Scenario #2 (Section 2.3): the truncated length is about 3/4 of the full one."""
    for n in (2**16, 2**20, 2**24):
        ratio = P.choose("lo", n)["N"] / P.choose("full", n)["N"]
        assert 0.6 < ratio < 0.9
