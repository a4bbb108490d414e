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


def test_measured_bounds_reduce_to_the_worst_case():
    """With the worst-case norms (every digit at 2^(b-1), top digit 2^b) the
    measured-norm bounds equal the planner's worst-case bounds."""
    import math
    for n, b, N in [(1 << 16, 11, 6144), (1 << 20, 9, 122880), (1 << 24, 8, 2097152)]:
        w = 2.0 ** (b - 1) * math.sqrt(N)
        assert P.bound_lo_measured(b, N, w, w) == pytest.approx(P.bound_lo(n, b, N)[0], rel=1e-12)
    for n, b, N in [(1 << 16, 10, 6912), (1 << 24, 7, 2408448)]:
        w = 2.0 ** (b - 1) * math.sqrt(N)
        t = 2.0 ** b
        assert P.bound_hi_measured(b, N, w, w, t, t) == pytest.approx(P.bound_hi(n, b, N)[0],
                                                                      rel=1e-12)
    for n, b, L in [(1 << 16, 17, 8192), (1 << 24, 12, 2867200)]:
        w = 2.0 ** (b - 1) * math.sqrt(P.full_digits(n, b))
        assert P.bound_full_measured(L, w, w) == pytest.approx(P.bound_full(n, b, L)[0],
                                                               rel=1e-12)


def test_adaptive_choice_bounds():
    """The data-dependent choice: worst-case operands keep the planner's b;
    random operands take b + 1 only where the measured bound certifies it, and
    every accepted bound is <= the target."""
    import random
    rng = random.Random(3)
    for n in (1 << 12, 1 << 16, 123457):
        for kind in ("lo", "hi", "full"):
            base = P.choose(kind, n)
            # every (b+1)-bit chunk 100...0: balanced digits of magnitude ~2^b, the
            # worst case for b + 1 (all-ones operands have balanced digits near 0)
            b1 = base["b"] + 1
            s0 = 0
            if kind == "hi":               # the high product splits u 2^s0
                s0 = (P.measured_length(kind, n, b1) + 1) * b1 - n
            worst = sum(1 << (i * b1 + b1 - 1 - s0) for i in range((n + s0) // b1)
                        if 0 <= i * b1 + b1 - 1 - s0 < n)
            assert P.adaptive_choice(kind, n, worst, worst)["b"] == base["b"]
            u, v = rng.getrandbits(n), rng.getrandbits(n)
            c = P.adaptive_choice(kind, n, u, v)
            assert c["b"] in (base["b"], base["b"] + 1)
            assert c["e_max"] <= P.E_TARGET
            if c["b"] != base["b"]:
                assert c["N"] < base["N"]
