"""Pins for oracle.trace: the digit splits, the exact coefficient identities of
Propositions 3.1 and 4.1 and the overlap-add steps, checked against the
definitions of the low, high and full products by brute force on small n."""
import random

import numpy as np
import pytest

from oracle import trace as T


def _hi_ok(n, b, N):
    return (N + 1) * b >= n + max(0, (N - 1).bit_length()) + 2


def test_brute_force_n8_all_pairs():
    """Every pair of 8-bit operands (N = 3, b = 4 as in Theorems 2.2 / 2.3)."""
    n, b = 8, 4
    Nl, Nh = 3, 3
    assert _hi_ok(n, b, Nh)
    for u in range(256):
        for v in range(256):
            assert T.trace("lo", u, v, n, b, Nl)["out"] == (u * v) % 256
            w = T.trace("hi", u, v, n, b, Nh)["out"]
            assert 0 <= w <= 256 and abs(u * v - (w << n)) < 256


def test_brute_force_n12_sampled():
    n, b = 12, 4
    Nh = 3
    while not _hi_ok(n, b, Nh):
        Nh += 1
    rnd = random.Random(12)
    pairs = [(rnd.getrandbits(n), rnd.getrandbits(n)) for _ in range(4000)]
    pairs += [(0, 0), (4095, 4095), (2048, 2048), (0x888, 0x888), (1, 4095)]
    for u, v in pairs:
        assert T.trace("lo", u, v, n, b, 3)["out"] == (u * v) % 4096
        w = T.trace("hi", u, v, n, b, Nh)["out"]
        assert 0 <= w <= 4096 and abs(u * v - (w << n)) < 4096
        assert T.trace("full", u, v, n, b, 4)["out"] == u * v


def test_figure1_cancellation_N3():
    """Figure 1 / Proposition 3.1 with N = 3: the rows of diagram (B) sum to
    L(2^b) = w0 + w1 2^b + w2 2^2b, the shaded copies of w3, w4 cancelling."""
    b, N = 5, 3
    rnd = random.Random(1)
    for _ in range(50):
        w = np.array([rnd.randint(-500, 500) for _ in range(2 * N - 1)], dtype=np.int64)
        c = T.low_coeffs(w, N, b)
        # diagram (B): constant row w0 + w3, X row -w3 + w1 + w4 (scaled), X^2 row -w4 + w2
        assert c[0] == (w[0] + w[3]) << b
        assert c[1] == ((w[1] + w[4]) << b) - w[3]
        assert c[2] == (w[2] << b) - w[4]
        L_at = sum(int(c[i]) << (i * b) for i in range(N))          # 2^b L(2^b)
        assert L_at == sum(int(w[i]) << (i * b + b) for i in range(N))


def test_coefficient_identities_against_polynomial_division():
    """c_i = 2^b (W mod A)_i and 2^b ((1 - 2^-b X) W mod B)_i, by long division."""
    from fractions import Fraction
    from oracle import series as S
    rnd = random.Random(2)
    for N in (3, 4, 7):
        for b in (4, 6):
            w = [rnd.randint(-999, 999) for _ in range(2 * N - 1)]
            L = S.poly_mod([Fraction(x) for x in w], S.A_poly(N, b))
            assert [int(x * (1 << b)) for x in L] == list(T.low_coeffs(np.array(w), N, b))
            assert all((x * (1 << b)).denominator == 1 for x in L)
            w = [rnd.randint(0, 999) for _ in range(2 * N + 1)]
            P = S.poly_mul([Fraction(1), Fraction(-1, 1 << b)], [Fraction(x) for x in w])
            H = S.poly_mod(P, S.B_poly(N, b))
            assert [int(x * (1 << b)) for x in H] == list(T.high_coeffs(np.array(w), N, b))


@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_balanced_split(kind):
    rnd = random.Random(hash(kind) & 0xFFFF)
    for _ in range(200):
        b = rnd.randint(4, 20)
        n = rnd.randint(1, 500)
        u = rnd.getrandbits(n)
        if kind == "lo":
            N = -(-n // b)
        elif kind == "full":
            N = -(-(n + 1) // b)
        else:
            N = 3
            while not _hi_ok(n, b, N):
                N += 1
        U = T.split(kind, u, n, b, N)
        half = 1 << (b - 1)
        if kind == "hi":
            assert all(-half <= x <= half for x in U[:-1]) and 0 <= U[-1] <= (1 << b)
            assert T.eval_poly(U, 1 << b) == u << ((N + 1) * b - n)
        else:
            assert all(-half <= x <= half for x in U)
            if kind == "full":
                assert T.eval_poly(U, 1 << b) == u
            else:
                assert T.eval_poly(U, 1 << b) % (1 << (N * b)) == u


def test_poly_mul_exact_against_direct_convolution():
    rnd = random.Random(9)
    for size in (1, 2, 5, 64, 300, 2100):
        U = [rnd.randint(-(1 << 20), 1 << 20) for _ in range(size)]
        V = [rnd.randint(-(1 << 20), 1 << 20) for _ in range(size + 1)]
        w = T.poly_mul_exact(U, V, bigmul_threshold=1000)
        if size <= 300:
            direct = np.convolve(np.array(U, dtype=object), np.array(V, dtype=object))
            assert [int(x) for x in w] == [int(x) for x in direct]
        assert T.eval_poly(w, 1 << 50) == T.eval_poly(U, 1 << 50) * T.eval_poly(V, 1 << 50)


def test_c0_divisible_and_random_products():
    rnd = random.Random(4)
    for n in (100, 1000, 3000):
        for b in (7, 11):
            N = -(-n // b)
            u, v = rnd.getrandbits(n), rnd.getrandbits(n)
            r = T.trace("lo", u, v, n, b, N)
            assert int(r["c"][0]) % (1 << b) == 0 and r["out"] == (u * v) % (1 << n)
            Nh = 3
            while not _hi_ok(n, b, Nh):
                Nh += 1
            r = T.trace("hi", u, v, n, b, Nh)
            assert int(r["c"][0]) % (1 << b) == 0
            assert abs(u * v - (r["out"] << n)) < (1 << n)
