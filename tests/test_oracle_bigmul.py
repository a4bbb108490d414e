"""Pins for oracle.bigmul: the C schoolbook/Karatsuba product against Python's
own big-integer multiply (an independent implementation), and the low/high
products against the definitions of Section 1."""
import random

import numpy as np
import pytest

from oracle import bigmul as bm


@pytest.mark.parametrize("nl", [1, 2, 3, 15, 31, 32, 33, 63, 64, 65, 127, 200, 513, 1031])
@pytest.mark.parametrize("depth", [0, 2])
def test_full_product_matches_python_ints(nl, depth):
    rng = np.random.default_rng(nl * 7 + depth)
    for pattern in ("random", "ones", "sparse"):
        if pattern == "random":
            u = rng.integers(0, 2**64, nl, dtype=np.uint64)
            v = rng.integers(0, 2**64, nl, dtype=np.uint64)
        elif pattern == "ones":
            u = np.full(nl, 2**64 - 1, dtype=np.uint64)
            v = u.copy()
        else:
            u = np.zeros(nl, dtype=np.uint64); u[-1] = 1
            v = np.zeros(nl, dtype=np.uint64); v[0] = 2**63
        got = bm.to_int(bm.mul_full(u, v, depth))
        assert got == bm.to_int(u) * bm.to_int(v)


def test_low_and_high_definitions_small_n_exhaustive():
    """All pairs for n <= 5: lo is uv mod 2^n; the high accept-set {q, q+1} is
    exactly the set of 0 <= w <= 2^n with |uv - 2^n w| < 2^n (Section 1)."""
    for n in range(1, 6):
        for u in range(1 << n):
            for v in range(1 << n):
                U = bm.from_int(u, 1); V = bm.from_int(v, 1)
                lo = bm.to_int(bm.mul_lo(U, V, n))
                assert 0 <= lo < (1 << n) and (u * v - lo) % (1 << n) == 0
                q_limbs, q1_ok = bm.mul_hi_floor(U, V, n)
                q = bm.to_int(q_limbs)
                admissible = {w for w in range(0, (1 << n) + 1) if abs(u * v - (w << n)) < (1 << n)}
                assert admissible == ({q, q + 1} if q1_ok else {q})


@pytest.mark.parametrize("n", [1, 63, 64, 65, 127, 128, 1000, 4097, 65536])
def test_low_high_random(n):
    rnd = random.Random(n)
    nl = (n + 63) // 64
    for _ in range(3):
        u, v = rnd.getrandbits(n), rnd.getrandbits(n)
        U, V = bm.from_int(u, nl), bm.from_int(v, nl)
        assert bm.to_int(bm.mul_lo(U, V, n)) == (u * v) % (1 << n)
        q, ok = bm.mul_hi_floor(U, V, n)
        assert bm.to_int(q) == (u * v) >> n
        assert ok == ((u * v) % (1 << n) != 0)
        assert q.size == n // 64 + 1


def test_high_product_can_be_two_to_the_n():
    """w = 2^n is admissible when uv > 2^2n - 2^n (Section 1 allows w = 2^n)."""
    n = 64
    u = v = (1 << n) - 1
    q, ok = bm.mul_hi_floor(bm.from_int(u, 1), bm.from_int(v, 1), n)
    q = bm.to_int(q)
    assert ok and abs(u * v - ((q + 1) << n)) < (1 << n) and q + 1 <= (1 << n)
