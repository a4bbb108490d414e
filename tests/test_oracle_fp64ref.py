"""Pins for oracle.fp64_ref: Algorithms 1-3 in float64 must reproduce the exact
trace (Propositions 3.1 / 4.1) and the product definitions, and the paper's own
Table 2 parameters must give correct products on uniformly random inputs
(Section 5: they "consistently" did so with balanced digits)."""
import random

import numpy as np
import pytest

from conftest import golden
from oracle import bigmul as bm
from oracle import fp64_ref as R
from oracle import plan as P
from oracle import trace as T


def _operands(pattern, n, rnd, b):
    if pattern == "random":
        return rnd.getrandbits(n), rnd.getrandbits(n)
    if pattern == "ones":
        x = (1 << n) - 1
        return x, x
    if pattern == "balanced_worst":      # every b-bit chunk = 2^(b-1): digits of maximal size
        x = sum(1 << (i * b + b - 1) for i in range(n // b)) & ((1 << n) - 1)
        return x, x
    if pattern == "alternating":
        x = int("10" * (n // 2) + "1" * (n % 2), 2)
        return x, x ^ ((1 << n) - 1)
    raise ValueError(pattern)


@pytest.mark.parametrize("n", [1, 17, 64, 100, 999, 4096, 20000])
@pytest.mark.parametrize("pattern", ["random", "ones", "balanced_worst", "alternating"])
def test_fp64_reference_matches_exact_trace(n, pattern):
    rnd = random.Random(n)
    for kind in ("lo", "hi", "full"):
        p = P.choose(kind, n)
        u, v = _operands(pattern, n, rnd, p["b"])
        if kind == "lo":
            r = R.mul_lo(u, v, n, p["b"], p["N"], p["lam_fwd"], p["lam_bwd"])
            ex = T.trace("lo", u, v, n, p["b"], p["N"])
            assert np.array_equal(r["c"], ex["c"]) and r["out"] == (u * v) % (1 << n)
        elif kind == "hi":
            r = R.mul_hi(u, v, n, p["b"], p["N"], p["lam_fwd"], p["lam_bwd"])
            ex = T.trace("hi", u, v, n, p["b"], p["N"])
            assert np.array_equal(r["c"], ex["c"]) and r["out"] == ex["out"]
            assert abs(u * v - (r["out"] << n)) < (1 << n)
        else:
            r = R.mul_full(u, v, n, p["b"], p["N"], p["n_digits"])
            assert r["out"] == u * v
        assert r["margin"] <= p["e_max"]


@pytest.mark.parametrize("row", golden("table2_params.txt")[:3])
def test_table2_replay(row):
    """Table 2, n = 10^6 (N = 71680 = 2^11 * 35, b = 14, lambda = 4 for both truncated
    products; 2N = 98304, b = 21 for the full product), 2154434 and 4641588."""
    n, N, b, lam, L, bf = map(int, row)
    rnd = random.Random(2017)
    nl = (n + 63) // 64
    for _ in range(2):
        u, v = rnd.getrandbits(n), rnd.getrandbits(n)
        U, V = bm.from_int(u, nl), bm.from_int(v, nl)
        lo = R.mul_lo(u, v, n, b, N, lam, lam)
        assert lo["out"] == bm.to_int(bm.mul_lo(U, V, n, par_depth=2))
        assert (N + 1) * b >= n + (N - 1).bit_length() + 2
        hi = R.mul_hi(u, v, n, b, N, lam, lam)
        q, ok = bm.mul_hi_floor(U, V, n, par_depth=2)
        assert hi["out"] in ({bm.to_int(q), bm.to_int(q) + 1} if ok else {bm.to_int(q)})
        Nd = -(-(n + 1) // bf)
        assert 2 * Nd - 1 <= L
        full = R.mul_full(u, v, n, bf, L, Nd)
        assert full["out"] == u * v
        for r in (lo, hi, full):
            assert r["margin"] < 0.5


def test_stage_maps_against_exact_series():
    """The float64 maps agree with the exact-rational maps of oracle.series."""
    from fractions import Fraction
    from oracle import series as S
    rnd = random.Random(11)
    N, b, lam = 9, 5, 9
    F = [rnd.randint(-16, 16) for _ in range(N)]
    Fx = [Fraction(x) for x in F]
    a = R.alpha_star(np.array(F, float), N, b, lam)
    assert np.allclose(a, [float(x) for x in S.alpha_star(Fx, N, b, lam)], rtol=0, atol=1e-13)
    be = R.beta_star(np.array(F, float), N, b, lam)
    assert np.allclose(be, [float(x) for x in S.beta_star(Fx, N, b, lam)], rtol=0, atol=1e-13)
    rho = S.rho(N, b)
    Fb = [rnd.randint(-16, 16) for _ in range(N + 1)]
    g, th = R.gamma_dagger(np.array(Fb, float), N, b, lam, float(rho))
    ge, the = S.gamma_dagger([Fraction(x) for x in Fb], N, b, lam, rho)
    assert np.allclose(g, [float(x) for x in ge], atol=1e-12) and abs(th - float(the)) < 1e-12
    d = R.delta_dagger(np.array(F, float), 3.25, N, b, lam, float(rho))
    de = S.delta_dagger(Fx, Fraction(13, 4), N, b, lam, rho)
    assert np.allclose(d, [float(x) for x in de], atol=1e-11)
