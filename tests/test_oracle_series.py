"""Pins for oracle.series: the printed first terms of the four series, the
Lagrange-inversion property, the coefficient bounds of Lemmas 3.5 and 4.7,
the root pictures of Figures 2 and 3, the rho expansion after Lemma 4.2, and
the ring-map identities of Corollaries 3.14 and 4.14 and Lemma 4.15."""
import cmath
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import golden
from oracle import series as S

COEF = {"alpha": S.alpha_coef, "beta": S.beta_coef, "gamma": S.gamma_coef, "delta": S.delta_coef}


@pytest.mark.parametrize("N", [3, 4, 7, 12, 1000])
@pytest.mark.parametrize("b", [1, 4, 9])
def test_printed_first_terms(N, b):
    for name, r, expr in golden("series_first_terms.txt"):
        r = int(r)
        want = eval(expr, {"__builtins__": {}}, {"N": Fraction(N)}) * Fraction(1, 1 << (r * b))
        assert COEF[name](1, r, N, b) == want, (name, r)


def _compose(outer, inner, N, b, R):
    """Coefficients of z^(1+s), s < R, in outer(inner(z)) as formal series, where
    f(z)^k = z^k sum_r f_{k,r} z^r supplies the powers of the inner series."""
    out = [Fraction(0)] * R
    for r in range(R):
        a = outer(1, r, N, b)            # outer(w) = sum_r a_r w^(1+r)
        if a == 0:
            continue
        for s in range(R - r):           # inner(z)^(1+r) = z^(1+r) sum_s inner_{1+r,s} z^s
            out[r + s] += a * inner(1 + r, s, N, b)
    return out


@pytest.mark.parametrize("N,b", [(3, 4), (5, 2), (12, 1), (17, 6)])
def test_lagrange_inversion(N, b):
    """alpha(beta(z)) = z and gamma(delta(z)) = z as formal series (Lemmas 3.4, 4.6)."""
    R = 8
    for outer, inner in ((S.alpha_coef, S.beta_coef), (S.beta_coef, S.alpha_coef),
                         (S.gamma_coef, S.delta_coef), (S.delta_coef, S.gamma_coef)):
        comp = _compose(outer, inner, N, b, R)
        assert comp[0] == 1 and all(c == 0 for c in comp[1:])


@pytest.mark.parametrize("N,b", [(3, 4), (8, 5), (31, 4)])
def test_coefficient_bounds(N, b):
    """Lemma 3.5 and Lemma 4.7."""
    for k in range(N):
        for r in range(10):
            lim = Fraction(1, 1 << (r * b))
            assert abs(S.alpha_coef(k, r, N, b)) <= lim
            assert abs(S.beta_coef(k, r, N, b)) <= lim
            assert abs(S.delta_coef(k, r, N, b)) <= lim
            assert abs(S.gamma_coef(k, r, N, b)) <= Fraction(1 << (2 * r), 1 << (r * b))
            # the sharper form carried through the proof of Lemma 4.7
            assert float(abs(S.gamma_coef(k, r, N, b))) <= float(lim) * math.exp(
                (r - 1) * sum(1 / j for j in range(1, r + 1)) / N) * (1 + 1e-12) if r else True


def _points(name):
    return sorted((round(float(x), 3), round(float(y), 3)) for x, y in golden(name))


def test_figure2_roots_of_A():
    """alpha maps the 12th roots of unity onto the roots of A (Corollary 3.7);
    summing the series reproduces the printed filled circles of Figure 2."""
    N, b = 12, 1
    pts = []
    for k in range(N):
        z = S.series_value(S.alpha_coef, 1, cmath.exp(2j * math.pi * k / N), N, b, 400)
        pts.append((round(z.real, 3) + 0.0, round(z.imag, 3) + 0.0))
    assert sorted(pts) == _points("fig2_roots_A.txt")
    roots = np.roots([1] + [0] * 10 + [0.5, -1])           # X^12 + X/2 - 1
    assert sorted((round(r.real, 3) + 0.0, round(r.imag, 3) + 0.0) for r in roots) == _points("fig2_roots_A.txt")


def test_figure3_roots_of_B():
    """gamma maps the 12th roots of unity onto the roots of C (Corollary 4.9); with
    rho (Lemma 4.2) these are the printed roots of B in Figure 3."""
    N, b = 12, 1
    pts = []
    for k in range(N):
        z = S.series_value(S.gamma_coef, 1, cmath.exp(2j * math.pi * k / N), N, b, 400)
        pts.append((round(z.real, 3) + 0.0, round(z.imag, 3) + 0.0))
    pts.append((round(float(S.rho(N, b)), 3), 0.0))
    assert sorted(pts) == _points("fig3_roots_B.txt")


@pytest.mark.parametrize("N,b", [(3, 4), (5, 4), (12, 1), (4, 9)])
def test_rho(N, b):
    """Lemma 4.2 interval (4.1), identity (4.3) and the expansion
    rho = 2^b (1 - eps - N eps^2 - ...), eps = 2^-Nb."""
    r = S.rho(N, b)
    two_b = Fraction(1 << b)
    eps = Fraction(1, 1 << (N * b))
    if b >= 4:
        assert two_b * (1 - 2 * eps) < r < two_b
    assert abs(1 - r / two_b - 1 / r ** N) < Fraction(1, 1 << 300)
    dev = r / two_b - (1 - eps - N * eps ** 2)
    assert abs(dev) <= 4 * N * N * eps ** 3
    if b == 1:
        assert abs(float(r) - 2.0) < 1e-3


def _rand_poly(rnd, N, scale=16):
    return [Fraction(rnd.randint(-scale, scale)) for _ in range(N)]


def _maxdiff(P, Q):
    return max(abs(a - b) for a, b in zip(P, Q))


def test_alpha_beta_inverse_homomorphisms():
    """Corollary 3.14: beta* alpha* = id and alpha*(FG mod A) = alpha*F alpha*G
    (mod X^N - 1), up to the truncation tails of Lemmas 3.10 / 3.11."""
    import random
    rnd = random.Random(3)
    N, b, lam = 5, 4, 14
    tol = Fraction(1, 1 << 40)
    for _ in range(3):
        F, G = _rand_poly(rnd, N), _rand_poly(rnd, N)
        assert _maxdiff(S.beta_star(S.alpha_star(F, N, b, lam), N, b, lam), F) < tol
        assert _maxdiff(S.alpha_star(S.beta_star(F, N, b, lam), N, b, lam), F) < tol
        FG = S.poly_mod(S.poly_mul(F, G), S.A_poly(N, b))
        lhs = S.alpha_star(FG, N, b, lam)
        rhs = S.cyclic_mul(S.alpha_star(F, N, b, lam), S.alpha_star(G, N, b, lam), N)
        assert _maxdiff(lhs, rhs) < tol * 1000


def test_alpha_star_evaluates_at_roots():
    """Lemma 3.12: (alpha* F)(z) = F(alpha(z)) for z^N = 1, alpha(z) a root of A."""
    N, b, lam = 6, 4, 16
    F = [Fraction(x) for x in (3, -1, 4, 1, -5, 9)]
    G = [complex(float(x)) for x in S.alpha_star(F, N, b, lam)]
    for k in range(N):
        z = cmath.exp(2j * math.pi * k / N)
        a = S.series_value(S.alpha_coef, 1, z, N, b, 30)
        assert abs(a ** N + a / 16 - 1) < 1e-12                     # a is a root of A
        lhs = sum(g * z ** i for i, g in enumerate(G))
        rhs = sum(float(f) * a ** i for i, f in enumerate(F))
        assert abs(lhs - rhs) < 1e-10


def test_gamma_delta_inverse_and_lemma_4_15():
    """Corollary 4.14 (gamma*, delta* inverse on R[X]/C) and Lemma 4.15:
    delta-dagger(gamma-dagger F . gamma-dagger G) = (1 - 2^-b X) F G mod B."""
    import random
    rnd = random.Random(7)
    N, b, lam = 5, 6, 14
    r = S.rho(N, b)
    tol = Fraction(1, 1 << 36)
    C = S.C_poly(N, b, r)
    for _ in range(2):
        F = _rand_poly(rnd, N)
        back = S.delta_star(S.gamma_star(F, N, b, lam), N, b, lam, r)
        assert _maxdiff(back, S.poly_mod(F, C)) < tol
        Fb, Gb = _rand_poly(rnd, N + 1), _rand_poly(rnd, N + 1)
        gF, tF = S.gamma_dagger(Fb, N, b, lam, r)
        gG, tG = S.gamma_dagger(Gb, N, b, lam, r)
        lhs = S.delta_dagger(S.cyclic_mul(gF, gG, N), tF * tG, N, b, lam, r)
        P = S.poly_mul([Fraction(1), Fraction(-1, 1 << b)], S.poly_mul(Fb, Gb))
        rhs = S.poly_mod(P, S.B_poly(N, b))
        assert _maxdiff(lhs, rhs) < tol * 1000
