"""Exact rational coefficient series and ring maps (test infrastructure only).

Section 3.2: beta_{k,r} = binom(-k/N, r) (-2^-b)^r and, by Lagrange inversion
(Lemma 3.4), alpha_{k,0} = 1, alpha_{k,r} = k/(k+r) binom((k+r)/N, r) (-2^-b)^r.
Section 4.2: delta_{k,r} = binom(k/N, r) (-2^-b)^r and (Lemma 4.6)
gamma_{k,0} = 1, gamma_{k,r} = k/(k+r) binom(-(k+r)/N, r) (-2^-b)^r.
Lemma 4.2: rho is the real root of B(X) = X^(N+1) - 2^b X^N + 2^b in
2^b (1 - 2 * 2^-Nb) < rho < 2^b, found by Newton's method from 2^b (proof of
Proposition 4.18).
Sections 3.3 / 4.3: the truncated maps sum_{r<lambda} alpha*_r etc., written out
with exact Fractions and plain polynomial long division, for small N only.
"""
from fractions import Fraction


def gbinom(x: Fraction, r: int) -> Fraction:
    """Generalised binomial coefficient x (x-1) ... (x-r+1) / r!."""
    acc = Fraction(1)
    for j in range(r):
        acc = acc * (x - j) / (j + 1)
    return acc


def _m2b(b: int) -> Fraction:
    return Fraction(-1, 1 << b)


def beta_coef(k: int, r: int, N: int, b: int) -> Fraction:
    return gbinom(Fraction(-k, N), r) * _m2b(b) ** r


def alpha_coef(k: int, r: int, N: int, b: int) -> Fraction:
    if r == 0:
        return Fraction(1)
    return Fraction(k, k + r) * gbinom(Fraction(k + r, N), r) * _m2b(b) ** r


def delta_coef(k: int, r: int, N: int, b: int) -> Fraction:
    return gbinom(Fraction(k, N), r) * _m2b(b) ** r


def gamma_coef(k: int, r: int, N: int, b: int) -> Fraction:
    if r == 0:
        return Fraction(1)
    return Fraction(k, k + r) * gbinom(Fraction(-(k + r), N), r) * _m2b(b) ** r


# ------------------------------------------------------------------ rho

def _round_dyadic(x: Fraction, bits: int) -> Fraction:
    return Fraction(round(x * (1 << bits)), 1 << bits)


def B_poly(N: int, b: int) -> list:
    """Coefficients (low to high) of B(X) = X^(N+1) - 2^b X^N + 2^b (Prop. 4.1)."""
    c = [Fraction(0)] * (N + 2)
    c[0] = Fraction(1 << b)
    c[N] = Fraction(-(1 << b))
    c[N + 1] = Fraction(1)
    return c


def A_poly(N: int, b: int) -> list:
    """Coefficients of A(X) = X^N + 2^-b X - 1 (Proposition 3.1)."""
    c = [Fraction(0)] * (N + 1)
    c[0] = Fraction(-1)
    c[1] += Fraction(1, 1 << b)
    c[N] += Fraction(1)
    return c


def rho(N: int, b: int, bits: int = 400) -> Fraction:
    """Real root of B in (2^b (1 - 2^(1-Nb)), 2^b) by Newton iteration from 2^b
    (proof of Proposition 4.18), each iterate rounded to `bits` fractional bits."""
    z = Fraction(1 << b)
    for _ in range(200):
        zN = z ** N
        f = zN * z - (1 << b) * zN + (1 << b)
        df = (N + 1) * zN - (1 << b) * N * z ** (N - 1)
        z_new = _round_dyadic(z - f / df, bits)
        if z_new == z:
            break
        z = z_new
    return z


def C_poly(N: int, b: int, rho_: Fraction) -> list:
    """C(X) = B(X)/(X - rho) = X^N - (2^b/rho) sum_{i<N} (X/rho)^i (eq. 4.4)."""
    c = [-(Fraction(1 << b) / rho_) / rho_ ** i for i in range(N)]
    c.append(Fraction(1))
    return c


# ------------------------------------------------------- polynomial helpers

def poly_mod(P: list, M: list) -> list:
    """Remainder of P modulo the monic polynomial M (long division), length deg M."""
    P = [Fraction(x) for x in P]
    d = len(M) - 1
    assert M[-1] == 1
    for top in range(len(P) - 1, d - 1, -1):
        q = P[top]
        if q:
            for j in range(d + 1):
                P[top - d + j] -= q * M[j]
    out = P[:d] + [Fraction(0)] * max(0, d - len(P))
    return out[:d]


def poly_mul(P: list, Q: list) -> list:
    out = [Fraction(0)] * (len(P) + len(Q) - 1)
    for i, p in enumerate(P):
        if p:
            for j, q in enumerate(Q):
                out[i + j] += p * q
    return out


def poly_eval(P: list, z):
    acc = 0
    for c in reversed(P):
        acc = acc * z + c
    return acc


def cyclic_mul(F: list, G: list, N: int) -> list:
    out = [Fraction(0)] * N
    for i, f in enumerate(F):
        for j, g in enumerate(G):
            out[(i + j) % N] += f * g
    return out


# ------------------------------------------------------------- the maps

def alpha_star(F: list, N: int, b: int, lam: int) -> list:
    """sum_{r<lam} alpha*_r F: R[X]/A -> R[X]/(X^N - 1) (Section 3.3)."""
    G = [Fraction(0)] * N
    for r in range(lam):
        for k in range(N):
            G[(k + r) % N] += alpha_coef(k, r, N, b) * F[k]
    return G


def beta_star(F: list, N: int, b: int, lam: int) -> list:
    """sum_{r<lam} beta*_r F: R[X]/(X^N - 1) -> R[X]/A (Section 3.3)."""
    P = [Fraction(0)] * (N + lam)
    for r in range(lam):
        for k in range(N):
            P[k + r] += beta_coef(k, r, N, b) * F[k]
    return poly_mod(P, A_poly(N, b))


def gamma_star(F: list, N: int, b: int, lam: int) -> list:
    """sum_{r<lam} gamma*_r F: R[X]/C -> R[X]/(X^N - 1) (Section 4.3)."""
    G = [Fraction(0)] * N
    for r in range(lam):
        for k in range(N):
            G[(k + r) % N] += gamma_coef(k, r, N, b) * F[k]
    return G


def delta_star(F: list, N: int, b: int, lam: int, rho_: Fraction) -> list:
    """sum_{r<lam} delta*_r F: R[X]/(X^N - 1) -> R[X]/C (Section 4.3)."""
    P = [Fraction(0)] * (N + lam)
    for r in range(lam):
        for k in range(N):
            P[k + r] += delta_coef(k, r, N, b) * F[k]
    return poly_mod(P, C_poly(N, b, rho_))


def gamma_dagger(F: list, N: int, b: int, lam: int, rho_: Fraction):
    """gamma-dagger F = (gamma*(F mod C), rho^-N F(rho)) for F in R[X]/B, len(F) = N+1
    (Section 4.3)."""
    assert len(F) == N + 1
    G = gamma_star(poly_mod(F, C_poly(N, b, rho_)), N, b, lam)
    theta = poly_eval(F, rho_) / rho_ ** N
    return G, theta


def delta_dagger(F: list, theta: Fraction, N: int, b: int, lam: int, rho_: Fraction) -> list:
    """delta-dagger(F, theta) by the explicit CRT formula (eqs. 4.6 and 4.7):
    H = delta* F (degree < N), psi = (rho^N theta - rho^-N H(rho)) / C(rho),
    result = (1 - 2^-b X) H + psi C(X), of degree <= N."""
    H = delta_star(F, N, b, lam, rho_)
    C = C_poly(N, b, rho_)
    psi = (rho_ ** N * theta - poly_eval(H, rho_) / rho_ ** N) / poly_eval(C, rho_)
    J = [Fraction(0)] * (N + 1)
    for i, h in enumerate(H):
        J[i] += h
        J[i + 1] -= h / (1 << b)
    for i, c in enumerate(C):
        J[i] += psi * c
    return J


def series_value(coef, k: int, z: complex, N: int, b: int, terms: int) -> complex:
    """z^k sum_{r<terms} coef(k, r) z^r evaluated in complex floating point."""
    acc = 0j
    for r in range(terms):
        acc += complex(float(coef(k, r, N, b))) * z ** (k + r)
    return acc
