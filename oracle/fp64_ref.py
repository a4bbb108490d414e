"""Algorithms 1-3 of the paper step by step in numpy float64 (test
infrastructure only). numpy's FFT (rfft / irfft) plays the Convolution black
box of Section 2.1; every other step is written from its definition:

- alpha* / gamma*:   sum_{r<lambda} coef_{k,r} F_k X^((k+r) mod N)      (Sections 3.3, 4.3)
- beta* / delta*:    sum_{r<lambda} coef_{k,r} F_k X^(k+r), reduced mod A or C
- F mod C, theta:    eq. (4.5) and rho^-N F(rho) = F_N + rho^-1 F_(N-1) + ...
- delta-dagger:      eqs. (4.6)-(4.7), with psi in the scaled form
                     psi = (theta - rho^-2N H(rho)) / (1 - N 2^b rho^-(N+1)),
                     which is (4.6) divided through by rho^N
- rounding:          round(2^b Wbar_i) (overlap-add step of Algorithms 2 and 3)

Results: the rounded coefficients, the final integer and the largest distance
to the nearest integer ("margin").
"""
import math

import numpy as np

from . import trace


def _gbinom_vec(x: np.ndarray, r: int) -> np.ndarray:
    acc = np.ones_like(x)
    for j in range(r):
        acc = acc * (x - j) / (j + 1)
    return acc


def coef_table(which: str, N: int, b: int, lam: int) -> np.ndarray:
    """tab[r, k] = coef_{k,r} for k < N, r < lam, in float64 from the definitions."""
    k = np.arange(N, dtype=np.float64)
    tab = np.zeros((lam, N))
    for r in range(lam):
        s = (-(2.0 ** -b)) ** r
        if which == "beta":
            tab[r] = _gbinom_vec(-k / N, r) * s
        elif which == "delta":
            tab[r] = _gbinom_vec(k / N, r) * s
        elif which == "alpha":
            tab[r] = 1.0 if r == 0 else k / (k + r) * _gbinom_vec((k + r) / N, r) * s
        elif which == "gamma":
            tab[r] = 1.0 if r == 0 else k / (k + r) * _gbinom_vec(-(k + r) / N, r) * s
        else:
            raise ValueError(which)
    return tab


def cyclic_map(F: np.ndarray, tab: np.ndarray) -> np.ndarray:
    """sum_r tab[r, k] F_k X^((k+r) mod N): alpha* or gamma*."""
    G = np.zeros_like(F)
    for r in range(tab.shape[0]):
        G += np.roll(tab[r] * F, r)
    return G


def shifted_terms(F: np.ndarray, tab: np.ndarray) -> np.ndarray:
    """P = sum_r tab[r, k] F_k X^(k+r), as a length N + lam - 1 vector."""
    N, lam = F.size, tab.shape[0]
    P = np.zeros(N + lam - 1)
    for r in range(lam):
        P[r:r + N] += tab[r] * F
    return P


def reduce_mod_A(P: np.ndarray, N: int, b: int) -> np.ndarray:
    """P mod A(X), A = X^N + 2^-b X - 1: X^(N+m) = X^m - 2^-b X^(m+1)."""
    P = P.copy()
    for j in range(P.size - 1, N - 1, -1):
        P[j - N] += P[j]
        P[j - N + 1] -= P[j] * 2.0 ** -b
        P[j] = 0.0
    return P[:N]


def kappa(N: int, b: int, rho: float) -> np.ndarray:
    """kappa_i = 2^b / rho^(i+1), i < N: C(X) = X^N - sum kappa_i X^i (eq. 4.4)."""
    i = np.arange(N, dtype=np.float64)
    return np.exp(b * math.log(2.0) - (i + 1) * math.log(rho))


def reduce_mod_C(P: np.ndarray, N: int, kap: np.ndarray) -> np.ndarray:
    """P mod C(X): X^(N+m) = X^m sum_i kappa_i X^i."""
    P = P.copy()
    nz = int(np.count_nonzero(kap))
    for j in range(P.size - 1, N - 1, -1):
        m = j - N
        t = min(nz, j - m)            # positions m .. j-1 receive contributions
        P[m:m + t] += P[j] * kap[:t]
        P[j] = 0.0
    return P[:N]


def convolution(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """The Convolution black box (Section 2.1) with numpy's real FFT."""
    L = x.size
    return np.fft.irfft(np.fft.rfft(x) * np.fft.rfft(y), L)


def _round(Wbar: np.ndarray, scale: float):
    s = Wbar * scale
    c = np.rint(s)
    return c.astype(np.int64), float(np.max(np.abs(s - c))) if s.size else 0.0


def mul_full(u: int, v: int, n: int, b: int, L: int, Nd: int) -> dict:
    """Algorithm 1 (balanced digits, cyclic length L >= 2 Nd - 1)."""
    U = np.array(trace.split("full", u, n, b, Nd), dtype=np.float64)
    V = np.array(trace.split("full", v, n, b, Nd), dtype=np.float64)
    x = np.zeros(L); x[:Nd] = U
    y = np.zeros(L); y[:Nd] = V
    W = convolution(x, y)
    c, margin = _round(W, 1.0)
    return {"c": c, "margin": margin, "out": trace.eval_at_2b(c, b)}


def alpha_star(U: np.ndarray, N: int, b: int, lam: int) -> np.ndarray:
    return cyclic_map(U, coef_table("alpha", N, b, lam))


def beta_star(W: np.ndarray, N: int, b: int, lam: int) -> np.ndarray:
    return reduce_mod_A(shifted_terms(W, coef_table("beta", N, b, lam)), N, b)


def mul_lo(u: int, v: int, n: int, b: int, N: int, lam_a: int, lam_b: int) -> dict:
    """Algorithm 2."""
    U = np.array(trace.split("lo", u, n, b, N), dtype=np.float64)
    V = np.array(trace.split("lo", v, n, b, N), dtype=np.float64)
    Ut = alpha_star(U, N, b, lam_a)                       # convert to cyclic convolution
    Vt = alpha_star(V, N, b, lam_a)
    Wt = convolution(Ut, Vt)                              # perform convolution
    Wbar = beta_star(Wt, N, b, lam_b)                     # convert back
    c, margin = _round(Wbar, 2.0 ** b)                    # overlap-add (rounding)
    return {"Ut": Ut, "Vt": Vt, "Wt": Wt, "Wbar": Wbar, "c": c, "margin": margin,
            "out": trace.low_output(c, n, b)}


def gamma_dagger(F: np.ndarray, N: int, b: int, lam: int, rho: float):
    """gamma-dagger (Proposition 4.18): F mod C by eq. (4.5), gamma*, theta."""
    kap = kappa(N, b, rho)
    Fc = F[:N] + kap * F[N]
    G = cyclic_map(Fc, coef_table("gamma", N, b, lam))
    j = np.arange(N + 1, dtype=np.float64)
    w = np.exp(-j * math.log(rho))                        # rho^-j
    theta = float(np.sum(w * F[::-1]))                    # sum_j rho^-j F_(N-j)
    return G, theta


def delta_dagger(Wt: np.ndarray, theta: float, N: int, b: int, lam: int, rho: float) -> np.ndarray:
    """delta-dagger (Proposition 4.19, eqs. 4.6-4.7)."""
    kap = kappa(N, b, rho)
    H = reduce_mod_C(shifted_terms(Wt, coef_table("delta", N, b, lam)), N, kap)
    i = np.arange(N, dtype=np.float64)
    lr = math.log(rho)
    Hrho = float(np.sum(H * np.exp((i - 2 * N) * lr)))    # rho^-2N H(rho)
    psi = (theta - Hrho) / (1.0 - N * math.exp(b * math.log(2.0) - (N + 1) * lr))
    J = np.zeros(N + 1)
    J[:N] += H
    J[1:] -= H * 2.0 ** -b
    J[:N] -= psi * kap
    J[N] += psi
    return J


def rho_float(N: int, b: int) -> float:
    """rho by Newton from 2^b in the scaled variable y = rho/2^b (Lemma 4.2)."""
    eps = 2.0 ** (-N * b)
    y = 1.0
    for _ in range(100):
        f = y ** N * (y - 1.0) + eps
        df = y ** (N - 1) * ((N + 1) * y - N)
        yn = y - f / df
        if yn == y:
            break
        y = yn
    return y * 2.0 ** b


def mul_hi(u: int, v: int, n: int, b: int, N: int, lam_g: int, lam_d: int) -> dict:
    """Algorithm 3."""
    rho = rho_float(N, b)
    U = np.array(trace.split("hi", u, n, b, N), dtype=np.float64)
    V = np.array(trace.split("hi", v, n, b, N), dtype=np.float64)
    Ut, thU = gamma_dagger(U, N, b, lam_g, rho)          # convert to cyclic convolution
    Vt, thV = gamma_dagger(V, N, b, lam_g, rho)
    Wt = convolution(Ut, Vt)                              # perform convolution
    thW = thU * thV
    Wbar = delta_dagger(Wt, thW, N, b, lam_d, rho)        # convert back
    c, margin = _round(Wbar, 2.0 ** b)                    # overlap-add (rounding)
    return {"Ut": Ut, "Vt": Vt, "thU": thU, "thV": thV, "Wt": Wt, "Wbar": Wbar, "c": c,
            "margin": margin, "out": trace.high_output(c, n, N, b)}
