"""The truncated-FFT question left open at the end of Section 2.2 ("The full
product"), as a CPU experiment (test infrastructure only; the library has no
counterpart).

A truncated Fourier transform (TFT) of length N, 2^(k-1) < N <= 2^k, evaluates a
polynomial of degree < N at the N points omega^rev_k(i), i < N, where omega =
exp(2 pi i / 2^k) and rev_k reverses k bits; its inverse interpolates at the same
points. Multiplying two such transforms pointwise therefore computes the product
modulo g_N(X) = prod_{i<N} (X - omega^rev_k(i)). That is X^N - 1 only when N is a
power of two. For any other N the N points are all 2^(k-1)-th roots of unity
plus part of the odd 2^k-th roots, an uneven set.

Algorithm 2 needs the product modulo X^N - 1: alpha* and beta* (Section 3.3) are
the ring isomorphisms between R[X]/A(X), A = X^N + 2^-b X - 1, and R[X]/(X^N - 1)
induced by the analytic maps alpha, beta that carry the N roots of A to the N-th
roots of unity (Lemma 3.4, Corollary 3.14). They are short (lambda terms) because
beta(z) = z (1 - 2^-b z)^(-1/N) moves each root by a relative 2^-b / N. Any
bijection between the roots of A and the TFT points also induces a ring
isomorphism R[X]/A -> R[X]/g_N, but the TFT points are not the image of A's
roots under a map close to the identity, so this isomorphism has no short form.

The functions below measure that: the matrix of the induced isomorphism (roots
paired by angle) for the two targets, its profile along cyclic diagonals, and
Algorithm 2 run with the Convolution step replaced by the product modulo g_N.
"""
import numpy as np

from . import fp64_ref
from . import trace


def bit_reverse(i: int, k: int) -> int:
    return int(format(i, f"0{k}b")[::-1], 2) if k else 0


def tft_points(N: int) -> np.ndarray:
    """omega^rev_k(i), i < N, with 2^(k-1) < N <= 2^k: the evaluation points of a
    truncated Fourier transform of length N."""
    k = max(0, (N - 1).bit_length())
    return np.exp(2j * np.pi * np.array([bit_reverse(i, k) for i in range(N)]) / 2 ** k)


def cyclic_points(N: int) -> np.ndarray:
    """The N-th roots of unity: the points of a length-N DFT (roots of X^N - 1)."""
    return np.exp(2j * np.pi * np.arange(N) / N)


def low_roots(N: int, b: int) -> np.ndarray:
    """The roots of A(X) = X^N + 2^-b X - 1 (Section 3.2), by Newton's method from
    the N-th roots of unity (Lemma 3.3 puts one root near each)."""
    z = cyclic_points(N).astype(complex)
    for _ in range(60):
        z = z - (z ** N + 2.0 ** -b * z - 1) / (N * z ** (N - 1) + 2.0 ** -b)
    return z


def _by_angle(z: np.ndarray) -> np.ndarray:
    return z[np.argsort(np.mod(np.angle(z), 2 * np.pi))]


def ring_map(src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Matrix T of the ring isomorphism R[X]/prod(X - src) -> R[X]/prod(X - dst)
    that sends F to the G of degree < N with G(d_i) = F(s_i), the points paired in
    order of angle: T = V(dst)^-1 V(src) on coefficient vectors."""
    s, d = _by_angle(src), _by_angle(dst)
    N = s.size
    return np.linalg.solve(np.vander(d, N, increasing=True), np.vander(s, N, increasing=True))


def diagonal_profile(T: np.ndarray) -> np.ndarray:
    """prof[r] = max |T[j, k]| over (j - k) mod N = r: alpha* only fills the
    diagonals r < lambda (its term r sends F_k to X^(k+r))."""
    N = T.shape[0]
    j, k = np.indices(T.shape)
    prof = np.zeros(N)
    np.maximum.at(prof, (j - k) % N, np.abs(T))
    return prof


def product_at_points(x: np.ndarray, y: np.ndarray, points: np.ndarray) -> np.ndarray:
    """The product of x and y (coefficient vectors of length N) modulo
    prod(X - p): values at the points, pointwise product, interpolation - what a
    transform evaluating at `points` and its inverse compute."""
    N = x.size
    V = np.vander(points, N, increasing=True)
    w = np.linalg.solve(V, (V @ x) * (V @ y))
    return w.real


def mul_lo_with(u: int, v: int, n: int, b: int, N: int, lam_a: int, lam_b: int,
                points: np.ndarray) -> dict:
    """Algorithm 2 with the Convolution step replaced by the product at `points`
    (the N-th roots of unity give the cyclic convolution; TFT points give the
    product modulo g_N)."""
    U = np.array(trace.split("lo", u, n, b, N), dtype=np.float64)
    V = np.array(trace.split("lo", v, n, b, N), dtype=np.float64)
    Ut = fp64_ref.alpha_star(U, N, b, lam_a)
    Vt = fp64_ref.alpha_star(V, N, b, lam_a)
    Wt = product_at_points(Ut, Vt, points)
    Wbar = fp64_ref.beta_star(Wt, N, b, lam_b)
    s = Wbar * 2.0 ** b
    c = np.rint(s).astype(np.int64)
    # the overlap-add needs 2^b | c_0 (Proposition 3.1); a wrong product may break it
    out = trace.low_output(c, n, b) if c[0] % (1 << b) == 0 else None
    return {"c": c, "margin": float(np.max(np.abs(s - c))), "out": out}
