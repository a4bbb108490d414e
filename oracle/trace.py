"""Exact integer trace of the truncated-product method (test infrastructure only).

Everything here is exact integer arithmetic (Python ints and int64 numpy arrays
whose ranges are checked). Given the split parameters (b, N), the trace gives:

- the digits of the "Split inputs" step of Algorithms 1-3, in the balanced form the
  paper's implementation uses (Section 5: |U_i| <= 2^(b-1)); the reading for
  the high product keeps its top digit U_N unbalanced, 0 <= U_N <= 2^b;
- w_i, the coefficients of W = U V (proofs of Theorems 2.1-2.3), by Kronecker
  substitution X = 2^64 through the exact big-integer product;
- c_i = 2^b L_i (Proposition 3.1) for the low product and c_i = 2^b H_i
  (Proposition 4.1) for the high product: the integers that the overlap-add
  steps of Algorithms 2 and 3 obtain as round(2^b * Wbar_i);
- the overlap-add outputs of Algorithms 1, 2 and 3 (with the round-half-up
  reading of Algorithm 3's final round(t)).
"""
import numpy as np

from . import bigmul

# ---------------------------------------------------------------- digit split

def unsigned_digits(x: int, count: int, b: int) -> list:
    """d_i = bits [ib, ib+b) of x, i = 0..count-1 (x >= 0). The bits are read from
    the binary string of x once (least significant first), so the cost is linear
    in the length of x."""
    assert x >= 0
    bits = bin(x)[2:][::-1]
    return [int(bits[i * b:(i + 1) * b][::-1] or "0", 2) for i in range(count)]


def balanced_digits(x: int, count: int, b: int, balance_top: bool) -> list:
    """Digits u_i with sum u_i 2^(ib) == x (mod 2^(count*b)) and |u_i| <= 2^(b-1).

    u_i = d_i - 2^b [d_i >= 2^(b-1)] + [d_(i-1) >= 2^(b-1)] (Section 5, signed
    coefficients). With balance_top=False the top digit is left as d + carry in
    [0, 2^b], which makes the sum exact whenever x < 2^(count*b).
    """
    d = unsigned_digits(x, count, b)
    half = 1 << (b - 1)
    out, carry = [], 0
    for i, di in enumerate(d):
        if i == count - 1 and not balance_top:
            out.append(di + carry)
            carry = 0
            break
        top = 1 if di >= half else 0
        out.append(di - (top << b) + carry)
        carry = top
    return out


def split(kind: str, u: int, n: int, b: int, N: int) -> list:
    """The "Split inputs" step of Algorithms 1-3 with balanced digits.

    full: N digits, requires N*b >= n+1 so that the top digit never carries out;
    lo:   N digits with U(2^b) == u (mod 2^(Nb)) (Algorithm 2 only needs that);
    hi:   N+1 digits of u * 2^((N+1)b - n) (Algorithm 3), top digit unbalanced.
    """
    if kind == "full":
        assert N * b >= n + 1
        return balanced_digits(u, N, b, balance_top=True)
    if kind == "lo":
        assert N * b >= n
        return balanced_digits(u, N, b, balance_top=True)
    if kind == "hi":
        s0 = (N + 1) * b - n
        assert s0 >= 0
        return balanced_digits(u << s0, N + 1, b, balance_top=False)
    raise ValueError(kind)


def eval_poly(coeffs, x: int) -> int:
    """sum coeffs[i] x^i (Horner), exact."""
    acc = 0
    for c in reversed(list(coeffs)):
        acc = acc * x + int(c)
    return acc


# ------------------------------------------------ exact polynomial product

def _signed_to_int_at_2_64(digits) -> int:
    """U(2^64) for signed digits |u_i| < 2^63, via two's complement limbs."""
    a = np.asarray(digits, dtype=np.int64)
    as_u = a.view(np.uint64)
    pos = bigmul.to_int(as_u)                 # sum (u_i mod 2^64) 2^(64 i)
    neg = (a < 0).astype(np.uint64)
    # each negative digit was read as u_i + 2^64, i.e. contributes an extra 2^(64(i+1))
    correction = bigmul.to_int(np.concatenate([np.zeros(1, np.uint64), neg]))
    return pos - correction


def poly_mul_exact(U, V, bigmul_threshold: int = 2048) -> np.ndarray:
    """w = U * V as int64 coefficients (|w_i| < 2^62 is asserted).

    Kronecker substitution: W(2^64) = U(2^64) V(2^64), then read the 64-bit
    fields of W(2^64) + sum_i 2^63 2^(64 i), each of which is w_i + 2^63.
    """
    U = [int(x) for x in U]
    V = [int(x) for x in V]
    bound = len(U) * max(1, max(abs(x) for x in U)) * max(1, max(abs(x) for x in V))
    assert bound < (1 << 62), "coefficients too large for the 64-bit Kronecker slots"
    count = len(U) + len(V) - 1
    a = _signed_to_int_at_2_64(U)
    c = _signed_to_int_at_2_64(V)
    if max(len(U), len(V)) < bigmul_threshold:
        prod = a * c
    else:   # magnitudes through the C oracle product, sign by hand
        nl = max(len(U), len(V)) + 1
        ma = bigmul.from_int(abs(a), nl)
        mc = bigmul.from_int(abs(c), nl)
        prod = bigmul.to_int(bigmul.mul_full(ma, mc, par_depth=3))
        if (a < 0) != (c < 0):
            prod = -prod
    offset = bigmul.to_int(np.full(count, 1 << 63, dtype=np.uint64))
    shifted = prod + offset
    assert 0 <= shifted < (1 << (64 * count))
    fields = bigmul.from_int(shifted, count)
    return (fields ^ np.uint64(1 << 63)).view(np.int64).copy()


# ------------------------------------------------------- c_i and outputs

def low_coeffs(w: np.ndarray, N: int, b: int) -> np.ndarray:
    """c_i = 2^b L_i, L = W mod A(X), A = X^N + 2^-b X - 1 (Proposition 3.1):
    L_i = w_i + w_(N+i) - 2^-b w_(N+i-1), with w_j = 0 for j > 2N-2."""
    w = np.asarray(w, dtype=np.int64)
    assert w.size == 2 * N - 1
    hi = np.zeros(N, dtype=np.int64)
    hi[: N - 1] = w[N:]                       # w_(N+i), i = 0..N-2
    prev = np.zeros(N, dtype=np.int64)
    prev[1:] = w[N:]                          # w_(N+i-1), i = 1..N-1
    assert np.abs(w).max(initial=0) < (1 << (62 - b))
    return (w[:N] + hi) * (1 << b) - prev


def high_coeffs(w: np.ndarray, N: int, b: int) -> np.ndarray:
    """c_i = 2^b H_i, H = (1 - 2^-b X) W mod B(X), B = X^(N+1) - 2^b X^N + 2^b
    (Proposition 4.1): H_i = [i<N] w_i - 2^-b [i>=1] w_(i-1) + w_(N+i), i = 0..N."""
    w = np.asarray(w, dtype=np.int64)
    assert w.size == 2 * N + 1
    low = np.zeros(N + 1, dtype=np.int64)
    low[:N] = w[:N]
    prev = np.zeros(N + 1, dtype=np.int64)
    prev[1:] = w[:N]
    assert np.abs(w).max(initial=0) < (1 << (62 - b))
    return (low + w[N:]) * (1 << b) - prev


def eval_at_2b(c, b: int) -> int:
    """sum c_i 2^(ib) for integer c_i, by pairwise combination."""
    vals = [int(x) for x in c]
    if not vals:
        return 0
    shift = b
    while len(vals) > 1:
        nxt = [vals[j] + (vals[j + 1] << shift) for j in range(0, len(vals) - 1, 2)]
        if len(vals) % 2:
            nxt.append(vals[-1])
        vals = nxt
        shift *= 2
    return vals[0]


def low_output(c: np.ndarray, n: int, b: int) -> int:
    """Algorithm 2, overlap-add: sum 2^-b c_i 2^(ib) mod 2^n. c_0 is divisible by 2^b
    (c_0 = 2^b (w_0 + w_N)), so the sum is an integer."""
    c0 = int(c[0])
    assert c0 % (1 << b) == 0
    return eval_at_2b(c, b) >> b & ((1 << n) - 1)


def high_t_numerator(c: np.ndarray, n: int, N: int, b: int):
    """Algorithm 3, overlap-add: t = S / 2^s with S = sum c_i 2^(ib), s = (N+3)b - n."""
    return eval_at_2b(c, b), (N + 3) * b - n


def high_output(c: np.ndarray, n: int, N: int, b: int) -> int:
    """Algorithm 3, returned value round(t), read as round half up: floor(t + 1/2)."""
    S, s = high_t_numerator(c, n, N, b)
    return (S + (1 << (s - 1))) >> s


# ----------------------------------------------------------- whole traces

def trace(kind: str, u: int, v: int, n: int, b: int, N: int) -> dict:
    """Exact trace for one product; returns digits, w, c and the final output."""
    U = split(kind, u, n, b, N)
    V = split(kind, v, n, b, N)
    w = poly_mul_exact(U, V)
    if kind == "full":
        c = w
        out = eval_at_2b(c, b)
    elif kind == "lo":
        c = low_coeffs(w, N, b)
        out = low_output(c, n, b)
    else:
        c = high_coeffs(w, N, b)
        out = high_output(c, n, N, b)
    return {"U": U, "V": V, "w": w, "c": c, "out": out}
