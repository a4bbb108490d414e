"""Division by a k-bit divisor, by definition (test infrastructure only).

Section 1 of the paper names Barrett's reduction as an application of the high
product. The GPU library divides with Newton's iteration and Barrett's quotient;
here the results are their definitions, on Python integers:

- ``reciprocal(m, k)``: R = floor((2^(2k) - 1) / m) for 2^(k-1) <= m < 2^k, the
  reciprocal the library's Barrett context keeps (k + 1 bits);
- ``divrem(x, m)``: q = floor(x / m), r = x - q m;
- ``is_divrem(x, m, q, r)``: the same pair recognised by x = q m + r, 0 <= r < m.

``long_division`` is a second, independent evaluation (binary restoring division,
one quotient bit per step) that the CPU tests compare with the definitions.
"""


def reciprocal(m: int, k: int) -> int:
    """floor((2^(2k) - 1) / m) for a divisor of exactly k bits."""
    if not (1 << (k - 1)) <= m < (1 << k):
        raise ValueError("m must have exactly k bits")
    return ((1 << (2 * k)) - 1) // m


def divrem(x: int, m: int):
    """(floor(x / m), x mod m) for x >= 0, m >= 1."""
    if x < 0 or m < 1:
        raise ValueError("x >= 0 and m >= 1 required")
    return x // m, x % m


def is_divrem(x: int, m: int, q: int, r: int) -> bool:
    """Euclidean division is unique: (q, r) == divrem(x, m) exactly when x = q m + r
    and 0 <= r < m. One product instead of a division, for very long operands."""
    return 0 <= r < m and q * m + r == x


def long_division(x: int, m: int):
    """Binary restoring division: bit i of the quotient from the partial remainder."""
    q, r = 0, 0
    for i in range(x.bit_length() - 1, -1, -1):
        r = 2 * r + ((x >> i) & 1)
        q *= 2
        if r >= m:
            r -= m
            q += 1
    return q, r
