"""High-precision cos and sin of rational multiples of 2 pi with the standard
library's decimal module (about 200 bits), for checking tables against exact
values on machines without mpmath. pi from Machin's formula
pi/4 = 4 atan(1/5) - atan(1/239); cos and sin from their Taylor series after
reduction to [0, pi/4]."""
from decimal import Decimal, localcontext

PREC = 70


def _atan_inv(x: int) -> Decimal:
    """atan(1/x) for an integer x > 1 by its alternating series."""
    x2 = x * x
    term = Decimal(1) / x
    total, k, sign = term, 1, 1
    eps = Decimal(10) ** -(PREC + 5)
    while term > eps:
        term /= x2
        k += 2
        sign = -sign
        total += sign * term / k
    return total


def _pi() -> Decimal:
    with localcontext() as ctx:
        ctx.prec = PREC + 10
        return 4 * (4 * _atan_inv(5) - _atan_inv(239))


_PI = None


def pi() -> Decimal:
    global _PI
    if _PI is None:
        _PI = _pi()
    return _PI


def _sincos_small(x: Decimal):
    """sin x, cos x for 0 <= x <= pi/4 (Taylor series)."""
    with localcontext() as ctx:
        ctx.prec = PREC + 10
        x2 = x * x
        s, c = x, Decimal(1)
        ts, tc = x, Decimal(1)
        eps = Decimal(10) ** -(PREC + 8)
        j = 1
        while abs(ts) > eps or abs(tc) > eps:
            ts = -ts * x2 / ((2 * j) * (2 * j + 1))
            tc = -tc * x2 / ((2 * j - 1) * (2 * j))
            s += ts
            c += tc
            j += 1
        return s, c


def cossin_2pi(m: int, length: int):
    """(cos, sin) of 2 pi m / length as Decimals."""
    with localcontext() as ctx:
        ctx.prec = PREC + 10
        m %= length
        q, r = divmod(4 * m, length)              # angle = pi/2 (q + r/length)
        swap = 2 * r > length
        if swap:
            r = length - r
        s, c = _sincos_small(pi() / 2 * Decimal(r) / Decimal(length))
        if swap:
            s, c = c, s
        return [(c, s), (-s, c), (-c, -s), (s, -c)][q]
