"""A float64 model of the FFT kernels' arithmetic (test infrastructure).

The FP64 error bound of the convolution (eta_conv in the oracle's planner and the
library's) is derived for the operations the CUDA kernels perform: the Stockham
butterflies of radix 2, 3, 4 (plain and tangent form), 5 and 7, the table-twiddle
products, the four-step twiddles between passes, and the fused real-FFT twist and
pointwise product. This module performs the same operation sequences in the same
order on Python floats (IEEE binary64 with rounding to nearest, as on the GPU),
with a correctly rounded fused multiply-add, and with the tables' values (each
the nearest double to its exact value), so that the tests can measure the exact
rounding error of that arithmetic on chosen inputs and hold the bound against it.

Complex numbers are pairs (re, im) of floats. S = -1 is the forward direction,
S = +1 the inverse.
"""
import math

import hp_trig

_SPLIT = 134217729.0          # 2^27 + 1, Veltkamp's splitting constant


def _split(a: float):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def fma(a: float, b: float, c: float) -> float:
    """a * b + c rounded once: Dekker's exact product (p + e = a b) and a
    correctly rounded sum of p, e and c (math.fsum)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return math.fsum((p, e, c))


def cadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def csub(a, b):
    return (a[0] - b[0], a[1] - b[1])


def cmul(a, w):
    return (fma(a[0], w[0], -(a[1] * w[1])), fma(a[0], w[1], a[1] * w[0]))


def cmulc(a, w):              # a * conj(w)
    return (fma(a[0], w[0], a[1] * w[1]), fma(a[1], w[0], -(a[0] * w[1])))


def mul_si(a, S):             # a * (S i)
    return (a[1], -a[0]) if S < 0 else (-a[1], a[0])


def conj(a):
    return (a[0], -a[1])


# ------------------------------------------------------------ constants and tables

def nearest(x) -> float:
    return float(x)


C5 = [nearest(hp_trig.cossin_2pi(k, 5)[0]) for k in (1, 2)]
S5 = [nearest(hp_trig.cossin_2pi(k, 5)[1]) for k in (1, 2)]
C7 = [nearest(hp_trig.cossin_2pi(k, 7)[0]) for k in (1, 2, 3)]
S7 = [nearest(hp_trig.cossin_2pi(k, 7)[1]) for k in (1, 2, 3)]
SQRT3_2 = nearest(hp_trig.cossin_2pi(1, 3)[1])


def twiddle(m: int, length: int):
    """exp(-2 pi i m / length), each component the nearest double."""
    c, s = hp_trig.cossin_2pi(m, length)
    return (nearest(c), nearest(-s))


def tan_record(k: int, Ns: int):
    """(t1, c1, t2, c2s) of the tangent-form radix-4 butterfly: c the nearest
    double to the cosine, t the nearest double to sin / c."""
    from decimal import Decimal, localcontext
    with localcontext() as ctx:
        ctx.prec = 80
        c1d, s1d = hp_trig.cossin_2pi(k, 4 * Ns)
        c1 = nearest(c1d)
        t1 = nearest(s1d / Decimal(c1))
        rot = 2 * k >= Ns
        c2d, s2d = hp_trig.cossin_2pi(2 * k - Ns if rot else 2 * k, 4 * Ns)
        c2 = nearest(c2d)
        t2 = nearest(s2d / Decimal(c2))
    return (t1, c1, t2, -c2 if rot else c2)


def twist_coef(k: int, N: int):
    """cos(2 pi k / N) exp(-2 pi i k / N) / N, each component the nearest double."""
    from decimal import localcontext
    with localcontext() as ctx:
        ctx.prec = 80
        c, s = hp_trig.cossin_2pi(k, N)
        return (nearest(c * c / N), nearest(-c * s / N))


# ------------------------------------------------------------ butterflies

def dft2(x, S):
    return [cadd(x[0], x[1]), csub(x[0], x[1])]


def dft4(x, S):
    t0, t1 = cadd(x[0], x[2]), csub(x[0], x[2])
    t2, t3 = cadd(x[1], x[3]), mul_si(csub(x[1], x[3]), S)
    return [cadd(t0, t2), cadd(t1, t3), csub(t0, t2), csub(t1, t3)]


def dft3(x, S):
    t = cadd(x[1], x[2])
    m = (fma(t[0], -0.5, x[0][0]), fma(t[1], -0.5, x[0][1]))
    d = csub(x[1], x[2])
    sd = mul_si((d[0] * SQRT3_2, d[1] * SQRT3_2), S)
    return [cadd(x[0], t), cadd(m, sd), csub(m, sd)]


def dft5(x, S):
    t1, t2 = cadd(x[1], x[4]), cadd(x[2], x[3])
    d1, d2 = csub(x[1], x[4]), csub(x[2], x[3])
    x0 = x[0]
    a1 = tuple(fma(C5[0], t1[i], fma(C5[1], t2[i], x0[i])) for i in (0, 1))
    a2 = tuple(fma(C5[1], t1[i], fma(C5[0], t2[i], x0[i])) for i in (0, 1))
    b1 = mul_si(tuple(fma(S5[0], d1[i], S5[1] * d2[i]) for i in (0, 1)), S)
    b2 = mul_si(tuple(fma(S5[1], d1[i], -S5[0] * d2[i]) for i in (0, 1)), S)
    return [cadd(x0, cadd(t1, t2)), cadd(a1, b1), cadd(a2, b2), csub(a2, b2), csub(a1, b1)]


def dft7(x, S):
    t1, t2, t3 = cadd(x[1], x[6]), cadd(x[2], x[5]), cadd(x[3], x[4])
    d1, d2, d3 = csub(x[1], x[6]), csub(x[2], x[5]), csub(x[3], x[4])
    x0 = x[0]
    c1, c2, c3 = C7
    s1, s2, s3 = S7
    a1 = tuple(fma(c1, t1[i], fma(c2, t2[i], fma(c3, t3[i], x0[i]))) for i in (0, 1))
    a2 = tuple(fma(c2, t1[i], fma(c3, t2[i], fma(c1, t3[i], x0[i]))) for i in (0, 1))
    a3 = tuple(fma(c3, t1[i], fma(c1, t2[i], fma(c2, t3[i], x0[i]))) for i in (0, 1))
    b1 = mul_si(tuple(fma(s1, d1[i], fma(s2, d2[i], s3 * d3[i])) for i in (0, 1)), S)
    b2 = mul_si(tuple(fma(s2, d1[i], fma(-s3, d2[i], -s1 * d3[i])) for i in (0, 1)), S)
    b3 = mul_si(tuple(fma(s3, d1[i], fma(-s1, d2[i], s2 * d3[i])) for i in (0, 1)), S)
    return [cadd(x0, cadd(t1, cadd(t2, t3))), cadd(a1, b1), cadd(a2, b2), cadd(a3, b3),
            csub(a3, b3), csub(a2, b2), csub(a1, b1)]


DFT = {2: dft2, 3: dft3, 4: dft4, 5: dft5, 7: dft7}


def tan_bracket(z, t, S):
    if S < 0:
        return (fma(t, z[1], z[0]), fma(-t, z[0], z[1]))
    return (fma(-t, z[1], z[0]), fma(t, z[0], z[1]))


def radix4_tan(x, rec, S):
    t1, c1, t2, c2s = rec
    rot = math.copysign(1.0, c2s) < 0
    mag = abs(c2s)
    ca = -mag if (rot and S > 0) else mag
    cq = -mag if (rot and S < 0) else mag
    x2, x3 = tan_bracket(x[2], t2, S), tan_bracket(x[3], t2, S)
    p2, q2 = (x2[1], x2[0]) if rot else x2
    p3, q3 = (x3[1], x3[0]) if rot else x3
    x0, x1 = x[0], x[1]
    A = (fma(ca, p2, x0[0]), fma(cq, q2, x0[1]))
    B = (fma(-ca, p2, x0[0]), fma(-cq, q2, x0[1]))
    E = tan_bracket((fma(ca, p3, x1[0]), fma(cq, q3, x1[1])), t1, S)
    F = tan_bracket((fma(-ca, p3, x1[0]), fma(-cq, q3, x1[1])), t1, S)
    y0 = (fma(c1, E[0], A[0]), fma(c1, E[1], A[1]))
    y2 = (fma(-c1, E[0], A[0]), fma(-c1, E[1], A[1]))
    if S < 0:
        y1 = (fma(c1, F[1], B[0]), fma(-c1, F[0], B[1]))
        y3 = (fma(-c1, F[1], B[0]), fma(c1, F[0], B[1]))
    else:
        y1 = (fma(-c1, F[1], B[0]), fma(c1, F[0], B[1]))
        y3 = (fma(c1, F[1], B[0]), fma(-c1, F[0], B[1]))
    return [y0, y1, y2, y3]


# ------------------------------------------------------------ stages and passes

def radices(L: int):
    """Stages of a sub-FFT of length L, in the kernels' order: 7, 5, 3, then 4s and
    at most one 2."""
    out, rest = [], L
    for r in (7, 5, 3):
        while rest % r == 0:
            out.append(r)
            rest //= r
    twos = 0
    while rest % 2 == 0:
        rest //= 2
        twos += 1
    assert rest == 1, L
    out += [4] * (twos // 2) + [2] * (twos % 2)
    return out


def sub_fft(seq, S, tables):
    """One Stockham sub-FFT of length L = len(seq), natural order in and out: stage
    with radix R reads butterfly j's inputs at j + t L / R, multiplies input t by
    the table twiddle omega_L^(t (j mod Ns) L / (Ns R)) (the tangent form for
    radix 4 with Ns > 1), and writes output t at (j / Ns) Ns R + (j mod Ns) + t Ns."""
    L = len(seq)
    buf = list(seq)
    Ns = 1
    for R in radices(L):
        out = [None] * L
        nb = L // R
        step = L // (Ns * R)
        for j in range(nb):
            x = [buf[j + t * nb] for t in range(R)]
            kk = j % Ns
            if R == 4 and Ns > 1:
                y = radix4_tan(x, tables.tan(kk, Ns), S)
            else:
                if Ns > 1:
                    for t in range(1, R):
                        w = tables.tw(kk * t * step, L)
                        x[t] = cmul(x[t], w) if S < 0 else cmulc(x[t], w)
                y = DFT[R](x, S)
            base = (j // Ns) * Ns * R + kk
            for t in range(R):
                out[base + t * Ns] = y[t]
        buf = out
        Ns *= R
    return buf


class Tables:
    """The tables' values, computed once per entry."""

    def __init__(self):
        self._tw, self._tan, self._tc = {}, {}, {}

    def tw(self, m, length):
        key = (m % length, length)
        if key not in self._tw:
            self._tw[key] = twiddle(*key)
        return self._tw[key]

    def tan(self, k, Ns):
        if (k, Ns) not in self._tan:
            self._tan[(k, Ns)] = tan_record(k, Ns)
        return self._tan[(k, Ns)]

    def tc(self, k, N):
        if (k, N) not in self._tc:
            self._tc[(k, N)] = twist_coef(k, N)
        return self._tc[(k, N)]


def fft(z, S, split, tables):
    """Complex FFT of length M = len(z) in one pass (split = (M,)) or two passes
    (split = (L1, L2), M = L1 L2): L2 column transforms of length L1, the
    four-step twiddle omega_M^(q k) on output k of column q, then L1 row
    transforms of length L2."""
    M = len(z)
    if len(split) == 1:
        return sub_fft(z, S, tables)
    L1, L2 = split
    assert L1 * L2 == M
    mid = [None] * M
    for q in range(L2):
        col = sub_fft([z[q + j * L2] for j in range(L1)], S, tables)
        for k in range(L1):
            w = tables.tw(q * k, M)
            mid[q + k * L2] = cmul(col[k], w) if S < 0 else cmulc(col[k], w)
    out = [None] * M
    for q in range(L1):
        row = sub_fft([mid[q * L2 + j] for j in range(L2)], S, tables)
        for k in range(L2):
            out[q + k * L1] = row[k]
    return out


def twist(Zu, Zv, N, tables):
    """The fused real-FFT twist, pointwise product and inverse pre-twist for every
    pair (k, M - k), as the twist kernel computes it."""
    M = N // 2
    two_over_N = 2.0 / N
    Q = [None] * M
    for k in range(M // 2 + 1):
        km = 0 if k == 0 else M - k
        c = tables.tc(k, N)
        A0, B0 = Zu[k], conj(Zu[km])
        A1, B1 = Zv[k], conj(Zv[km])
        D0, D1 = csub(A0, B0), csub(A1, B1)
        AA, BB, DD = cmul(A0, A1), cmul(B0, B1), cmul(D0, D1)
        H = cmul(DD, c)
        Q[k] = (fma(two_over_N, AA[0], -H[0]), fma(two_over_N, AA[1], -H[1]))
        if k != 0 and km != k:
            Q[km] = (fma(two_over_N, BB[0], -H[0]), fma(-two_over_N, BB[1], H[1]))
    return Q


def convolution(x, y, split=None, tables=None):
    """The FP64 cyclic convolution of the real sequences x, y (floats, even length
    N) as the kernels compute it: pack, forward FFTs, twist, inverse FFT, unpack."""
    N = len(x)
    M = N // 2
    tables = tables or Tables()
    split = split or (M,)
    zu = [(float(x[2 * j]), float(x[2 * j + 1])) for j in range(M)]
    zv = [(float(y[2 * j]), float(y[2 * j + 1])) for j in range(M)]
    Zu = fft(zu, -1, split, tables)
    Zv = fft(zv, -1, split, tables)
    q = fft(twist(Zu, Zv, N, tables), 1, split, tables)
    out = []
    for v in q:
        out += [v[0], v[1]]
    return out


def exact_cyclic(x, y):
    """The exact cyclic convolution of integer sequences."""
    N = len(x)
    return [sum(int(x[i]) * int(y[(k - i) % N]) for i in range(N)) for k in range(N)]
