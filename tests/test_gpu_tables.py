"""Accuracy of the FFT kernels' twiddle tables (marked gpu).

The FFT error bound takes every table component within 2^-53 (1 + 2^-40) of its
exact value: a twiddle (cos, -sin)(2 pi m / len) and a twist coefficient
cos(2 pi k / N) (cos, -sin)(2 pi k / N) / N rounded once to the nearest double,
and a tangent-form radix-4 record (t, c) with c the nearest double to the cosine
and t the nearest double to sin / c. tm_table_values writes the tables with the
kernels the plans use; every sampled entry is compared with its exact value to
about 200 bits (tests/hp_trig.py, standard-library decimals): it must be the
nearest double, unless the exact value lies within 2^-30 of an ulp of a
rounding tie."""
from decimal import Decimal, localcontext

import numpy as np
import pytest

import hp_trig

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1703_00640_gb300 as p
    p.build()
    p.load()
    return p


def _nearest_ok(got: float, exact: Decimal) -> bool:
    """got is the double nearest to `exact` (or exact is within 2^-30 ulp of a tie)."""
    want = float(exact)                          # correctly rounded conversion
    if got == want:
        return True
    lo, hi = sorted((float(got), want))
    if np.nextafter(lo, np.inf) != hi:
        return False                             # more than one ulp apart
    with localcontext() as ctx:
        ctx.prec = 80
        tie = (Decimal(lo) + Decimal(hi)) / 2
        return abs(exact - tie) <= (Decimal(hi) - Decimal(lo)) * Decimal(2) ** -30


def _sample(count, k=1500, seed=0):
    if count <= k:
        return np.arange(count)
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([np.arange(40), count - 1 - np.arange(40),
                                     rng.integers(0, count, k)]))


@pytest.mark.parametrize("length", [4, 6, 8, 12, 20, 28, 60, 105, 1024, 3 * 2 ** 11,
                                    5 * 2 ** 13, 189 * 2 ** 9, 2 ** 20 * 5])
def test_twiddles_are_correctly_rounded(pkg, length):
    tab = pkg.table_values(0, length, length).reshape(-1, 2)
    for m in _sample(length, seed=length):
        c, s = hp_trig.cossin_2pi(int(m), length)
        assert _nearest_ok(tab[m, 0], c), (length, m, "cos")
        assert _nearest_ok(tab[m, 1], -s), (length, m, "sin")


@pytest.mark.parametrize("N", [8, 12, 40, 6144, 2 ** 21, 2621440])
def test_twist_coefficients_are_correctly_rounded(pkg, N):
    count = N // 4 + 1
    tab = pkg.table_values(2, N, count).reshape(-1, 2)
    with localcontext() as ctx:
        ctx.prec = 80
        for k in _sample(count, seed=N):
            c, s = hp_trig.cossin_2pi(int(k), N)
            assert _nearest_ok(tab[k, 0], c * c / N), (N, k)
            assert _nearest_ok(tab[k, 1], -c * s / N), (N, k)


OUTER = [(12, 3), (12, 4), (40, 8), (4096, 64), (6144, 48), (2 ** 20, 1024),
         (9 * 2 ** 17, 1152), (5 * 2 ** 20, 5120), (45 * 2 ** 15, 1440), (7 * 2 ** 12, 7)]


@pytest.mark.parametrize("Mp,Qc", OUTER, ids=[f"{m}x{q}" for m, q in OUTER])
def test_outer_twiddles_in_output_order(pkg, Mp, Qc):
    """The four-step table entry k Qc + qc is the double nearest to
    exp(-2 pi i (qc k mod Mp) / Mp) (sampled against 200-bit values), and every
    entry equals the plain table's entry at qc k mod Mp, bit for bit."""
    tab = pkg.table_values(3, Mp, Qc).reshape(-1, 2)
    plain = pkg.table_values(0, Mp, Mp).reshape(-1, 2)
    e = np.arange(Mp, dtype=np.int64)
    k, qc = e // Qc, e % Qc
    m = (qc * k) % Mp
    assert np.array_equal(tab.view(np.int64), plain[m].view(np.int64)), (Mp, Qc)
    for i in _sample(Mp, k=600, seed=Mp + Qc):
        c, s = hp_trig.cossin_2pi(int(m[i]), Mp)
        assert _nearest_ok(tab[i, 0], c), (Mp, Qc, int(i), "cos")
        assert _nearest_ok(tab[i, 1], -s), (Mp, Qc, int(i), "sin")


def test_outer_twiddles_argument_checked(pkg):
    with pytest.raises(pkg.TruncMulError):
        pkg.table_values(3, 40, 7)


@pytest.mark.parametrize("Ns", [1, 2, 4, 16, 64, 256, 1024])
def test_tangent_records(pkg, Ns):
    """c is the nearest double to the cosine and t the nearest double to sin / c,
    so c (1 - i t) is within 2^-53 (1 + 2^-30) of the twiddle; the records of
    angles at or above pi/2 carry -c and describe -i c (1 - i t)."""
    tab = pkg.table_values(1, Ns, Ns).reshape(-1, 4)
    bound = Decimal(2) ** -53 * (1 + Decimal(2) ** -30)
    with localcontext() as ctx:
        ctx.prec = 80
        for k in range(Ns):
            t1, c1, t2, c2s = (float(x) for x in tab[k])
            cth, sth = hp_trig.cossin_2pi(k, 4 * Ns)
            assert _nearest_ok(c1, cth) and _nearest_ok(t1, sth / Decimal(c1)), (Ns, k)
            rot = 2 * k >= Ns
            cph, sph = hp_trig.cossin_2pi(2 * k - Ns if rot else 2 * k, 4 * Ns)
            c2 = abs(c2s)
            assert (c2s < 0) == rot, (Ns, k)
            assert _nearest_ok(c2, cph) and _nearest_ok(t2, sph / Decimal(c2)), (Ns, k)
            # the twiddles the butterfly applies: c (1 - i t) against exp(-i angle)
            dr, di = Decimal(c1) - cth, Decimal(c1) * Decimal(t1) - sth
            assert (dr * dr + di * di).sqrt() <= bound, (Ns, k, "w1")
            dr, di = Decimal(c2) - cph, Decimal(c2) * Decimal(t2) - sph
            assert (dr * dr + di * di).sqrt() <= bound, (Ns, k, "w2")
