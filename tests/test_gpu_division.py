"""Division on the GPU (tm_reciprocal, tm_barrett_*), through the C ABI (marked gpu).

The reciprocal floor((2^(2k) - 1) / m) and the quotient and remainder of Barrett's
division must equal their definitions (oracle.division) exactly, for divisors of
every width class (one limb, limb boundaries, the Newton path above 60 bits, the
large configurations) and for the extreme dividends and divisors."""
import numpy as np
import pytest

import workloads
from gpu_util import dev, host
from oracle import bigmul
from oracle import division as D

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


def _limbs(x: int, n_bits: int) -> np.ndarray:
    return bigmul.from_int(x, (n_bits + 63) // 64)


def _divisor(k: int, seed: int, kind: str = "random") -> int:
    if kind == "min":
        return 1 << (k - 1)
    if kind == "max":
        return (1 << k) - 1
    if kind == "min+1":
        return (1 << (k - 1)) + (1 if k > 1 else 0)
    return bigmul.to_int(workloads.random_limbs(k, seed)) | (1 << (k - 1))


RECIP_K = [1, 2, 3, 7, 59, 60, 61, 63, 64, 65, 100, 127, 128, 129, 1000, 4097, 65536, 100003]


@pytest.mark.parametrize("k", RECIP_K)
@pytest.mark.parametrize("kind", ["random", "min", "max", "min+1"])
def test_reciprocal(pkg, k, kind):
    m = _divisor(k, seed=k, kind=kind)
    R = pkg.reciprocal(dev(_limbs(m, k)), k)
    assert bigmul.to_int(host(R)) == D.reciprocal(m, k)


@pytest.mark.parametrize("k", [1 << 20, (1 << 21) + 17])
def test_reciprocal_large(pkg, k):
    m = _divisor(k, seed=3)
    R = pkg.reciprocal(dev(_limbs(m, k)), k)
    assert bigmul.to_int(host(R)) == D.reciprocal(m, k)


def _dividends(k: int, m: int, seed: int):
    rng = np.random.default_rng(seed)
    top = (1 << (2 * k)) - 1
    t = bigmul.to_int(workloads.random_limbs(k, seed + 1))
    xs = [0, 1, m - 1, m, top, bigmul.to_int(workloads.random_limbs(2 * k, seed)),
          min(m * t, top), max(min(m * t, top) - 1, 0), (m * ((top // m) - 1)) if k > 1 else 0]
    return xs + [int(rng.integers(0, 1 << 62)) % (top + 1)]


@pytest.mark.parametrize("k", [1, 2, 5, 60, 61, 64, 65, 1000, 4097, 65536, 250001])
@pytest.mark.parametrize("kind", ["random", "min", "max"])
def test_barrett_divrem(pkg, k, kind):
    m = _divisor(k, seed=100 + k, kind=kind)
    b = pkg.Barrett(dev(_limbs(m, k)), k)
    try:
        assert bigmul.to_int(host(b.reciprocal())) == D.reciprocal(m, k)
        for x in _dividends(k, m, seed=k):
            q, r, rep = b.divrem(dev(_limbs(x, 2 * k)))
            assert rep["status"] == 0
            assert (bigmul.to_int(host(q)), bigmul.to_int(host(r))) == D.divrem(x, m), x
    finally:
        b.close()


def test_barrett_large(pkg):
    """k = 2^20: quotient and remainder of random dividends, and the remainder-only
    and quotient-only forms."""
    k = 1 << 20
    m = _divisor(k, seed=20)
    b = pkg.Barrett(dev(_limbs(m, k)), k)
    try:
        for seed in range(2):
            x = bigmul.to_int(workloads.random_limbs(2 * k, 40 + seed))
            dx = dev(_limbs(x, 2 * k))
            q, r, rep = b.divrem(dx)
            assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
            want = D.divrem(x, m)
            assert (bigmul.to_int(host(q)), bigmul.to_int(host(r))) == want
            _, r2, _ = b.divrem(dx, want=("r",))
            q2, _, _ = b.divrem(dx, want=("q",))
            assert bigmul.to_int(host(r2)) == want[1] and bigmul.to_int(host(q2)) == want[0]
    finally:
        b.close()


def test_barrett_config_2_24(pkg):
    """The served workload's divisor size: a 2^24-bit modulus. Python's division of a
    random 2^25-bit dividend takes minutes, so the pair is recognised by x = q m + r,
    0 <= r < m (unique), and the reciprocal by its defining inequality."""
    k = 1 << 24
    m = _divisor(k, seed=24)
    b = pkg.Barrett(dev(_limbs(m, k)), k)
    try:
        R = bigmul.to_int(host(b.reciprocal()))
        assert m * R <= (1 << (2 * k)) - 1 < m * (R + 1)
        x = bigmul.to_int(workloads.random_limbs(2 * k, 77))
        q, r, rep = b.divrem(dev(_limbs(x, 2 * k)))
        assert rep["status"] == 0
        assert D.is_divrem(x, m, bigmul.to_int(host(q)), bigmul.to_int(host(r)))
    finally:
        b.close()


def test_divisor_width_checked(pkg):
    k = 100
    m = (1 << (k - 2)) + 5                 # bit k-1 clear
    with pytest.raises(pkg.TruncMulError) as e:
        pkg.reciprocal(dev(_limbs(m, k)), k)
    assert e.value.code == pkg.TM_EINVAL
    with pytest.raises(pkg.TruncMulError) as e:
        pkg.Barrett(dev(_limbs(m, k)), k)
    assert e.value.code == pkg.TM_EINVAL
