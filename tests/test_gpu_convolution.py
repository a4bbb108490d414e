"""The Convolution step alone (tm_convolution) against its derived error bound
(marked gpu).

The CUDA kernels' cyclic convolution of integer sequences is compared with the
exact convolution (the oracle's integer polynomial product, folded cyclically):
every output must lie within eta ||x||_2 ||y||_2 of it, where eta is the error
bound derived for the kernels' arithmetic (the value the call reports, which
must equal the oracle planner's eta_conv). Inputs: extreme digits (every value
+-2^(b-1)), constant maximal digits, and uniform digits, at lengths with every
radix and one, two and three passes. With eta ||x|| ||y|| below 1/2 the rounded
outputs equal the exact convolution."""
import math

import numpy as np
import pytest

from oracle import plan as P
from oracle import trace as T

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


def _exact_cyclic(x, y):
    w = T.poly_mul_exact(x, y)
    N = len(x)
    out = w[:N].copy()
    out[: len(w) - N] += w[N:]
    return out


# every radix, one to three passes; the longest odd parts the library takes (2^8 x 189 =
# 3^3 x 7, 2^12 x 5^3, 2^10 x 147 = 3 x 7^2), and the high product's certified lengths
# at n = 2^24 (2^16 x 35, 2^14 x 135)
LENGTHS = [4, 6, 12, 40, 56, 210, 6144, 6720, 8192, 2 ** 15 * 3, 2 ** 14 * 35,
           2 ** 8 * 189, 2 ** 12 * 125, 2 ** 10 * 147,
           2 ** 17 * 5, 2 ** 20, 2 ** 14 * 135, 2 ** 16 * 35, 2 ** 21 * 3]


@pytest.mark.parametrize("N", LENGTHS)
def test_convolution_within_derived_bound(pkg, N):
    import torch
    rng = np.random.default_rng(N)
    b = 12 if N < 2 ** 20 else 9
    h = 2 ** (b - 1)
    worst = 0.0
    for trial in range(3):
        if trial == 0:
            x = rng.choice([-h, h], size=N)
            y = rng.choice([-h, h], size=N)
        elif trial == 1:
            x = np.full(N, h)
            y = np.full(N, -h)
        else:
            x = rng.integers(-h, h + 1, size=N)
            y = rng.integers(-h, h + 1, size=N)
        want = _exact_cyclic(x, y)
        dx = torch.from_numpy(x.astype(np.float64)).cuda()
        dy = torch.from_numpy(y.astype(np.float64)).cuda()
        out, eta = pkg.convolution(dx, dy)
        assert math.isclose(eta, P.eta_conv(N), rel_tol=1e-12), (eta, P.eta_conv(N))
        got = out.cpu().numpy()
        err = np.abs(got - want.astype(np.float64)).max()
        # the difference is formed in float64: allow its own rounding (half an ulp
        # of the largest |want|)
        slack = np.spacing(np.abs(want).max().astype(np.float64))
        bound = eta * np.linalg.norm(x.astype(np.float64)) * np.linalg.norm(y.astype(np.float64))
        assert err <= bound + slack, (N, trial, err, bound)
        worst = max(worst, err / bound)
        if bound < 0.5:
            assert np.array_equal(np.rint(got).astype(np.int64), want)
    print(f"N={N}: largest error {worst:.4f} of the bound")


def test_convolution_rejects_bad_lengths(pkg):
    import torch
    x = torch.zeros(22, dtype=torch.float64, device="cuda")      # 22 = 2 x 11
    with pytest.raises(pkg.TruncMulError) as e:
        pkg.convolution(x, x)
    assert e.value.code == pkg.TM_EINVAL
