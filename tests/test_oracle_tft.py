"""The truncated-FFT question at the end of Section 2.2, answered on the CPU for
Algorithm 2 (oracle/tft.py).

- Algorithm 2 needs a cyclic convolution of length N, not a smooth N: with a
  length-N cyclic product (the N-th roots of unity), the low product is exact for
  prime N and other non-smooth lengths.
- A truncated FFT of non-power-of-two length N evaluates at N points that are not
  the N-th roots of unity; Algorithm 2 with that product in place of the
  Convolution step gets every coefficient wrong.
- The ring isomorphism from R[X]/A(X) to the product ring of the TFT points has
  entries of size about 1 on diagonals far from the main one, while the one to
  R[X]/(X^N - 1) (alpha*) decays by about 2^-b per diagonal: alpha* and beta*
  have no short counterpart for the TFT points.
Powers of two, where the TFT points are the N-th roots of unity, give the same
results as the cyclic product (a check of the experiment itself)."""
import random

import numpy as np
import pytest

from oracle import plan as P
from oracle import tft
from oracle import trace

B = 10


def test_tft_points():
    for N in (5, 6, 12, 64, 100):
        k = (N - 1).bit_length()
        pts = tft.tft_points(N)
        roots = np.exp(2j * np.pi * np.arange(2 ** k) / 2 ** k)
        # a subset of the 2^k-th roots of unity containing every 2^(k-1)-th root
        assert all(np.min(np.abs(roots - p)) < 1e-12 for p in pts)
        half = np.exp(2j * np.pi * np.arange(2 ** (k - 1)) / 2 ** (k - 1))
        assert all(np.min(np.abs(pts - h)) < 1e-12 for h in half)
    pts = tft.tft_points(64)
    assert np.allclose(np.sort(np.angle(pts)), np.sort(np.angle(tft.cyclic_points(64))))


def test_product_at_points_is_the_ring_product():
    """Values, pointwise product, interpolation: the product modulo prod(X - p);
    for the N-th roots of unity that is the cyclic convolution."""
    rng = np.random.default_rng(1)
    N = 24
    x, y = rng.integers(-9, 10, N).astype(float), rng.integers(-9, 10, N).astype(float)
    cyc = np.array([sum(x[i] * y[(k - i) % N] for i in range(N)) for k in range(N)])
    assert np.allclose(tft.product_at_points(x, y, tft.cyclic_points(N)), cyc, atol=1e-9)
    # low-degree factors whose product fits below degree N: any N points give it
    x[N // 2:] = 0
    y[N // 2:] = 0
    lin = np.convolve(x, y)[:N]
    assert np.allclose(tft.product_at_points(x, y, tft.tft_points(N)), lin, atol=1e-8)


@pytest.mark.parametrize("N", [64, 96, 120, 128, 131, 200])
def test_algorithm2_with_cyclic_and_truncated_products(N):
    n = N * B
    rnd = random.Random(N)
    la, lb = P.lam_alpha(B), P.lam_beta(B)
    for _ in range(2):
        u, v = rnd.getrandbits(n), rnd.getrandbits(n)
        ex = trace.trace("lo", u, v, n, B, N)
        cyc = tft.mul_lo_with(u, v, n, B, N, la, lb, tft.cyclic_points(N))
        assert cyc["out"] == ex["out"] and np.array_equal(cyc["c"], ex["c"])
        assert cyc["margin"] < 1e-3
        trunc = tft.mul_lo_with(u, v, n, B, N, la, lb, tft.tft_points(N))
        if N & (N - 1) == 0:
            assert trunc["out"] == ex["out"]
        else:
            assert trunc["out"] != ex["out"]
            assert np.count_nonzero(trunc["c"] != ex["c"]) > N // 2


@pytest.mark.parametrize("N", [96, 120, 131, 200])
def test_ring_maps_short_only_for_the_cyclic_target(N):
    zA = tft.low_roots(N, B)
    assert np.max(np.abs(zA ** N + 2.0 ** -B * zA - 1)) < 1e-12
    lam = P.lam_alpha(B)
    cyc = tft.diagonal_profile(tft.ring_map(zA, tft.cyclic_points(N)))
    # alpha*: diagonal r of size about (2^-b)^r, nothing beyond lambda but rounding
    assert 1e-4 < cyc[1] < 2.0 ** -B * 1.1
    above = cyc[1:lam] > 1e-12          # float64 interpolation leaves ~1e-15 of noise
    assert np.all((cyc[2:lam + 1] < cyc[1:lam] * 2.0 ** -B * 1.5)[above])
    assert cyc[lam:].max() < 1e-12
    trunc = tft.diagonal_profile(tft.ring_map(zA, tft.tft_points(N)))
    assert trunc[lam:].max() > 0.5
