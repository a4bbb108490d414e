"""Seeded synthetic operands and workload recipes.

Holds none of the multiplication method's arithmetic: only random bits and
fixed bit patterns, laid out as little-endian uint64 limb arrays with the bits
at positions >= n cleared. Both the CUDA path's tests/bench and the oracle take
their inputs from here.

Patterns (the paper measures on uniformly random operands, Section 5; the
others are the adversarial structures of the method's error analysis):
  random          uniform random bits (numpy PCG64 seeded per call)
  ones            u = v = 2^n - 1
  balanced_worst  every b-bit chunk equal to 2^(b-1) (b given by the caller)
  alternating     u = 1010...b, v = its complement within n bits
  zero, one       u = 0 or 1, v random
  top             u = v = 2^(n-1)
"""
import math

import numpy as np


def nlimbs(n_bits: int) -> int:
    return (int(n_bits) + 63) // 64


def mask_top(limbs: np.ndarray, n_bits: int) -> np.ndarray:
    r = n_bits % 64
    if r and limbs.size:
        limbs[-1] &= np.uint64((1 << r) - 1)
    return limbs


def random_limbs(n_bits: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.integers(0, 2**64, nlimbs(n_bits), dtype=np.uint64)
    return mask_top(x, n_bits)


def _from_bits(bits: str, n_bits: int) -> np.ndarray:
    """bits[i] is bit i (little-endian string of '0'/'1' of length n_bits)."""
    arr = np.zeros(nlimbs(n_bits) * 64, dtype=np.uint8)
    arr[:n_bits] = np.frombuffer(bits.encode(), dtype=np.uint8) - ord("0")
    packed = np.packbits(arr, bitorder="little")
    return np.frombuffer(packed.tobytes(), dtype="<u8").astype(np.uint64)


def pattern_limbs(pattern: str, n_bits: int, seed: int = 0, b: int = 8):
    """(u, v) limb arrays for one of the patterns above."""
    L = nlimbs(n_bits)
    if pattern == "random":
        return random_limbs(n_bits, 2 * seed), random_limbs(n_bits, 2 * seed + 1)
    if pattern == "ones":
        x = mask_top(np.full(L, 2**64 - 1, dtype=np.uint64), n_bits)
        return x, x.copy()
    if pattern == "balanced_worst":
        bits = "".join("1" if (i % b) == b - 1 else "0" for i in range(n_bits))
        x = _from_bits(bits, n_bits)
        return x, x.copy()
    if pattern == "alternating":
        bits = "".join("1" if i % 2 == 0 else "0" for i in range(n_bits))
        x = _from_bits(bits, n_bits)
        y = mask_top(~x, n_bits)
        return x, y
    if pattern == "zero":
        return np.zeros(L, dtype=np.uint64), random_limbs(n_bits, seed)
    if pattern == "one":
        x = np.zeros(L, dtype=np.uint64); x[0] = 1
        return x, random_limbs(n_bits, seed)
    if pattern == "top":
        x = np.zeros(L, dtype=np.uint64)
        x[(n_bits - 1) // 64] = np.uint64(1 << ((n_bits - 1) % 64))
        return x, x.copy()
    raise ValueError(pattern)


def log_uniform_sizes(count: int, lo_exp: float, hi_exp: float, seed: int) -> np.ndarray:
    """n = floor(2^U(lo_exp, hi_exp)) bits, the batched / served size mix."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.floor(2.0 ** rng.uniform(lo_exp, hi_exp, count)).astype(np.int64)


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, count))


def barrett_reciprocal(k: int, seed: int):
    """A fixed k-bit modulus m (top bit set, uniform random below) and the
    Barrett-shaped reciprocal R = min(floor(2^(2k-1) / m), 2^k - 1), as uint64
    limb arrays (plain integer division; no part of the multiplication method)."""
    mbits = random_limbs(k, seed)
    mbits[(k - 1) // 64] |= np.uint64(1 << ((k - 1) % 64))
    m = int.from_bytes(mbits.astype("<u8").tobytes(), "little")
    R = min((1 << (2 * k - 1)) // m, (1 << k) - 1)
    nl = nlimbs(k)
    r = np.frombuffer(R.to_bytes(8 * nl, "little"), dtype="<u8").astype(np.uint64)
    return mbits, r


def top_bits(limbs: np.ndarray, k: int, n: int) -> np.ndarray:
    """The top n bits of the k-bit integer in `limbs`, as ceil(n/64) limbs."""
    s = k - n
    q, r = s // 64, s % 64
    out_n = nlimbs(n)
    src = np.concatenate([limbs, np.zeros(2, dtype=np.uint64)])
    lo = src[q:q + out_n] >> np.uint64(r)
    hi = (src[q + 1:q + 1 + out_n] << np.uint64(64 - r)) if r else np.zeros(out_n, np.uint64)
    return mask_top((lo | hi).astype(np.uint64), n)
