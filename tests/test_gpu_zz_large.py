"""The largest size in the GPU suite, n = 2^30 bits (2^24 limbs per operand, 3-pass
transforms of about 2^28 points), marked gpu. The oracle's full product would take too
long here, so the checks are properties that hold at any size: the full product's
residues modulo three primes equal the products of the operands' residues, the low
product is the full product's low n bits, and the high product is one of the two
admissible values read off the full product."""
import numpy as np
import pytest

import workloads
from gpu_util import dev, host

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


def residue(limbs: np.ndarray, p: int) -> int:
    """sum limbs[i] 2^(64 i) mod p (p < 2^31): blocks of 4096 limbs reduced with numpy,
    then combined by Horner's rule over the blocks."""
    x = limbs.astype(np.uint64)
    lo = (x & np.uint64(0xFFFFFFFF)) % np.uint64(p)
    hi = (x >> np.uint64(32)) % np.uint64(p)
    r = (hi * np.uint64(pow(2, 32, p)) + lo) % np.uint64(p)          # each limb mod p
    B = 4096
    w = np.ones(B, dtype=np.uint64)
    base = pow(2, 64, p)
    for j in range(1, B):
        w[j] = (int(w[j - 1]) * base) % p
    acc = 0
    step = pow(base, B, p)
    nblocks = (len(r) + B - 1) // B
    for k in range(nblocks - 1, -1, -1):
        seg = r[k * B:(k + 1) * B]
        s = int(((seg * w[:len(seg)]) % np.uint64(p)).sum(dtype=np.uint64) % np.uint64(p))
        acc = (acc * step + s) % p
    return acc


def test_residue_helper_small():
    rng = np.random.default_rng(1)
    x = rng.integers(0, 2**63, 10000, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    xi = int.from_bytes(x.astype("<u8").tobytes(), "little")
    for p in (1000000007, 998244353, 2147483647):
        assert residue(x, p) == xi % p


def test_size_2_30(pkg):
    n = 1 << 30
    u, v = workloads.pattern_limbs("random", n, seed=2030)
    du, dv = dev(u), dev(v)
    full, rf = pkg.mul_full(du, dv, n)
    lo, rl = pkg.mul_lo(du, dv, n)
    hi, rh = pkg.mul_hi(du, dv, n)
    for rep in (rf, rl, rh):
        assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
    F, L, H = host(full), host(lo), host(hi)
    del full, lo, hi, du, dv
    for p in (1000000007, 998244353, 2147483647):
        assert (residue(u, p) * residue(v, p) - residue(F, p)) % p == 0
    nl = n // 64
    assert np.array_equal(L, F[:nl])
    q = np.concatenate([F[nl:], np.zeros(len(H) - len(F[nl:]), dtype=np.uint64)])
    if not np.array_equal(H, q):                       # the admissible neighbour q + 1
        assert np.any(F[:nl])
        i = 0
        while q[i] == np.uint64(0xFFFFFFFFFFFFFFFF):
            q[i] = 0
            i += 1
        q[i] += np.uint64(1)
        assert np.array_equal(H, q)
    pkg.release()
