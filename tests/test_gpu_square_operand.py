"""Squares (u == v) and kept operand transforms (tm_operand_*), through the C ABI
(marked gpu).

Both paths run one forward map and one forward FFT per product instead of two;
their results must equal the oracle exactly as the two-operand path does: low and
full products bit for bit, high products the round-half-up round(t) of
Algorithm 3 (exact trace), coefficients c_i the exact 2^b L_i / 2^b H_i / w_i of
Propositions 3.1, 4.1 and Theorem 2.1."""
import numpy as np
import pytest

import workloads
from gpu_util import dev, hi_ok, host
from oracle import bigmul
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


def _expect(kind, u, v, n, exact_hi=True):
    """Oracle value of one product: low / full limbs, or the exact round(t)."""
    full = bigmul.mul_full(u, v, par_depth=3)
    nl = (n + 63) // 64
    if kind == "full":
        return full
    if kind == "lo":
        lo = full[:nl].copy()
        if n % 64:
            lo[-1] &= np.uint64((1 << (n % 64)) - 1)
        return lo
    if exact_hi:
        pl = P.choose("hi", n)
        return T.trace("hi", bigmul.to_int(u), bigmul.to_int(v), n, pl["b"], pl["N"])["out"]
    return ("accept", full)


def _check(kind, got, want, u, v, n):
    if kind == "hi":
        w = bigmul.to_int(host(got))
        if isinstance(want, tuple):
            assert hi_ok(w, u, v, n, full=want[1]), f"high n={n}"
        else:
            assert w == want, f"high round(t) n={n}"
    else:
        assert np.array_equal(host(got), want), f"{kind} n={n}"


SQUARE_N = [1, 2, 63, 64, 65, 129, 1000, 4097, 10000, 65535, 65536, 100003, 250001]


@pytest.mark.parametrize("n", SQUARE_N)
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_square_random(pkg, n, kind):
    u, _ = workloads.pattern_limbs("random", n, seed=n + 1)
    du = dev(u)
    out, rep = pkg.mul(kind, du, du, n)
    _check(kind, out, _expect(kind, u, u, n), u, u, n)
    assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]


@pytest.mark.parametrize("pattern", ["ones", "balanced_worst", "alternating", "top"])
@pytest.mark.parametrize("n", [64, 4097, 65536, 200000])
def test_square_adversarial(pkg, n, pattern):
    """All-ones and maximal balanced digits make the convolution's inputs as large
    as the error bound allows; u^2 keeps them in both factors."""
    b = P.choose("lo", n)["b"]
    u, _ = workloads.pattern_limbs(pattern, n, seed=5, b=b)
    du = dev(u)
    for kind in ("lo", "hi", "full"):
        out, rep = pkg.mul(kind, du, du, n)
        _check(kind, out, _expect(kind, u, u, n), u, u, n)
        assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]


@pytest.mark.parametrize("n", [100, 5000, 65536, 300001])
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_square_coefficients_exact(pkg, n, kind):
    u, _ = workloads.pattern_limbs("random", n, seed=13)
    pl = P.choose(kind, n)
    du = dev(u)
    c, rep = pkg.coeffs(kind, du, du, n)
    c = c.cpu().numpy()
    x = bigmul.to_int(u)
    ex = T.trace(kind, x, x, n, pl["b"], pl["n_digits"] if kind == "full" else pl["N"])
    want = np.zeros(c.size, dtype=np.int64)
    want[: ex["c"].size] = ex["c"][: c.size]
    assert np.array_equal(c, want)
    assert rep["margin"] <= rep["e_max"]


@pytest.mark.parametrize("n", [2**20, 2**24])
def test_square_config_sizes(pkg, n):
    u, _ = workloads.pattern_limbs("random", n, seed=24)
    du = dev(u)
    for kind in ("lo", "hi", "full"):
        out, rep = pkg.mul(kind, du, du, n)
        _check(kind, out, _expect(kind, u, u, n, exact_hi=(n <= 2**20)), u, u, n)
        assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]


@pytest.mark.parametrize("n", [1, 65, 1000, 4097, 65536, 100003, 2**20])
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_operand_matches_two_operand_path(pkg, n, kind):
    """A kept transform of v gives the oracle's product, and the same limbs as
    tm_mul, for several u; other products in between do not disturb it."""
    _, v = workloads.pattern_limbs("random", n, seed=31)
    dv = dev(v)
    op = pkg.Operand(kind, dv, n)
    try:
        for seed in range(3):
            u, _ = workloads.pattern_limbs("random", n, seed=100 + seed)
            du = dev(u)
            got, rep = op.mul(du)
            assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
            _check(kind, got, _expect(kind, u, v, n, exact_hi=(n <= 2**20)), u, v, n)
            ref, _ = pkg.mul(kind, du, dv, n)
            assert np.array_equal(host(got), host(ref))
            # an unrelated product of another size on the same stream
            a, b = workloads.pattern_limbs("random", 3000, seed=seed)
            pkg.mul("lo", dev(a), dev(b), 3000)
        # v itself: the kept transform against the square path
        got, _ = op.mul(dv)
        sq, _ = pkg.mul(kind, dv, dv, n)
        assert np.array_equal(host(got), host(sq))
    finally:
        op.close()


def test_operand_barrett_shape(pkg):
    """High products x R with R the top bits of a Barrett-shaped reciprocal: the
    served workload's fixed operand, kept once and reused."""
    n = 1 << 18
    _, R = workloads.barrett_reciprocal(n, seed=3)
    dR = dev(R)
    op = pkg.Operand("hi", dR, n)
    try:
        for seed in range(4):
            x, _ = workloads.pattern_limbs("random", n, seed=200 + seed)
            got, rep = op.mul(dev(x))
            assert rep["status"] == 0
            want = _expect("hi", x, R, n)
            assert bigmul.to_int(host(got)) == want
    finally:
        op.close()


def test_operand_survives_release(pkg):
    n = 5000
    u, v = workloads.pattern_limbs("random", n, seed=41)
    du, dv = dev(u), dev(v)
    op = pkg.Operand("lo", dv, n)
    try:
        pkg.release()                                   # frees the plan cache only
        got, _ = op.mul(du)
        assert np.array_equal(host(got), _expect("lo", u, v, n))
    finally:
        op.close()


def test_operand_alias_and_stream(pkg):
    import torch
    n = 3000
    u, v = workloads.pattern_limbs("random", n, seed=43)
    op = pkg.Operand("lo", dev(v), n)
    try:
        buf = torch.zeros(64, dtype=torch.int64, device="cuda")
        buf[:47].copy_(dev(u))
        with pytest.raises(pkg.TruncMulError) as e:      # out overlapping u
            op.mul(buf[:47], out=buf[10:57])
        assert e.value.code == pkg.TM_EALIAS
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            du = dev(u)
            got, rep = op.mul(du, stream=s, report=False)
        assert rep is None
        st = pkg.stream_status(s)
        assert st["rc"] == 0
        assert np.array_equal(host(got), _expect("lo", u, v, n))
    finally:
        op.close()


def test_square_with_host_buffers(pkg):
    n = 77777
    u, _ = workloads.pattern_limbs("random", n, seed=19)
    for kind in ("lo", "hi", "full"):
        out, rep = pkg.mul_host(kind, u, u, n)
        assert rep["status"] == 0
        d, _ = pkg.mul(kind, dev(u), dev(u), n)
        assert np.array_equal(out, host(d))


@pytest.mark.parametrize("n", [100003, 1 << 20])
def test_autotuned_layout_keeps_results(pkg, n):
    """tm_autotune only changes the FFT pass layout: products after it equal the
    oracle and the products before it, limb for limb."""
    u, v = workloads.pattern_limbs("random", n, seed=57)
    du, dv = dev(u), dev(v)
    before = {k: host(pkg.mul(k, du, dv, n)[0]) for k in ("lo", "hi", "full")}
    for k in ("lo", "hi", "full"):
        t = pkg.autotune(k, n)
        assert t["candidates"] >= 1 and 0 < t["ms_best"] <= t["ms_default"]
    for k in ("lo", "hi", "full"):
        out, rep = pkg.mul(k, du, dv, n)
        assert rep["status"] == 0
        assert np.array_equal(host(out), before[k])
        _check(k, out, _expect(k, u, v, n), u, v, n)
