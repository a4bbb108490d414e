"""Data-dependent digit size (tm_mul_adaptive), through the C ABI (marked gpu).

The plan that runs must be the oracle planner's adaptive choice (the worst-case b,
or b + 1 where the bound on the operands' measured digit norms certifies it; the
library may keep b where its own policy skips the measurement), and
the product must be exact as for tm_mul: low and full bit for bit, high the
round(t) of Algorithm 3 for the (b, N) that ran."""
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


# The library's policy (not the method's): it measures the digit norms only when
# b + 1's worst-case bound is within this factor of the target, since uniformly
# random digits lower the norm product by about 3.
MEASURE_SPAN = 3.5


def _library_measures(kind, n, b, N):
    count = P.full_digits(n, b) if kind == "full" else N
    w = 2.0 ** (b - 1) * np.sqrt(count)
    if kind == "lo":
        Ew = P.bound_lo_measured(b, N, w, w)
    elif kind == "hi":
        Ew = P.bound_hi_measured(b, N, w, w, 2.0 ** b, 2.0 ** b)
    else:
        Ew = P.bound_full_measured(N, w, w)
    return Ew <= MEASURE_SPAN * P.E_TARGET


def _check(pkg, kind, n, u, v, exact_hi=True):
    ui, vi = bigmul.to_int(u), bigmul.to_int(v)
    want_plan = P.adaptive_choice(kind, n, ui, vi)
    base = P.choose(kind, n)
    out, rep = pkg.mul_adaptive(kind, dev(u), dev(v), n)
    if want_plan["b"] > base["b"] and rep["b"] == base["b"]:
        # b + 1 is certified for these operands but the library did not measure
        assert not _library_measures(kind, n, want_plan["b"], want_plan["N"]), (kind, n)
        want_plan = base
    assert (rep["b"], rep["N"]) == (want_plan["b"], want_plan["N"]), (kind, n)
    assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
    assert rep["e_max"] == pytest.approx(want_plan["e_max"], rel=1e-9)
    full = bigmul.mul_full(u, v, par_depth=3)
    nl = (n + 63) // 64
    if kind == "full":
        assert np.array_equal(host(out), full)
    elif kind == "lo":
        lo = full[:nl].copy()
        if n % 64:
            lo[-1] &= np.uint64((1 << (n % 64)) - 1)
        assert np.array_equal(host(out), lo)
    else:
        w = bigmul.to_int(host(out))
        assert hi_ok(w, u, v, n, full=full)
        if exact_hi:
            ex = T.trace("hi", ui, vi, n, rep["b"], rep["N"])
            assert w == ex["out"]
    return rep


@pytest.mark.parametrize("n", [100, 4097, 65536, 123457, 1 << 20])
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_random_operands(pkg, kind, n):
    u, v = workloads.pattern_limbs("random", n, seed=n % 1000 + 1)
    _check(pkg, kind, n, u, v)


@pytest.mark.parametrize("n", [4097, 65536, 1 << 20])
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_worst_case_operands_keep_the_planner_b(pkg, kind, n):
    """Every (b+1)-bit chunk of the split is 100...0, so the balanced digits for
    b + 1 are all near 2^b: the measured bound is the worst case and b stays."""
    base = P.choose(kind, n)
    b1 = base["b"] + 1
    s0 = 0
    if kind == "hi":
        s0 = (P.measured_length(kind, n, b1) + 1) * b1 - n
    x = 0
    for i in range((n + s0) // b1):
        pos = i * b1 + b1 - 1 - s0
        if 0 <= pos < n:
            x |= 1 << pos
    u = bigmul.from_int(x, (n + 63) // 64)
    rep = _check(pkg, kind, n, u, u.copy())
    assert rep["b"] == base["b"]


def test_config_2_24(pkg):
    """n = 2^24, random operands: the full product takes b + 1 (a shorter
    transform); the low and high products keep their worst-case b = 8 (b = 9 is
    not certified by these operands' digit norms)."""
    n = 1 << 24
    u, v = workloads.pattern_limbs("random", n, seed=241)
    reps = {k: _check(pkg, k, n, u, v, exact_hi=False) for k in ("lo", "hi", "full")}
    assert reps["lo"]["b"] == P.choose("lo", n)["b"] == 8
    assert reps["hi"]["b"] == P.choose("hi", n)["b"] == 8
    assert reps["full"]["b"] == P.choose("full", n)["b"] + 1
