"""Caller-chosen digit size and transform length (tm_mul_params), through the C ABI
(marked gpu).

With the planner's own (b, N) the call must reproduce tm_mul limb for limb. With the
parameters of the paper's Table 2 (Section 5: b and N chosen by experiment for random
operands, not certified; the worst-case bound for them is above 1/2), uniformly random
operands must give the exact products (low and full bit for bit against the oracle,
high the round(t) of Algorithm 3 for that (b, N) and admissible); their margins are
printed (about 1/4 at n = 10^6, b = 14, against the default acceptance limit of 3/8).
Operands whose digits are all maximal push coefficients towards
half-integers at those digit sizes: every such call must either report TM_EPRECISION
or still return the exact product, never a wrong product with a success status."""
import numpy as np
import pytest

import workloads
from conftest import golden
from gpu_util import dev, hi_ok, host
from oracle import bigmul
from oracle import plan as P
from oracle import trace as T

pytestmark = pytest.mark.gpu

ROWS = [tuple(map(int, r)) for r in golden("table2_params.txt")]


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1703_00640_gb300 as p
    p.build()
    p.load()
    return p


@pytest.mark.parametrize("n", [1000, 65536, 100003])
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_planner_parameters_reproduce_tm_mul(pkg, kind, n):
    u, v = workloads.pattern_limbs("random", n, seed=n % 97)
    du, dv = dev(u), dev(v)
    ref, rep = pkg.mul(kind, du, dv, n)
    pl = P.choose(kind, n)
    out, rep_p = pkg.mul_params(kind, du, dv, n, b=pl["b"], N=pl["N"])
    assert np.array_equal(host(out), host(ref))
    for f in ("b", "N", "lam_fwd", "lam_bwd", "n_digits", "margin", "e_max", "status"):
        assert rep_p[f] == rep[f], f


def _exact(kind, u, v, n, b, N, full):
    """Exact expected value of the product as an int (high: the round(t) of
    Algorithm 3 for (b, N) when the trace is affordable, else None)."""
    if kind == "full":
        return bigmul.to_int(full)
    if kind == "lo":
        return bigmul.to_int(full) & ((1 << n) - 1)
    if n <= 5_000_000:
        return T.trace("hi", bigmul.to_int(u), bigmul.to_int(v), n, b, N)["out"]
    return None


@pytest.mark.parametrize("row", ROWS[:3], ids=[str(r[0]) for r in ROWS[:3]])
def test_table2_random_operands(pkg, row):
    n, N, b, lam, L, bf = row
    for seed in range(2):
        u, v = workloads.pattern_limbs("random", n, seed=900 + seed)
        du, dv = dev(u), dev(v)
        full = bigmul.mul_full(u, v, par_depth=3)
        for kind, (bb, NN) in (("lo", (b, N)), ("hi", (b, N)), ("full", (bf, L))):
            out, rep = pkg.mul_params(kind, du, dv, n, b=bb, N=NN, check=False)
            assert (rep["b"], rep["N"]) == (bb, NN)
            assert rep["status"] in (pkg.TM_UNCERTIFIED, pkg.TM_EPRECISION)
            assert rep["e_max"] >= 0.5                     # not certified by the bound
            print(f"n={n} {kind} b={bb} N={NN}: margin {rep['margin']:.3g}")
            got = bigmul.to_int(host(out))
            want = _exact(kind, u, v, n, bb, NN, full)
            if kind == "hi":
                assert hi_ok(got, u, v, n, full=full)
            if want is not None:
                assert got == want, (kind, n)


@pytest.mark.parametrize("row", ROWS[:2], ids=[str(r[0]) for r in ROWS[:2]])
@pytest.mark.parametrize("pattern", ["balanced_worst", "ones"])
def test_table2_large_digits_never_silently_wrong(pkg, row, pattern):
    n, N, b, lam, L, bf = row
    flagged = 0
    for kind, (bb, NN) in (("lo", (b, N)), ("hi", (b, N)), ("full", (bf, L))):
        u, v = workloads.pattern_limbs(pattern, n, seed=7, b=bb)
        full = bigmul.mul_full(u, v, par_depth=3)
        out, rep = pkg.mul_params(kind, dev(u), dev(v), n, b=bb, N=NN, check=False)
        assert rep["status"] in (pkg.TM_UNCERTIFIED, pkg.TM_EPRECISION)
        if rep["status"] == pkg.TM_EPRECISION:
            flagged += 1
            continue
        got = bigmul.to_int(host(out))
        if kind == "hi":
            assert hi_ok(got, u, v, n, full=full), (kind, pattern, rep)
            want = _exact(kind, u, v, n, bb, NN, full)
            assert want is None or got == want, (kind, pattern, rep)
        else:
            assert got == _exact(kind, u, v, n, bb, NN, full), (kind, pattern, rep)
    print(f"n={n} {pattern}: {flagged} of 3 products flagged")


def test_limit(pkg):
    """The acceptance limit is the caller's: a tiny limit flags a certified plan's
    product (the limbs are unchanged), 1/2 is accepted, outside [0, 1/2] is refused."""
    n = 100003
    u, v = workloads.pattern_limbs("random", n, seed=5)
    du, dv = dev(u), dev(v)
    pl = P.choose("lo", n)
    ref, _ = pkg.mul("lo", du, dv, n)
    out, rep = pkg.mul_params("lo", du, dv, n, b=pl["b"], N=pl["N"], limit=1e-15, check=False)
    assert rep["status"] == pkg.TM_EPRECISION and np.array_equal(host(out), host(ref))
    out, rep = pkg.mul_params("lo", du, dv, n, b=pl["b"], N=pl["N"], limit=0.5)
    assert rep["status"] == 0 and np.array_equal(host(out), host(ref))
    with pytest.raises(pkg.TruncMulError) as e:
        pkg.mul_params("lo", du, dv, n, b=pl["b"], N=pl["N"], limit=0.75)
    assert e.value.code == pkg.TM_EINVAL
