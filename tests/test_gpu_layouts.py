"""FFT pass layouts forced with tm_set_layout, through the C ABI (marked gpu).

A layout only changes how the transforms are split into passes and launched (points
per CTA, where the odd prime factors go, the pass count); the products must stay exact for every layout: low and full
products bit for bit against the oracle, high products the round(t) of Algorithm 3
for the plan's (b, N), and every rounding margin below the plan's bound."""
import numpy as np
import pytest

import workloads
from gpu_util import dev, host
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


def _expect(kind, u, v, n):
    if kind == "hi":
        pl = P.choose("hi", n)
        return T.trace("hi", bigmul.to_int(u), bigmul.to_int(v), n, pl["b"], pl["N"])["out"]
    full = bigmul.mul_full(u, v, par_depth=3)
    if kind == "full":
        return bigmul.to_int(full)
    return bigmul.to_int(full) & ((1 << n) - 1)


LAYOUTS = [dict(points=512), dict(points=2048), dict(passes=3), dict(passes=2),
           dict(split=1, passes=3), dict(split=2, points=2048), dict(split=1, points=512)]


@pytest.mark.parametrize("n", [65536, 100003, 1 << 20, (1 << 22) + 12345])
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_forced_layouts_exact(pkg, kind, n):
    u, v = workloads.pattern_limbs("random", n, seed=n % 977)
    du, dv = dev(u), dev(v)
    want = _expect(kind, u, v, n)
    try:
        for lay in LAYOUTS:
            try:
                pkg.set_layout(kind, n, **lay)
            except pkg.TruncMulError as e:       # no pass split of that many passes
                assert e.code == pkg.TM_ERANGE
                continue
            out, rep = pkg.mul(kind, du, dv, n)
            assert rep["status"] == 0 and rep["margin"] <= rep["e_max"], lay
            assert bigmul.to_int(host(out)) == want, (kind, n, lay)
    finally:
        pkg.set_layout(kind, n)


@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_reapplied_tuned_layout_config_2_24(pkg, kind):
    """n = 2^24: the layout tm_autotune picks, reapplied with tm_set_layout after the
    default was restored, gives the same limbs as the default layout."""
    n = 1 << 24
    u, v = workloads.pattern_limbs("random", n, seed=5)
    du, dv = dev(u), dev(v)
    ref, _ = pkg.mul(kind, du, dv, n)
    try:
        t = pkg.autotune(kind, n)
        pkg.set_layout(kind, n)
        pkg.set_layout(kind, n, points=t["points"], split=t["split"], passes=t["passes"])
        out, rep = pkg.mul(kind, du, dv, n)
        assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
        assert np.array_equal(host(out), host(ref))
        pkg.set_layout(kind, n, passes=3)
        out, rep = pkg.mul(kind, du, dv, n)
        assert np.array_equal(host(out), host(ref))
    finally:
        pkg.set_layout(kind, n)
    if kind == "lo":
        full = bigmul.mul_full(u, v, par_depth=3)
        assert np.array_equal(host(out), full[: n // 64])


def test_batch_with_forced_layout(pkg):
    """A batch built after tm_set_layout uses that layout; results equal the single
    products."""
    import torch
    n = 1 << 20
    pkg.set_layout("lo", n, passes=3, points=512)
    try:
        items = []
        for s in range(3):
            u, v = workloads.pattern_limbs("random", n, seed=70 + s)
            du, dv = dev(u), dev(v)
            items.append(("lo", n, torch.empty(n // 64, dtype=torch.int64, device="cuda"),
                          du, dv))
        b = pkg.Batch(items)
        try:
            b.launch()
            torch.cuda.synchronize()
            for k, nn, o, u, v in items:
                ref, _ = pkg.mul(k, u, v, nn)
                assert torch.equal(o, ref)
        finally:
            b.close()
    finally:
        pkg.set_layout("lo", n)


def _bound(kind, n, b, N):
    E = {"lo": P.bound_lo, "hi": P.bound_hi, "full": P.bound_full}[kind](n, b, N)
    return E[0] if isinstance(E, tuple) else (E["E"] if isinstance(E, dict) else E)


@pytest.mark.parametrize("n", [100003, 1 << 20, 1 << 22])
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_autotuned_plan_stays_exact(pkg, kind, n):
    """tm_autotune_plan picks a plan the oracle planner's own bound certifies; products
    with it are exact (high: the round(t) of Algorithm 3 for the chosen (b, N)), and
    tm_plan_set(0, 0) restores the planner's choice."""
    u, v = workloads.pattern_limbs("random", n, seed=n % 613)
    du, dv = dev(u), dev(v)
    try:
        t = pkg.autotune_plan(kind, n)
        assert 1 <= t["candidates"] <= 8 and 0 < t["ms_best"] <= t["ms_default"]
        q = pkg.plan(kind, n)
        assert (q["b"], q["N"]) == (t["b"], t["N"])
        assert _bound(kind, n, t["b"], t["N"]) <= P.E_TARGET
        out, rep = pkg.mul(kind, du, dv, n)
        assert (rep["b"], rep["N"]) == (t["b"], t["N"])
        assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
        got = bigmul.to_int(host(out))
        if kind == "hi":
            want = T.trace("hi", bigmul.to_int(u), bigmul.to_int(v), n, t["b"], t["N"])["out"]
        else:
            want = _expect(kind, u, v, n)
        assert got == want
    finally:
        pkg.plan_set(kind, n)
    base = P.choose(kind, n)
    q = pkg.plan(kind, n)
    assert (q["b"], q["N"]) == (base["b"], base["N"])


def test_autotune_plan_keeps_the_streams_status(pkg):
    """tm_autotune_plan runs trial products on the caller's stream: a status pending
    there before (here a flagged product) is still reported after, and the trials'
    own margins are not."""
    import torch
    n = 100003
    s = torch.cuda.Stream()
    u, v = workloads.pattern_limbs("random", n, seed=2)
    du, dv = dev(u), dev(v)
    pl = P.choose("lo", n)
    try:
        pkg.mul_params("lo", du, dv, n, b=pl["b"], N=pl["N"], limit=1e-15, stream=s,
                       report=False, check=False)
        pkg.autotune_plan("hi", n, stream=s)
        st = pkg.stream_status(s)
        assert st["rc"] == pkg.TM_EPRECISION
        pkg.autotune_plan("full", n, stream=s)          # nothing pending now
        assert pkg.stream_status(s)["rc"] == 0
        assert pkg.stream_status(s)["margin"] == 0.0
    finally:
        pkg.plan_set("hi", n)
        pkg.plan_set("full", n)
