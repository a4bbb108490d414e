"""tm_mul_static: full, low and high products for callers that cannot allocate
device memory (code running where the allocator belongs to someone else, or
that must not block on an allocation). Every device buffer of the call lives in
one fixed device array inside the library, so the checks are: the results equal
tm_mul's (these are exact integers, so equal means bit for bit) and the oracle's
(low and full products bit for bit, high products the exact round(t) of
Algorithm 3) on two calls in a row that reuse that array, oversize requests are
refused, the device's free memory does not change across calls, and a call made
without a report enqueues no host-to-device copy, so it can be recorded into a
CUDA graph after a first call on the device. This file is collected last on
purpose."""
import numpy as np
import pytest

import workloads
from gpu_util import check_product, dev, host

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


@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
@pytest.mark.parametrize("n", [1, 100, 4097, 40000, 65536])
def test_static_matches_tm_mul_on_two_calls(pkg, kind, n):
    import torch
    for call in range(2):
        u, v = workloads.pattern_limbs("random", n, seed=5000 + 11 * call + n % 89)
        du, dv = dev(u), dev(v)
        ref, _ = pkg.mul(kind, du, dv, n)
        out = torch.full((pkg.out_limbs(kind, n),), -1, dtype=torch.int64, device="cuda")
        rc, rep = pkg.mul_static(kind, du, dv, n, out)
        assert rc == pkg.TM_OK, pkg.strerror(rc)
        assert torch.equal(out, ref), (kind, n, call)
        assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
        plan = pkg.plan(kind, n)
        assert (rep["b"], rep["N"]) == (plan["b"], plan["N"])
        check_product(kind, host(out), u, v, n, rep["b"], rep["N"])


@pytest.mark.parametrize("pattern", ["ones", "balanced_worst", "top", "zero"])
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_static_adversarial_against_oracle(pkg, kind, pattern):
    import torch
    n = 65536
    b = pkg.plan(kind, n)["b"]
    u, v = workloads.pattern_limbs(pattern, n, seed=9, b=b)
    out = torch.full((pkg.out_limbs(kind, n),), -1, dtype=torch.int64, device="cuda")
    rc, rep = pkg.mul_static(kind, dev(u), dev(v), n, out)
    assert rc == pkg.TM_OK, pkg.strerror(rc)
    assert rep["margin"] <= rep["e_max"]
    check_product(kind, host(out), u, v, n, rep["b"], rep["N"])


def test_static_high_product_in_a_graph(pkg):
    """After a first call on the device, a high product without a report is
    recorded into a CUDA graph and replayed on new operand values."""
    import torch
    n = 50000
    u0, v0 = workloads.pattern_limbs("random", n, seed=41)
    du, dv = dev(u0), dev(v0)
    out = torch.zeros(pkg.out_limbs("hi", n), dtype=torch.int64, device="cuda")
    rc, rep = pkg.mul_static("hi", du, dv, n, out)           # set-up call, outside capture
    assert rc == pkg.TM_OK
    b, N = rep["b"], rep["N"]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc, _ = pkg.mul_static("hi", du, dv, n, out, stream=s, report=False)
    assert rc == pkg.TM_OK, pkg.strerror(rc)
    for seed in (42, 43):
        u, v = workloads.pattern_limbs("random", n, seed=seed)
        du.copy_(dev(u))
        dv.copy_(dev(v))
        out.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        check_product("hi", host(out), u, v, n, b, N)


def test_static_rejects_oversize(pkg):
    import torch
    n = pkg.STATIC_MAX_BITS + 1
    u, v = workloads.pattern_limbs("random", n, seed=1)
    out = torch.zeros(pkg.out_limbs("lo", n), dtype=torch.int64, device="cuda")
    rc, _ = pkg.mul_static("lo", dev(u), dev(v), n, out)
    assert rc == pkg.TM_ERANGE
    assert int(out.abs().sum()) == 0


def test_static_leaves_device_memory_unchanged(pkg):
    import torch
    n = 65536
    u, v = workloads.pattern_limbs("random", n, seed=2)
    du, dv = dev(u), dev(v)
    outs = {k: torch.empty(pkg.out_limbs(k, n), dtype=torch.int64, device="cuda")
            for k in ("lo", "hi", "full")}
    for k in outs:                      # first calls load the kernels
        assert pkg.mul_static(k, du, dv, n, outs[k])[0] == pkg.TM_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        for k in outs:
            rc, _ = pkg.mul_static(k, du, dv, n, outs[k], report=False)
            assert rc == pkg.TM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref, _ = pkg.mul("hi", du, dv, n)
    assert torch.equal(outs["hi"], ref)
