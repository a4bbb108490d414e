"""Serving layer (tm_server_*): results of requests served in a mixed stream
with continuous batching are the oracle's (low and full products bit for bit,
high products the exact round(t) of Algorithm 3) and equal the same products
computed alone with tm_mul, whatever the admission order, budget or arrival
pattern (marked gpu)."""
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


def _requests(pkg, count, lo_exp, hi_exp, seed, shared_v=True):
    import torch
    sizes = workloads.log_uniform_sizes(count, lo_exp, hi_exp, seed=seed)
    rng = np.random.default_rng(seed)
    vmax = int(sizes.max())
    # one shared operand, as a fixed reciprocal would be: requests use its low limbs
    _, vfix = workloads.pattern_limbs("random", vmax, seed=seed + 1)
    reqs = []
    for i, n in enumerate(sizes):
        n = int(n)
        kind = ["lo", "hi", "full"][int(rng.integers(0, 3))]
        u, v = workloads.pattern_limbs("random", n, seed=seed * 1000 + i)
        if shared_v and i % 5 < 2:
            v = workloads.mask_top(vfix[: (n + 63) // 64].copy(), n)
        out = torch.full((pkg.out_limbs(kind, n),), -1, dtype=torch.int64, device="cuda")
        reqs.append((kind, n, out, dev(u), dev(v)))
    return reqs


def _serve_all(srv, reqs, stagger=0):
    tickets, done = {}, {}
    i = 0
    while len(done) < len(reqs):
        step = len(reqs) if not stagger else stagger
        for _ in range(step):
            if i < len(reqs):
                kind, n, out, u, v = reqs[i]
                tickets[srv.submit(kind, out, u, v, n)] = i
                i += 1
        for t, st in srv.progress():
            done[tickets[t]] = st
    return done


def _check(pkg, reqs, done):
    """Each served result against the oracle (low and full bit for bit, high the
    exact round(t) of Algorithm 3 for n <= 2^18, else admissible) and against the
    same product computed alone with tm_mul."""
    import torch
    assert all(st == 0 for st in done.values())
    for kind, n, out, u, v in reqs:
        pl = pkg.plan(kind, n)
        check_product(kind, host(out), host(u), host(v), n, pl["b"], pl["N"])
        ref, _ = pkg.mul(kind, u, v, n)
        assert torch.equal(out, ref), (kind, n)


def test_server_mixed_stream(pkg):
    reqs = _requests(pkg, 300, 10, 20, seed=21)
    srv = pkg.Server(budget_bytes=1 << 34, slots=4)
    done = _serve_all(srv, reqs)
    srv.close()
    _check(pkg, reqs, done)


def test_server_tight_budget_and_staggered_arrivals(pkg):
    reqs = _requests(pkg, 120, 12, 22, seed=33)
    srv = pkg.Server(budget_bytes=8 << 20, slots=3)      # large requests wait for memory
    done = _serve_all(srv, reqs, stagger=3)
    assert srv.pending() == 0
    srv.close()
    _check(pkg, reqs, done)
