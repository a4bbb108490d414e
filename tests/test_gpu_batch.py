"""Batched products (tm_batch_*, tm_mul_batch): every product of a batch is the
oracle's (low and full products bit for bit, high products the exact round(t) of
Algorithm 3) and equals the same product computed alone with tm_mul, for mixed
kinds and uneven sizes, at the edge between the CTA-resident kernel and the
per-phase launches, and on adversarial operands; a recorded batch relaunched on
new operand values recomputes them (marked gpu)."""
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


def _make(pkg, sizes, kinds, seed):
    import torch
    items = []
    for i, (n, kind) in enumerate(zip(sizes, kinds)):
        u, v = workloads.pattern_limbs("random", int(n), seed=seed + i)
        out = torch.full((pkg.out_limbs(kind, int(n)),), -1, dtype=torch.int64, device="cuda")
        items.append((kind, int(n), out, dev(u), dev(v)))
    return items


def _check(pkg, items):
    """Each product against the oracle (low and full bit for bit, high the exact
    round(t) of Algorithm 3 for n <= 2^18, else admissible) and against the same
    product computed alone with tm_mul."""
    import torch
    for kind, n, out, u, v in items:
        pl = pkg.plan(kind, n)
        check_product(kind, host(out), host(u), host(v), n, pl["b"], pl["N"])
        ref, _ = pkg.mul(kind, u, v, n)
        assert torch.equal(out, ref), (kind, n)


def test_batch_mixed_sizes_matches_single(pkg):
    sizes = list(workloads.log_uniform_sizes(120, 6, 18, seed=4))
    sizes += [1, 64, 65, 5000, 5000, 5001, 65536]            # tiny, shared plans
    rng = np.random.default_rng(4)
    kinds = [["lo", "hi", "full"][k] for k in rng.integers(0, 3, len(sizes))]
    items = _make(pkg, sizes, kinds, seed=100)
    rep = pkg.mul_batch(items)
    assert rep["status"] == 0 and rep["margin"] <= 0.5
    _check(pkg, items)


def test_batch_relaunch_with_new_operands(pkg):
    import torch
    sizes = [3000, 3001, 40000, 100000, 777]
    kinds = ["lo", "hi", "lo", "hi", "full"]
    items = _make(pkg, sizes, kinds, seed=7)
    b = pkg.Batch(items)
    b.launch()
    assert b.status()["rc"] == 0
    _check(pkg, items)
    for i, (kind, n, out, u, v) in enumerate(items):     # new values in the same buffers
        nu, nv = workloads.pattern_limbs("random", n, seed=999 + i)
        u.copy_(dev(nu))
        v.copy_(dev(nv))
        out.fill_(-1)
    b.launch()
    st = b.status()
    assert st["rc"] == 0 and st["margin"] <= st["e_max"]
    _check(pkg, items)
    b.close()


def test_batch_config_shape_small(pkg):
    """The batched configuration's shape (log-uniform sizes in [2^12, 2^20],
    half low / half high), on 256 products."""
    sizes = workloads.log_uniform_sizes(256, 12, 20, seed=12)
    kinds = ["lo" if i % 2 == 0 else "hi" for i in range(len(sizes))]
    items = _make(pkg, sizes, kinds, seed=300)
    b = pkg.Batch(items)
    b.launch()
    assert b.status()["rc"] == 0
    _check(pkg, items)


def _edge_sizes(pkg, kind, M_max=2048):
    """The largest n whose plan has complex length M <= M_max (the last size the
    CTA-resident kernel takes) and the next n (the first size above it)."""
    lo, hi = 1, 1 << 20
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if pkg.plan(kind, mid)["N"] // 2 <= M_max:
            lo = mid
        else:
            hi = mid
    return [lo, hi]


def test_batch_edge_of_cta_resident_kernel(pkg):
    """Products at M = kSmallMaxM and just above, n = 1, ragged n and adversarial
    operands, all in one batch, against the oracle."""
    import torch
    items = []
    seed = 700
    for kind in ("lo", "hi", "full"):
        sizes = _edge_sizes(pkg, kind) + [1, 2, 63, 65, 4097]
        for n in sizes:
            b = pkg.plan(kind, n)["b"]
            for pattern in ("random", "ones", "balanced_worst", "top"):
                u, v = workloads.pattern_limbs(pattern, n, seed=seed, b=b)
                seed += 1
                out = torch.full((pkg.out_limbs(kind, n),), -1, dtype=torch.int64,
                                 device="cuda")
                items.append((kind, n, out, dev(u), dev(v)))
    for kind in ("lo", "hi", "full"):
        e = _edge_sizes(pkg, kind)
        assert pkg.plan(kind, e[0])["N"] // 2 <= 2048 < pkg.plan(kind, e[1])["N"] // 2
    rep = pkg.mul_batch(items)
    assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
    _check(pkg, items)
