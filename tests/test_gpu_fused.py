"""Single-launch products and the persistent batch (tm_set_fused; marked gpu).

Both run the per-phase kernels' block bodies inside one cooperative launch with
grid barriers between the phases, so their results must equal the per-phase
launches' limb for limb, and the oracle's: low and full products bit for bit, high
products the exact round(t) of Algorithm 3 (n <= 2^18) or admissible."""
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
    yield p
    p.set_fused(p.FUSED_AUTO)


SIZES = [1, 17, 100, 1000, 4097, 65536, 100003, 1 << 20, 3 << 20]


@pytest.mark.parametrize("n", SIZES)
def test_single_launch_equals_per_phase_and_oracle(pkg, n):
    for pattern in ("random", "ones", "balanced_worst"):
        b = pkg.plan("lo", n)["b"]
        u, v = workloads.pattern_limbs(pattern, n, seed=n % 101, b=b)
        du, dv = dev(u), dev(v)
        for kind in ("lo", "hi", "full"):
            pkg.set_fused(pkg.FUSED_NEVER)
            ref, _ = pkg.mul(kind, du, dv, n)
            sq_ref, _ = pkg.mul(kind, du, du, n)
            pkg.set_fused(pkg.FUSED_ALWAYS)
            got, rep = pkg.mul(kind, du, dv, n)
            sq, _ = pkg.mul(kind, du, du, n)
            pkg.set_fused(pkg.FUSED_AUTO)
            assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
            assert np.array_equal(host(got), host(ref)), (kind, n, pattern)
            assert np.array_equal(host(sq), host(sq_ref)), (kind, n, pattern, "square")
            check_product(kind, host(got), u, v, n, rep["b"], rep["N"])


def test_persistent_batch_equals_per_phase_graph(pkg):
    """The same batch as one persistent launch (mode 2) and as the per-phase
    graph: identical limbs, and a sample checked against the oracle."""
    import torch
    sizes = list(workloads.log_uniform_sizes(300, 4, 21, seed=77)) + [1, 2, 64, 65, 3000]
    rng = np.random.default_rng(77)
    kinds = [["lo", "hi", "full"][k] for k in rng.integers(0, 3, len(sizes))]
    items, hosts = [], []
    for i, (n, kind) in enumerate(zip(sizes, kinds)):
        n = int(n)
        u, v = workloads.pattern_limbs("random", n, seed=900 + i)
        out = torch.full((pkg.out_limbs(kind, n),), -1, dtype=torch.int64, device="cuda")
        items.append((kind, n, out, dev(u), dev(v)))
        hosts.append((u, v))
    results = {}
    for mode in (pkg.FUSED_NEVER, pkg.FUSED_ALWAYS):
        pkg.set_fused(mode)
        for it in items:
            it[2].fill_(-1)
        b = pkg.Batch(items)
        b.launch()
        st = b.status()
        assert st["rc"] == 0 and st["margin"] <= st["e_max"], (mode, st)
        b.launch()                              # a second launch recomputes the same
        assert b.status()["rc"] == 0
        b.close()
        results[mode] = [host(it[2]).copy() for it in items]
    pkg.set_fused(pkg.FUSED_AUTO)
    for a, c in zip(results[pkg.FUSED_NEVER], results[pkg.FUSED_ALWAYS]):
        assert np.array_equal(a, c)
    for i in range(0, len(items), 7):
        kind, n, out, _, _ = items[i]
        pl = pkg.plan(kind, n)
        check_product(kind, results[pkg.FUSED_ALWAYS][i], hosts[i][0], hosts[i][1], n,
                      pl["b"], pl["N"])


def test_mode_argument_checked(pkg):
    with pytest.raises(pkg.TruncMulError) as e:
        pkg.set_fused(3)
    assert e.value.code == pkg.TM_EINVAL
