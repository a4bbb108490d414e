"""Single products with complex length M <= 640 run whole in
the CTA-resident kernel (marked gpu): against the per-phase launches (tm_set_fused
mode 1) bit for bit, and against the oracle (low and full exact, high the exact
round(t) of Algorithm 3), on random, all-ones and balanced-worst operands, at
ragged sizes up to the largest length the kernel takes, with reports and margins."""
import numpy as np
import pytest

import workloads
from gpu_util import check_product, dev, host
from oracle import plan as P

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


SMALL_MAX_M = 640      # the library's threshold for one product in one CTA


def _largest_small_n(kind):
    """The largest n whose planner length keeps M <= SMALL_MAX_M (searched downward)."""
    n = 20000
    while P.choose(kind, n)["N"] // 2 > SMALL_MAX_M:
        n -= 37
    return n


@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_small_single_equals_per_phase_and_oracle(pkg, kind):
    sizes = [1, 2, 63, 64, 65, 100, 777, 4096, 9999, _largest_small_n(kind)]
    for n in sizes:
        assert P.choose(kind, n)["N"] // 2 <= SMALL_MAX_M, (kind, n)
        for pattern in ("random", "ones", "balanced_worst"):
            u, v = workloads.pattern_limbs(pattern, n, seed=n, b=P.choose(kind, n)["b"])
            du, dv = dev(u), dev(v)
            pkg.set_fused(pkg.FUSED_NEVER)
            ref, rep_ref = pkg.mul(kind, du, dv, n)
            pkg.set_fused(pkg.FUSED_AUTO)
            got, rep = pkg.mul(kind, du, dv, n)
            assert rep["status"] == 0 and rep["margin"] <= rep["e_max"], (kind, n, rep)
            assert (rep["b"], rep["N"]) == (rep_ref["b"], rep_ref["N"])
            assert np.array_equal(host(got), host(ref)), (kind, n, pattern)
            check_product(kind, host(got), u, v, n, rep["b"], rep["N"])


def test_small_single_square_and_status_cleared(pkg):
    """u == v through the one-CTA path, and the status word left clear for the next
    reported call."""
    n = 5000
    u, _ = workloads.pattern_limbs("random", n, seed=3)
    du = dev(u)
    for kind in ("lo", "hi", "full"):
        got, rep = pkg.mul(kind, du, du, n)
        assert rep["status"] == 0
        check_product(kind, host(got), u, u.copy(), n, rep["b"], rep["N"])
    z = dev(np.zeros_like(u))
    _, rep = pkg.mul("lo", z, z, n)
    assert rep["status"] == 0 and rep["margin"] == 0.0
