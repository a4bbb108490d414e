"""Parity of the CUDA path with the oracle, through the C ABI (marked gpu).

Low and full products must match the oracle bit for bit; high products must be
the round-half-up value round(t) that Algorithm 3 returns, as the exact trace
gives (and therefore lie in the admissible set of Section 1); the rounded
coefficients c_i (tm_coeffs) must equal the exact 2^b L_i, 2^b H_i and w_i of
Propositions 3.1, 4.1 and Theorem 2.1; every call's margin must stay below its
a-priori bound."""
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


def _check_all(pkg, n, u, v, exact_hi=True):
    du, dv = dev(u), dev(v)
    full_ref = bigmul.mul_full(u, v, par_depth=3)
    nl = (n + 63) // 64
    lo, rep = pkg.mul_lo(du, dv, n)
    lo_ref = full_ref[:nl].copy()
    if n % 64:
        lo_ref[-1] &= np.uint64((1 << (n % 64)) - 1)
    assert np.array_equal(host(lo), lo_ref), f"low n={n}"
    assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
    hi, rep = pkg.mul_hi(du, dv, n)
    w = bigmul.to_int(host(hi))
    assert hi_ok(w, u, v, n, full=full_ref), f"high n={n}"
    if exact_hi:
        pl = P.choose("hi", n)
        ex = T.trace("hi", bigmul.to_int(u), bigmul.to_int(v), n, pl["b"], pl["N"])
        assert w == ex["out"], f"high round(t) n={n}"
    assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
    full, rep = pkg.mul_full(du, dv, n)
    assert np.array_equal(host(full), full_ref), f"full n={n}"
    assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]


# sizes: tiny, ragged (n % 64 != 0), several radix stages, 1 / 2 pass boundaries
SMALL_N = [1, 2, 3, 17, 63, 64, 65, 100, 127, 129, 255, 257, 500, 999, 1000, 1023, 1025,
           2047, 3001, 4096, 4097, 8191, 10000, 12345, 20000, 40000, 65535, 65536, 65537,
           100003, 131072, 250001]


@pytest.mark.parametrize("n", SMALL_N)
def test_random(pkg, n):
    u, v = workloads.pattern_limbs("random", n, seed=n)
    _check_all(pkg, n, u, v)


SWEEP_N = sorted({int(x) for x in workloads.log_uniform_sizes(160, 0, 21, seed=1703)} | {1})


@pytest.mark.parametrize("chunk", range(8))
def test_random_size_sweep(pkg, chunk):
    """Seeded sizes, log-uniform in [1, 2^21] (132 distinct: ragged, every pass layout class):
    low and full bit for bit, high admissible and (n <= 2^18) the exact round(t)."""
    for n in SWEEP_N[chunk::8]:
        u, v = workloads.pattern_limbs("random", n, seed=50000 + n)
        _check_all(pkg, n, u, v, exact_hi=n <= 1 << 18)


@pytest.mark.parametrize("pattern", ["ones", "balanced_worst", "alternating", "zero", "one", "top"])
@pytest.mark.parametrize("n", [64, 1000, 4097, 65536, 200000])
def test_adversarial(pkg, n, pattern):
    b = P.choose("lo", n)["b"]
    u, v = workloads.pattern_limbs(pattern, n, seed=7, b=b)
    _check_all(pkg, n, u, v)


@pytest.mark.parametrize("n", [100, 5000, 65536, 300001])
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_coefficients_exact(pkg, n, kind):
    """tm_coeffs equals the exact trace coefficient by coefficient."""
    u, v = workloads.pattern_limbs("random", n, seed=3)
    pl = P.choose(kind, n)
    c, rep = pkg.coeffs(kind, dev(u), dev(v), n)
    c = c.cpu().numpy()
    ex = T.trace(kind, bigmul.to_int(u), bigmul.to_int(v), n, pl["b"],
                 pl["n_digits"] if kind == "full" else pl["N"])
    want = np.zeros(c.size, dtype=np.int64)
    want[: ex["c"].size] = ex["c"][: c.size]
    assert np.array_equal(c, want)
    assert rep["margin"] <= rep["e_max"]
    if kind != "full":
        assert c[0] % (1 << pl["b"]) == 0


def test_square_and_alias_rules(pkg):
    import torch
    n = 3000
    u, _ = workloads.pattern_limbs("random", n, seed=11)
    du = dev(u)
    lo, _ = pkg.mul_lo(du, du, n)                      # u == v is allowed
    assert np.array_equal(host(lo), bigmul.mul_lo(u, u, n))
    buf = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(pkg.TruncMulError) as e:       # out overlapping u
        pkg.mul_lo(buf[:47], buf[:47], n, out=buf[10:57])
    assert e.value.code == pkg.TM_EALIAS


def test_async_then_status(pkg):
    import torch
    n = 20000
    s = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(s):
        for seed in range(4):
            u, v = workloads.pattern_limbs("random", n, seed=seed)
            du, dv = dev(u), dev(v)
            out, rep = pkg.mul("lo", du, dv, n, stream=s, report=False)
            assert rep is None
            outs.append((out, u, v))
    st = pkg.stream_status(s)
    assert st["rc"] == 0 and 0 < st["margin"] < 0.5
    for out, u, v in outs:
        assert np.array_equal(host(out), bigmul.mul_lo(u, v, n))


def test_host_buffers(pkg):
    n = 77777
    u, v = workloads.pattern_limbs("random", n, seed=5)
    for kind in ("lo", "hi", "full"):
        out, rep = pkg.mul_host(kind, u, v, n)
        d, _ = pkg.mul(kind, dev(u), dev(v), n)
        assert np.array_equal(out, host(d))
        assert rep["status"] == 0


def test_deterministic(pkg):
    n = 123457
    u, v = workloads.pattern_limbs("random", n, seed=9)
    a, _ = pkg.mul_hi(dev(u), dev(v), n)
    b, _ = pkg.mul_hi(dev(u), dev(v), n)
    assert np.array_equal(host(a), host(b))


@pytest.mark.parametrize("n", [2**20, 2**24])
@pytest.mark.parametrize("pattern", ["random", "ones", "balanced_worst"])
def test_config_sizes(pkg, n, pattern):
    """The single-product configurations at n = 2^20 and 2^24 (uniform random and
    the adversarial all-ones / maximal-digit operands)."""
    b = P.choose("lo", n)["b"]
    u, v = workloads.pattern_limbs(pattern, n, seed=20, b=b)
    _check_all(pkg, n, u, v, exact_hi=(n <= 2**20))


def test_config_2_28(pkg):
    """n = 2^28 (32 MiB operands): low / high / full against the oracle product."""
    n = 2**28
    u, v = workloads.pattern_limbs("random", n, seed=28)
    _check_all(pkg, n, u, v, exact_hi=False)


def test_host_buffers_on_a_stream_repeated(pkg):
    """tm_mul_host on a created stream records its sequence once and then only points
    the copies at new buffers: repeated calls with other (page-locked and pageable)
    buffers, other kinds and sizes in between, all give the device path's limbs."""
    import torch
    s = torch.cuda.Stream()
    n = 40000
    for kind in ("lo", "hi", "full"):
        for rep in range(3):
            u, v = workloads.pattern_limbs("random", n, seed=300 + rep)
            if rep == 1:      # page-locked host tensors
                hu = torch.from_numpy(u.view(np.int64)).pin_memory()
                hv = torch.from_numpy(v.view(np.int64)).pin_memory()
                out = torch.empty(pkg.out_limbs(kind, n), dtype=torch.int64).pin_memory()
                got, rep_d = pkg.mul_host(kind, hu, hv, n, out=out, stream=s)
                got = got.numpy().view(np.uint64)
            else:
                got, rep_d = pkg.mul_host(kind, u, v, n, stream=s)
            assert rep_d["status"] == 0
            d, _ = pkg.mul(kind, dev(u), dev(v), n)
            assert np.array_equal(got, host(d)), (kind, rep)
            # another size on the same stream between the calls
            a, b = workloads.pattern_limbs("random", 999, seed=rep)
            pkg.mul_host("lo", a, b, 999, stream=s)
    # squares through the same stream
    u, _ = workloads.pattern_limbs("random", n, seed=310)
    hu = torch.from_numpy(u.view(np.int64)).pin_memory()
    for _ in range(2):
        got, _ = pkg.mul_host("lo", hu, hu, n, stream=s)
        d, _ = pkg.mul("lo", dev(u), dev(u), n)
        assert np.array_equal(np.asarray(got).view(np.uint64), host(d))


@pytest.mark.parametrize("n", [1, 64, 65, 4097, 100003, 1 << 20])
def test_host_buffers_mapped(pkg, n):
    """Page-locked operands and output: the kernels read and write the host buffers
    in place (no staging copies). Interior pointers of one page-locked block, squares,
    a page-locked input with a pageable output, and an output that overlaps an input
    (which takes the staged path) all give the device path's limbs."""
    import torch
    nl = (n + 63) // 64
    u, v = workloads.pattern_limbs("random", n, seed=n % 1000 + 400)
    for kind in ("lo", "hi", "full"):
        no = pkg.out_limbs(kind, n)
        ref = {k: host(pkg.mul(kind, dev(a), dev(b), n)[0])
               for k, (a, b) in (("uv", (u, v)), ("uu", (u, u)))}
        block = torch.zeros(1 + 2 * nl + no + 3, dtype=torch.int64).pin_memory()
        bu = block[1:1 + nl]                             # odd-limb offset
        bv = block[1 + nl:1 + 2 * nl]
        bo = block[1 + 2 * nl:1 + 2 * nl + no]
        bu.copy_(torch.from_numpy(u.view(np.int64)))
        bv.copy_(torch.from_numpy(v.view(np.int64)))
        for stream in (None, torch.cuda.Stream()):
            bo.fill_(-1)
            got, rep = pkg.mul_host(kind, bu, bv, n, out=bo, stream=stream)
            assert rep["status"] == 0 and rep["margin"] <= rep["e_max"]
            assert np.array_equal(bo.numpy().view(np.uint64), ref["uv"]), (kind, n)
            assert block[0].item() == 0 and bool((block[1 + 2 * nl + no:] == 0).all())
            got, _ = pkg.mul_host(kind, bu, bu, n, out=bo, stream=stream)
            assert np.array_equal(bo.numpy().view(np.uint64), ref["uu"]), (kind, n)
        pageable = np.zeros(no, dtype=np.uint64)
        got, _ = pkg.mul_host(kind, bu, bv, n, out=pageable)
        assert np.array_equal(got, ref["uv"])
        if no <= 2 * nl:                                  # out over u and v: staged
            both = torch.cat([torch.from_numpy(u.view(np.int64)),
                              torch.from_numpy(v.view(np.int64))]).pin_memory()
            got, _ = pkg.mul_host(kind, both[:nl], both[nl:], n, out=both[:no])
            assert np.array_equal(both[:no].numpy().view(np.uint64), ref["uv"])


@pytest.mark.parametrize("n", [1, 65, 127, 1000, 4097, 100003, (1 << 20) + 5])
def test_bits_above_n_are_ignored(pkg, n):
    """Bits at positions >= n of the operands' top limb are ignored: set at random,
    every entry point (tm_mul, tm_mul_adaptive, squares, host buffers, kept operands,
    a batch) gives the product of the masked operands."""
    import torch
    if n % 64 == 0:
        return
    u, v = workloads.pattern_limbs("random", n, seed=n % 991)
    rng = np.random.default_rng(n)
    junk = np.uint64(~((1 << (n % 64)) - 1) & (2**64 - 1))
    ud, vd = u.copy(), v.copy()
    ud[-1] |= rng.integers(0, 2**63, dtype=np.uint64) * np.uint64(2) & junk
    vd[-1] |= junk                                         # every bit above n set
    assert (ud[-1] & junk) != 0 or n % 64 > 60
    for kind in ("lo", "hi", "full"):
        clean, rep = pkg.mul(kind, dev(u), dev(v), n)
        want = host(clean)
        dirty, rep_d = pkg.mul(kind, dev(ud), dev(vd), n)
        assert np.array_equal(host(dirty), want), kind
        assert rep_d["margin"] == rep["margin"]
        a_c, ra = pkg.mul_adaptive(kind, dev(u), dev(v), n)
        a_d, rd = pkg.mul_adaptive(kind, dev(ud), dev(vd), n)
        assert (ra["b"], ra["N"]) == (rd["b"], rd["N"]) and np.array_equal(host(a_c), host(a_d))
        sq_c, _ = pkg.mul(kind, dev(v), dev(v), n)
        sq_d, _ = pkg.mul(kind, dev(vd), dev(vd), n)
        assert np.array_equal(host(sq_c), host(sq_d))
        pu = torch.from_numpy(ud.view(np.int64)).pin_memory()
        pv = torch.from_numpy(vd.view(np.int64)).pin_memory()
        po = torch.empty(pkg.out_limbs(kind, n), dtype=torch.int64).pin_memory()
        pkg.mul_host(kind, pu, pv, n, out=po)
        assert np.array_equal(po.numpy().view(np.uint64), want)
        got, _ = pkg.mul_host(kind, ud, vd, n)
        assert np.array_equal(got, want)
        op = pkg.Operand(kind, dev(vd), n)
        try:
            got, _ = op.mul(dev(ud))
            assert np.array_equal(host(got), want)
        finally:
            op.close()
        o = torch.empty(pkg.out_limbs(kind, n), dtype=torch.int64, device="cuda")
        b = pkg.Batch([(kind, n, o, dev(ud), dev(vd))])
        try:
            b.launch()
            torch.cuda.synchronize()
            assert np.array_equal(host(o), want)
        finally:
            b.close()
    # and the oracle agrees with the masked operands
    assert np.array_equal(host(pkg.mul("lo", dev(ud), dev(vd), n)[0]), bigmul.mul_lo(u, v, n))


def test_concurrent_streams(pkg):
    """Products enqueued on three streams without waits between them (each stream has
    its own workspace and side stream) equal the oracle."""
    import torch
    streams = [torch.cuda.Stream() for _ in range(3)]
    jobs = []
    for i, s in enumerate(streams):
        for j, kind in enumerate(("lo", "hi", "full")):
            n = [30001, 65536, 200003][(i + j) % 3]
            u, v = workloads.pattern_limbs("random", n, seed=400 + 3 * i + j)
            with torch.cuda.stream(s):
                du, dv = dev(u), dev(v)
                out, _ = pkg.mul(kind, du, dv, n, stream=s, report=False)
            jobs.append((kind, n, u, v, out, du, dv))
    torch.cuda.synchronize()
    for s in streams:
        assert pkg.stream_status(s)["rc"] == 0
    for kind, n, u, v, out, _, _ in jobs:
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
            assert hi_ok(bigmul.to_int(host(out)), u, v, n, full=full)
