"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
function include/truncmul.h declares, its tm_report layout matches the header,
its host-only planner agrees with the oracle's independent planner, and bad
arguments are rejected before any device work."""
import ctypes
import os
import re
import subprocess

import pytest

from oracle import plan as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "truncmul.h")


@pytest.fixture(scope="module")
def pkg():
    import paper_1703_00640_gb300 as p
    p.build()
    p.load()
    return p


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(tm_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(pkg):
    names = _declared()
    assert len(names) >= 10
    out = subprocess.check_output(["nm", "-D", "--defined-only", pkg.library_path()], text=True)
    exported = set(re.findall(r" T (tm_\w+)$", out, re.M))
    assert set(names) <= exported, set(names) - exported
    assert set(names) == set(pkg.EXPORTS)
    lib = pkg.load()
    for n in names:
        getattr(lib, n)


def test_report_layout_matches_header(tmp_path, pkg):
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "truncmul.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(tm_report),'
                   ' offsetof(tm_report, margin), offsetof(tm_report, e_max),'
                   ' offsetof(tm_report, table_bytes)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    size, om, oe, ot = map(int, subprocess.check_output([str(exe)], text=True).split())
    R = pkg.Report
    assert (size, om, oe, ot) == (ctypes.sizeof(R), R.margin.offset, R.e_max.offset,
                                  R.table_bytes.offset)


def test_tune_layout_matches_header(tmp_path, pkg):
    src = tmp_path / "tune.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "truncmul.h"\n'
                   'int main(void){printf("%zu %zu %zu\\n", sizeof(tm_tune),'
                   ' offsetof(tm_tune, ms_default), offsetof(tm_tune, ms_best)); return 0;}\n')
    exe = tmp_path / "tune"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    size, od, ob = map(int, subprocess.check_output([str(exe)], text=True).split())
    T = pkg.Tune
    assert (size, od, ob) == (ctypes.sizeof(T), T.ms_default.offset, T.ms_best.offset)


NS = [1, 2, 7, 63, 64, 65, 100, 999, 1000, 4096, 5000, 65536, 100003, 2**20, 10**6, 2**24,
      21544346, 2**28]


@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_plan_matches_oracle_plan(pkg, n, kind):
    from oracle import plan as P
    mine = pkg.plan(kind, n)
    ref = P.choose(kind, n)
    assert (mine["b"], mine["N"], mine["n_digits"]) == (ref["b"], ref["N"], ref["n_digits"])
    assert (mine["lam_fwd"], mine["lam_bwd"]) == (ref["lam_fwd"], ref["lam_bwd"])
    assert mine["e_max"] == pytest.approx(ref["e_max"], rel=1e-9)
    assert mine["e_max"] < 0.5


@pytest.mark.parametrize("kind", ["lo", "hi", "full"])
def test_forward_stream_choice(pkg, kind):
    # u's and v's forward transforms go to two streams only where one transform's
    # passes fill the GPU (152 SMs, 1024 threads each): the headline size, not below
    for n in (1000, 65536, 2**20, 2**22):
        assert pkg.plan(kind, n)["fwd_streams"] == 1, n
    assert pkg.plan(kind, 2**24)["fwd_streams"] == 2


def test_host_side_errors(pkg):
    lib = pkg.load()
    rep = pkg.Report()
    assert lib.tm_plan_query(1, 0, ctypes.byref(rep)) == pkg.TM_EINVAL
    assert lib.tm_plan_query(7, 100, ctypes.byref(rep)) == pkg.TM_EINVAL
    assert lib.tm_plan_query(1, (1 << 31) + 1, ctypes.byref(rep)) == pkg.TM_ERANGE
    assert lib.tm_plan_query(1, 100, None) == pkg.TM_EINVAL
    # null operands are rejected before any CUDA call
    assert lib.tm_mul(1, None, None, None, 100, None, None) == pkg.TM_EINVAL
    assert lib.tm_mul_lo(None, None, None, 0, None, None) == pkg.TM_EINVAL
    assert lib.tm_autotune(1, 100, None, None) == pkg.TM_EINVAL
    assert lib.tm_autotune(5, 100, None, ctypes.byref(pkg.Tune())) == pkg.TM_EINVAL
    assert lib.tm_autotune(1, (1 << 31) + 1, None, ctypes.byref(pkg.Tune())) == pkg.TM_ERANGE
    # explicit parameters: checked before any CUDA call
    fp = ctypes.c_void_p(0x1000)
    fq = ctypes.c_void_p(0x100000)
    n = 1000000
    ok = dict(b=14, N=71680, limit=0.0)               # a Table 2 row (low product)
    assert lib.tm_mul_params(1, fq, fp, fp, n, None, None, None) == pkg.TM_EINVAL
    for bad in (dict(b=3), dict(b=25), dict(N=71681), dict(N=71680 * 11), dict(N=2),
                dict(b=13, N=71680),                  # N b < n: Theorem 2.2 fails
                dict(limit=-0.1), dict(limit=0.6), dict(limit=float("nan"))):
        prm = pkg.Params(**{**ok, **bad})
        assert lib.tm_mul_params(1, fq, fp, fp, n, ctypes.byref(prm), None, None) == \
            pkg.TM_EINVAL, bad
    hi_bad = pkg.Params(b=14, N=65536, limit=0.0)    # (N + 1) b < n + lg N + 2
    assert lib.tm_mul_params(2, fq, fp, fp, n, ctypes.byref(hi_bad), None, None) == pkg.TM_EINVAL
    full_bad = pkg.Params(b=21, N=65536, limit=0.0)   # below 2 ceil((n+1)/b) - 1
    assert lib.tm_mul_params(0, fq, fp, fp, n, ctypes.byref(full_bad), None, None) == \
        pkg.TM_EINVAL
    prm = pkg.Params(**ok)
    assert lib.tm_mul_params(1, fq, fp, fp, 0, ctypes.byref(prm), None, None) == pkg.TM_EINVAL
    assert lib.tm_mul_params(1, fq, fp, fp, (1 << 31) + 1, ctypes.byref(prm), None,
                             None) == pkg.TM_ERANGE
    assert lib.tm_mul_params(1, fp, fp, fp, n, ctypes.byref(prm), None, None) == pkg.TM_EALIAS
    # plan choice: checked (and, for tm_plan_set, applied) without a GPU
    T = pkg.PlanTune()
    assert lib.tm_autotune_plan(1, 1000, None, None) == pkg.TM_EINVAL
    assert lib.tm_autotune_plan(5, 1000, None, ctypes.byref(T)) == pkg.TM_EINVAL
    assert lib.tm_autotune_plan(1, 0, None, ctypes.byref(T)) == pkg.TM_EINVAL
    assert lib.tm_autotune_plan(1, (1 << 31) + 1, None, ctypes.byref(T)) == pkg.TM_ERANGE
    assert lib.tm_plan_set(7, 1000000, 9, 122880) == pkg.TM_EINVAL
    assert lib.tm_plan_set(1, 0, 9, 122880) == pkg.TM_EINVAL
    assert lib.tm_plan_set(1, 1000000, 9, 122881) == pkg.TM_EINVAL        # not a length
    assert lib.tm_plan_set(1, 1000000, 14, 71680) == pkg.TM_ERANGE        # not certified
    assert lib.tm_plan_set(1, 1000000, 0, 0) == pkg.TM_OK
    # layouts: checked before any CUDA call
    good = pkg.Tune(points=512, split=0, passes=3)
    assert lib.tm_set_layout(1, 100, None) == pkg.TM_EINVAL
    assert lib.tm_set_layout(4, 100, ctypes.byref(good)) == pkg.TM_EINVAL
    assert lib.tm_set_layout(1, 0, ctypes.byref(good)) == pkg.TM_EINVAL
    assert lib.tm_set_layout(1, (1 << 31) + 1, ctypes.byref(good)) == pkg.TM_ERANGE
    for bad in (dict(points=16), dict(points=8192), dict(split=3), dict(split=-1),
                dict(passes=1), dict(passes=4)):
        t = pkg.Tune(**{**dict(points=1024, split=0, passes=0), **bad})
        assert lib.tm_set_layout(1, 1 << 20, ctypes.byref(t)) == pkg.TM_EINVAL, bad
    assert lib.tm_mul_adaptive(1, None, None, None, 100, None, None) == pkg.TM_EINVAL
    assert lib.tm_mul_adaptive(9, fake_ptr := ctypes.c_void_p(0x1000), fake_ptr, fake_ptr, 100,
                               None, None) == pkg.TM_EINVAL
    assert lib.tm_mul_adaptive(1, fake_ptr, fake_ptr, fake_ptr, (1 << 31) + 1, None,
                               None) == pkg.TM_ERANGE
    # kept operands: argument checks precede any CUDA call
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    assert lib.tm_operand_create(1, 100, None, None, ctypes.byref(h)) == pkg.TM_EINVAL
    assert lib.tm_operand_create(1, 100, fake, None, None) == pkg.TM_EINVAL
    assert lib.tm_operand_create(7, 100, fake, None, ctypes.byref(h)) == pkg.TM_EINVAL
    assert lib.tm_operand_create(1, 0, fake, None, ctypes.byref(h)) == pkg.TM_EINVAL
    assert lib.tm_operand_create(2, (1 << 31) + 1, fake, None, ctypes.byref(h)) == pkg.TM_ERANGE
    assert not h.value                                   # no handle on error
    assert lib.tm_mul_operand(None, fake, fake, None, None) == pkg.TM_EINVAL
    assert lib.tm_mul_operand(fake, fake, None, None, None) == pkg.TM_EINVAL
    assert lib.tm_operand_destroy(None) == pkg.TM_OK
    # division: argument checks precede any CUDA call
    assert lib.tm_reciprocal(None, fake, 100, None) == pkg.TM_EINVAL
    assert lib.tm_reciprocal(fake, None, 100, None) == pkg.TM_EINVAL
    assert lib.tm_reciprocal(fake, fake, 0, None) == pkg.TM_EINVAL
    assert lib.tm_reciprocal(fake, fake, 1 << 31, None) == pkg.TM_ERANGE
    assert lib.tm_barrett_create(fake, 100, None, None) == pkg.TM_EINVAL
    assert lib.tm_barrett_create(None, 100, None, ctypes.byref(h)) == pkg.TM_EINVAL
    assert lib.tm_barrett_create(fake, 0, None, ctypes.byref(h)) == pkg.TM_EINVAL
    assert not h.value
    assert lib.tm_barrett_divrem(None, fake, fake, fake, None, None) == pkg.TM_EINVAL
    assert lib.tm_barrett_reciprocal(None, fake, None) == pkg.TM_EINVAL
    assert lib.tm_barrett_destroy(None) == pkg.TM_OK
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, 99):
        assert pkg.strerror(code)


def test_plan_set_changes_the_plan(pkg):
    """tm_plan_set makes a certified (b, N) the plan of (kind, n) (tm_plan_query shows
    it) and b = N = 0 restores the planner's choice; certification comes from the
    oracle planner's independent bound."""
    n = 1000000
    for kind in ("lo", "hi", "full"):
        base = P.choose(kind, n)
        cand = None
        for N in P.smooth_lengths_from(base["N"] + 1):
            if kind == "hi" and not P.hi_ok(n, base["b"], N):
                continue
            E = {"lo": P.bound_lo, "hi": P.bound_hi, "full": P.bound_full}[kind](n, base["b"], N)
            E = E[0] if isinstance(E, tuple) else (E["E"] if isinstance(E, dict) else E)
            if E <= P.E_TARGET:
                cand = N
                break
        assert cand is not None
        pkg.plan_set(kind, n, base["b"], cand)
        try:
            q = pkg.plan(kind, n)
            assert (q["b"], q["N"]) == (base["b"], cand)
        finally:
            pkg.plan_set(kind, n)
        q = pkg.plan(kind, n)
        assert (q["b"], q["N"]) == (base["b"], base["N"])



@pytest.mark.parametrize("n", [1000, 65536, 1000003, 1 << 24])
def test_plan_set_certification_matches_oracle_bound(pkg, n):
    """tm_plan_set accepts (b, N) exactly when the oracle planner's independent
    worst-case bound for (b, N) is within the target (and rejects lengths that
    break the hypotheses of Theorems 2.1-2.3 as invalid)."""
    lib = pkg.load()
    bound = {"lo": P.bound_lo, "hi": P.bound_hi, "full": P.bound_full}
    kinds = {"lo": 1, "hi": 2, "full": 0}
    checked = 0
    for kind in ("lo", "hi", "full"):
        base = P.choose(kind, n)
        for b in (base["b"] - 1, base["b"], base["b"] + 1):
            if kind == "lo":
                x = P.min_len_lo(n, b)
            elif kind == "hi":
                x = P.min_len_hi(n, b)
            else:
                x = 2 * P.full_digits(n, b) - 1
            for N in list(P.smooth_lengths_from(x))[:4]:
                if kind == "hi" and not P.hi_ok(n, b, N):
                    continue
                E = bound[kind](n, b, N)
                E = E[0] if isinstance(E, tuple) else (E["E"] if isinstance(E, dict) else E)
                if abs(E - P.E_TARGET) < 1e-9 * P.E_TARGET:
                    continue                      # too close to call across two codes
                rc = lib.tm_plan_set(kinds[kind], n, b, N)
                assert rc == (pkg.TM_OK if E <= P.E_TARGET else pkg.TM_ERANGE), (kind, b, N, E)
                checked += 1
        lib.tm_plan_set(kinds[kind], n, 0, 0)
    assert checked >= 12


def test_plan_matches_oracle_plan_random_sizes(pkg):
    """The C++ planner and the oracle's planner agree on (b, N, lambda, e_max) for 200
    seeded sizes, log-uniform over [1, 2^31]."""
    import random
    rnd = random.Random(1703)
    for _ in range(200):
        n = int(2 ** rnd.uniform(0, 31))
        kind = rnd.choice(("lo", "hi", "full"))
        mine = pkg.plan(kind, n)
        ref = P.choose(kind, n)
        assert (mine["b"], mine["N"], mine["n_digits"]) == \
            (ref["b"], ref["N"], ref["n_digits"]), (kind, n)
        assert (mine["lam_fwd"], mine["lam_bwd"]) == (ref["lam_fwd"], ref["lam_bwd"]), (kind, n)
        assert mine["e_max"] == pytest.approx(ref["e_max"], rel=1e-9), (kind, n)


def test_dft_constants_are_the_nearest_doubles():
    """The radix-3/5/7 DFT constants written in the kernels are the doubles
    nearest to cos / sin of 2 pi k / R (the FFT error bound takes each within
    2^-53 of its exact value)."""
    import hp_trig
    src = open(os.path.join(ROOT, "paper_1703_00640_gb300", "csrc", "kernels.cu")).read()
    vals = dict(re.findall(r"constexpr double (k[CS]\d_\d|kSqrt3_2) = "
                           r"(-?0x[0-9a-fp.+-]+);", src))
    want = {"kSqrt3_2": hp_trig.cossin_2pi(1, 3)[1]}
    for R, count in ((5, 2), (7, 3)):
        for k in range(1, count + 1):
            c, s = hp_trig.cossin_2pi(k, R)
            want[f"kC{R}_{k}"], want[f"kS{R}_{k}"] = c, s
    assert set(vals) == set(want), set(want) ^ set(vals)
    for name, text in vals.items():
        assert float.fromhex(text) == float(want[name]), name


def test_double_double_constants():
    """The double-double constants of the table kernels: cos and sin of j pi / 32
    and 1/k! (hi + lo within 2^-104 of the exact value, hi the nearest double), and
    pi / 2."""
    from decimal import Decimal, localcontext
    from math import factorial
    import hp_trig
    src = open(os.path.join(ROOT, "paper_1703_00640_gb300", "csrc", "kernels.cu")).read()
    hexnum = r"(-?0x[0-9a-fp.+-]+)"
    trig = re.findall(r"\{" + r",\s*".join([hexnum] * 4) + r"\}", src.split("kTrig32")[1].split(";")[0])
    fact = re.findall(r"\{" + hexnum + r",\s*" + hexnum + r"\}", src.split("kInvFact")[1].split(";")[0])
    assert len(trig) == 9 and len(fact) == 16

    def close(hi, lo, exact):
        with localcontext() as ctx:
            ctx.prec = 80
            v = Decimal(float.fromhex(hi)) + Decimal(float.fromhex(lo))
            assert float.fromhex(hi) == float(exact)
            assert abs(v - exact) <= abs(exact) * Decimal(2) ** -104 + Decimal(10) ** -70

    for j, (ch, cl, sh, sl) in enumerate(trig):
        c, s = hp_trig.cossin_2pi(j, 64)                     # angle j pi / 32
        close(ch, cl, c)
        close(sh, sl, s)
    with localcontext() as ctx:
        ctx.prec = 80
        for k, (h, l) in enumerate(fact):
            close(h, l, Decimal(1) / Decimal(factorial(k)))
        hi = re.search(r"kPi2Hi = " + hexnum, src).group(1)
        lo = re.search(r"kPi2Lo = " + hexnum, src).group(1)
        close(hi, lo, hp_trig.pi() / 2)
