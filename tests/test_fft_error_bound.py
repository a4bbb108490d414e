"""Pins of the FP64 convolution error bound (oracle.plan.eta_conv and its stage
constants) against the arithmetic the FFT kernels perform, on the CPU.

tests/fft_model.py performs the kernels' operation sequences (butterflies,
table-twiddle products, four-step twiddles, the fused twist) on binary64 floats
with a correctly rounded FMA and the tables' values. Here:
- every butterfly kind's exact rounding error (against its exact result, with the
  exact twiddles and DFT constants, to about 200 bits) stays within the oracle's
  local constants, per output in the 1-norm of the inputs and for the whole
  butterfly in the 2-norm, over every twiddle angle of several stages, both
  directions and inputs of mixed magnitudes;
- the model convolution's exact error (integer inputs: the exact convolution is
  an integer) stays within eta_conv(N) ||x||_2 ||y||_2 on extreme-digit inputs,
  for one- and two-pass layouts and every radix;
- the two norm facts the bound composes with are checked at inputs that attain
  them: a forward error dZ acts on each output as the convolution of a real
  vector of norm ||dZ|| / sqrt(M) (Cauchy-Schwarz, attained by a reversed copy),
  and the inverse FFT's input Q has ||Q||_1 <= 2 ||x||_2 ||y||_2, with inputs that
  come close to 2 (so the factor cannot be 1).
Worst-case rounding alignment is not reached by sampling (the measured errors
are about a third of the per-butterfly constants and a hundredth of eta), so these
pins establish validity on what they sample and the exact norm algebra, not
sharpness of the rounding constants."""
import math
import random
from decimal import Decimal, localcontext

import numpy as np
import pytest

import fft_model as F
import hp_trig
from oracle import plan as P

U = P.U


def _dexp(num, den):
    c, s = hp_trig.cossin_2pi(num % den, den)
    return (c, -s)


def _dmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def _exact_butterfly(x, R, S, tw):
    """sum_t exp(2 pi i S j t / R) tw_t x_t for every j (tw_t the exact twiddle
    multipliers of the direction S)."""
    out = []
    for j in range(R):
        acc = (Decimal(0), Decimal(0))
        for t in range(R):
            root = _dexp(j * t, R)
            if S > 0:
                root = (root[0], -root[1])
            w = _dmul(tw[t], root)
            v = _dmul((Decimal(x[t][0]), Decimal(x[t][1])), w)
            acc = (acc[0] + v[0], acc[1] + v[1])
        out.append(acc)
    return out


def _errors(y, ex):
    return [float(((Decimal(a[0]) - b[0]) ** 2 + (Decimal(a[1]) - b[1]) ** 2).sqrt())
            for a, b in zip(y, ex)]


def _inputs(rnd, R):
    kind = rnd.randrange(4)
    if kind == 0:
        return [(rnd.uniform(-1, 1), rnd.uniform(-1, 1)) for _ in range(R)]
    if kind == 1:                     # mixed magnitudes
        return [(rnd.uniform(-1, 1) * 2.0 ** rnd.randint(-30, 0),
                 rnd.uniform(-1, 1) * 2.0 ** rnd.randint(-30, 0)) for _ in range(R)]
    if kind == 2:                     # extreme digits
        return [(float(rnd.choice([-2048, 2048])), float(rnd.choice([-2048, 2048])))
                for _ in range(R)]
    return [(rnd.uniform(0.5, 1), 0.0) for _ in range(R)]


KINDS = [("r2tw", 2), ("r4tan", 4), ("r3tw", 3), ("r5tw", 5), ("r7tw", 7)]


@pytest.mark.parametrize("key,R", KINDS, ids=[k for k, _ in KINDS])
def test_butterflies_within_local_constants(key, R):
    """Twiddled butterflies (and the same radix without twiddles, which the bound
    prices at the twiddled constant) within the oracle's LOCAL_L1 / LOCAL_L2."""
    rnd = random.Random(R)
    tables = F.Tables()
    worst1 = worst2 = 0.0
    with localcontext() as ctx:
        ctx.prec = 60
        for Ns in (1, 2, 8, 32):
            for kk in range(Ns):
                for S in (-1, 1):
                    x = _inputs(rnd, R)
                    if R == 4 and Ns > 1:
                        y = F.radix4_tan(x, tables.tan(kk, Ns), S)
                        tw = [_dexp(0, 1)] + [_dexp(kk * t, 4 * Ns) for t in (1, 2, 3)]
                    else:
                        xs = list(x)
                        if Ns > 1:
                            for t in range(1, R):
                                w = tables.tw(kk * t, Ns * R)
                                xs[t] = F.cmul(xs[t], w) if S < 0 else F.cmulc(xs[t], w)
                        y = F.DFT[R](xs, S)
                        tw = [_dexp(kk * t, Ns * R) for t in range(R)]
                    if S > 0:
                        tw = [(t[0], -t[1]) for t in tw]
                    ex = _exact_butterfly(x, R, S, tw)
                    err = _errors(y, ex)
                    n1 = sum(math.hypot(*v) for v in x)
                    n2 = math.sqrt(sum(a * a + b * b for a, b in x))
                    r1 = max(err) / (U * n1)
                    r2 = math.sqrt(sum(e * e for e in err)) / (U * math.sqrt(R) * n2)
                    assert r1 <= P.LOCAL_L1[key], (key, Ns, kk, S, r1)
                    assert r2 <= P.LOCAL_L2[key], (key, Ns, kk, S, r2)
                    if Ns == 1:          # a pass's first stage: no twiddle
                        assert r1 <= P.LOCAL_L1[key] - P.FIRST_STAGE_L1, (key, S, r1)
                        assert r2 <= P.LOCAL_L2[key] - P.FIRST_STAGE_L2, (key, S, r2)
                    worst1, worst2 = max(worst1, r1), max(worst2, r2)
    print(f"{key}: worst per-output {worst1:.2f} U (bound {P.LOCAL_L1[key]:.2f}), "
          f"worst 2-norm {worst2:.2f} U (bound {P.LOCAL_L2[key]:.2f})")


def _dft3_first_order(x, S, twiddled):
    """The output-error vectors of dft3's roundings to first order, one per real
    rounding (a unit relative error there, every other operation exact), in the
    kernel's order: t = x1 + x2, m = x0 - t/2 (FMA), d = x1 - x2, the constant
    sqrt(3)/2 (one relative error for both components), d times it, the three
    final additions. The twiddle products' error, at most 3 U |x_t| in any
    direction, enters through the DFT (norm sqrt 3) and is returned apart."""
    x0, x1, x2 = (complex(*v) for v in x)
    c = math.sqrt(3) / 2
    si = 1j * S

    def outputs(eps):
        def r(v, *keys):            # v with relative errors on its real / imaginary parts
            return complex(v.real * (1 + eps.get(keys[0], 0)),
                           v.imag * (1 + eps.get(keys[1], 0)))
        t = r(x1 + x2, "tr", "ti")
        m = r(x0 - t / 2, "mr", "mi")
        d = r(x1 - x2, "dr", "di")
        k = c * (1 + eps.get("k", 0))
        sd = si * r(d * k, "pr", "pi")
        return np.array([r(x0 + t, "y0r", "y0i"), r(m + sd, "y1r", "y1i"),
                         r(m - sd, "y2r", "y2i")])

    base = outputs({})
    h = 2.0 ** -20
    keys = ["tr", "ti", "mr", "mi", "dr", "di", "k", "pr", "pi",
            "y0r", "y0i", "y1r", "y1i", "y2r", "y2i"]
    vecs = []
    for key in keys:
        dv = (outputs({key: h}) - base) / h
        vecs.append(np.concatenate([dv.real, dv.imag]))
    tw = math.sqrt(3) * 3 * math.hypot(abs(x1), abs(x2)) if twiddled else 0.0
    return np.array(vecs), tw


def test_radix3_two_norm_constant_brute_force():
    """The radix-3 2-norm constant (LOCAL_L2["r3tw"], and with the first-stage
    saving for the untwiddled butterfly) against the worst first-order error of
    dft3's operation sequence: every sign pattern of its 15 real roundings, on
    random and hill-climbed unit inputs. A dropped or undercounted term in the
    derivation shows as a pattern above the constant."""
    signs = np.array([[1 - 2 * ((p >> i) & 1) for i in range(15)] for p in range(1 << 15)],
                     dtype=np.float64)
    rng = np.random.default_rng(3)

    def worst(x, S, twiddled):
        V, tw = _dft3_first_order(x, S, twiddled)
        return (np.max(np.linalg.norm(signs @ V, axis=1)) + tw) / math.sqrt(3)

    found = {}
    for twiddled in (True, False):
        limit = P.LOCAL_L2["r3tw"] - (0.0 if twiddled else P.FIRST_STAGE_L2)
        best, bx = 0.0, None
        for _ in range(60):
            v = rng.normal(size=6)
            v /= np.linalg.norm(v)
            x = [(v[2 * i], v[2 * i + 1]) for i in range(3)]
            w = worst(x, -1, twiddled)
            if w > best:
                best, bx = w, v
        step = 0.3
        for _ in range(120):            # hill-climb from the best random start
            v = bx + step * rng.normal(size=6)
            v /= np.linalg.norm(v)
            w = worst([(v[2 * i], v[2 * i + 1]) for i in range(3)], -1, twiddled)
            if w > best:
                best, bx = w, v
            else:
                step *= 0.97
        for S in (-1, 1):
            w = worst([(bx[2 * i], bx[2 * i + 1]) for i in range(3)], S, twiddled)
            assert w <= limit, (twiddled, S, w, limit)
        assert best <= limit, (twiddled, best, limit)
        found[twiddled] = (best, limit)
    print("radix 3 first-order worst (twiddled, untwiddled):",
          {k: (round(a, 3), round(b, 3)) for k, (a, b) in found.items()})


def _round_model(eps):
    """r(v, key): v with relative errors eps[key + "r"], eps[key + "i"] on its real and
    imaginary parts (a componentwise rounding, to first order)."""
    def r(v, key):
        return complex(v.real * (1 + eps.get(key + "r", 0)), v.imag * (1 + eps.get(key + "i", 0)))
    return r


def _dft5_outputs(x, S, eps):
    """dft5's operation sequence (sums and differences, two FMA chains per cosine
    half, a product and an FMA per sine half, the final additions) with relative
    errors eps on every rounding and on the four constants."""
    r = _round_model(eps)
    x0, x1, x2, x3, x4 = x
    c1, c2 = math.cos(2 * math.pi / 5), math.cos(4 * math.pi / 5)
    s1, s2 = math.sin(2 * math.pi / 5), math.sin(4 * math.pi / 5)
    C1, C2 = c1 * (1 + eps.get("c1", 0)), c2 * (1 + eps.get("c2", 0))
    S1, S2 = s1 * (1 + eps.get("s1", 0)), s2 * (1 + eps.get("s2", 0))
    si = 1j * S
    t1, t2 = r(x1 + x4, "t1"), r(x2 + x3, "t2")
    d1, d2 = r(x1 - x4, "d1"), r(x2 - x3, "d2")
    a1 = r(C1 * t1 + r(C2 * t2 + x0, "a1i"), "a1o")
    a2 = r(C2 * t1 + r(C1 * t2 + x0, "a2i"), "a2o")
    b1 = si * r(S1 * d1 + r(S2 * d2, "p1"), "b1")
    b2 = si * r(S2 * d1 + r(-S1 * d2, "p2"), "b2")
    y0 = r(x0 + r(t1 + t2, "s12"), "y0")
    return np.array([y0, r(a1 + b1, "y1"), r(a2 + b2, "y2"), r(a2 - b2, "y3"), r(a1 - b1, "y4")])


def _dft7_outputs(x, S, eps):
    """dft7's operation sequence: sums and differences, a_m by three chained FMAs
    (innermost k = 3), b_m by a product (k = 3) and two FMAs, y0 = x0 + (t1 + (t2 + t3)),
    the final additions; relative errors eps on every rounding and constant."""
    r = _round_model(eps)
    x0 = x[0]
    c = [math.cos(2 * math.pi * k / 7) * (1 + eps.get(f"c{k}", 0)) for k in (1, 2, 3)]
    s_ = [math.sin(2 * math.pi * k / 7) * (1 + eps.get(f"s{k}", 0)) for k in (1, 2, 3)]
    cm = {1: (c[0], c[1], c[2]), 2: (c[1], c[2], c[0]), 3: (c[2], c[0], c[1])}
    sm = {1: (s_[0], s_[1], s_[2]), 2: (s_[1], -s_[2], -s_[0]), 3: (s_[2], -s_[0], s_[1])}
    t = [r(x[k] + x[7 - k], f"t{k}") for k in (1, 2, 3)]
    d = [r(x[k] - x[7 - k], f"d{k}") for k in (1, 2, 3)]
    si = 1j * S
    y = [None] * 7
    for m in (1, 2, 3):
        C, Sn = cm[m], sm[m]
        a = r(C[0] * t[0] + r(C[1] * t[1] + r(C[2] * t[2] + x0, f"a{m}i"), f"a{m}m"), f"a{m}o")
        b = si * r(Sn[0] * d[0] + r(Sn[1] * d[1] + r(Sn[2] * d[2], f"p{m}"), f"b{m}i"), f"b{m}o")
        y[m], y[7 - m] = r(a + b, f"y{m}"), r(a - b, f"y{7 - m}")
    y[0] = r(x0 + r(t[0] + r(t[1] + t[2], "s23"), "s123"), "y0")
    return np.array(y)


def _dft3_outputs(x, S, eps):
    r = _round_model(eps)
    x0, x1, x2 = x
    k = math.sqrt(3) / 2 * (1 + eps.get("k", 0))
    t = r(x1 + x2, "t")
    m = r(x0 - t / 2, "m")
    sd = 1j * S * r(r(x1 - x2, "d") * k, "p")
    return np.array([r(x0 + t, "y0"), r(m + sd, "y1"), r(m - sd, "y2")])


def _first_order_vectors(outputs, x, S, keys):
    """Output-error vectors (complex, one per rounding) of a unit relative error at
    each key, by a one-sided difference (the outputs are linear in each error)."""
    base = outputs(x, S, {})
    h = 2.0 ** -24
    return np.array([(outputs(x, S, {key: h}) - base) / h for key in keys])


def _keys(names, scalars=()):
    return [n + c for n in names for c in ("r", "i")] + list(scalars)


R5_KEYS = _keys(["t1", "t2", "d1", "d2", "a1i", "a1o", "a2i", "a2o", "p1", "b1", "p2", "b2",
                 "s12", "y0", "y1", "y2", "y3", "y4"], ["c1", "c2", "s1", "s2"])
R3_KEYS = _keys(["t", "m", "d", "p", "y0", "y1", "y2"], ["k"])
R7_KEYS = _keys([f"{v}{k}" for v in "td" for k in (1, 2, 3)]
                + [f"a{m}{w}" for m in (1, 2, 3) for w in "imo"]
                + [f"{v}{m}{w}" for m in (1, 2, 3) for v, w in (("p", ""), ("b", "i"), ("b", "o"))]
                + ["s23", "s123"] + [f"y{j}" for j in range(7)],
                [f"{v}{k}" for v in "cs" for k in (1, 2, 3)])


def _worst_per_output(V, x, R, twiddled):
    """max over outputs j of the largest first-order error of y_j over all rounding
    errors in [-U, U] (max over directions phi of sum |Re(e^-i phi v_ij)|), plus the
    twiddle products' 3 U |x_t| (t >= 1) aligned; relative to ||x||_1."""
    phis = np.linspace(0, 2 * np.pi, 721)
    rot = np.exp(-1j * phis)
    tw = 3 * sum(abs(v) for v in x[1:]) if twiddled else 0.0
    worst = max(float(np.max(np.abs(np.real(rot[:, None] * V[None, :, j])).sum(axis=1)))
                for j in range(R))
    return (worst + tw) / sum(abs(v) for v in x)


def _worst_two_norm(V, x, R, twiddled, rng):
    """A large ||sum theta_i v_i|| over signs theta (random starts, then single-sign
    flips while they help), plus the twiddles' 3 sqrt(R) ||x_1..||; relative to
    sqrt(R) ||x||. The exact maximum over 2^K patterns is out of reach for radix 5;
    the derivation bounds every pattern."""
    Vr = np.concatenate([V.real, V.imag], axis=1)
    best = 0.0
    for _ in range(12):
        th = rng.choice([-1.0, 1.0], size=len(Vr))
        val = np.linalg.norm(th @ Vr)
        improved = True
        while improved:
            improved = False
            for i in range(len(th)):
                th[i] = -th[i]
                nv = np.linalg.norm(th @ Vr)
                if nv > val + 1e-15:
                    val, improved = nv, True
                else:
                    th[i] = -th[i]
        best = max(best, val)
    tw = 3 * math.sqrt(R) * np.linalg.norm(x[1:]) if twiddled else 0.0
    return (best + tw) / (math.sqrt(R) * np.linalg.norm(x))


@pytest.mark.parametrize("R,outputs,keys,kind", [(5, _dft5_outputs, R5_KEYS, "r5tw"),
                                                 (7, _dft7_outputs, R7_KEYS, "r7tw"),
                                                 (3, _dft3_outputs, R3_KEYS, "r3tw")],
                         ids=["radix5", "radix7", "radix3"])
def test_odd_radix_constants_first_order(R, outputs, keys, kind):
    """The radix-3, 5 and 7 constants (per output LOCAL_L1, and for radix 5 and 7 the
    2-norm LOCAL_L2), with and without twiddles, against the first-order error of the
    butterfly's own operation sequence: per output the exact worst case over all
    rounding errors, in the 2-norm a local search over sign patterns; inputs from
    random starts improved by hill-climbing. A term dropped from the derivations
    shows as an error above its constant."""
    rng = np.random.default_rng(R)

    def scores(v, tw):
        x = v[:R] + 1j * v[R:]
        V = _first_order_vectors(outputs, x, -1, keys)
        return _worst_per_output(V, x, R, tw), (_worst_two_norm(V, x, R, tw, rng) if R > 3 else 0.0)

    for tw in (True, False):
        lim1 = P.LOCAL_L1[kind] - (0.0 if tw else P.FIRST_STAGE_L1)
        lim2 = P.LOCAL_L2[kind] - (0.0 if tw else P.FIRST_STAGE_L2)
        best1 = best2 = 0.0
        x1 = x2 = None
        for _ in range(40):
            v = rng.normal(size=2 * R)
            s1_, s2_ = scores(v, tw)
            if s1_ > best1:
                best1, x1 = s1_, v
            if s2_ > best2:
                best2, x2 = s2_, v
        for target in (1, 2) if R > 3 else (1,):
            xb = x1 if target == 1 else x2
            step = 0.3
            for _ in range(60):
                v = xb + step * rng.normal(size=2 * R)
                sc = scores(v, tw)[target - 1]
                if sc > (best1 if target == 1 else best2):
                    xb = v
                    if target == 1:
                        best1 = sc
                    else:
                        best2 = sc
                else:
                    step *= 0.95
        assert best1 <= lim1, (kind, tw, best1, lim1)
        assert best2 <= lim2, (kind, tw, best2, lim2)
        two = f", 2-norm {best2:.3f} U (constant {lim2:.2f})" if R > 3 else ""
        print(f"{kind} {'twiddled' if tw else 'first stage'}: per output {best1:.3f} U "
              f"(constant {lim1:.2f}){two}")


def test_first_stage_discount_is_conservative():
    """eta_conv with the discount taken from the dearest stages is at least eta_conv
    with the discount on any other choice of P stages (the layout decides which
    stages open a pass), checked for lengths with every mix of radices."""
    import itertools
    for M in (1260, 2520 * 7, 4608, 3 * 5 * 7 * 64):
        for stages, passes in P.stage_lists(M):
            radix = [P.LOCAL_L2[k] for k in stages if k != "outer"]
            mine = math.prod(1 + c * U for c in
                             P._with_first_stages(P.LOCAL_L2, stages, passes, P.FIRST_STAGE_L2)
                             if True)
            for pick in itertools.combinations(range(len(radix)), min(passes, len(radix))):
                other = [c - (P.FIRST_STAGE_L2 if i in pick else 0.0)
                         for i, c in enumerate(radix)]
                other += [P.LOCAL_L2["outer"]] * stages.count("outer")
                assert math.prod(1 + c * U for c in other) <= mine * (1 + 1e-15)


def test_twiddle_product_within_constant():
    """The four-step twiddle product (one table entry, one complex product)."""
    rnd = random.Random(3)
    tables = F.Tables()
    with localcontext() as ctx:
        ctx.prec = 60
        for length in (12, 40, 96, 1000):
            for m in range(0, length, max(1, length // 50)):
                for S in (-1, 1):
                    a = (rnd.uniform(-1, 1), rnd.uniform(-1, 1))
                    w = tables.tw(m, length)
                    got = F.cmul(a, w) if S < 0 else F.cmulc(a, w)
                    e = _dexp(m, length)
                    if S > 0:
                        e = (e[0], -e[1])
                    want = _dmul((Decimal(a[0]), Decimal(a[1])), e)
                    err = _errors([got], [want])[0]
                    assert err <= P.TWIDDLE_PRODUCT * U * math.hypot(*a)


CONV_CASES = [(8, None), (12, None), (20, None), (28, None), (40, None), (56, None),
              (96, (4, 12)), (120, (12, 5)), (168, (12, 7)), (256, (8, 16)),
              (420, (14, 15)), (250, None), (486, (27, 9)), (686, (7, 49)),
              (1250, (25, 25))]


@pytest.mark.parametrize("N,split", CONV_CASES, ids=[f"N{n}" for n, _ in CONV_CASES])
def test_model_convolution_within_eta(N, split):
    rnd = random.Random(N)
    tables = F.Tables()
    b = 13
    worst = 0.0
    for trial in range(4):
        if trial == 0:
            x = [2 ** (b - 1)] * N
            y = [-(2 ** (b - 1))] * N
        elif trial == 1:
            x = [rnd.choice([-1, 1]) * 2 ** (b - 1) for _ in range(N)]
            y = [rnd.choice([-1, 1]) * 2 ** (b - 1) for _ in range(N)]
        else:
            x = [rnd.randint(-2 ** (b - 1), 2 ** (b - 1)) for _ in range(N)]
            y = [rnd.randint(-2 ** (b - 1), 2 ** (b - 1)) for _ in range(N)]
        got = F.convolution(x, y, split, tables)
        want = F.exact_cyclic(x, y)
        err = max(abs(Decimal(g) - w) for g, w in zip(got, want))
        norm = math.sqrt(sum(v * v for v in x)) * math.sqrt(sum(v * v for v in y))
        ratio = float(err) / (P.eta_conv(N) * norm)
        assert ratio <= 1.0, (N, trial, ratio)
        worst = max(worst, ratio)
    print(f"N={N}: largest error {worst:.4f} of eta ||x|| ||y||")


def _pack(x):
    return x[0::2] + 1j * x[1::2]


def _twist_exact(Zu, Zv, N):
    """The twist formula in complex128 (the norm facts need no rounding model)."""
    M = N // 2
    k = np.arange(M)
    km = (-k) % M
    w = np.exp(-2j * np.pi * k / N)
    c = (1 + w * w) / (2 * N)
    A, B = Zu, np.conj(Zu[km])
    A1, B1 = Zv, np.conj(Zv[km])
    Q = (2 / N) * A * A1 - c * (A - B) * (A1 - B1)
    return Q


@pytest.mark.parametrize("N", [16, 60, 256])
def test_twist_is_the_packed_product_spectrum(N):
    """F*_M Q(Z_x, Z_y) is the packed cyclic convolution of x and y for real x, y
    (the identity the bound's composition rests on), and Q_k =
    ((1 + i w^-k) P_k + (1 - i w^-k) P_(k+M)) / N with P = X X'."""
    rng = np.random.default_rng(N)
    x, y = rng.normal(size=N), rng.normal(size=N)
    M = N // 2
    Q = _twist_exact(np.fft.fft(_pack(x)), np.fft.fft(_pack(y)), N)
    q = np.fft.ifft(Q) * M
    conv = np.real(np.fft.ifft(np.fft.fft(x) * np.fft.fft(y)))
    assert np.allclose(q, _pack(conv), atol=1e-9 * np.abs(conv).max())
    X, Y = np.fft.fft(x), np.fft.fft(y)
    Pk = X * Y
    k = np.arange(M)
    wi = np.exp(2j * np.pi * k / N)
    assert np.allclose(Q, ((1 + 1j * wi) * Pk[:M] + (1 - 1j * wi) * Pk[M:]) / N,
                       atol=1e-9 * np.abs(Q).max())


@pytest.mark.parametrize("N", [16, 64, 240])
def test_forward_error_acts_as_a_real_convolution(N):
    """A spectrum error dZ (any complex vector) changes the packed result by the
    convolution of the real vector dx with pack(dx) = F^-1 dZ, ||dx|| =
    ||dZ|| / sqrt(M): each output changes by at most ||dZ|| ||y|| / sqrt(M), and a
    reversed copy of y attains it."""
    rng = np.random.default_rng(N)
    M = N // 2
    y = rng.normal(size=N)
    Zy = np.fft.fft(_pack(y))
    for trial in range(3):
        if trial < 2:
            dZ = rng.normal(size=M) + 1j * rng.normal(size=M)
        else:                                  # dx = y reversed: output 0 attains it
            dx = np.roll(y[::-1], 1)
            dZ = np.fft.fft(_pack(dx))
        dq = np.fft.ifft(_twist_exact(dZ, Zy, N)) * M
        change = np.concatenate([dq.real[:, None], dq.imag[:, None]], axis=1).ravel()
        bound = np.linalg.norm(dZ) / math.sqrt(M) * np.linalg.norm(y)
        assert np.abs(change).max() <= bound * (1 + 1e-12)
        if trial == 2:
            assert np.abs(change).max() >= bound * (1 - 1e-9)


@pytest.mark.parametrize("N", [64, 256, 1024])
def test_inverse_input_one_norm(N):
    """||Q||_1 <= 2 ||x||_2 ||y||_2 on random and extremal inputs; a pure tone at
    the frequency where |1 - i w^-k| is largest comes within a few percent of 2."""
    rng = np.random.default_rng(N)
    M = N // 2
    worst = 0.0
    cases = [(rng.normal(size=N), rng.normal(size=N)) for _ in range(5)]
    n = np.arange(N)
    for f in (N // 4 + 1, N // 4 + N // 16, 3 * N // 8):
        tone = np.cos(2 * np.pi * f * n / N + 0.3)
        cases.append((tone, tone))
    for x, y in cases:
        Q = _twist_exact(np.fft.fft(_pack(x)), np.fft.fft(_pack(y)), N)
        ratio = np.abs(Q).sum() / (np.linalg.norm(x) * np.linalg.norm(y))
        assert ratio <= P.Q_NORM * (1 + 1e-12)
        worst = max(worst, ratio)
    assert worst > 1.3, worst            # the factor 2 is needed, 1 would be wrong
