"""The oracle's own choice of (b, N, lambda) from an FP64 error bound
(test infrastructure only; written independently of the library's planner).

Rule (a reading of the paper, which leaves b and lambda to the implementer;
Section 2.3 Scenario #2 asks for 3b + lg N + beta_N <= 53, Section 5 picks b
empirically, and the bounds below replace that by a proof-style budget):

- digits are balanced (Section 5), |U_i| <= 2^(b-1); the high product's top
  digit is unbalanced, 0 <= U_N <= 2^b;
- transform lengths are even and smooth, L = 2^a m with odd part m in ODD_PARTS
  (Section 5 restricts N to 2^e2 3^e3 5^e5 7^e7); the smallest such length that
  satisfies the method's hypothesis is used: N >= n/b (Theorem 2.2),
  (N+1) b >= n + lg N + 2 (Theorem 2.3), L >= 2 N_d - 1 with N_d b >= n + 1
  (full product, Theorem 2.1 with any cyclic length that holds the product);
- the convolution error is ||x||_2 ||y||_2 eta_conv(L), derived for the
  arithmetic of the FFT kernels (Section 2.1 leaves the Convolution step's
  explicit bound to the implementation; see eta_conv below);
- the maps' coefficient bounds follow Lemmas 3.5 and 4.7 (with the proof of
  Lemma 4.7 carried to |gamma_{k,r}| <= 2^-rb exp((r-1) H_r / N)), their norm
  growth Lemmas 3.8/3.9 and 4.8/4.9 (with ||X H|| <= (1 + 2^-b)||H|| mod A
  and <= (1 + 2^(1-b))||H|| mod C, as shown inside those proofs);
- lambda is the smallest number of terms whose truncation tail is at most u/4
  relative (Lemmas 3.10, 3.11, 4.10, 4.11);
- b is the largest value in [4, 24] whose total bound, times 2^b for the
  truncated products, is <= E_TARGET < 1/2 (Theorems 2.2 / 2.3 need < 1/2).
"""
import math

U = 2.0 ** -53
E_TARGET = 0.45
B_MIN, B_MAX = 4, 24
ODD_PARTS = (1, 3, 5, 7, 9, 15, 21, 25, 27, 35, 45, 49, 63, 75, 81, 105, 125, 135, 147,
             175, 189)
SEARCH_SPAN = 1.25   # candidate lengths up to SEARCH_SPAN x the minimal one


def ceil_log2(x: int) -> int:
    return max(0, (int(x) - 1).bit_length())


def odd_prime_factor_count(L: int) -> int:
    c = 0
    for p in (3, 5, 7):
        while L % p == 0:
            L //= p
            c += 1
    return c


def is_valid_length(L: int) -> bool:
    if L < 4 or L % 2:
        return False
    m = L
    while m % 2 == 0:
        m //= 2
    return m in ODD_PARTS


def smooth_at_least(x: int) -> int:
    x = max(4, int(x))
    best = None
    for m in ODD_PARTS:
        L = 2 * m
        while L < x:
            L *= 2
        if best is None or L < best:
            best = L
    return best


# ---------------------------------------------- error of the FP64 convolution
#
# The convolution of real length L runs as two forward complex FFTs of length
# M = L/2, the fused twist / pointwise product and one inverse FFT. Rounding model:
# every floating-point operation (and FMA) is exact times (1 + e), |e| <= U, and
# every twiddle-table entry and DFT constant is within U of its exact value.
# Per stage kind, with the butterfly input x (R complex values):
#   LOCAL_L2[kind]: ||error of the stage outputs||_2 <= c U sqrt(R) ||x||_2,
#   LOCAL_L1[kind]: |error of any one output|        <= c U ||x||_1,
# for a radix-R butterfly whose inputs 1..R-1 are first multiplied by table
# twiddles ("tw": each product within 3U |x|: U from the table, 2U from the
# complex product), the tangent-form radix-4 butterfly, and the four-step
# twiddle product between passes.
TWIDDLE_PRODUCT = 3.0
LOCAL_L1 = {"r2tw": TWIDDLE_PRODUCT + 1.0, "r4tan": 6.0, "outer": TWIDDLE_PRODUCT}
LOCAL_L2 = {"r2tw": TWIDDLE_PRODUCT + 1.0, "r4tan": (math.sqrt(112.0) + 2.0) / 2.0,
            "outer": TWIDDLE_PRODUCT}
for _R in (3, 5, 7):
    # symmetric sums / differences (1 rounding each, twiddle errors on their
    # inputs), constants within U, then (R-1)/2 roundings in each half's FMA chain
    # and one final addition: per output sqrt(2) (3 + 2) U + (R - 1) U + U of ||x||_1
    LOCAL_L1[f"r{_R}tw"] = math.sqrt(2.0) * (TWIDDLE_PRODUCT + 2.0) + (_R - 1) + 1.0
    LOCAL_L2[f"r{_R}tw"] = math.sqrt(_R) * LOCAL_L1[f"r{_R}tw"]
# Radix 3 in the 2-norm directly: with x12 = (x1, x2) the twiddle products add
# sqrt3 3U ||x12|| (through the DFT, norm sqrt3), the rounding of t = x1 + x2
# sqrt(3/2) U |t| <= sqrt3 U ||x12||, the difference d, the constant sqrt(3)/2 and
# its product each sqrt2 (sqrt3/2) U |d| <= sqrt3 U ||x12||, the FMA m = x0 - t/2
# sqrt2 U (|x0| + ||x12|| / sqrt2), the final additions U sqrt3 ||x||: in all
# 13.12 U ||x12|| + 1.415 U |x0| + 1.733 U ||x||, at most 14.93 U ||x||, which is
# 8.6213 U relative to sqrt3 ||x||, rounded up.
LOCAL_L2["r3tw"] = 8.63
# Radix 3 per output, directly. Output y1 = m + S i (sqrt3/2) d takes the twiddle
# errors 3U (|x1| + |x2|), the rounding of t through the factor 1/2, of d, of the
# constant and of its product each through sqrt3/2, the FMA m (|m| <= |x0| + |t|/2)
# and the final addition (|y1| <= ||x||_1, an output of the DFT): on |x1|, |x2| at most
# 3 + 1/2 + 3 sqrt3/2 + 1/2 + 1 = 7.598, on |x0| 2; y0 takes 3 + 1 + 1 on |x1|, |x2|.
LOCAL_L1["r3tw"] = 7.6
# Radix 5 (cos / sin of 2 pi / 5 and 4 pi / 5: c1, s1, c2, s2). Per output, y1 =
# a1 + b1 with a1 = fma(c1, t1, fma(c2, t2, x0)), b1 = S i fma(s1, d1, s2 d2),
# t_k, d_k the sums and differences of x_k and x_(5-k): on |x2|, |x3| the twiddles 3,
# the roundings of t2 and d2 (|c2| + |s2|), the constants c2 and s2 (|c2| + |s2|),
# the inner and outer FMAs (2 |c2|), the product s2 d2 and the FMA of b1 (2 |s2|), the
# final addition 1: 9.588 in all, the largest coefficient of any output (y2: 9.04 on
# |x2|, |x3|; y0: 6). In the 2-norm: the twiddles through the DFT, 3 sqrt5 ||x14||;
# the roundings of t1, t2, d1, d2 enter the outputs along orthogonal columns of norm
# sqrt(5/2), with ||(t, d)|| = sqrt2 ||x14||: sqrt5 ||x14||; the four constants
# sqrt2 (|c1| + |c2|) ||t|| + sqrt2 (|s1| + |s2|) ||d|| <= 3.805 ||x14||; each FMA or
# product rounding reaches two outputs (sqrt2) times the norm of the linear form it
# rounds (Cauchy-Schwarz): 15.715 ||x|| for the eight; t1 + t2 for y0, 2 ||x14||; the
# final roundings sqrt5 ||x||: at most 32.70 U ||x||, 14.62 U relative to sqrt5 ||x||.
LOCAL_L1["r5tw"] = 9.59
LOCAL_L2["r5tw"] = 14.63
# Radix 7 in the same way (a_m = x0 + sum_k C_mk t_k by three chained FMAs, innermost
# k = 3; b_m = S i sum_k S_mk d_k by a product and two FMAs). Per output, over each pair
# (x_k, x_(7-k)): the twiddles 3, the rounding of t_k and d_k and the errors of the two
# constants 2 (|C_mk| + |S_mk|), every FMA or product whose form contains t_k or d_k
# |C_mk| or |S_mk| each, the final addition 1: at most 11.027 (on x0: 4; y0: 7). In the
# 2-norm: twiddles 3 sqrt7 ||x16||; t, d roundings along six orthogonal columns of
# norm sqrt(7/2), sqrt7 ||x16||; the six constants, each meeting every t_k (or d_k)
# once, sqrt2 (sum |c| ||t|| + sum |s| ||d||) <= 4.98 ||x16||; the eighteen FMA and
# product roundings, sqrt2 times the norms of their forms, 39.55 ||x||; y0's two
# partial sums 2 + sqrt6; the final roundings sqrt7 ||x||: 62.50 U ||x||, 23.622 U
# relative to sqrt7 ||x||.
LOCAL_L1["r7tw"] = 11.03
LOCAL_L2["r7tw"] = 23.63
# The first stage of every pass (Ns = 1) multiplies by no twiddle. Its constants are
# at least FIRST_STAGE_L2 / FIRST_STAGE_L1 below the twiddled ones: plain radix 4
# has 2 / 2 against 6.3 / 6, radix 2 1 / 1 against 4 / 4, radix 3 5.65 / 4.6 against
# 8.63 / 7.6, radix 5 11.62 / 6.59 against 14.63 / 9.59, radix 7 20.62 / 8.03 against
# 23.63 / 11.03 (the twiddle terms, 3 sqrt(R) ||x_1..|| and 3, drop).
FIRST_STAGE_L2 = 2.9
FIRST_STAGE_L1 = 3.0
TWIST = 20.0          # roundings of the twist, relative to ||x||_2 ||y||_2 (1 + eF)^2
Q_NORM = 2.0          # ||Q||_1 <= 2 ||x||_2 ||y||_2 for the inverse FFT's input
SECOND_ORDER = 1.0 + 2.0 ** -20


def stage_lists(M: int):
    """Every stage multiset a layout of the complex FFT of length M can have, priced
    at the dearer variant (with twiddles), with its pass count: for 1, 2 and 3
    passes, the odd primes of M one stage each, the factor 2^a as radix-4 stages
    plus as many radix-2 stages as passes allow (at most one per pass, same parity
    as a), and passes - 1 four-step twiddle stages."""
    a, m = 0, M
    while m % 2 == 0:
        m //= 2
        a += 1
    odd = []
    for R in (3, 5, 7):
        while m % R == 0:
            m //= R
            odd.append(f"r{R}tw")
    assert m == 1, M
    lists = []
    for passes in (1, 2, 3):
        r2 = min(passes, a)
        if (a - r2) % 2:
            r2 -= 1
        lists.append((odd + ["r4tan"] * ((a - r2) // 2) + ["r2tw"] * r2
                      + ["outer"] * (passes - 1), passes))
    return lists


def _with_first_stages(consts, stages, passes, saving):
    """Stage constants with the first stage of each pass untwiddled. Which stages
    come first depends on the layout; taking the saving from the dearest radix
    stages leaves the largest product, so the bound holds for every layout."""
    radix = sorted((consts[k] for k in stages if k != "outer"), reverse=True)
    outer = [consts[k] for k in stages if k == "outer"]
    for i in range(min(passes, len(radix))):
        radix[i] -= saving
    return radix + outer


def eta_conv(L: int) -> float:
    """Bound eta with |computed_k - (x*y)_k| <= eta ||x||_2 ||y||_2 for the FP64 cyclic
    convolution of real length L (Section 2.1's Convolution step) as the FFT kernels
    compute it: the forward errors eF (2-norm) of both operands, the twist's
    roundings, and the inverse FFT's per-output error on an input of 1-norm
    Q_NORM (1 + eF)^2 ||x|| ||y||; the worst of the possible layouts, each pass's
    first stage untwiddled."""
    worst = 0.0
    for stages, passes in stage_lists(L // 2):
        g = _with_first_stages(LOCAL_L2, stages, passes, FIRST_STAGE_L2)
        d = _with_first_stages(LOCAL_L1, stages, passes, FIRST_STAGE_L1)
        eF = math.prod(1.0 + SECOND_ORDER * c * U for c in g) - 1.0
        eI = math.prod(1.0 + SECOND_ORDER * c * U for c in d) - 1.0
        grow = (1.0 + eF) ** 2
        twist = SECOND_ORDER * TWIST * U * grow
        worst = max(worst, 2.0 * eF + eF * eF + twist + (Q_NORM * grow + twist) * eI)
    return worst


_H = [0.0]
for _j in range(1, 400):
    _H.append(_H[-1] + 1.0 / _j)


def harmonic(r: int) -> float:
    return _H[r]


def gamma_coef_bound(r: int, b: int, N: int) -> float:
    return 2.0 ** (-r * b) * math.exp((r - 1) * harmonic(r) / N) if r else 1.0


def lam_alpha(b: int) -> int:
    lam = 1
    while (16.0 / 15.0) * 2.0 ** (-lam * b) > U / 4:
        lam += 1
    return lam


def _lam_geometric(b: int, grow: float) -> int:
    q = grow * 2.0 ** -b
    lam = 1
    while q ** lam / (1 - q) > U / 4:
        lam += 1
    return lam


def lam_beta(b: int) -> int:
    return _lam_geometric(b, 1 + 2.0 ** -b)


def lam_delta(b: int) -> int:
    return _lam_geometric(b, 1 + 2.0 ** (1 - b))


def gamma_tail(lam: int, b: int, N: int) -> float:
    return sum(gamma_coef_bound(r, b, N) for r in range(lam, lam + 64))


def lam_gamma(b: int, N: int) -> int:
    lam = 1
    while gamma_tail(lam, b, N) > U / 4:
        lam += 1
    return lam


def rho_float(N: int, b: int) -> float:
    """Newton on B(z) = z^(N+1) - 2^b z^N + 2^b in the scaled form y = z/2^b:
    y^N (y - 1) + 2^-Nb = 0 (proof of Lemma 4.2); float is enough for the bound."""
    eps = 2.0 ** (-N * b)
    y = 1.0
    for _ in range(100):
        f = y ** N * (y - 1.0) + eps
        df = y ** (N - 1) * ((N + 1) * y - N)
        y_new = y - f / df
        if y_new == y:
            break
        y = y_new
    return y * 2.0 ** b


def min_len_lo(n: int, b: int) -> int:
    """Theorem 2.2: N >= n/b, N >= 3."""
    return max(3, -(-n // b))


def hi_ok(n: int, b: int, N: int) -> bool:
    """Theorem 2.3: (N + 1) b >= n + lg N + 2, N >= 3."""
    return N >= 3 and (N + 1) * b >= n + ceil_log2(N) + 2


def min_len_hi(n: int, b: int) -> int:
    N = max(3, -(-(n + 2) // b) - 1)      # ignores lg N, so it is a lower bound
    while not hi_ok(n, b, N):
        N += 1
    return N


def full_digits(n: int, b: int) -> int:
    """Balanced digits without a carry out of the top one need N_d b >= n + 1."""
    return max(2, -(-(n + 1) // b))


def bound_lo(n: int, b: int, N: int):
    la, lb = lam_alpha(b), lam_beta(b)
    eta = eta_conv(N)
    g = 1.0 / (1.0 - 2.0 ** -b)
    S = g * 2.0 ** (b - 1) * math.sqrt(N)
    MW = S * S
    d_in = ((la + 2) * U + (16.0 / 15.0) * 2.0 ** (-la * b)) * g * 2.0 ** (b - 1)
    E_in = 2.0 * math.sqrt(N) * d_in * S * (1.0 + eta)
    A = 1.0 / (1.0 - (1.0 + 2.0 ** -b) * 2.0 ** -b)
    q = (1.0 + 2.0 ** -b) * 2.0 ** -b
    tail = q ** lb / (1.0 - q)
    E_W = eta * MW + E_in
    E = 2.0 ** b * (A * E_W + (lb + 3) * U * A * MW + tail * MW)
    return E, N, la, lb


def bound_hi(n: int, b: int, N: int):
    rho = rho_float(N, b)
    lg, ld = lam_gamma(b, N), lam_delta(b)
    eta = eta_conv(N)
    g = sum(gamma_coef_bound(r, b, N) for r in range(0, 80))
    kappa0 = 2.0 ** b / rho
    K2 = kappa0 / math.sqrt(1.0 - rho ** -2)
    S = g * (2.0 ** (b - 1) * math.sqrt(N) + 2.0 ** b * K2)
    MW = S * S
    m_F = 2.0 ** (b - 1) + 2.0 ** b * kappa0
    d_in = ((lg + 4) * U + gamma_tail(lg, b, N)) * g * m_F
    E_in = 2.0 * math.sqrt(N) * d_in * S * (1.0 + eta)
    T = 2.0 ** b + 2.0 ** (b - 1) / (rho - 1.0)
    J = -(-60 // b) + 1
    E_theta = (2 * (J + 2) + 1) * U * T * T
    q = (1.0 + 2.0 ** (1 - b)) * 2.0 ** -b
    A = 1.01 * (1.0 + 2.0 ** -b) / (1.0 - q)
    tail = q ** ld / (1.0 - q)
    E_W = eta * MW + E_in
    E = 2.0 ** b * (A * (E_W + E_theta) + (ld + 4) * U * A * (MW + T * T) + tail * MW)
    return E, N, lg, ld


def bound_full(n: int, b: int, L: int):
    Nd = full_digits(n, b)
    eta = eta_conv(L)
    MW = 2.0 ** (2 * b - 2) * Nd
    E = eta * MW + 2.0 * U * MW
    return E, L, Nd


def smooth_lengths_from(x: int, span: float = SEARCH_SPAN):
    """Valid transform lengths in [x, span * x] (at least one), increasing."""
    x = max(4, int(x))
    first = smooth_at_least(x)
    out = set()
    top = max(first, int(span * x))
    for m in ODD_PARTS:
        L = 2 * m
        while L < x:
            L *= 2
        while L <= top:
            out.add(L)
            L *= 2
    return sorted(out)


def choose(kind: str, n: int) -> dict:
    """For each b in [B_MIN, B_MAX], the shortest valid length (searched up to
    SEARCH_SPAN x the minimal one) whose bound is <= E_TARGET; then the b whose
    length is shortest (ties: the larger b). Keys: kind, n, b, N (transform
    length), n_digits, lam_fwd, lam_bwd, e_max."""
    assert n >= 1
    best = None
    for b in range(B_MIN, B_MAX + 1):
        if kind == "lo":
            lmin = min_len_lo(n, b)
        elif kind == "hi":
            lmin = min_len_hi(n, b)
        elif kind == "full":
            lmin = 2 * full_digits(n, b) - 1
        else:
            raise ValueError(kind)
        for N in smooth_lengths_from(lmin):
            if kind == "hi" and not hi_ok(n, b, N):
                continue
            if kind == "lo":
                E, _, lf, lb = bound_lo(n, b, N)
                nd = N
            elif kind == "hi":
                E, _, lf, lb = bound_hi(n, b, N)
                nd = N + 1
            else:
                E, _, nd = bound_full(n, b, N)
                lf = lb = 0
            if E <= E_TARGET:
                cand = {"kind": kind, "n": n, "b": b, "N": N, "n_digits": nd,
                        "lam_fwd": lf, "lam_bwd": lb, "e_max": E}
                if best is None or N < best["N"] or (N == best["N"] and b > best["b"]):
                    best = cand
                break
    if best is None:
        raise ValueError(f"no FP64 plan for {kind} n={n}")
    return best


# ------------------------------------------------ measured digit norms

def bound_lo_measured(b: int, N: int, nu: float, nv: float) -> float:
    """bound_lo with the measured norms ||U||_2, ||V||_2 of the balanced digits in
    place of the worst case 2^(b-1) sqrt(N); per-coefficient terms unchanged."""
    la, lb = lam_alpha(b), lam_beta(b)
    eta = eta_conv(N)
    g = 1.0 / (1.0 - 2.0 ** -b)
    Su, Sv = g * nu, g * nv
    MW = Su * Sv
    d_in = ((la + 2) * U + (16.0 / 15.0) * 2.0 ** (-la * b)) * g * 2.0 ** (b - 1)
    E_in = math.sqrt(N) * d_in * (Su + Sv) * (1.0 + eta)
    q = (1.0 + 2.0 ** -b) * 2.0 ** -b
    A = 1.0 / (1.0 - q)
    tail = q ** lb / (1.0 - q)
    return 2.0 ** b * (A * (eta * MW + E_in) + (lb + 3) * U * A * MW + tail * MW)


def bound_hi_measured(b: int, N: int, nu: float, nv: float, tu: float, tv: float) -> float:
    """bound_hi with ||F_0..F_(N-1)||_2 measured and the top digits F_N measured."""
    rho = rho_float(N, b)
    lg, ld = lam_gamma(b, N), lam_delta(b)
    eta = eta_conv(N)
    g = sum(gamma_coef_bound(r, b, N) for r in range(0, 80))
    kappa0 = 2.0 ** b / rho
    K2 = kappa0 / math.sqrt(1.0 - rho ** -2)
    Su, Sv = g * (nu + tu * K2), g * (nv + tv * K2)
    MW = Su * Sv
    m_F = 2.0 ** (b - 1) + 2.0 ** b * kappa0
    d_in = ((lg + 4) * U + gamma_tail(lg, b, N)) * g * m_F
    E_in = math.sqrt(N) * d_in * (Su + Sv) * (1.0 + eta)
    T = 2.0 ** b + 2.0 ** (b - 1) / (rho - 1.0)
    J = -(-60 // b) + 1
    E_theta = (2 * (J + 2) + 1) * U * T * T
    q = (1.0 + 2.0 ** (1 - b)) * 2.0 ** -b
    A = 1.01 * (1.0 + 2.0 ** -b) / (1.0 - q)
    tail = q ** ld / (1.0 - q)
    return 2.0 ** b * (A * (eta * MW + E_in + E_theta) + (ld + 4) * U * A * (MW + T * T)
                       + tail * MW)


def bound_full_measured(L: int, nu: float, nv: float) -> float:
    MW = nu * nv
    return eta_conv(L) * MW + 2.0 * U * MW


def measured_length(kind: str, n: int, b: int) -> int:
    """The shortest admissible length for digit size b (hypotheses only)."""
    if kind == "lo":
        return smooth_at_least(min_len_lo(n, b))
    if kind == "hi":
        N = smooth_at_least(min_len_hi(n, b))
        while not hi_ok(n, b, N):
            N = smooth_at_least(N + 1)
        return N
    return smooth_at_least(2 * full_digits(n, b) - 1)


def adaptive_choice(kind: str, n: int, u: int, v: int) -> dict:
    """The plan of the data-dependent digit size: the worst-case plan's b plus one,
    at its shortest admissible length, when the bound on the operands' measured
    digit norms is <= E_TARGET and that length is shorter (b + 1 is then
    certified for these operands); else the worst-case plan. Norms come from the
    balanced digits of the split step (trace.split). A caller may still keep the
    worst-case plan where b + 1 is admissible (for example to skip measuring)."""
    from . import trace
    base = choose(kind, n)
    b = base["b"] + 1
    if b > B_MAX:
        return base
    N = measured_length(kind, n, b)
    if N >= base["N"]:
        return base
    count = full_digits(n, b) if kind == "full" else N
    du = trace.split(kind, u, n, b, count)
    dv = trace.split(kind, v, n, b, count)
    if kind == "hi":
        nu = math.sqrt(sum(d * d for d in du[:N]))
        nv = math.sqrt(sum(d * d for d in dv[:N]))
        E = bound_hi_measured(b, N, nu, nv, float(abs(du[N])), float(abs(dv[N])))
        lf, lb, nd = lam_gamma(b, N), lam_delta(b), N + 1
    else:
        nu = math.sqrt(sum(d * d for d in du))
        nv = math.sqrt(sum(d * d for d in dv))
        if kind == "lo":
            E = bound_lo_measured(b, N, nu, nv)
            lf, lb, nd = lam_alpha(b), lam_beta(b), N
        else:
            E = bound_full_measured(N, nu, nv)
            lf, lb, nd = 0, 0, count
    if E > E_TARGET:
        return base
    return {"kind": kind, "n": n, "b": b, "N": N, "n_digits": nd, "lam_fwd": lf,
            "lam_bwd": lb, "e_max": E}
