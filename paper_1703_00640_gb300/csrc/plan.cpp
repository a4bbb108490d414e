// Parameter selection for the three products and the FFT pass layout.
//
// Digits are balanced, |U_i| <= 2^(b-1) (the variant of Section 5); the high
// product's top digit keeps the final carry, 0 <= U_N <= 2^b. A candidate
// (b, N) must satisfy the hypotheses of Theorem 2.1 (cyclic length >= 2 N_d - 1
// with N_d b >= n + 1, so no digit carries out of the top), Theorem 2.2
// (N b >= n, N >= 3) or Theorem 2.3 ((N+1) b >= n + lg N + 2, N >= 3), and a
// worst-case FP64 error bound: (bound on |W~_i - (exact)_i|) x 2^b <= kTarget
// for the truncated products (Theorems 2.2 / 2.3 need < 1/2 after scaling by
// 2^b), or the bound itself <= kTarget for the full product. The convolution
// term is ||x||_2 ||y||_2 eta with eta = (1+u)^3K (1+sqrt5 u)^(3K+1) (1+tau)^3K - 1,
// the explicit FFT bound the paper cites in Section 2.1 (Brent-Zimmermann,
// Thm 3.6), K counting radix-2-equivalent levels of one transform. Map growth
// and truncation follow Lemmas 3.5, 3.8-3.11 and 4.7-4.11. Lengths are
// 2^a * m with m in kOddParts (Section 5 uses 2^e2 3^e3 5^e5 7^e7 with odd part
// below 200); the shortest length meeting the bound wins, ties to the larger b.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "../../include/truncmul.h"

namespace tmul {
namespace {

constexpr double kU = 1.0 / 9007199254740992.0;  // 2^-53
constexpr double kTarget = 0.45;
constexpr int kBMin = 4, kBMax = 24;
constexpr double kSpan = 1.25;
const int kOddParts[] = {1, 3, 5, 7, 9, 15, 21, 25, 27, 35, 45, 49, 63, 75, 81, 105, 125,
                         135, 147, 175, 189};

int ceil_lg(int64_t x) {  // ceil(log2 x), x >= 1
  int k = 0;
  while ((int64_t(1) << k) < x) ++k;
  return k;
}

int odd_factor_count(int64_t L) {
  int c = 0;
  for (int p : {3, 5, 7})
    while (L % p == 0) { L /= p; ++c; }
  return c;
}

// Error of one FP64 cyclic convolution of real length L as the kernels compute it:
// two forward complex FFTs of length M = L/2 (Stockham stages of radix 2, 3, 4, 5, 7
// in one to three passes, four-step twiddles between passes), the fused twist and
// pointwise product, one inverse FFT. For real inputs x, y every output satisfies
// |computed_k - (x*y)_k| <= eta_conv(L) ||x||_2 ||y||_2. Derivation (Section 2.1's
// Convolution step, with the rounding model fl(a op b) = (a op b)(1 + e), |e| <= u,
// and every table entry and DFT constant within u of its exact value):
//  - a stage's local error per butterfly is at most gamma sqrt(R) ||in||_2 in the
//    2-norm and at most delta ||in||_1 in each output (constants below, units of
//    u); the forward FFT's relative 2-norm error is eF = prod(1 + gamma_s) - 1;
//  - a forward error dZ of the packed spectrum is the spectrum of a real vector
//    of norm ||dZ|| / sqrt(M), so its effect on each output is at most
//    eF ||x|| ||y|| (Cauchy-Schwarz on the cyclic convolution), for each operand;
//  - the twist's roundings add at most kTwist (1 + eF)^2 ||x|| ||y|| to the
//    1-norm of the inverse FFT's input Q, whose 1-norm is at most
//    2 (1 + eF)^2 ||x|| ||y|| (Q_k = ((1 + i w^-k) P_k + (1 - i w^-k) P_(k+M)) / N
//    with P = X X', and |1 + i w^-k|^2 + |1 - i w^-k|^2 = 4);
//  - each inverse output's error is at most ||Q||_1 (prod(1 + delta_s) - 1): a
//    stage-s node reaches an output along one path of unit-modulus factors, and
//    the nodes of stage s that reach one output hold partial sums of disjoint
//    parts of Q.
// The layout (passes, placement of the odd primes) is the autotuner's, so the
// bound takes the worst one: every stage priced with twiddles, as many radix-2
// stages as the pass count allows, two four-step twiddle stages, except that the
// first stage of each pass multiplies by no twiddle, which every radix turns into
// a saving of at least kFirstG / kFirstD.
namespace fftbound {
constexpr double kMu = 3.0;             // product by a table twiddle: table u, cmul 2u
constexpr double kR2 = kMu + 1.0;       // radix 2 with a twiddle (both norms)
constexpr double kR4tG = 6.3;           // tangent-form radix 4: 2-norm, (sqrt(112) + 2) / 2
constexpr double kR4tD = 6.0;           // tangent-form radix 4: per output
constexpr double kR3G = 8.63;           // radix 3 in the 2-norm, derived on its own
constexpr double kR3D = 7.6;            // radix 3 per output: 3 + 1/2 + 3 sqrt3/2 + 1/2 + 1
constexpr double kR5G = 14.63;          // radix 5 in the 2-norm, derived on its own
constexpr double kR5D = 9.59;           // radix 5 per output (largest coefficient, on |x2|, |x3|)
constexpr double kR7G = 23.63;          // radix 7 in the 2-norm, derived on its own
constexpr double kR7D = 11.03;          // radix 7 per output
constexpr double kOuter = kMu;          // four-step twiddle product
constexpr double kTwist = 20.0;         // twist + pointwise roundings, relative to ||x|| ||y||
constexpr double kSlack = 1.0 + 1.0 / (1 << 20);   // second-order terms
// The first stage of a pass multiplies by no twiddle; every radix saves at least
// this much there (2-norm, per output).
constexpr double kFirstG = 2.9;
constexpr double kFirstD = 3.0;
// radix 3, 5 and 7 with twiddles: the constants of the analyses of the butterflies'
// own operation sequences
double odd_delta(int R) { return R == 3 ? kR3D : (R == 5 ? kR5D : kR7D); }
double odd_gamma(int R) { return R == 3 ? kR3G : (R == 5 ? kR5G : kR7G); }

// prod (1 + c u) over the radix stages (count[i] stages of constant c[i], the
// constants in decreasing order), the first `firsts` of them discounted by `save`:
// which stages open a pass depends on the layout, and discounting the dearest
// gives the largest product.
double radix_product(const double* c, const int* count, int kinds, int firsts, double save) {
  double p = 1.0;
  for (int i = 0; i < kinds; ++i)
    for (int j = 0; j < count[i]; ++j) {
      const double ci = firsts > 0 ? c[i] - save : c[i];
      if (firsts > 0) --firsts;
      p *= 1.0 + kSlack * ci * kU;
    }
  return p;
}
}  // namespace fftbound

double eta_conv(int64_t L) {
  using namespace fftbound;
  int64_t m = L / 2;
  int a = 0;
  while (m % 2 == 0) { m /= 2; ++a; }
  int odd[3] = {0, 0, 0};                           // stages of radix 7, 5, 3
  const int radix[3] = {7, 5, 3};
  for (int i = 0; i < 3; ++i)
    while (m % radix[i] == 0) { m /= radix[i]; ++odd[i]; }
  const double cG[5] = {odd_gamma(7), odd_gamma(5), odd_gamma(3), kR4tG, kR2};
  const double cD[5] = {odd_delta(7), odd_delta(5), odd_delta(3), kR4tD, kR2};
  double worst = 0.0;
  for (int P = 1; P <= 3; ++P) {
    int r2 = std::min(P, a);
    if ((a - r2) % 2) --r2;                         // radix-2 stages: one per pass at most
    const int count[5] = {odd[0], odd[1], odd[2], (a - r2) / 2, r2};
    const double outer = std::pow(1.0 + kSlack * kOuter * kU, P - 1);
    const double g = radix_product(cG, count, 5, P, kFirstG) * outer;
    const double d = radix_product(cD, count, 5, P, kFirstD) * outer;
    const double eF = g - 1.0, eI = d - 1.0, grow = (1.0 + eF) * (1.0 + eF);
    const double e = 2.0 * eF + eF * eF + kSlack * kTwist * kU * grow +
                     (2.0 * grow + kSlack * kTwist * kU * grow) * eI;
    worst = std::max(worst, e);
  }
  return worst;
}

// |gamma_{k,r}| <= 2^-rb exp((r-1) H_r / N): the proof of Lemma 4.7 with
// (k+r)/N + j <= (j+1)(1 + (r-1)/((j+1) N)) in place of the final estimate.
double gamma_bound(int r, int b, int64_t N) {
  if (r == 0) return 1.0;
  double h = 0;
  for (int j = 1; j <= r; ++j) h += 1.0 / j;
  return std::ldexp(std::exp((r - 1) * h / double(N)), -r * b);
}

double gamma_tail(int lam, int b, int64_t N) {
  double s = 0;
  for (int r = lam; r < lam + 64; ++r) s += gamma_bound(r, b, N);
  return s;
}

// Lemma 3.10 tail: (16/15) 2^(-lam b) <= u/4.
int lambda_alpha(int b) {
  int lam = 1;
  while (16.0 / 15.0 * std::ldexp(1.0, -lam * b) > kU / 4) ++lam;
  return lam;
}

// Tails of beta* / delta*: sum_{r>=lam} q^r with q = (1 + g) 2^-b, where
// ||X H|| <= (1 + g) ||H|| is the growth of one multiplication by X modulo A
// (g = 2^-b, inside the proof of Lemma 3.9) or C (g = 2^(1-b), Lemma 4.9).
int lambda_geometric(int b, double g) {
  const double q = (1.0 + g) * std::ldexp(1.0, -b);
  int lam = 1;
  while (std::pow(q, lam) / (1.0 - q) > kU / 4) ++lam;
  return lam;
}

int lambda_gamma(int b, int64_t N) {
  int lam = 1;
  while (gamma_tail(lam, b, N) > kU / 4) ++lam;
  return lam;
}

// rho of Lemma 4.2 by Newton's method from 2^b on y = rho / 2^b:
// y^N (y - 1) + 2^(-N b) = 0.
double rho_of(int64_t N, int b) {
  const double eps = std::ldexp(1.0, -int(std::min<int64_t>(N * b, 2000)));
  double y = 1.0;
  for (int it = 0; it < 100; ++it) {
    const double yN1 = std::pow(y, double(N - 1));
    const double f = yN1 * y * (y - 1.0) + eps;
    const double df = yN1 * ((N + 1) * y - N);
    const double yn = y - f / df;
    if (yn == y) break;
    y = yn;
  }
  return std::ldexp(y, b);
}

bool hi_hypothesis(uint64_t n, int b, int64_t N) {
  return N >= 3 && uint64_t(N + 1) * b >= n + ceil_lg(N) + 2;
}

int64_t full_digit_count(uint64_t n, int b) {
  return std::max<int64_t>(2, int64_t((n + 1 + b - 1) / b));
}

struct Bound { double E; int lf, lb; };

Bound bound_lo(int b, int64_t N) {
  const int la = lambda_alpha(b), lb = lambda_geometric(b, std::ldexp(1.0, -b));
  const double eta = eta_conv(N);
  const double g = 1.0 / (1.0 - std::ldexp(1.0, -b));           // alpha* growth
  const double S = g * std::ldexp(1.0, b - 1) * std::sqrt(double(N));  // ||U~||_2
  const double MW = S * S;                                       // |W~_i| bound
  const double din = ((la + 2) * kU + 16.0 / 15.0 * std::ldexp(1.0, -la * b)) * g *
                     std::ldexp(1.0, b - 1);                      // error of one U~_i
  const double Ein = 2.0 * std::sqrt(double(N)) * din * S * (1.0 + eta);
  const double q = (1.0 + std::ldexp(1.0, -b)) * std::ldexp(1.0, -b);
  const double A = 1.0 / (1.0 - q);                              // beta* growth
  const double tail = std::pow(q, lb) / (1.0 - q);
  const double EW = eta * MW + Ein;
  const double E = std::ldexp(A * EW + (lb + 3) * kU * A * MW + tail * MW, b);
  return {E, la, lb};
}

Bound bound_hi(int b, int64_t N) {
  const double rho = rho_of(N, b);
  const int lg = lambda_gamma(b, N), ld = lambda_geometric(b, std::ldexp(1.0, 1 - b));
  const double eta = eta_conv(N);
  double g = 0;
  for (int r = 0; r < 80; ++r) g += gamma_bound(r, b, N);       // gamma* growth
  const double kappa0 = std::ldexp(1.0, b) / rho;
  const double K2 = kappa0 / std::sqrt(1.0 - 1.0 / (rho * rho));  // ||kappa||_2
  const double S = g * (std::ldexp(1.0, b - 1) * std::sqrt(double(N)) + std::ldexp(K2, b));
  const double MW = S * S;
  const double mF = std::ldexp(1.0, b - 1) + std::ldexp(kappa0, b);  // |(F mod C)_i|
  const double din = ((lg + 4) * kU + gamma_tail(lg, b, N)) * g * mF;
  const double Ein = 2.0 * std::sqrt(double(N)) * din * S * (1.0 + eta);
  const double T = std::ldexp(1.0, b) + std::ldexp(1.0, b - 1) / (rho - 1.0);  // |theta|
  const int J = (60 + b - 1) / b + 1;
  const double Etheta = (2 * (J + 2) + 1) * kU * T * T;
  const double q = (1.0 + std::ldexp(1.0, 1 - b)) * std::ldexp(1.0, -b);
  const double A = 1.01 * (1.0 + std::ldexp(1.0, -b)) / (1.0 - q);  // delta-dagger growth
  const double tail = std::pow(q, ld) / (1.0 - q);
  const double EW = eta * MW + Ein;
  const double E =
      std::ldexp(A * (EW + Etheta) + (ld + 4) * kU * A * (MW + T * T) + tail * MW, b);
  return {E, lg, ld};
}

double bound_full(uint64_t n, int b, int64_t L) {
  const double MW = std::ldexp(double(full_digit_count(n, b)), 2 * b - 2);
  return eta_conv(L) * MW + 2.0 * kU * MW;
}

// The same bounds with measured digit norms in place of the worst case: nu, nv are
// ||U||_2, ||V||_2 of the balanced digits (high product: of F_0 .. F_(N-1)), tu, tv
// the high product's top digits F_N. Every use of the worst-case norm
// 2^(b-1) sqrt(N) (or sqrt(N_d 2^(2b-2)) for the full product) becomes the
// measured one; per-coefficient magnitudes (din, |theta|) keep their worst case.
Bound bound_lo_measured(int b, int64_t N, double nu, double nv) {
  const int la = lambda_alpha(b), lb = lambda_geometric(b, std::ldexp(1.0, -b));
  const double eta = eta_conv(N);
  const double g = 1.0 / (1.0 - std::ldexp(1.0, -b));
  const double Su = g * nu, Sv = g * nv;
  const double MW = Su * Sv;
  const double din = ((la + 2) * kU + 16.0 / 15.0 * std::ldexp(1.0, -la * b)) * g *
                     std::ldexp(1.0, b - 1);
  const double Ein = std::sqrt(double(N)) * din * (Su + Sv) * (1.0 + eta);
  const double q = (1.0 + std::ldexp(1.0, -b)) * std::ldexp(1.0, -b);
  const double A = 1.0 / (1.0 - q);
  const double tail = std::pow(q, lb) / (1.0 - q);
  const double EW = eta * MW + Ein;
  const double E = std::ldexp(A * EW + (lb + 3) * kU * A * MW + tail * MW, b);
  return {E, la, lb};
}

Bound bound_hi_measured(int b, int64_t N, double nu, double nv, double tu, double tv) {
  const double rho = rho_of(N, b);
  const int lg = lambda_gamma(b, N), ld = lambda_geometric(b, std::ldexp(1.0, 1 - b));
  const double eta = eta_conv(N);
  double g = 0;
  for (int r = 0; r < 80; ++r) g += gamma_bound(r, b, N);
  const double kappa0 = std::ldexp(1.0, b) / rho;
  const double K2 = kappa0 / std::sqrt(1.0 - 1.0 / (rho * rho));   // ||kappa||_2 / 2^b
  const double Su = g * (nu + tu * K2), Sv = g * (nv + tv * K2);
  const double MW = Su * Sv;
  const double mF = std::ldexp(1.0, b - 1) + std::ldexp(kappa0, b);
  const double din = ((lg + 4) * kU + gamma_tail(lg, b, N)) * g * mF;
  const double Ein = std::sqrt(double(N)) * din * (Su + Sv) * (1.0 + eta);
  const double T = std::ldexp(1.0, b) + std::ldexp(1.0, b - 1) / (rho - 1.0);
  const int J = (60 + b - 1) / b + 1;
  const double Etheta = (2 * (J + 2) + 1) * kU * T * T;
  const double q = (1.0 + std::ldexp(1.0, 1 - b)) * std::ldexp(1.0, -b);
  const double A = 1.01 * (1.0 + std::ldexp(1.0, -b)) / (1.0 - q);
  const double tail = std::pow(q, ld) / (1.0 - q);
  const double EW = eta * MW + Ein;
  const double E =
      std::ldexp(A * (EW + Etheta) + (ld + 4) * kU * A * (MW + T * T) + tail * MW, b);
  return {E, lg, ld};
}

double bound_full_measured(int64_t L, double nu, double nv) {
  const double MW = nu * nv;
  return eta_conv(L) * MW + 2.0 * kU * MW;
}

std::vector<int64_t> candidate_lengths(int64_t x) {
  x = std::max<int64_t>(4, x);
  const int64_t first = smooth_at_least(x);
  const int64_t top = std::max<int64_t>(first, int64_t(kSpan * double(x)));
  std::vector<int64_t> out;
  for (int m : kOddParts) {
    int64_t L = 2 * int64_t(m);
    while (L < x) L *= 2;
    for (; L <= top; L *= 2) out.push_back(L);
  }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
  return out;
}

}  // namespace

bool is_valid_length(int64_t L) {
  if (L < 4 || L % 2) return false;
  while (L % 2 == 0) L /= 2;
  for (int m : kOddParts)
    if (L == m) return true;
  return false;
}

int64_t smooth_at_least(int64_t x) {
  x = std::max<int64_t>(4, x);
  int64_t best = -1;
  for (int m : kOddParts) {
    int64_t L = 2 * int64_t(m);
    while (L < x) L *= 2;
    if (best < 0 || L < best) best = L;
  }
  return best;
}

// No heap allocation (tm_mul_static plans with it): for each b the candidate
// lengths are walked per odd part, stopping at the first certified one or at the
// shortest found so far, which gives the shortest certified length up to kSpan x
// the minimal one.
int choose_params(int kind, uint64_t n, PlanParams* out) {
  if (n == 0 || (kind != TM_FULL && kind != TM_LO && kind != TM_HI)) return TM_EINVAL;
  if (n > TM_MAX_BITS) return TM_ERANGE;
  bool found = false;
  PlanParams best;
  for (int b = kBMin; b <= kBMax; ++b) {
    int64_t lmin;
    if (kind == TM_LO) {
      lmin = std::max<int64_t>(3, int64_t((n + b - 1) / b));
    } else if (kind == TM_HI) {
      lmin = std::max<int64_t>(3, int64_t((n + 2 + b - 1) / b) - 1);
      while (!hi_hypothesis(n, b, lmin)) ++lmin;
    } else {
      lmin = 2 * full_digit_count(n, b) - 1;
    }
    const int64_t x = std::max<int64_t>(4, lmin);
    const int64_t top = std::max<int64_t>(smooth_at_least(x), int64_t(kSpan * double(x)));
    PlanParams cand;
    bool have = false;
    for (int m : kOddParts) {
      int64_t N = 2 * int64_t(m);
      while (N < x) N *= 2;
      for (; N <= top; N *= 2) {
        if (have && N >= cand.N) break;
        if (kind == TM_HI && !hi_hypothesis(n, b, N)) continue;
        double E;
        int lf = 0, lb = 0;
        int64_t nd;
        if (kind == TM_LO) {
          Bound B = bound_lo(b, N);
          E = B.E; lf = B.lf; lb = B.lb; nd = N;
        } else if (kind == TM_HI) {
          Bound B = bound_hi(b, N);
          E = B.E; lf = B.lf; lb = B.lb; nd = N + 1;
        } else {
          E = bound_full(n, b, N);
          nd = full_digit_count(n, b);
        }
        if (E <= kTarget) {
          cand.kind = kind; cand.n = n; cand.b = b; cand.N = N; cand.n_digits = nd;
          cand.lam_fwd = lf; cand.lam_bwd = lb; cand.e_max = E;
          cand.rho = kind == TM_HI ? rho_of(N, b) : 0.0;
          have = true;
          break;
        }
      }
    }
    if (have && (!found || cand.N < best.N || (cand.N == best.N && b > best.b))) {
      best = cand;
      found = true;
    }
  }
  if (!found) return TM_ERANGE;
  *out = best;
  return TM_OK;
}

int explicit_params(int kind, uint64_t n, int b, int64_t N, PlanParams* out) {
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n == 0) return TM_EINVAL;
  if (n > TM_MAX_BITS) return TM_ERANGE;
  if (b < kBMin || b > kBMax || !is_valid_length(N) || N > (int64_t(1) << 31))
    return TM_EINVAL;
  PlanParams p;
  p.kind = kind; p.n = n; p.b = b; p.N = N;
  if (kind == TM_LO) {
    if (N < 3 || uint64_t(N) * uint64_t(b) < n) return TM_EINVAL;     // Theorem 2.2
    const Bound B = bound_lo(b, N);
    p.e_max = B.E; p.lam_fwd = B.lf; p.lam_bwd = B.lb; p.n_digits = N;
  } else if (kind == TM_HI) {
    if (!hi_hypothesis(n, b, N)) return TM_EINVAL;                     // Theorem 2.3
    const Bound B = bound_hi(b, N);
    p.e_max = B.E; p.lam_fwd = B.lf; p.lam_bwd = B.lb; p.n_digits = N + 1;
    p.rho = rho_of(N, b);
  } else {
    p.n_digits = full_digit_count(n, b);
    if (N < 2 * p.n_digits - 1) return TM_EINVAL;                      // Theorem 2.1
    p.e_max = bound_full(n, b, N);
  }
  *out = p;
  return TM_OK;
}

int certified_candidates(int kind, uint64_t n, double span, int max_count,
                         std::vector<PlanParams>* out) {
  out->clear();
  PlanParams best;
  int rc = choose_params(kind, n, &best);
  if (rc) return rc;
  out->push_back(best);
  const double top = span * double(best.N);
  std::vector<PlanParams> rest;
  for (int b = kBMin; b <= kBMax; ++b) {
    int64_t lmin;
    if (kind == TM_LO) lmin = std::max<int64_t>(3, int64_t((n + b - 1) / b));
    else if (kind == TM_HI) lmin = std::max<int64_t>(3, int64_t((n + 2 + b - 1) / b) - 1);
    else lmin = 2 * full_digit_count(n, b) - 1;
    if (double(lmin) > top) continue;
    for (int64_t N : candidate_lengths(lmin)) {
      if (double(N) > top || (b == best.b && N == best.N)) continue;
      PlanParams p;
      if (explicit_params(kind, n, b, N, &p) == TM_OK && p.e_max <= kTarget) rest.push_back(p);
    }
  }
  std::sort(rest.begin(), rest.end(), [](const PlanParams& x, const PlanParams& y) {
    return x.N != y.N ? x.N < y.N : x.b > y.b;
  });
  for (const PlanParams& p : rest) {
    if (int(out->size()) >= max_count) break;
    out->push_back(p);
  }
  return TM_OK;
}

int64_t measured_length(int kind, uint64_t n, int b) {
  if (b < kBMin || b > kBMax) return -1;
  int64_t lmin;
  if (kind == TM_LO) {
    lmin = std::max<int64_t>(3, int64_t((n + b - 1) / b));
  } else if (kind == TM_HI) {
    lmin = std::max<int64_t>(3, int64_t((n + 2 + b - 1) / b) - 1);
    while (!hi_hypothesis(n, b, lmin)) ++lmin;
  } else {
    lmin = 2 * full_digit_count(n, b) - 1;
  }
  int64_t N = smooth_at_least(lmin);
  while (kind == TM_HI && !hi_hypothesis(n, b, N)) N = smooth_at_least(N + 1);
  return N;
}

double bound_target() { return kTarget; }

double conv_error_bound(int64_t L) { return eta_conv(L); }

DigitNorms worst_norms(int kind, uint64_t n, int b, int64_t N) {
  DigitNorms w;
  const double count = kind == TM_FULL ? double(full_digit_count(n, b)) : double(N);
  w.nu = w.nv = std::ldexp(std::sqrt(count), b - 1);
  w.tu = w.tv = kind == TM_HI ? std::ldexp(1.0, b) : 0.0;
  return w;
}

int measured_params(int kind, uint64_t n, int b, int64_t N, const DigitNorms& dn,
                    PlanParams* out) {
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (b < kBMin || b > kBMax || N < 4) return TM_ERANGE;
  PlanParams p;
  p.kind = kind; p.n = n; p.b = b; p.N = N;
  if (kind == TM_LO) {
    const Bound B = bound_lo_measured(b, N, dn.nu, dn.nv);
    p.e_max = B.E; p.lam_fwd = B.lf; p.lam_bwd = B.lb; p.n_digits = N;
  } else if (kind == TM_HI) {
    if (!hi_hypothesis(n, b, N)) return TM_ERANGE;
    const Bound B = bound_hi_measured(b, N, dn.nu, dn.nv, dn.tu, dn.tv);
    p.e_max = B.E; p.lam_fwd = B.lf; p.lam_bwd = B.lb; p.n_digits = N + 1;
    p.rho = rho_of(N, b);
  } else {
    p.n_digits = full_digit_count(n, b);
    if (N < 2 * p.n_digits - 1) return TM_ERANGE;
    p.e_max = bound_full_measured(N, dn.nu, dn.nv);
  }
  *out = p;                      // e_max filled even when above the target
  return p.e_max <= kTarget ? TM_OK : TM_ERANGE;
}

// ---------------------------------------------------------------- FFT plan

namespace {

// Radix stages of one sub-FFT: 7, 5, 3 for the odd part, then 4s and at most
// one 2. Radix 4 costs the same FP64 instructions per point and level as radix 8
// (3.5) and keeps one butterfly's points per thread small.
void radices_of(int L, FftPass* p) {
  p->nstages = 0;
  int rest = L;
  for (int r : {7, 5, 3})
    while (rest % r == 0) { p->radix[p->nstages++] = r; rest /= r; }
  int twos = 0;
  while (rest % 2 == 0) { rest /= 2; ++twos; }
  for (; twos >= 2; twos -= 2) p->radix[p->nstages++] = 4;
  if (twos) p->radix[p->nstages++] = 2;
}

void shape(FftPass* p, int64_t ctas_wanted, int points) {
  // sequences per CTA: fill about `points` points (default 1024, measured best
  // against 512, 2048 and 4096 at M = 2^20; the autotuner tries others), keeping
  // >= ctas_wanted CTAs; one radix-4 butterfly per thread
  int C = std::max(1, points / p->L);
  while (C > 1 && (p->Q + C - 1) / C < ctas_wanted) C /= 2;
  C = int(std::min<int64_t>(C, p->Q));
  while (int64_t(C) * p->L > kMaxCL) --C;
  p->C = std::max(1, C);
  const int t = (p->C * p->L / 4 + 31) / 32 * 32;   // one radix-4 butterfly per thread
  p->threads = std::max(32, std::min(1024, t));
}

}  // namespace

int make_fft_plan(int64_t M, FftPlan* out, bool single, const FftShape* shape_in) {
  const FftShape sh = shape_in ? *shape_in : FftShape{};
  FftPlan f;
  f.M = M;
  int primes[64];                 // no heap allocation (tm_mul_static plans with it)
  int nprimes = 0;
  int64_t rest = M;
  for (int p : {7, 5, 3, 2})
    while (rest % p == 0 && nprimes < 64) { primes[nprimes++] = p; rest /= p; }
  if (rest != 1) return TM_EINVAL;
  int np = single ? 1 : (M <= 64 ? 1 : (M <= (int64_t(1) << 22) ? 2 : 3));
  if (!single && M > 64 && (sh.passes == 2 || sh.passes == 3)) np = sh.passes;
  int64_t Ls[kMaxPasses] = {1, 1, 1};
  for (int ip = 0; ip < nprimes; ++ip) {
    const int p = primes[ip];
    int best = 0;
    if (p != 2 && sh.split == 1) {
      best = 0;                             // odd primes to the first pass
    } else if (p != 2 && sh.split == 2) {
      best = np - 1;                        // odd primes to the last pass
    } else {                                // largest first, each to the shortest
      for (int i = 1; i < np; ++i)
        if (Ls[i] < Ls[best]) best = i;
    }
    Ls[best] *= p;
  }
  for (int i = 0; i < np; ++i)
    if (Ls[i] > kMaxSubLen || (np > 1 && Ls[i] < 2)) return TM_ERANGE;
  f.npass = np;
  const int64_t want = 2 * 152;
  if (np == 1) {
    FftPass& p = f.pass[0];
    p.L = int(M); p.Q = 1; p.Qc = 1; p.IS = 1; p.OS = 1; p.Mp = 0;
  } else if (np == 2) {
    const int64_t L1 = Ls[0], L2 = Ls[1];
    FftPass& a = f.pass[0];
    a.L = int(L1); a.Q = L2; a.Qc = L2; a.IA = 0; a.IC = 1; a.IS = L2;
    a.OA = 0; a.OC = 1; a.OS = L2; a.Mp = M;
    FftPass& c = f.pass[1];
    c.L = int(L2); c.Q = L1; c.Qc = L1; c.IA = 0; c.IC = L2; c.IS = 1;
    c.OA = 0; c.OC = 1; c.OS = L1; c.Mp = 0;
  } else {
    const int64_t L1 = Ls[0], L2 = Ls[1], L3 = Ls[2], Mq = L2 * L3;
    FftPass& a = f.pass[0];
    a.L = int(L1); a.Q = Mq; a.Qc = Mq; a.IA = 0; a.IC = 1; a.IS = Mq;
    a.OA = 0; a.OC = 1; a.OS = Mq; a.Mp = M;
    FftPass& b = f.pass[1];
    b.L = int(L2); b.Q = L3 * L1; b.Qc = L3; b.IA = Mq; b.IC = 1; b.IS = L3;
    b.OA = Mq; b.OC = 1; b.OS = L3; b.Mp = Mq;
    FftPass& c = f.pass[2];
    c.L = int(L3); c.Q = L1 * L2; c.Qc = L1; c.IA = L3; c.IC = Mq; c.IS = 1;
    c.OA = L1; c.OC = 1; c.OS = L1 * L2; c.Mp = 0;
  }
  for (int i = 0; i < np; ++i) {
    radices_of(f.pass[i].L, &f.pass[i]);
    shape(&f.pass[i], want, std::max(32, sh.points));
  }
  *out = f;
  return TM_OK;
}

}  // namespace tmul
