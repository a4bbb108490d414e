// Device kernels of the truncated-product pipeline (sm_103a).
//
// On GB300 the FP64 pipe is the scarce resource (about 1/37 of the integer
// rate), so every step that does not need FP64 arithmetic runs on the integer
// pipe: digit extraction, int -> double conversion (built from the IEEE-754
// fields), double -> int64 rounding with its distance to the integer, and the
// carry scan. FP64 is spent on the maps and the FFT.
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "../../include/truncmul.h"

namespace tmul {

// ------------------------------------------------------------ constants

// The radix-3/5/7 and radix-8 DFT constants, each the double nearest to its exact
// value (hex literals; the error bound takes every constant within 2^-53 of it).
constexpr double kC5_1 = 0x1.3c6ef372fe950p-2;    // cos(2 pi/5)   0.30901699437494745
constexpr double kC5_2 = -0x1.9e3779b97f4a8p-1;   // cos(4 pi/5)  -0.8090169943749475
constexpr double kS5_1 = 0x1.e6f0e134454ffp-1;    // sin(2 pi/5)   0.9510565162951535
constexpr double kS5_2 = 0x1.2cf2304755a5ep-1;    // sin(4 pi/5)   0.5877852522924731
constexpr double kC7_1 = 0x1.3f3a0e28bedd1p-1;    // cos(2 pi k/7), k = 1, 2, 3
constexpr double kC7_2 = -0x1.c7b90e3024582p-3;
constexpr double kC7_3 = -0x1.cd4bca9cb5c71p-1;
constexpr double kS7_1 = 0x1.904c37505de4bp-1;    // sin(2 pi k/7)
constexpr double kS7_2 = 0x1.f329c0558e969p-1;
constexpr double kS7_3 = 0x1.bc4c04d71abc1p-2;
constexpr double kSqrt3_2 = 0x1.bb67ae8584caap-1; // sqrt(3)/2

// ------------------------------------------------------- complex helpers

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 w) {
  return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 w) {  // a * conj(w)
  return make_double2(fma(a.x, w.x, a.y * w.y), fma(a.y, w.x, -a.x * w.y));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// a * (S i): S = -1 gives -i a = (a.y, -a.x); S = +1 gives i a = (-a.y, a.x)
template <int S>
__device__ __forceinline__ double2 mul_si(double2 a) {
  return S < 0 ? make_double2(a.y, -a.x) : make_double2(-a.y, a.x);
}

// ------------------------------------------- integer <-> double, exactly

// |x| < 2^53: the double with value x, built from its sign, exponent and
// mantissa fields on the integer pipe.
__device__ __forceinline__ double i2d_exact(long long x) {
  const unsigned long long sgn = (unsigned long long)x & 0x8000000000000000ull;
  const unsigned long long a = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  const int e = 63 - __clzll(a | 1ull);               // a in [2^e, 2^(e+1)); a = 0 -> e = 0
  const unsigned long long m = (a << (52 - e)) & 0xFFFFFFFFFFFFFull;
  const unsigned long long bits = sgn | ((unsigned long long)(e + 1023) << 52) | m;
  return a ? __longlong_as_double((long long)bits) : 0.0;
}

// x * 2^k for finite x (result stays normal): add k to the exponent field.
__device__ __forceinline__ double scale2(double x, int k) {
  const long long bits = __double_as_longlong(x);
  return (bits & 0x7FF0000000000000ll) ? __longlong_as_double(bits + ((long long)k << 52)) : x;
}

// Rounds x (|x| < 2^62) to the nearest integer c (ties to even) and returns the
// distance |x - c| in units of 2^-63 (<= 2^62). Integer pipe only.
__device__ __forceinline__ long long round_dist(double x, unsigned long long* dist) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ef = int((bits >> 52) & 0x7FF);
  const int e = ef - 1023;
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
  unsigned long long q, d;
  if (e < -1) {                       // |x| < 1/2 (or zero / subnormal)
    q = 0;
    const int sh = e + 11;            // x = mant 2^(e-52) = mant 2^(sh-63)
    d = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
  } else if (e >= 52) {               // already an integer
    q = mant << (e - 52);
    d = 0;
  } else {
    const int shift = 52 - e;         // 1 .. 53
    q = mant >> shift;
    const unsigned long long rem = mant & ((1ull << shift) - 1ull);
    const unsigned long long half = 1ull << (shift - 1);
    const bool up = rem > half || (rem == half && (q & 1ull));
    q += up ? 1ull : 0ull;
    d = (up ? (1ull << shift) - rem : rem) << (63 - shift);
  }
  *dist = d;
  return (bits >> 63) ? -(long long)q : (long long)q;
}

// -------------------------------------------------------- table kernels

// Every twiddle table entry is computed in double-double arithmetic and rounded
// once, so each stored component is within 2^-53 (1 + 2^-40) of its exact value;
// the FFT error bound relies on that. Error-free transformations: Knuth's
// two-sum and the FMA form of Dekker's exact product; double-double sums,
// products and quotients after Dekker (1971), each with relative error below
// 2^-100 for the operands used here.
struct DD {
  double hi, lo;
};

// (The operations use the _rn intrinsics, which the compiler never contracts
// into FMAs: the transformations need every sum and product rounded as written.)
__device__ __forceinline__ DD dd_two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  return DD{s, __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb))};
}

__device__ __forceinline__ DD dd_fast_two_sum(double a, double b) {   // |a| >= |b| or a = 0
  const double s = __dadd_rn(a, b);
  return DD{s, __dsub_rn(b, __dsub_rn(s, a))};
}

__device__ __forceinline__ DD dd_add(DD x, DD y) {
  DD s = dd_two_sum(x.hi, y.hi);
  const DD t = dd_two_sum(x.lo, y.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = dd_fast_two_sum(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return dd_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ DD dd_mul(DD x, DD y) {
  const double p = __dmul_rn(x.hi, y.hi);
  const double e = __fma_rn(x.hi, y.hi, -p);
  const double c = __dadd_rn(__dmul_rn(x.hi, y.lo), __dmul_rn(x.lo, y.hi));
  return dd_fast_two_sum(p, __dadd_rn(e, c));
}

// x / y for a double y != 0: the quotient of the leading parts, then one
// correction from the remainder (x.hi - q1 y is formed exactly)
__device__ __forceinline__ DD dd_div_d(DD x, double y) {
  const double q1 = __ddiv_rn(x.hi, y);
  const double p = __dmul_rn(q1, y);
  const double pe = __fma_rn(q1, y, -p);     // q1 y = p + pe exactly
  DD r = dd_two_sum(x.hi, -p);
  r.lo = __dadd_rn(r.lo, __dsub_rn(x.lo, pe));
  const double q2 = __ddiv_rn(__dadd_rn(r.hi, r.lo), y);
  return dd_fast_two_sum(q1, q2);
}

__device__ __forceinline__ DD dd_neg(DD x) { return DD{-x.hi, -x.lo}; }

// pi / 2 to 2^-109 relative
__device__ __constant__ const double kPi2Hi = 0x1.921fb54442d18p+0;
__device__ __constant__ const double kPi2Lo = 0x1.1a62633145c07p-54;

__device__ __forceinline__ DD dd_mul_d(DD x, double y) {
  const double p = __dmul_rn(x.hi, y);
  const double e = __fma_rn(x.hi, y, -p);
  return dd_fast_two_sum(p, __dadd_rn(e, __dmul_rn(x.lo, y)));
}

// cos and sin of j pi / 32, j = 0..8, as double-double (cos hi, lo, sin hi, lo), and
// 1/k!, k = 0..15 (hi, lo): constants written out to 2^-106
__device__ __constant__ const double kTrig32[9][4] = {
    {0x1.0000000000000p+0, 0x0.0p+0, 0x0.0p+0, 0x0.0p+0},
    {0x1.fd88da3d12526p-1, -0x1.87df6378811c7p-55, 0x1.917a6bc29b42cp-4, -0x1.e2718d26ed688p-60},
    {0x1.f6297cff75cb0p-1, 0x1.562172a361fd3p-56, 0x1.8f8b83c69a60bp-3, -0x1.26d19b9ff8d82p-57},
    {0x1.e9f4156c62ddap-1, 0x1.760b1e2e3f81ep-55, 0x1.294062ed59f06p-2, -0x1.5d28da2c4612dp-56},
    {0x1.d906bcf328d46p-1, 0x1.457e610231ac2p-56, 0x1.87de2a6aea963p-2, -0x1.72cedd3d5a610p-57},
    {0x1.c38b2f180bdb1p-1, -0x1.6e0b1757c8d07p-56, 0x1.e2b5d3806f63bp-2, 0x1.e0d891d3c6841p-58},
    {0x1.a9b66290ea1a3p-1, 0x1.9f630e8b6dac8p-60, 0x1.1c73b39ae68c8p-1, 0x1.b25dd267f6600p-55},
    {0x1.8bc806b151741p-1, -0x1.2c5e12ed1336dp-55, 0x1.44cf325091dd6p-1, 0x1.8076a2cfdc6b3p-57},
    {0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55, 0x1.6a09e667f3bcdp-1, -0x1.bdd3413b26456p-55}};
__device__ __constant__ const double kInvFact[16][2] = {
    {0x1.0000000000000p+0, 0x0.0p+0},          {0x1.0000000000000p+0, 0x0.0p+0},
    {0x1.0000000000000p-1, 0x0.0p+0},          {0x1.5555555555555p-3, 0x1.5555555555555p-57},
    {0x1.5555555555555p-5, 0x1.5555555555555p-59}, {0x1.1111111111111p-7, 0x1.1111111111111p-63},
    {0x1.6c16c16c16c17p-10, -0x1.f49f49f49f49fp-65}, {0x1.a01a01a01a01ap-13, 0x1.a01a01a01a01ap-73},
    {0x1.a01a01a01a01ap-16, 0x1.a01a01a01a01ap-76}, {0x1.71de3a556c734p-19, -0x1.c154f8ddc6c00p-73},
    {0x1.27e4fb7789f5cp-22, 0x1.cbbc05b4fa99ap-76}, {0x1.ae64567f544e4p-26, -0x1.c062e06d1f209p-80},
    {0x1.1eed8eff8d898p-29, -0x1.2aec959e14c06p-83}, {0x1.6124613a86d09p-33, 0x1.f28e0cc748ebep-87},
    {0x1.93974a8c07c9dp-37, 0x1.05d6f8a2efd1fp-92}, {0x1.ae7f3e733b81fp-41, 0x1.1d8656b0ee8cbp-97}};

// sin x and cos x for 0 <= x <= pi/4: x = j pi/32 + y with |y| <= pi/64, the Taylor
// series of sin y and cos y to the terms of degree 15 / 14 by Horner's rule in y^2
// (the next terms are below 2^-110 of the sums), then the angle-addition formulas
// with the table's cos and sin of j pi/32.
__device__ void dd_sincos_small(DD x, DD* sn, DD* cs) {
  int j = int(rint(x.hi * (32.0 / 3.141592653589793)));
  j = j < 0 ? 0 : (j > 8 ? 8 : j);
  const DD pi32 = DD{kPi2Hi * 0.0625, kPi2Lo * 0.0625};          // exact: a power of two
  const DD y = dd_add(x, dd_neg(dd_mul_d(pi32, double(j))));
  const DD z = dd_mul(y, y);
  DD S = DD{-kInvFact[15][0], -kInvFact[15][1]};                  // sum (-z)^i / (2i+1)!
  DD C = DD{-kInvFact[14][0], -kInvFact[14][1]};                  // sum (-z)^i / (2i)!
  for (int i = 6; i >= 0; --i) {
    const double sg = (i & 1) ? -1.0 : 1.0;
    S = dd_add(dd_mul(S, z), DD{sg * kInvFact[2 * i + 1][0], sg * kInvFact[2 * i + 1][1]});
    C = dd_add(dd_mul(C, z), DD{sg * kInvFact[2 * i][0], sg * kInvFact[2 * i][1]});
  }
  const DD sy = dd_mul(y, S), cy = C;
  const DD cj = DD{kTrig32[j][0], kTrig32[j][1]}, sj = DD{kTrig32[j][2], kTrig32[j][3]};
  *cs = dd_add(dd_mul(cj, cy), dd_neg(dd_mul(sj, sy)));
  *sn = dd_add(dd_mul(sj, cy), dd_mul(cj, sy));
}

// cos and sin of 2 pi m / len in double-double. The angle is reduced with
// integers to a quadrant and a complement, leaving pi/2 (r / len) with
// r / len in [0, 1/2].
__device__ void dd_cossin_2pi(long long m, long long len, DD* cs, DD* sn) {
  const long long m4 = 4 * m;
  const long long q = m4 / len;              // quadrant 0..3
  long long r = m4 - q * len;                // angle = pi/2 (q + r/len)
  bool swap = false;
  if (2 * r > len) { r = len - r; swap = true; }   // use the complement angle
  const DD frac = dd_div_d(DD{double(r), 0.0}, double(len));
  DD s, c;
  dd_sincos_small(dd_mul(DD{kPi2Hi, kPi2Lo}, frac), &s, &c);
  if (swap) { const DD t = s; s = c; c = t; }
  switch (q) {
    case 0: *cs = c; *sn = s; break;
    case 1: *cs = dd_neg(s); *sn = c; break;
    case 2: *cs = dd_neg(c); *sn = dd_neg(s); break;
    default: *cs = s; *sn = dd_neg(c); break;
  }
}

// The table kernels take runs of kTwRun consecutive entries per thread: the run's
// first angle from the Taylor series, the others by rotation with the one-step
// twiddle (double-double complex products; after a run the error stays below
// 2^-95, far below the rounding to double). Entries whose cosine or sine is
// exactly 0 or +-1 (4m a multiple of len) take the exact values.
constexpr int kTwRun = 16;
constexpr int kTwThreads = 64;

// (c + i s) <- (c + i s)(c1 + i s1)
__device__ __forceinline__ void dd_rotate(DD& c, DD& s, const DD c1, const DD s1) {
  const DD cc = dd_add(dd_mul(c, c1), dd_neg(dd_mul(s, s1)));
  const DD ss = dd_add(dd_mul(s, c1), dd_mul(c, s1));
  c = cc;
  s = ss;
}

__device__ __forceinline__ void dd_exact_axes(long long m, long long len, DD* c, DD* s) {
  if ((4 * m) % len == 0) {
    const int q = int(((4 * m) / len) & 3);
    *c = DD{q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0), 0.0};
    *s = DD{q == 1 ? 1.0 : (q == 3 ? -1.0 : 0.0), 0.0};
  }
}

// cos and sin of 2 pi / len for the whole block (thread 0 computes, all read)
__device__ void dd_block_step(long long step, long long len, DD* c1, DD* s1) {
  __shared__ DD sc, ss;
  if (threadIdx.x == 0) dd_cossin_2pi(step, len, &sc, &ss);
  __syncthreads();
  *c1 = sc;
  *s1 = ss;
}

// tab[m] = exp(-2 pi i m / len), m < count, each component rounded once.
__global__ void __launch_bounds__(kTwThreads) k_init_twiddles(double2* tab, long long len,
                                                                long long count) {
  DD c1, s1;
  dd_block_step(1, len, &c1, &s1);
  const long long m0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * kTwRun;
  if (m0 >= count) return;
  DD c, s;
  dd_cossin_2pi(m0, len, &c, &s);
  for (int i = 0; i < kTwRun && m0 + i < count; ++i) {
    if (i) dd_rotate(c, s, c1, s1);
    DD cc = c, ss = s;
    dd_exact_axes(m0 + i, len, &cc, &ss);
    tab[m0 + i] = make_double2(cc.hi, -ss.hi);
  }
}

// tab[k Qc + qc] = exp(-2 pi i (qc k mod Mp) / Mp), qc < Qc, k < Mp / Qc: the four-step
// twiddles in the order a pass stores its outputs (output k of sequence qc), so
// that the consecutive sequences of a warp read consecutive entries. Along a row
// the exponent steps by k: a run rotates by exp(-2 pi i k / Mp) and starts over
// where it enters the next row.
__global__ void __launch_bounds__(kTwThreads) k_init_outer(double2* tab, long long Mp,
                                                             long long Qc) {
  const long long e0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * kTwRun;
  if (e0 >= Mp) return;
  long long k = e0 / Qc, qc = e0 - k * Qc;
  DD c, s, c1, s1;
  for (int i = 0; i < kTwRun && e0 + i < Mp; ++i) {
    const long long m = (qc * k) % Mp;
    if (i == 0 || qc == 0) {
      dd_cossin_2pi(m, Mp, &c, &s);
      dd_cossin_2pi(k, Mp, &c1, &s1);
    } else {
      dd_rotate(c, s, c1, s1);
    }
    DD cc = c, ss = s;
    dd_exact_axes(m, Mp, &cc, &ss);
    tab[e0 + i] = make_double2(cc.hi, -ss.hi);
    if (++qc == Qc) { qc = 0; ++k; }
  }
}

// tab[k] = (1 + w^2) / (2N) = cos(2 pi k / N) w / N, w = exp(-2 pi i k / N), k < count:
// the one twiddle of the fused real-FFT twist (see twist_pair), each component
// rounded once.
__global__ void __launch_bounds__(kTwThreads) k_init_twist_coef(double2* tab, long long N,
                                                                  long long count) {
  DD c1, s1;
  dd_block_step(1, N, &c1, &s1);
  const long long k0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * kTwRun;
  if (k0 >= count) return;
  DD c, s;
  dd_cossin_2pi(k0, N, &c, &s);
  for (int i = 0; i < kTwRun && k0 + i < count; ++i) {
    if (i) dd_rotate(c, s, c1, s1);
    DD cs = c, sn = s;
    dd_exact_axes(k0 + i, N, &cs, &sn);
    const DD re = dd_div_d(dd_mul(cs, cs), double(N));
    const DD im = dd_div_d(dd_mul(cs, sn), double(N));
    tab[k0 + i] = make_double2(re.hi, -im.hi);
  }
}

// Tangent-form twiddles of a radix-4 stage (see launch_init_tw4). The cosine c is
// rounded first and the tangent is taken as the double nearest to sin / c (with
// the rounded c), so the twiddle c (1 - i t) the butterfly applies is within
// 2^-53 (1 + 2^-40) of exp(-i theta), as for a rounded (cos, sin) pair.
__global__ void __launch_bounds__(kTwThreads) k_init_tw4(Tan4* tab, int Ns) {
  const long long len = 4LL * Ns;
  DD a1, b1, a2, b2;                                  // steps of theta and of 2 theta
  dd_block_step(1, len, &a1, &b1);
  __syncthreads();
  dd_block_step(2, len, &a2, &b2);
  const long long k0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) * kTwRun;
  if (k0 >= Ns) return;
  DD c1, s1, c2, s2;
  dd_cossin_2pi(k0, len, &c1, &s1);                   // theta = 2 pi k / (4 Ns) < pi/2
  dd_cossin_2pi(2 * k0, len, &c2, &s2);               // 2 theta
  for (int i = 0; i < kTwRun && k0 + i < Ns; ++i) {
    const long long k = k0 + i;
    if (i) {
      dd_rotate(c1, s1, a1, b1);
      dd_rotate(c2, s2, a2, b2);
    }
    DD x1 = c1, y1 = s1, x2 = c2, y2 = s2;
    dd_exact_axes(k, len, &x1, &y1);
    dd_exact_axes(2 * k, len, &x2, &y2);
    const bool rot = 2 * k >= Ns;                     // 2 theta >= pi/2: use 2 theta - pi/2
    const DD cw = rot ? y2 : x2;                      // cos(2 theta - pi/2) = sin 2 theta
    const DD sw = rot ? dd_neg(x2) : y2;              // sin(2 theta - pi/2) = -cos 2 theta
    Tan4 e;
    e.c1 = x1.hi;
    e.t1 = dd_div_d(y1, e.c1).hi;
    e.t2 = dd_div_d(sw, cw.hi).hi;
    e.c2s = rot ? -cw.hi : cw.hi;
    tab[k] = e;
  }
}

// Coefficient rows of the ring maps (Sections 3.2 and 4.2), tab[(r-1) N + k]:
//   alpha_{k,r} = k/(k+r) binom((k+r)/N, r) (-2^-b)^r
//   beta_{k,r}  = binom(-k/N, r) (-2^-b)^r
//   gamma_{k,r} = k/(k+r) binom(-(k+r)/N, r) (-2^-b)^r
//   delta_{k,r} = binom(k/N, r) (-2^-b)^r
// and for the high product's back map the combined rows
//   delta'_{k,r} = delta_{k,r} - 2^-b delta_{k,r-1}, r = 1..rows (delta_{k,rows} := 0),
// the coefficients of (1 - 2^-b X) delta*.
__device__ double binom_scaled(double x, int r, int b) {
  double acc = 1.0;
  for (int j = 0; j < r; ++j) acc *= (x - j) / (j + 1);
  return acc * ((r & 1) ? -1.0 : 1.0) * scale2(1.0, -r * b);
}

__global__ void k_init_maptab(double* tab, int which, long long N, int b, int rows) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= N) return;
  const double dk = (double)k, dN = (double)N;
  for (int r = 1; r <= rows; ++r) {
    double v;
    switch (which) {
      case kTabAlpha: v = dk / (dk + r) * binom_scaled((dk + r) / dN, r, b); break;
      case kTabBeta: v = binom_scaled(-dk / dN, r, b); break;
      case kTabGamma: v = dk / (dk + r) * binom_scaled(-(dk + r) / dN, r, b); break;
      case kTabDelta: v = binom_scaled(dk / dN, r, b); break;
      default: {  // delta'
        const double cur = r < rows ? binom_scaled(dk / dN, r, b) : 0.0;
        const double prev = binom_scaled(dk / dN, r - 1, b);
        v = cur - scale2(prev, -b);
      }
    }
    tab[(long long)(r - 1) * N + k] = v;
  }
}

__global__ void k_init_maptab_fx(long long* tab, int which, long long N, int b, int rows, int Q) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= N) return;
  const double dk = (double)k, dN = (double)N;
  for (int r = 1; r <= rows; ++r) {
    const double v = which == kTabAlpha ? dk / (dk + r) * binom_scaled((dk + r) / dN, r, b)
                                        : dk / (dk + r) * binom_scaled(-(dk + r) / dN, r, b);
    tab[(long long)(r - 1) * N + k] = __double2ll_rn(scale2(v, Q + r * b));
  }
}

// High product: tab[i] = kappa_i = 2^b / rho^(i+1) (eq. 4.4), i < nkappa, then
// tab[nkappa + j] = rho^-j, j < ntheta, from lr = ln rho; the host planner's
// formula, evaluated on the device so that a call needs no host-to-device copy.
__global__ void k_init_rho_powers(double* tab, int nkappa, int ntheta, int b, double lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nkappa) tab[i] = exp(b * 0.6931471805599453 - (i + 1) * lr);
  else if (i < nkappa + ntheta) tab[i] = exp(-(i - nkappa) * lr);
}

// ------------------------------------------------------------ digits

// bits [pos, pos + cnt) of the n-bit integer in `limbs` (cnt <= 32, pos may be
// negative: bits below 0 read as zero; bits >= n read as zero).
__device__ __forceinline__ unsigned get_bits(const unsigned long long* limbs, long long nlimbs,
                                             unsigned long long n, long long pos, int cnt) {
  if (pos + cnt <= 0) return 0u;
  int lead = 0;                       // zero bits below position 0
  if (pos < 0) { lead = int(-pos); cnt -= lead; pos = 0; }
  if ((unsigned long long)pos >= n) return 0u;
  const long long i = pos >> 6;
  const int off = int(pos & 63);
  unsigned long long lo = __ldg(limbs + i) >> off;
  if (off + cnt > 64 && i + 1 < nlimbs) lo |= __ldg(limbs + i + 1) << (64 - off);
  unsigned long long valid = n - (unsigned long long)pos;   // bits below n
  int keep = cnt;
  if (valid < (unsigned long long)keep) keep = int(valid);
  lo &= (keep >= 64) ? ~0ull : ((1ull << keep) - 1ull);
  return (unsigned)(lo << lead);
}

// Balanced digit p of x = limbs * 2^shift (Section 5 variant):
// u_p = d_p - 2^b [d_p >= 2^(b-1)] + [d_(p-1) >= 2^(b-1)], d_p = bits [pb, pb+b) of x.
// With top_unbalanced, digit p = top keeps d_p + carry (high product, u_N).
__device__ __forceinline__ int balanced_digit(const unsigned long long* limbs, long long nlimbs,
                                              unsigned long long n, long long shift, int b,
                                              long long p, long long top, bool top_unbalanced) {
  const long long pos = p * b - shift;
  const unsigned d = get_bits(limbs, nlimbs, n, pos, b);
  const unsigned half = 1u << (b - 1);
  const int carry_in = p > 0 ? int(get_bits(limbs, nlimbs, n, pos - 1, 1)) : 0;
  if (top_unbalanced && p == top) return int(d) + carry_in;
  return int(d) - ((d >= half) ? (1 << b) : 0) + carry_in;
}

// ----------------------------------------------------- digit norms

// sums[0] += sum of u_p^2, sums[1] += sum of v_p^2 over the balanced digits p < count
// of u 2^shift and v 2^shift (digit size b; the digit `top` unbalanced when
// top_unbalanced); block 0 stores |u_top|, |v_top| in sums[2], sums[3] when
// top_unbalanced. Exact: |digit| <= 2^b, count < 2^26.
__global__ void k_digit_norms(const unsigned long long* u, const unsigned long long* v,
                              long long nlimbs, unsigned long long n, long long shift, int b,
                              long long count, long long top, int top_unbalanced,
                              unsigned long long* sums) {
  unsigned long long su = 0, sv = 0;
  const long long pend = top_unbalanced ? (count < top ? count : top) : count;
  const unsigned half = 1u << (b - 1);
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < pend;
       p += (long long)gridDim.x * blockDim.x) {
    // balanced digit p (p < top when the top is unbalanced) of u and v: b bits at
    // p b - shift and the carry bit below, from two or three cached limb reads
    const long long pos = p * b - shift;
    long long d[2];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      const unsigned long long* x = o ? v : u;
      unsigned dp, c;
      if (pos >= 1 && (unsigned long long)(pos + b) <= n) {
        const long long w = pos >> 6;
        const int off = int(pos & 63);
        const unsigned long long l0 = __ldg(x + w);
        const unsigned long long l1 = (off + b > 64) ? __ldg(x + w + 1) : 0ull;
        dp = unsigned(((l0 >> off) | ((l1 << 1) << (63 - off))) & ((1ull << b) - 1ull));
        const long long pc = pos - 1;
        c = unsigned((__ldg(x + (pc >> 6)) >> (pc & 63)) & 1ull);
      } else {
        dp = get_bits(x, nlimbs, n, pos, b);
        c = p > 0 ? get_bits(x, nlimbs, n, pos - 1, 1) : 0u;
      }
      d[o] = (long long)dp - (dp >= half ? (1ll << b) : 0) + c;
    }
    su += (unsigned long long)(d[0] * d[0]);
    sv += (unsigned long long)(d[1] * d[1]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    su += __shfl_xor_sync(~0u, su, o);
    sv += __shfl_xor_sync(~0u, sv, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sums, su);
    atomicAdd(sums + 1, sv);
  }
  if (top_unbalanced && blockIdx.x == 0 && threadIdx.x == 0) {
    const long long tu = balanced_digit(u, nlimbs, n, shift, b, top, top, true);
    const long long tv = balanced_digit(v, nlimbs, n, shift, b, top, top, true);
    sums[2] = (unsigned long long)(tu < 0 ? -tu : tu);
    sums[3] = (unsigned long long)(tv < 0 ? -tv : tv);
  }
}

void launch_digit_norms(const unsigned long long* u, const unsigned long long* v,
                        long long nlimbs, unsigned long long n, long long shift, int b,
                        long long count, long long top, bool top_unbalanced,
                        unsigned long long* sums, cudaStream_t s) {
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  k_digit_norms<<<unsigned(blocks), 256, 0, s>>>(u, v, nlimbs, n, shift, b, count, top,
                                                  top_unbalanced ? 1 : 0, sums);
}

// ----------------------------------------------------- forward maps

// Launches KERNEL<ROWS> with ROWS = rows for the map row counts the planner
// produces (3..12 for b = 5..14), else KERNEL<0> (any count up to kMaxLam).
#define TM_LAUNCH_ROWS(R, KERNEL, CFG, ARGS) \
  case R: launch_pdl(KERNEL<R>, TM_UNPAREN CFG, TM_UNPAREN ARGS); break;
#define TM_UNPAREN(...) __VA_ARGS__
#define TM_ROWS_DISPATCH(rows, KERNEL, CFG, ARGS)                                     \
  switch (rows) {                                                                    \
    TM_LAUNCH_ROWS(3, KERNEL, CFG, ARGS) TM_LAUNCH_ROWS(4, KERNEL, CFG, ARGS)        \
    TM_LAUNCH_ROWS(5, KERNEL, CFG, ARGS) TM_LAUNCH_ROWS(6, KERNEL, CFG, ARGS)        \
    TM_LAUNCH_ROWS(7, KERNEL, CFG, ARGS) TM_LAUNCH_ROWS(8, KERNEL, CFG, ARGS)        \
    TM_LAUNCH_ROWS(9, KERNEL, CFG, ARGS) TM_LAUNCH_ROWS(10, KERNEL, CFG, ARGS)       \
    TM_LAUNCH_ROWS(11, KERNEL, CFG, ARGS) TM_LAUNCH_ROWS(12, KERNEL, CFG, ARGS)      \
    default: launch_pdl(KERNEL<0>, TM_UNPAREN CFG, TM_UNPAREN ARGS); break;          \
  }

constexpr int kFwdThreads = 256;
constexpr int kMaxLam = 24;
constexpr int kMaxB = 24;
// limbs holding the bits of one tile's digits (plus the carry bit below them)
constexpr int kStageLimbs = ((kFwdTile + kMaxLam) * kMaxB + 64) / 64 + 4;

// Limbs of x = u 2^shift staged in shared memory for the digits p in [p_lo, p_hi):
// st[i] = limb w0 + i of u (bits at and above n cleared, zero outside the limbs).
struct DigitStage {
  long long w0;
  bool ok;            // false: the range did not fit; digits come from get_bits
};

__device__ DigitStage stage_digits(unsigned long long* st, const unsigned long long* limbs,
                                   long long nlimbs, unsigned long long n, long long shift,
                                   int b, long long p_lo, long long p_hi) {
  DigitStage g{0, true};
  if (p_hi <= p_lo) return g;
  const long long ulo = p_lo * b - 1 - shift, uhi = p_hi * b - shift;   // bits of u
  g.w0 = ulo >= 0 ? ulo / 64 : -((-ulo + 63) / 64);
  const long long cnt = (uhi - 1 - 64 * g.w0) / 64 + 2;
  if (cnt > kStageLimbs) {
    g.ok = false;
    return g;
  }
  for (long long t = threadIdx.x; t < cnt; t += blockDim.x) {
    const long long w = g.w0 + t;
    unsigned long long x = 0;
    if (w >= 0 && w < nlimbs && (unsigned long long)(64 * w) < n) {
      x = __ldg(limbs + w);
      const unsigned long long rem = n - (unsigned long long)(64 * w);
      if (rem < 64) x &= (1ull << rem) - 1ull;
    }
    st[t] = x;
  }
  return g;
}

// cnt <= 32 bits of the staged limbs from local bit lb
__device__ __forceinline__ unsigned stage_bits(const unsigned long long* st, long long lb,
                                               int cnt) {
  const long long w = lb >> 6;
  const int off = int(lb & 63);
  const unsigned long long x = (st[w] >> off) | ((st[w + 1] << 1) << (63 - off));
  return unsigned(x & ((1ull << cnt) - 1ull));
}

// Balanced digits d[t] of positions p = j0 - halo + t (cyclic mod N), t < span, of
// x = u 2^shift: positions below `limit` get the digit of Section 5, the others 0.
// Staged limbs serve positions p >= 0; wrapped positions (first tile) use get_bits.
__device__ void fill_digits(int* d, const unsigned long long* st, DigitStage g,
                            const unsigned long long* limbs, long long nlimbs,
                            unsigned long long n, long long shift, int b, long long N,
                            long long limit, long long top, bool top_unbalanced, long long j0,
                            int halo, int span) {
  const unsigned half = 1u << (b - 1);
  for (int t = threadIdx.x; t < span; t += blockDim.x) {
    long long p = j0 - halo + t;
    int x = 0;
    if (p < 0 || !g.ok) {
      if (p < 0) p += N;
      if (p < limit) x = balanced_digit(limbs, nlimbs, n, shift, b, p, top, top_unbalanced);
    } else if (p < limit) {
      const long long lb = p * b - shift - 64 * g.w0;
      const unsigned dp = stage_bits(st, lb, b);
      const int c = p > 0 ? int(stage_bits(st, lb - 1, 1)) : 0;
      x = int(dp) - (dp >= half ? (1 << b) : 0) + c;
    }
    d[t] = x;
  }
}

// Low product: U~ = sum_{r<lam} alpha*_r U (Algorithm 2, convert step; Proposition 3.15),
// U~_j = U_j + sum_{r=1}^{lam-1} alpha_{(j-r) mod N, r} U_{(j-r) mod N}, evaluated in
// fixed point on the integer pipe: with A_{k,r} = round(alpha_{k,r} 2^(Q+rb)),
// S_j = U_j 2^Q + sum_r (A_{k,r} U_k) >> rb is exact up to the table rounding and
// the shifts, |S_j| < 2^61, and U~_j = S_j 2^-Q after one rounding conversion.
// Full product (lam = 0): X_j = U_j for j < nd, 0 for nd <= j < N (Algorithm 1, split step).
// Shared memory of one forward-map block (one instance per kernel: the bodies are
// also run inside the single-launch kernels, where one union serves every phase).
struct FwdLoShared {
  int du[kFwdTile + kMaxLam], dv[kFwdTile + kMaxLam];
  unsigned long long stu[kStageLimbs], stv[kStageLimbs];
};
struct FwdHiShared {
  int du[kFwdTile + kMaxLam], dv[kFwdTile + kMaxLam];
  double fu[kFwdTile + kMaxLam], fv[kFwdTile + kMaxLam];
  unsigned long long stu[kStageLimbs], stv[kStageLimbs];
  double topu, topv;
};
union FwdShared {
  FwdLoShared lo;
  FwdHiShared hi;
};

template <int ROWS>
__device__ __forceinline__ void fwd_lo_full_body(FwdArgs a0, int kind, const uint3 bid, const uint3 gdim,
                                                 FwdLoShared& sh) {
  FwdArgs a = a0;
  if (a0.items) {
    const FwdItem it = a0.items[bid.y];
    a.u = it.u; a.v = it.v; a.n = it.n; a.nlimbs = it.nlimbs; a.nd = it.nd; a.s0 = it.s0;
    a.X = it.X; a.theta = it.theta;
  }
  pdl_trigger();
  pdl_wait();
  int* du = sh.du;
  int* dv = sh.dv;
  unsigned long long* stu = sh.stu;
  unsigned long long* stv = sh.stv;
  const bool two = !a.one_operand;
  const int tile = a.tile ? a.tile : kFwdTile;
  const long long j0 = (long long)bid.x * tile;
  const int halo = a.lam > 0 ? a.lam - 1 : 0;
  const int span = tile + halo;
  const long long limit = a.N < a.nd ? a.N : a.nd;
  {
    const long long p_lo = j0 - halo > 0 ? j0 - halo : 0;
    const long long p_hi = j0 + tile < limit ? j0 + tile : limit;
    const DigitStage gu = stage_digits(stu, a.u, a.nlimbs, a.n, 0, a.b, p_lo, p_hi);
    DigitStage gv{0, true};
    if (two) gv = stage_digits(stv, a.v, a.nlimbs, a.n, 0, a.b, p_lo, p_hi);
    __syncthreads();
    fill_digits(du, stu, gu, a.u, a.nlimbs, a.n, 0, a.b, a.N, limit, a.nd - 1, false, j0, halo,
                span);
    if (two)
      fill_digits(dv, stv, gv, a.v, a.nlimbs, a.n, 0, a.b, a.N, limit, a.nd - 1, false, j0,
                  halo, span);
  }
  __syncthreads();
  const int Q = fx_q(a.b);
  for (int t = threadIdx.x; t < tile; t += blockDim.x) {
    const long long j = j0 + t;
    if (j >= a.N) break;
    if (a.lam == 0) {
      a.X[j] = i2d_exact(du[t]);
      if (two) a.X[a.N + j] = i2d_exact(dv[t]);
      continue;
    }
    long long su = (long long)du[t + halo] << Q, sv = (long long)dv[t + halo] << Q;
    if (j >= halo) {                 // no wrap: row r, index j - r; loads first
      const long long* tp = a.tab + (j - 1);
      constexpr int RM = ROWS > 0 ? ROWS : kMaxLam;
      long long A[RM + 1];
#pragma unroll
      for (int r = 1; r <= RM; ++r)
        A[r] = (ROWS > 0 || r < a.lam) ? __ldg(tp + (long long)(r - 1) * (a.N - 1)) : 0;
#pragma unroll
      for (int r = 1; r <= RM; ++r) {
        if (ROWS > 0 || r < a.lam) {
          su += (A[r] * du[t + halo - r]) >> (r * a.b);
          if (two) sv += (A[r] * dv[t + halo - r]) >> (r * a.b);
        }
      }
    } else {
      for (int r = 1; r < a.lam; ++r) {
        long long k = j - r;
        if (k < 0) k += a.N;
        const long long A = __ldg(a.tab + (long long)(r - 1) * a.N + k);
        su += (A * du[t + halo - r]) >> (r * a.b);
        if (two) sv += (A * dv[t + halo - r]) >> (r * a.b);
      }
    }
    a.X[j] = scale2(__ll2double_rn(su), -Q);
    if (two) a.X[a.N + j] = scale2(__ll2double_rn(sv), -Q);
  }
}

template <int ROWS>
__global__ void __launch_bounds__(kFwdThreads) k_fwd_lo_full(FwdArgs a0, int kind) {
  __shared__ FwdLoShared sh;
  fwd_lo_full_body<ROWS>(a0, kind, blockIdx, gridDim, sh);
}

// High product: gamma-dagger (Algorithm 3, convert step; Proposition 4.18).
// F' = F mod C: F'_i = F_i + kappa_i F_N (eq. 4.5), then
// U~_j = sum_{r<lam} gamma_{(j-r) mod N, r} F'_{(j-r) mod N}, and
// theta = rho^-N F(rho) = sum_j rho^-j F_(N-j).
// Outputs that read a kappa-corrected F'_i or wrap around (j < nkappa + lam - 1,
// all in the first tile) are evaluated in FP64; the others read integer digits
// only and use the fixed-point form of the low product's map.
__device__ __forceinline__ double fx_coef(const long long* tab, long long N, int r, long long k,
                                          int Q, int b) {
  return scale2(__ll2double_rn(__ldg(tab + (long long)(r - 1) * N + k)), -(Q + r * b));
}

template <int ROWS>
__device__ __forceinline__ void fwd_hi_body(FwdArgs a0, const uint3 bid, const uint3 gdim,
                                            FwdHiShared& sh) {
  FwdArgs a = a0;
  if (a0.items) {
    const FwdItem it = a0.items[bid.y];
    a.u = it.u; a.v = it.v; a.n = it.n; a.nlimbs = it.nlimbs; a.nd = it.nd; a.s0 = it.s0;
    a.X = it.X; a.theta = it.theta;
  }
  pdl_trigger();
  pdl_wait();
  int* du = sh.du;
  int* dv = sh.dv;
  double* fu = sh.fu;
  double* fv = sh.fv;
  unsigned long long* stu = sh.stu;
  unsigned long long* stv = sh.stv;
  double& topu = sh.topu;
  double& topv = sh.topv;
  const bool two = !a.one_operand;
  const int tile = a.tile ? a.tile : kFwdTile;
  const long long j0 = (long long)bid.x * tile;
  const int halo = a.lam - 1;
  const int span = tile + halo;
  const long long N = a.N;
  const bool head = bid.x == 0;
  const int Q = fx_q(a.b);
  if (threadIdx.x == 0) {
    topu = i2d_exact(balanced_digit(a.u, a.nlimbs, a.n, a.s0, a.b, N, N, true));
    topv = two ? i2d_exact(balanced_digit(a.v, a.nlimbs, a.n, a.s0, a.b, N, N, true)) : 0.0;
  }
  {
    const long long p_lo = j0 - halo > 0 ? j0 - halo : 0;
    const long long p_hi = j0 + tile < N ? j0 + tile : N;
    const DigitStage gu = stage_digits(stu, a.u, a.nlimbs, a.n, a.s0, a.b, p_lo, p_hi);
    DigitStage gv{0, true};
    if (two) gv = stage_digits(stv, a.v, a.nlimbs, a.n, a.s0, a.b, p_lo, p_hi);
    __syncthreads();
    fill_digits(du, stu, gu, a.u, a.nlimbs, a.n, a.s0, a.b, N, N, N, true, j0, halo, span);
    if (two) fill_digits(dv, stv, gv, a.v, a.nlimbs, a.n, a.s0, a.b, N, N, N, true, j0, halo, span);
    else
      for (int t = threadIdx.x; t < span; t += blockDim.x) dv[t] = 0;
  }
  __syncthreads();
  if (head) {
    for (int t = threadIdx.x; t < span; t += blockDim.x) {
      long long p = j0 - halo + t;
      if (p < 0) p += N;
      double yu = i2d_exact(du[t]), yv = i2d_exact(dv[t]);
      if (p < a.nkappa) {
        const double kp = __ldg(a.kappa + p);
        yu = fma(kp, topu, yu);
        yv = fma(kp, topv, yv);
      }
      fu[t] = yu;
      fv[t] = yv;
    }
    __syncthreads();
  }
  const long long head_end = head ? (long long)a.nkappa + a.lam - 1 : 0;
  for (int t = threadIdx.x; t < tile; t += blockDim.x) {
    const long long j = j0 + t;
    if (j >= N) break;
    if (j < head_end) {             // reads a kappa-corrected F'_i or wraps: FP64
      double su = fu[t + halo], sv = fv[t + halo];
      for (int r = 1; r < a.lam; ++r) {
        long long k = j - r;
        if (k < 0) k += N;
        const double g = fx_coef(a.tab, N, r, k, Q, a.b);
        su = fma(g, fu[t + halo - r], su);
        sv = fma(g, fv[t + halo - r], sv);
      }
      a.X[j] = su;
      if (two) a.X[N + j] = sv;
    } else {
      long long su = (long long)du[t + halo] << Q, sv = (long long)dv[t + halo] << Q;
      const long long* tp = a.tab + (j - 1);
      constexpr int RM = ROWS > 0 ? ROWS : kMaxLam;
      long long A[RM + 1];
#pragma unroll
      for (int r = 1; r <= RM; ++r)
        A[r] = (ROWS > 0 || r < a.lam) ? __ldg(tp + (long long)(r - 1) * (N - 1)) : 0;
#pragma unroll
      for (int r = 1; r <= RM; ++r) {
        if (ROWS > 0 || r < a.lam) {
          su += (A[r] * du[t + halo - r]) >> (r * a.b);
          if (two) sv += (A[r] * dv[t + halo - r]) >> (r * a.b);
        }
      }
      a.X[j] = scale2(__ll2double_rn(su), -Q);
      if (two) a.X[N + j] = scale2(__ll2double_rn(sv), -Q);
    }
  }
  // theta: block 0, two threads (u and v), ntheta terms of rho^-j F_(N-j); with one
  // operand theta_V is copied (a kept transform), equals theta_U (a square) or is
  // left to the other operand's launch
  if (head && !two && threadIdx.x == 32) {
    if (a.theta_v) a.theta[1] = *a.theta_v;
  } else if (head && (threadIdx.x == 0 || threadIdx.x == 32)) {
    const unsigned long long* src = threadIdx.x == 0 ? a.u : a.v;
    double th = 0.0;
    for (int j = a.ntheta - 1; j >= 0; --j) {
      const long long p = N - j;
      if (p < 0) continue;
      const double f = i2d_exact(balanced_digit(src, a.nlimbs, a.n, a.s0, a.b, p, N, true));
      th = fma(__ldg(a.rho_pow + j), f, th);
    }
    a.theta[threadIdx.x == 0 ? 0 : 1] = th;
    if (!two && a.square_theta && threadIdx.x == 0) a.theta[1] = th;
  }
}

template <int ROWS>
__global__ void __launch_bounds__(kFwdThreads) k_fwd_hi(FwdArgs a0) {
  __shared__ FwdHiShared sh;
  fwd_hi_body<ROWS>(a0, blockIdx, gridDim, sh);
}

// SMs of the current device (read once). A map launch takes 256-position tiles (one
// position per thread instead of four) when their grid fits in two CTAs per SM: at
// n = 2^16 and 2^18 bits that cuts 4-30 us from a single product; at 2^20 the 480
// small CTAs take a second wave and cost 6-9 us, so the 1024-position tiles stay.
int map_sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      (void)cudaGetLastError();
      return 0;
    }
    return v;
  }();
  return n;
}
constexpr int kSmallTile = 256;
bool small_tile_fits(long long N) {
  return (N + kSmallTile - 1) / kSmallTile <= 2LL * map_sm_count();
}
// the high product's head positions (fewer than nkappa + lam, nkappa <= 3 + 128 / b
// for N < 2^64) stay in block 0, as the map bodies require
static_assert(kSmallTile >= 131 + kMaxLam, "head positions outside block 0");

void launch_fwd(int kind, const FwdArgs& a0, int batch, cudaStream_t s) {
  FwdArgs a = a0;
  if (!a.items && a.tile == 0 && small_tile_fits(a.N)) a.tile = kSmallTile;
  const int tile = a.tile ? a.tile : kFwdTile;
  const dim3 grid(unsigned((a.N + tile - 1) / tile), unsigned(batch));
  const int rows = a.lam - 1;                    // map rows r = 1..lam-1
  if (kind == TM_HI) {
    TM_ROWS_DISPATCH(rows, k_fwd_hi, (grid, kFwdThreads, 0, s), (a));
  } else {
    TM_ROWS_DISPATCH(rows, k_fwd_lo_full, (grid, kFwdThreads, 0, s), (a, kind));
  }
}

// ------------------------------------------------------------ FFT pass

// Radix-R DFT of x[0..R) in place, sign S of the exponent (-1 forward).
template <int R, int S>
__device__ __forceinline__ void dft(double2* x);

template <>
__device__ __forceinline__ void dft<2, -1>(double2* x) { const double2 a = x[0]; x[0] = cadd(a, x[1]); x[1] = csub(a, x[1]); }
template <>
__device__ __forceinline__ void dft<2, 1>(double2* x) { const double2 a = x[0]; x[0] = cadd(a, x[1]); x[1] = csub(a, x[1]); }

template <int S>
__device__ __forceinline__ void dft4(double2& x0, double2& x1, double2& x2, double2& x3) {
  const double2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
  const double2 t2 = cadd(x1, x3), t3 = mul_si<S>(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}
template <>
__device__ __forceinline__ void dft<4, -1>(double2* x) { dft4<-1>(x[0], x[1], x[2], x[3]); }
template <>
__device__ __forceinline__ void dft<4, 1>(double2* x) { dft4<1>(x[0], x[1], x[2], x[3]); }

template <int S>
__device__ __forceinline__ void dft3(double2* x) {
  const double2 t = cadd(x[1], x[2]);
  const double2 m = make_double2(fma(t.x, -0.5, x[0].x), fma(t.y, -0.5, x[0].y));
  const double2 d = csub(x[1], x[2]);
  const double2 sd = mul_si<S>(make_double2(d.x * kSqrt3_2, d.y * kSqrt3_2));
  x[0] = cadd(x[0], t);
  x[1] = cadd(m, sd);
  x[2] = csub(m, sd);
}
template <>
__device__ __forceinline__ void dft<3, -1>(double2* x) { dft3<-1>(x); }
template <>
__device__ __forceinline__ void dft<3, 1>(double2* x) { dft3<1>(x); }

template <int S>
__device__ __forceinline__ void dft5(double2* x) {
  const double2 t1 = cadd(x[1], x[4]), t2 = cadd(x[2], x[3]);
  const double2 d1 = csub(x[1], x[4]), d2 = csub(x[2], x[3]);
  const double2 x0 = x[0];
  const double2 a1 = make_double2(fma(kC5_1, t1.x, fma(kC5_2, t2.x, x0.x)), fma(kC5_1, t1.y, fma(kC5_2, t2.y, x0.y)));
  const double2 a2 = make_double2(fma(kC5_2, t1.x, fma(kC5_1, t2.x, x0.x)), fma(kC5_2, t1.y, fma(kC5_1, t2.y, x0.y)));
  const double2 b1 = mul_si<S>(make_double2(fma(kS5_1, d1.x, kS5_2 * d2.x), fma(kS5_1, d1.y, kS5_2 * d2.y)));
  const double2 b2 = mul_si<S>(make_double2(fma(kS5_2, d1.x, -kS5_1 * d2.x), fma(kS5_2, d1.y, -kS5_1 * d2.y)));
  x[0] = cadd(x0, cadd(t1, t2));
  x[1] = cadd(a1, b1); x[4] = csub(a1, b1);
  x[2] = cadd(a2, b2); x[3] = csub(a2, b2);
}
template <>
__device__ __forceinline__ void dft<5, -1>(double2* x) { dft5<-1>(x); }
template <>
__device__ __forceinline__ void dft<5, 1>(double2* x) { dft5<1>(x); }

template <int S>
__device__ __forceinline__ void dft7(double2* x) {
  const double2 t1 = cadd(x[1], x[6]), t2 = cadd(x[2], x[5]), t3 = cadd(x[3], x[4]);
  const double2 d1 = csub(x[1], x[6]), d2 = csub(x[2], x[5]), d3 = csub(x[3], x[4]);
  const double2 x0 = x[0];
  // a_m = x0 + sum_k cos(2 pi m k / 7) t_k ;  b_m = S i sum_k sin(2 pi m k / 7) d_k
  const double2 a1 = make_double2(fma(kC7_1, t1.x, fma(kC7_2, t2.x, fma(kC7_3, t3.x, x0.x))),
                                  fma(kC7_1, t1.y, fma(kC7_2, t2.y, fma(kC7_3, t3.y, x0.y))));
  const double2 a2 = make_double2(fma(kC7_2, t1.x, fma(kC7_3, t2.x, fma(kC7_1, t3.x, x0.x))),
                                  fma(kC7_2, t1.y, fma(kC7_3, t2.y, fma(kC7_1, t3.y, x0.y))));
  const double2 a3 = make_double2(fma(kC7_3, t1.x, fma(kC7_1, t2.x, fma(kC7_2, t3.x, x0.x))),
                                  fma(kC7_3, t1.y, fma(kC7_1, t2.y, fma(kC7_2, t3.y, x0.y))));
  // sin(2 pi m k/7): m=1: s1 s2 s3 ; m=2: s2 -s3 -s1 ; m=3: s3 -s1 s2
  const double2 b1 = mul_si<S>(make_double2(fma(kS7_1, d1.x, fma(kS7_2, d2.x, kS7_3 * d3.x)),
                                            fma(kS7_1, d1.y, fma(kS7_2, d2.y, kS7_3 * d3.y))));
  const double2 b2 = mul_si<S>(make_double2(fma(kS7_2, d1.x, fma(-kS7_3, d2.x, -kS7_1 * d3.x)),
                                            fma(kS7_2, d1.y, fma(-kS7_3, d2.y, -kS7_1 * d3.y))));
  const double2 b3 = mul_si<S>(make_double2(fma(kS7_3, d1.x, fma(-kS7_1, d2.x, kS7_2 * d3.x)),
                                            fma(kS7_3, d1.y, fma(-kS7_1, d2.y, kS7_2 * d3.y))));
  x[0] = cadd(x0, cadd(t1, cadd(t2, t3)));
  x[1] = cadd(a1, b1); x[6] = csub(a1, b1);
  x[2] = cadd(a2, b2); x[5] = csub(a2, b2);
  x[3] = cadd(a3, b3); x[4] = csub(a3, b3);
}
template <>
__device__ __forceinline__ void dft<7, -1>(double2* x) { dft7<-1>(x); }
template <>
__device__ __forceinline__ void dft<7, 1>(double2* x) { dft7<1>(x); }

// One Stockham stage of radix R over C sequences of length L held in shared
// memory, in place: butterfly j reads buf[j + t L/R], applies
// omega_(Ns R)^(t (j mod Ns)) and writes buf[(j/Ns) Ns R + (j mod Ns) + t Ns];
// after all stages the result is in natural order. Each thread owns up to
// ceil(4/R) butterflies (the CTA has C L / 4 threads): it reads all of their
// inputs, the CTA synchronises, then it writes all of their outputs.
template <int R, int S>
__device__ __forceinline__ void stockham_stage(double2* buf, int L, int C, int Ns,
                                               const double2* tw, double2 (&xs)[8],
                                               int (&base)[4], int (&kk)[4]) {
  constexpr int MB = (4 + R - 1) / R;
  const int nb = L / R;
  const int total = C * nb;
  const int twstep = L / (Ns * R);
#pragma unroll
  for (int i = 0; i < MB; ++i) {
    const int g = threadIdx.x + i * blockDim.x;
    base[i] = -1;
    if (g < total) {
      const int c = g / nb, j = g - c * nb;
      const double2* s = buf + c * L + j;
#pragma unroll
      for (int t = 0; t < R; ++t) xs[i * R + t] = s[t * nb];
      kk[i] = j % Ns;
      base[i] = c * L + (j / Ns) * Ns * R + kk[i];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MB; ++i) {
    if (base[i] < 0) continue;
    double2* x = xs + i * R;
    if (Ns > 1) {
#pragma unroll
      for (int t = 1; t < R; ++t) {
        const double2 w = tw[kk[i] * t * twstep];
        x[t] = S < 0 ? cmul(x[t], w) : cmulc(x[t], w);
      }
    }
    dft<R, S>(x);
    double2* d = buf + base[i];
#pragma unroll
    for (int t = 0; t < R; ++t) d[t * Ns] = x[t];
  }
}

// Radix-4 Stockham stage with tangent-form twiddles, 24 FMAs per butterfly in
// place of 12 for the three twiddle products and 16 additions. With
// w_t = omega^(t k) (t = 1, 2, 3), w3 = w1 w2, so for the DFT of
// (x0, w1 x1, w2 x2, w3 x3):  A, B = x0 +- w2 x2,  E, F = x1 +- w2 x3,
// y0, y2 = A +- w1 E,  y1, y3 = B +- S i w1 F.  Each w z is c (z -+ i t z):
// one FMA per component for the bracket, and the factor c folds into the FMA
// that adds it. When the angle of w2 reaches pi/2, w2 = -+i c (1 -+ i t): the
// real and imaginary parts trade places, selected on the integer pipe.
template <int S>
__device__ __forceinline__ double2 tan_bracket(double2 z, double t) {
  // z (1 - i t) for the forward direction, z (1 + i t) for the inverse
  return S < 0 ? make_double2(fma(t, z.y, z.x), fma(-t, z.x, z.y))
               : make_double2(fma(-t, z.y, z.x), fma(t, z.x, z.y));
}

template <int S>
__device__ __forceinline__ void radix4_tan(double2* x, Tan4 w) {
  const double t1 = w.t1, c1 = w.c1, t2 = w.t2;
  const long long cb = __double_as_longlong(w.c2s);
  const bool rot = cb < 0;
  const long long mag = cb & 0x7FFFFFFFFFFFFFFFll;
  const long long neg = mag | (long long)0x8000000000000000ull;
  // coefficient of the real part and of the imaginary part of w2 z
  const double ca = __longlong_as_double(rot && S > 0 ? neg : mag);
  const double cq = __longlong_as_double(rot && S < 0 ? neg : mag);
  const double2 x2 = tan_bracket<S>(x[2], t2), x3 = tan_bracket<S>(x[3], t2);
  const double p2 = rot ? x2.y : x2.x, q2 = rot ? x2.x : x2.y;
  const double p3 = rot ? x3.y : x3.x, q3 = rot ? x3.x : x3.y;
  const double2 x0 = x[0], x1 = x[1];
  const double2 A = make_double2(fma(ca, p2, x0.x), fma(cq, q2, x0.y));
  const double2 B = make_double2(fma(-ca, p2, x0.x), fma(-cq, q2, x0.y));
  const double2 E = tan_bracket<S>(make_double2(fma(ca, p3, x1.x), fma(cq, q3, x1.y)), t1);
  const double2 F = tan_bracket<S>(make_double2(fma(-ca, p3, x1.x), fma(-cq, q3, x1.y)), t1);
  x[0] = make_double2(fma(c1, E.x, A.x), fma(c1, E.y, A.y));
  x[2] = make_double2(fma(-c1, E.x, A.x), fma(-c1, E.y, A.y));
  if (S < 0) {   // B -+ i c1 F
    x[1] = make_double2(fma(c1, F.y, B.x), fma(-c1, F.x, B.y));
    x[3] = make_double2(fma(-c1, F.y, B.x), fma(c1, F.x, B.y));
  } else {       // B +- i c1 F
    x[1] = make_double2(fma(-c1, F.y, B.x), fma(c1, F.x, B.y));
    x[3] = make_double2(fma(c1, F.y, B.x), fma(-c1, F.x, B.y));
  }
}

template <int S>
__device__ __forceinline__ void stockham_stage4t(double2* buf, int L, int C, int Ns,
                                                 const Tan4* tw, double2 (&xs)[8],
                                                 int (&base)[4], int (&kk)[4]) {
  const int nb = L / 4;
  const int total = C * nb;
  const int g = threadIdx.x;
  base[0] = -1;
  if (g < total) {
    const int c = g / nb, j = g - c * nb;
    const double2* s = buf + c * L + j;
#pragma unroll
    for (int t = 0; t < 4; ++t) xs[t] = s[t * nb];
    kk[0] = j % Ns;
    base[0] = c * L + (j / Ns) * Ns * 4 + kk[0];
  }
  __syncthreads();
  if (base[0] >= 0) {
    radix4_tan<S>(xs, tw[kk[0]]);
    double2* d = buf + base[0];
#pragma unroll
    for (int t = 0; t < 4; ++t) d[t * Ns] = xs[t];
  }
}

// The split of the full product (Algorithm 1, split step) at the positions 2m and
// 2m + 1, for a first pass that computes its input as it loads it: the same
// balanced digits as fwd_lo_full_body gives the full product (0 from the digit
// count on), so the values are identical.
__device__ __forceinline__ double2 split_pair(const unsigned long long* limbs,
                                               unsigned long long n, long long nlimbs,
                                               long long limit, int b, long long m) {
  auto digit = [&](long long q) -> int {
    return q < limit ? balanced_digit(limbs, nlimbs, n, 0, b, q, limit - 1, false) : 0;
  };
  return make_double2(i2d_exact(digit(2 * m)), i2d_exact(digit(2 * m + 1)));
}

template <int S, bool MAP = false>
__device__ __forceinline__ void fft_pass_body(const double2* __restrict__ in, double2* __restrict__ out, PassArgs p, const uint3 bid, const uint3 gdim) {
  extern __shared__ double2 smem[];
  const int L = p.L, C = p.C;
  double2* buf = smem;
  const int off4 = (C * L + 1) & ~1;    // 32-byte aligned
  Tan4* tw4s = reinterpret_cast<Tan4*>(smem + off4);
  double2* tws = smem + off4 + 2 * p.tw4_len;   // omega_L^k, k < L (when needed)
  pdl_trigger();
  for (int t = threadIdx.x; t < p.tw4_len; t += blockDim.x) tw4s[t] = p.tw4[t];
  if (p.need_wL)
    for (int t = threadIdx.x; t < L; t += blockDim.x) tws[t] = __ldg(p.tw_sub + t);
  pdl_wait();                       // the plan's tables above; the data below
  const long long q0 = (long long)bid.x * C;
  const long long boff = (long long)bid.y * p.batch_stride;
  in += boff;
  out += boff;
  const int CL = C * L;
  const bool rowload = p.IS == 1;
  for (int e = threadIdx.x; e < CL; e += blockDim.x) {
    int c, j;
    if (rowload) { c = e / L; j = e - c * L; } else { j = e / C; c = e - j * C; }
    const long long q = q0 + c;
    double2 val = make_double2(0.0, 0.0);
    if (q < p.Q) {
      const long long qa = q / p.Qc, qc = q - qa * p.Qc;
      const long long m = qa * p.IA + qc * p.IC + (long long)j * p.IS;
      val = MAP ? split_pair(bid.y ? p.map_limbs2 : p.map_limbs, p.map_n, p.map_nlimbs,
                             p.map_limit, p.map_b, m)
                : in[m];
    }
    buf[c * L + j] = val;
  }
  __syncthreads();
  int Ns = 1;
  double2 xs[8];                        // one register array shared by every radix case
  int base[4], kk[4];
  for (int st = 0; st < p.nstages; ++st) {
    const int R = p.radix[st];
    switch (R) {
      case 2: stockham_stage<2, S>(buf, L, C, Ns, tws, xs, base, kk); break;
      case 3: stockham_stage<3, S>(buf, L, C, Ns, tws, xs, base, kk); break;
      case 4:
        if (Ns > 1) stockham_stage4t<S>(buf, L, C, Ns, tw4s + p.tw4_off[st], xs, base, kk);
        else stockham_stage<4, S>(buf, L, C, Ns, tws, xs, base, kk);
        break;
      case 5: stockham_stage<5, S>(buf, L, C, Ns, tws, xs, base, kk); break;
      default: stockham_stage<7, S>(buf, L, C, Ns, tws, xs, base, kk); break;
    }
    __syncthreads();
    Ns *= R;
  }
  const bool rowstore = p.OS == 1;
  for (int e = threadIdx.x; e < CL; e += blockDim.x) {
    int c, k;
    if (rowstore) { c = e / L; k = e - c * L; } else { k = e / C; c = e - k * C; }
    const long long q = q0 + c;
    if (q >= p.Q) continue;
    const long long qa = q / p.Qc, qc = q - qa * p.Qc;
    double2 val = buf[c * L + k];
    if (p.Mp) {
      const double2 w = __ldg(p.tw_outer + k * p.Qc + qc);
      val = S < 0 ? cmul(val, w) : cmulc(val, w);
    }
    out[qa * p.OA + qc * p.OC + (long long)k * p.OS] = val;
  }
}

template <int S>
__global__ void k_fft_pass(const double2* __restrict__ in, double2* __restrict__ out, PassArgs p) {
  fft_pass_body<S>(in, out, p, blockIdx, gridDim);
}

// First forward pass with the full product's split computed on load (PassArgs::map_limbs).
__global__ void k_fft_pass_map(double2* __restrict__ out, PassArgs p) {
  fft_pass_body<-1, true>(nullptr, out, p, blockIdx, gridDim);
}

void set_small_smem_attribute(int bytes);

// Shared memory above 48 KB per CTA needs the opt-in; set once before any launch
// (outside stream capture).
void set_fft_smem_attribute() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncSetAttribute(k_fft_pass<-1>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  cudaFuncSetAttribute(k_fft_pass<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  cudaFuncSetAttribute(k_fft_pass_map, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  set_small_smem_attribute(optin);
  set_fused_smem_attribute(optin);
}

void launch_fft_pass(int dir, const double2* in, double2* out, const PassArgs& p, int batch,
                     int threads, cudaStream_t s) {
  const unsigned blocks = unsigned((p.Q + p.C - 1) / p.C);
  const size_t smem = (size_t((p.C * p.L + 1) & ~1) + 2 * size_t(p.tw4_len) +
                      (p.need_wL ? size_t(p.L) : 0)) * sizeof(double2);
  dim3 grid(blocks, batch);
  if (p.map_limbs)
    launch_pdl(k_fft_pass_map, grid, dim3(threads), smem, s, out, p);
  else if (dir < 0)
    launch_pdl(k_fft_pass<-1>, grid, dim3(threads), smem, s, in, out, p);
  else
    launch_pdl(k_fft_pass<1>, grid, dim3(threads), smem, s, in, out, p);
}

// ------------------------------------------------ twist + pointwise product

// Real-FFT twist, pointwise product and inverse pre-twist in one step, for the
// pair (k, M-k) of the half-length spectra Z (u) and Z' (v) (Z = DFT_M of the
// real input packed as x_2j + i x_2j+1). With A = Z_k, B = conj(Z_(M-k)),
// D = A - B and w = omega_N^k, the real input's spectrum is (A + B - i w D) / 2 at
// k and conj(A + B + i w D) / 2 at M - k; multiplying the two inputs' spectra and
// packing the product back into a half-length spectrum (scaled by 1/N for the
// inverse transform) reduces, with |w| = 1, to
//   Q_k     = (2/N) A A' - c_k D D',
//   Q_(M-k) = conj((2/N) B B' - c_k D D'),   c_k = (1 + w^2) / (2N),
// 24 FP64 instructions per pair (a square: A' = A, B' = B, D' = D).
template <bool SQ>
__device__ __forceinline__ void twist_pair(const double2* Zu, const double2* Zv, double2* Q,
                                           long long M, long long k,
                                           const double2* __restrict__ tc, double two_over_N) {
  const long long km = k == 0 ? 0 : M - k;
  const double2 c = __ldg(tc + k);
  const double2 A0 = Zu[k], B0 = cconj(Zu[km]);
  const double2 D0 = csub(A0, B0);
  double2 AA, BB, DD;
  if (SQ) {
    AA = cmul(A0, A0);
    BB = cmul(B0, B0);
    DD = cmul(D0, D0);
  } else {
    const double2 A1 = Zv[k], B1 = cconj(Zv[km]);
    const double2 D1 = csub(A1, B1);
    AA = cmul(A0, A1);
    BB = cmul(B0, B1);
    DD = cmul(D0, D1);
  }
  const double2 H = cmul(DD, c);
  // (reads of Z precede the writes, so Q may alias Zu)
  Q[k] = make_double2(fma(two_over_N, AA.x, -H.x), fma(two_over_N, AA.y, -H.y));
  if (k != 0 && km != k)
    Q[km] = make_double2(fma(two_over_N, BB.x, -H.x), fma(-two_over_N, BB.y, H.y));
}

template <bool SQ>
__device__ __forceinline__ void twist_body(const double2* __restrict__ Zu, const double2* __restrict__ Zv,
                        double2* __restrict__ Q, long long M,
                        const double2* __restrict__ tc, double two_over_N, long long zstride,
                        long long qstride, const uint3 bid, const uint3 gdim) {
  pdl_trigger();
  pdl_wait();
  const long long k = bid.x * (long long)blockDim.x + threadIdx.x;
  if (k > M / 2) return;
  twist_pair<SQ>(Zu + bid.y * zstride, Zv + bid.y * zstride, Q + bid.y * qstride,
                 M, k, tc, two_over_N);
}

template <bool SQ>
__global__ void k_twist(const double2* __restrict__ Zu, const double2* __restrict__ Zv,
                        double2* __restrict__ Q, long long M,
                        const double2* __restrict__ tc, double two_over_N, long long zstride,
                        long long qstride) {
  twist_body<SQ>(Zu, Zv, Q, M, tc, two_over_N, zstride, qstride, blockIdx, gridDim);
}

void launch_twist(const double2* Zu, const double2* Zv, double2* Q, long long M,
                  const double2* tc, long long N, int batch, long long zstride,
                  long long qstride, cudaStream_t s) {
  const long long n = M / 2 + 1;
  const dim3 grid(unsigned((n + 255) / 256), unsigned(batch));
  const double two_over_N = 2.0 / double(N);
  if (Zv == Zu)
    launch_pdl(k_twist<true>, grid, dim3(256), 0, s, Zu, Zv, Q, M, tc, two_over_N, zstride,
               qstride);
  else
    launch_pdl(k_twist<false>, grid, dim3(256), 0, s, Zu, Zv, Q, M, tc, two_over_N, zstride,
               qstride);
}

// ------------------------------------------------ back maps and rounding

constexpr int kBackThreads = 256;

__device__ __forceinline__ void note_distance(unsigned long long d, unsigned long long* bmax) {
  // block-local max in shared memory, folded into the status at the end
  atomicMax(bmax, d);
}

__device__ __forceinline__ void finish_block(unsigned long long* bmax, unsigned* bflags,
                                             const BackArgs& a) {
  __syncthreads();
  if (threadIdx.x == 0) {
    if (*bmax) atomicMax(&a.status->margin_fx, *bmax);
    unsigned f = *bflags;
    if (*bmax > a.emax_fx) f |= kFlagPrecision;
    if (f) atomicOr(&a.status->flags, f);
  }
}

__device__ __forceinline__ void emit(const BackArgs& a, long long i, double x, bool scaled,
                                     unsigned long long* bmax) {
  unsigned long long d;
  const long long c = round_dist(scaled ? scale2(x, a.b) : x, &d);
  a.c[i] = c;
  note_distance(d, bmax);
}

// Full product (Algorithm 1, overlap-add): c_i = round(W_i).
__device__ void back_full_loop(const BackArgs& a, long long start, long long stride,
                               unsigned long long* bmax) {
  for (long long i = start; i < a.count; i += stride) emit(a, i, a.w[i], false, bmax);
}

__device__ __forceinline__ void back_full_body(BackArgs a0, const uint3 bid, const uint3 gdim) {
  BackArgs a = a0;
  if (a0.items) {
    const BackItem it = a0.items[bid.y];
    a.w = it.w; a.c = it.c; a.theta = it.theta; a.emax_fx = it.emax_fx;
  }
  pdl_trigger();
  pdl_wait();
  __shared__ unsigned long long bmax;
  __shared__ unsigned bflags;
  if (threadIdx.x == 0) { bmax = 0; bflags = 0; }
  __syncthreads();
  back_full_loop(a, bid.x * (long long)blockDim.x + threadIdx.x,
                 (long long)gdim.x * blockDim.x, &bmax);
  finish_block(&bmax, &bflags, a);
}

__global__ void __launch_bounds__(kBackThreads) k_back_full(BackArgs a0) {
  back_full_body(a0, blockIdx, gridDim);
}

// Low product (Algorithm 2, convert back and rounding; Proposition 3.16): Wbar = sum_{r<lam} beta*_r W~
// reduced mod A(X) = X^N + 2^-b X - 1, then c_i = round(2^b Wbar_i).
// Interior positions i >= lam receive no wrapped terms. Head positions i < lam
// add P_(N+i) and subtract 2^-b P_(N+i-1), where P_(N+m) =
// sum_{r=m+1}^{lam-1} beta_{N+m-r, r} W~_(N+m-r) are the coefficients of X^(N+m)
// before reduction (X^(N+m) = X^m - 2^-b X^(m+1) mod A). Requires N >= 2 lam + 2;
// smaller N take k_back_small.
__device__ __forceinline__ double beta_at(const BackArgs& a, long long k, int r) {
  return r == 0 ? 1.0 : __ldg(a.tab + (long long)(r - 1) * a.N + k);
}

__device__ double lo_overflow(const BackArgs& a, int m) {   // P_(N+m)
  double acc = 0.0;
  for (int r = m + 1; r < a.lam; ++r) {
    const long long k = a.N + m - r;
    acc = fma(beta_at(a, k, r), a.w[k], acc);
  }
  return acc;
}

__device__ void back_lo_loop(const BackArgs& a, long long start, long long stride,
                             unsigned long long* bmax, unsigned* bflags) {
  const long long N = a.N;
  for (long long i = start; i < N; i += stride) {
    double acc = a.w[i];
    const int rmax = i < a.lam ? int(i) + 1 : a.lam;
    for (int r = 1; r < rmax; ++r) acc = fma(beta_at(a, i - r, r), a.w[i - r], acc);
    if (i < a.lam) {
      if (i <= a.lam - 2) acc += lo_overflow(a, int(i));
      if (i >= 1) acc = fma(-scale2(1.0, -a.b), lo_overflow(a, int(i) - 1), acc);
    }
    unsigned long long d;
    const long long c = round_dist(scale2(acc, a.b), &d);
    a.c[i] = c;
    note_distance(d, bmax);
    if (i == 0 && (c & ((1ll << a.b) - 1)) != 0) atomicOr(bflags, kFlagC0);
  }
}

// Largest rounding distance of the block (every thread passes its own maximum).
__device__ __forceinline__ void block_note_distance(unsigned long long d,
                                                    unsigned long long* bmax) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long e = __shfl_xor_sync(~0u, d, o);
    d = e > d ? e : d;
  }
  if ((threadIdx.x & 31) == 0 && d) atomicMax(bmax, d);
}


// Tiles of kBackTile coefficients; every thread issues the loads of all map rows
// and W~ values of an output before the FMAs, unrolled for ROWS = lam - 1 rows
// (ROWS = 0: any count up to kMaxLam, predicated). Head positions i < lam (block 0)
// take back_lo_loop's path with the wrapped terms.
template <int ROWS>
__device__ __forceinline__ void back_lo_body(BackArgs a0, const uint3 bid, const uint3 gdim) {
  BackArgs a = a0;
  if (a0.items) {
    const BackItem it = a0.items[bid.y];
    a.w = it.w; a.c = it.c; a.theta = it.theta; a.emax_fx = it.emax_fx;
  }
  pdl_trigger();
  pdl_wait();
  __shared__ unsigned long long bmax;
  __shared__ unsigned bflags;
  const long long N = a.N;
  const int tile = a.tile ? a.tile : kBackTile;
  const long long i0 = (long long)bid.x * tile;
  if (threadIdx.x == 0) { bmax = 0; bflags = 0; }
  __syncthreads();
  unsigned long long dmax = 0;
  for (int t = threadIdx.x; t < tile; t += blockDim.x) {
    const long long i = i0 + t;
    if (i >= N) break;
    if (i < a.lam) {
      back_lo_loop(a, i, N, &bmax, &bflags);       // this one position
      continue;
    }
    constexpr int RM = ROWS > 0 ? ROWS : kMaxLam;
    double B[RM + 1], W[RM + 1];
    const double* tp = a.tab + (i - 1);            // row r, index i - r
#pragma unroll
    for (int r = 1; r <= RM; ++r) {
      const bool on = ROWS > 0 || r < a.lam;
      B[r] = on ? __ldg(tp + (long long)(r - 1) * (N - 1)) : 0.0;
      W[r] = on ? __ldg(a.w + (i - r)) : 0.0;
    }
    double acc = __ldg(a.w + i);
#pragma unroll
    for (int r = 1; r <= RM; ++r)
      if (ROWS > 0 || r < a.lam) acc = fma(B[r], W[r], acc);
    unsigned long long d;
    a.c[i] = round_dist(scale2(acc, a.b), &d);
    dmax = d > dmax ? d : dmax;
  }
  block_note_distance(dmax, &bmax);
  finish_block(&bmax, &bflags, a);
}

template <int ROWS>
__global__ void __launch_bounds__(kBackThreads) k_back_lo(BackArgs a0) {
  back_lo_body<ROWS>(a0, blockIdx, gridDim);
}

// High product (Algorithm 3, convert back and rounding; Proposition 4.19 with Remark 4.20 for
// large N): H = sum_{r<lam} delta*_r W~ reduced mod C(X), whose X^N = sum_i
// kappa_i X^i (eq. 4.4), and then by eq. (4.7)
//   J_i = H_i - 2^-b H_(i-1) - psi kappa_i (i < N),  J_N = -2^-b H_(N-1) + psi,
// with psi = theta_U theta_V: for N > 64 the other terms of eq. (4.6) lie far
// below the last bit of psi. Interior i >= lam + nkappa: one stencil with the
// combined rows delta' (tab). Head i < lam + nkappa and J_N: warp 0 of block 0.
__device__ __forceinline__ double delta_at(const BackArgs& a, long long k, int r) {
  return r == 0 ? 1.0 : __ldg(a.tab2 + (long long)(r - 1) * a.N + k);
}

__device__ double hi_H(const BackArgs& a, long long i, const double* P) {   // reduced H_i
  double acc = 0.0;
  const int rmax = i < a.lam ? int(i) + 1 : a.lam;
  for (int r = 0; r < rmax; ++r) acc = fma(delta_at(a, i - r, r), a.w[i - r], acc);
  // wrapped terms: P_(N+m) kappa_(i-m), m <= lam-2, 0 <= i-m < nkappa
  for (int m = 0; m <= a.lam - 2; ++m) {
    const long long t = i - m;
    if (t >= 0 && t < a.nkappa) acc = fma(__ldg(a.kappa + t), P[m], acc);
  }
  return acc;
}

// Interior J_i, i >= lam + nkappa, one stencil with the delta' rows.
__device__ void back_hi_interior(const BackArgs& a, long long start, long long stride,
                                 unsigned long long* bmax) {
  const long long N = a.N;
  const int head = a.lam + a.nkappa;
  for (long long i = head + start; i < N; i += stride) {
    double acc = a.w[i];
    for (int r = 1; r <= a.lam; ++r)
      acc = fma(__ldg(a.tab + (long long)(r - 1) * N + (i - r)), a.w[i - r], acc);
    unsigned long long d;
    a.c[i] = round_dist(scale2(acc, a.b), &d);
    note_distance(d, bmax);
  }
}

// Head J_i, i < lam + nkappa, and J_N: one warp (lane 0..31), shared P and Hh.
__device__ void back_hi_head(const BackArgs& a, int lane, double* P, double* Hh,
                             unsigned long long* bmax, unsigned* bflags) {
  const long long N = a.N;
  const int head = a.lam + a.nkappa;
  const double twmb = scale2(1.0, -a.b);
  const double psi = a.theta[0] * a.theta[1];
  // overflow coefficients P_(N+m), m = 0..lam-2
  for (int m = lane; m <= a.lam - 2; m += 32) {
    double acc = 0.0;
    for (int r = m + 1; r < a.lam; ++r) {
      const long long k = N + m - r;
      acc = fma(delta_at(a, k, r), a.w[k], acc);
    }
    P[m] = acc;
  }
  __syncwarp();
  for (int i = lane; i < head; i += 32) Hh[i] = hi_H(a, i, P);
  __syncwarp();
  for (int i = lane; i < head; i += 32) {
    double J = Hh[i];
    if (i >= 1) J = fma(-twmb, Hh[i - 1], J);
    if (i < a.nkappa) J = fma(-psi, __ldg(a.kappa + i), J);
    unsigned long long d;
    const long long c = round_dist(scale2(J, a.b), &d);
    a.c[i] = c;
    note_distance(d, bmax);
    if (i == 0 && (c & ((1ll << a.b) - 1)) != 0) atomicOr(bflags, kFlagC0);
  }
  if (lane == 0) {   // J_N = -2^-b H_(N-1) + psi (H_(N-1) is an interior value)
    double H = 0.0;
    for (int r = 0; r < a.lam; ++r) H = fma(delta_at(a, N - 1 - r, r), a.w[N - 1 - r], H);
    const double J = fma(-twmb, H, psi);
    unsigned long long d;
    a.c[N] = round_dist(scale2(J, a.b), &d);
    note_distance(d, bmax);
  }
}

// Tiles as in k_back_lo, ROWS = lam rows of delta'. Head positions and J_N are
// warp 0 of block 0 (back_hi_head).
template <int ROWS>
__device__ __forceinline__ void back_hi_body(BackArgs a0, const uint3 bid, const uint3 gdim) {
  BackArgs a = a0;
  if (a0.items) {
    const BackItem it = a0.items[bid.y];
    a.w = it.w; a.c = it.c; a.theta = it.theta; a.emax_fx = it.emax_fx;
  }
  pdl_trigger();
  pdl_wait();
  __shared__ unsigned long long bmax;
  __shared__ unsigned bflags;
  __shared__ double P[kMaxLam];
  __shared__ double Hh[kMaxLam + 64 + 1];
  const long long N = a.N;
  const int tile = a.tile ? a.tile : kBackTile;
  const long long i0 = (long long)bid.x * tile;
  const long long head = a.lam + a.nkappa;
  if (threadIdx.x == 0) { bmax = 0; bflags = 0; }
  __syncthreads();
  unsigned long long dmax = 0;
  for (int t = threadIdx.x; t < tile; t += blockDim.x) {
    const long long i = i0 + t;
    if (i >= N) break;
    if (i < head) continue;
    constexpr int RM = ROWS > 0 ? ROWS : kMaxLam;
    double D[RM + 1], W[RM + 1];
    const double* tp = a.tab + (i - 1);
#pragma unroll
    for (int r = 1; r <= RM; ++r) {
      const bool on = ROWS > 0 || r <= a.lam;
      D[r] = on ? __ldg(tp + (long long)(r - 1) * (N - 1)) : 0.0;
      W[r] = on ? __ldg(a.w + (i - r)) : 0.0;
    }
    double acc = __ldg(a.w + i);
#pragma unroll
    for (int r = 1; r <= RM; ++r)
      if (ROWS > 0 || r <= a.lam) acc = fma(D[r], W[r], acc);
    unsigned long long d;
    a.c[i] = round_dist(scale2(acc, a.b), &d);
    dmax = d > dmax ? d : dmax;
  }
  block_note_distance(dmax, &bmax);
  if (bid.x == 0 && threadIdx.x < 32) back_hi_head(a, threadIdx.x, P, Hh, &bmax, &bflags);
  finish_block(&bmax, &bflags, a);
}

template <int ROWS>
__global__ void __launch_bounds__(kBackThreads) k_back_hi(BackArgs a0) {
  back_hi_body<ROWS>(a0, blockIdx, gridDim);
}

// Small transforms (any N): one thread evaluates the back map from the
// definitions, reducing the shifted terms modulo A or C from the top degree
// down, and for the high product psi by eq. (4.6) in the scaled form
// psi = (theta - rho^-2N H(rho)) / (1 - N 2^b rho^-(N+1)).
constexpr int kSmallMax = 160;
// One thread; reports into the status word directly.
__device__ void back_small_body(const BackArgs& a, int kind) {
  double P[kSmallMax + kMaxLam];
  const long long N = a.N;
  const int tot = int(N) + a.lam - 1;
  for (int i = 0; i < tot; ++i) P[i] = 0.0;
  for (long long k = 0; k < N; ++k)
    for (int r = 0; r < a.lam; ++r) {
      const double co = kind == TM_LO ? beta_at(a, k, r) : delta_at(a, k, r);
      P[k + r] = fma(co, a.w[k], P[k + r]);
    }
  const double twmb = scale2(1.0, -a.b);
  for (int j = tot - 1; j >= N; --j) {       // reduce X^j, j >= N
    const double pj = P[j];
    P[j] = 0.0;
    const int m = j - int(N);
    if (kind == TM_LO) {                     // X^(N+m) = X^m - 2^-b X^(m+1)
      P[m] += pj;
      P[m + 1] = fma(-twmb, pj, P[m + 1]);
    } else {                                 // X^(N+m) = X^m sum_i kappa_i X^i
      for (int i = 0; i < a.nkappa && i < N; ++i) P[m + i] = fma(__ldg(a.kappa + i), pj, P[m + i]);
    }
  }
  unsigned long long bm = 0, d;
  unsigned flags = 0;
  if (kind == TM_LO) {
    for (long long i = 0; i < N; ++i) {
      const long long c = round_dist(scale2(P[i], a.b), &d);
      a.c[i] = c;
      bm = d > bm ? d : bm;
      if (i == 0 && (c & ((1ll << a.b) - 1)) != 0) flags |= kFlagC0;
    }
  } else {
    const double rho = a.rho;
    // rho^-2N H(rho) = sum_i H_i rho^(i - 2N), by Horner on rho^-1 from the top
    // h = sum_i H_i rho^(i-(N-1)) by Horner in 1/rho; rho^-2N H(rho) = h rho^-(N+1)
    double h = 0.0;
    const double ir = 1.0 / rho;
    for (long long i = 0; i < N; ++i) h = fma(h, ir, P[i]);
    const double rnp1 = pow(ir, double(N + 1));
    const double psi = (a.theta[0] * a.theta[1] - h * rnp1) /
                       (1.0 - double(N) * scale2(1.0, a.b) * rnp1);
    for (long long i = 0; i <= N; ++i) {
      double J = i < N ? P[i] : 0.0;
      if (i >= 1) J = fma(-twmb, P[i - 1], J);
      if (i < N) {
        if (i < a.nkappa) J = fma(-psi, __ldg(a.kappa + i), J);
      } else {
        J += psi;
      }
      const long long c = round_dist(scale2(J, a.b), &d);
      a.c[i] = c;
      bm = d > bm ? d : bm;
      if (i == 0 && (c & ((1ll << a.b) - 1)) != 0) flags |= kFlagC0;
    }
  }
  if (bm) atomicMax(&a.status->margin_fx, bm);
  if (bm > a.emax_fx) flags |= kFlagPrecision;
  if (flags) atomicOr(&a.status->flags, flags);
}


__device__ __forceinline__ void back_small_body_k(BackArgs a0, int kind, const uint3 bid, const uint3 gdim) {
  pdl_trigger();
  pdl_wait();
  if (threadIdx.x != 0 || bid.x != 0) return;
  BackArgs a = a0;
  if (a0.items) {
    const BackItem it = a0.items[bid.y];
    a.w = it.w; a.c = it.c; a.theta = it.theta; a.emax_fx = it.emax_fx;
  }
  back_small_body(a, kind);
}

__global__ void k_back_small(BackArgs a0, int kind) {
  back_small_body_k(a0, kind, blockIdx, gridDim);
}

void launch_back(int kind, const BackArgs& a0, int batch, cudaStream_t s) {
  BackArgs a = a0;
  if (!a.items && a.tile == 0 && small_tile_fits(a.N)) a.tile = kSmallTile;
  const long long n = a.count;
  unsigned blocks = unsigned((n + kBackThreads - 1) / kBackThreads);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks == 0) blocks = 1;
  const dim3 grid(blocks, unsigned(batch));
  if (kind == TM_FULL) {
    launch_pdl(k_back_full, grid, dim3(kBackThreads), 0, s, a);
  } else if (a.N <= 64 || a.N < 2 * a.lam + a.nkappa + 2) {
    launch_pdl(k_back_small, dim3(1, unsigned(batch)), dim3(32), 0, s, a, kind);
  } else {
    const int rows = kind == TM_LO ? a.lam - 1 : a.lam;
    const int tile = a.tile ? a.tile : kBackTile;
    const dim3 tgrid(unsigned((a.N + tile - 1) / tile), unsigned(batch));
    if (kind == TM_LO) {
      TM_ROWS_DISPATCH(rows, k_back_lo, (tgrid, kBackThreads, 0, s), (a));
    } else {
      TM_ROWS_DISPATCH(rows, k_back_hi, (tgrid, kBackThreads, 0, s), (a));
    }
  }
}

// ------------------------------------------------------------ carry scan

// S = sum_i t_i 2^(p_i) with signed 54-bit terms t_i: c_i at i b (full, high),
// c_i at (i-1) b for i >= 1 and c_0 / 2^b at 0 (low, Algorithm 2 overlap-add), plus
// 2^(s-1) for the high product's returned round(t) (Algorithm 3, half up).
// A_L = sum over terms starting in limb L of t_i 2^(p_i - 64 L) (int128);
// r_L = (A_L mod 2^64) + floor(A_(L-1) / 2^64) lies in (-2^60, 2^64 + 2^60), so
// the carry into each limb is -1, 0 or +1 and each limb acts on it through a
// 3-entry function f_L(cin) = floor((r_L + cin) / 2^64). The scan composes
// these functions: per block, over blocks, then applied per limb.
constexpr int kCarryThreads = 512;

__device__ __forceinline__ long long ceil_div_ll(long long a, long long b) {
  return a >= 0 ? (a + b - 1) / b : -((-a) / b);
}

__device__ __int128 limb_sum(const CarryArgs& a, long long L) {
  if (L < 0) return 0;
  __int128 acc = 0;
  const long long base = 64 * L;
  const long long off = a.kind == TM_LO ? -a.b : 0;          // p_i = i b + off
  long long ilo = ceil_div_ll(base - off, a.b), ihi = ceil_div_ll(base + 64 - off, a.b);
  if (a.kind == TM_LO) {
    if (ilo < 1) ilo = 1;
    if (L == 0) acc += (__int128)(a.c[0] >> a.b);
  }
  if (ilo < 0) ilo = 0;
  if (ihi > a.K) ihi = a.K;
  for (long long i = ilo; i < ihi; ++i) {
    const int sh = int(i * a.b + off - base);
    acc += (__int128)((unsigned __int128)(__int128)a.c[i] << sh);
  }
  if (a.round_bit >= 0 && (a.round_bit >> 6) == L)
    acc += (__int128)((unsigned __int128)1 << (a.round_bit & 63));
  return acc;
}

// f encoded as 3 x 2 bits: bits [2t, 2t+2) hold f(t-1) + 1, t = 0, 1, 2.
__device__ __forceinline__ unsigned carry_fn(__int128 r) {
  unsigned f = 0;
  for (int t = 0; t < 3; ++t) {
    const __int128 x = r + (t - 1);
    const long long co = (long long)(x >> 64);               // -1, 0 or 1
    f |= unsigned(co + 1) << (2 * t);
  }
  return f;
}
__device__ __forceinline__ int apply_fn(unsigned f, int cin) { return int((f >> (2 * (cin + 1))) & 3u) - 1; }
// (g o f)(c) = g(f(c))
__device__ __forceinline__ unsigned compose(unsigned g, unsigned f) {
  unsigned h = 0;
  for (int t = 0; t < 3; ++t) h |= unsigned(apply_fn(g, apply_fn(f, t - 1)) + 1) << (2 * t);
  return h;
}
constexpr unsigned kIdentityFn = 0u | (1u << 2) | (2u << 4);

// inclusive scan of functions in shared memory: s[i] = f_i o ... o f_0
__device__ void block_compose_scan(unsigned* s, int n) {
  for (int d = 1; d < n; d <<= 1) {
    unsigned v = 0;
    const int i = threadIdx.x;
    if (i < n && i >= d) v = compose(s[i], s[i - d]);
    __syncthreads();
    if (i < n && i >= d) s[i] = v;
    __syncthreads();
  }
}

// Exclusive and total composition of the block's functions in thread order:
// *ex = f_(t-1) o ... o f_0 (identity for thread 0), *tot = f_last o ... o f_0.
// NT threads, every thread calls it.
template <int NT>
__device__ void block_fn_scan(unsigned f, unsigned* ex, unsigned* tot) {
  __shared__ unsigned wsum[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned inc = f;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned g = __shfl_up_sync(~0u, inc, o);
    if (lane >= o) inc = compose(inc, g);
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    unsigned w = lane < NT / 32 ? wsum[lane] : kIdentityFn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned g = __shfl_up_sync(~0u, w, o);
      if (lane >= o) w = compose(w, g);
    }
    if (lane < NT / 32) wsum[lane] = w;
  }
  __syncthreads();
  const unsigned prev = __shfl_up_sync(~0u, inc, 1);
  const unsigned ex_lane = lane ? prev : kIdentityFn;
  const unsigned before = wid ? wsum[wid - 1] : kIdentityFn;
  *ex = compose(ex_lane, before);
  *tot = wsum[NT / 32 - 1];
  __syncthreads();
}

// r_L of every limb and the block's composed carry function. Word 2L of r holds
// r_L mod 2^64; word 2L+1 holds floor(r_L / 2^64) (-1, 0 or 1) in its low byte and
// the block-exclusive prefix of carry functions in bits 8..13.
__device__ __forceinline__ void carry_local_body(CarryArgs a0, const uint3 bid, const uint3 gdim) {
  CarryArgs a = a0;
  if (a0.items) {
    const CarryItem it = a0.items[bid.y];
    a.c = it.c; a.nS = it.nS; a.round_bit = it.round_bit; a.shift_bits = it.shift_bits;
    a.nout = it.nout; a.top_mask = it.top_mask; a.out = it.out; a.r = it.r;
    a.fblock = it.fblock; a.cin_block = it.cin_block;
  }
  pdl_trigger();
  pdl_wait();
  const long long my_blocks = (a.nS + kCarryThreads - 1) / kCarryThreads;
  if (bid.x >= my_blocks) return;     // uniform per block
  __shared__ long long hs[kCarryThreads];
  const long long L = bid.x * (long long)kCarryThreads + threadIdx.x;
  const __int128 AL = L < a.nS ? limb_sum(a, L) : (__int128)0;
  hs[threadIdx.x] = (long long)(AL >> 64);
  __syncthreads();
  const long long hp = threadIdx.x ? hs[threadIdx.x - 1] : (long long)(limb_sum(a, L - 1) >> 64);
  const __int128 r = (__int128)(unsigned long long)AL + hp;
  const unsigned f = L < a.nS ? carry_fn(r) : kIdentityFn;
  unsigned ex, tot;
  block_fn_scan<kCarryThreads>(f, &ex, &tot);
  if (L < a.nS) {
    a.r[2 * L] = (unsigned long long)r;
    a.r[2 * L + 1] = (unsigned long long)((unsigned)(int)(long long)(r >> 64) & 0xFFu) |
                     ((unsigned long long)ex << 8);
  }
  if (threadIdx.x == 0) a.fblock[bid.x] = (unsigned char)tot;
}

__global__ void __launch_bounds__(kCarryThreads) k_carry_local(CarryArgs a0) {
  carry_local_body(a0, blockIdx, gridDim);
}

// carry into every block: cin_0 = 0, cin_(B+1) = F_B(cin_B)
// NT threads scan the blocks' carry functions (one CTA).
template <int NT>
__device__ __forceinline__ void carry_blocks_body(CarryArgs a0, const uint3 bid) {
  CarryArgs a = a0;
  if (a0.items) {
    const CarryItem it = a0.items[bid.y];
    a.c = it.c; a.nS = it.nS; a.round_bit = it.round_bit; a.shift_bits = it.shift_bits;
    a.nout = it.nout; a.top_mask = it.top_mask; a.out = it.out; a.r = it.r;
    a.fblock = it.fblock; a.cin_block = it.cin_block;
  }
  pdl_trigger();
  pdl_wait();
  const long long nblocks = (a.nS + kCarryThreads - 1) / kCarryThreads;
  const long long per = (nblocks + NT - 1) / NT;
  const long long b0 = threadIdx.x * per;
  unsigned f = kIdentityFn;
  for (long long i = b0; i < b0 + per && i < nblocks; ++i) f = compose(a.fblock[i], f);
  unsigned ex, tot;
  block_fn_scan<NT>(f, &ex, &tot);
  int cin = apply_fn(ex, 0);
  for (long long i = b0; i < b0 + per && i < nblocks; ++i) {
    a.cin_block[i] = (unsigned char)(cin + 1);
    cin = apply_fn(a.fblock[i], cin);
  }
}

__global__ void __launch_bounds__(1024) k_carry_blocks(CarryArgs a0) {
  carry_blocks_body<1024>(a0, blockIdx);
}

// r_L + cin mod 2^64 for limb L (0 beyond the resolved limbs)
__device__ __forceinline__ unsigned long long resolved_lo(const CarryArgs& a, long long L,
                                                          int cin) {
  return L < a.nS ? a.r[2 * L] + (unsigned long long)(long long)cin : 0ull;
}

// Carry into block bidx: the composition of the carry functions of blocks 0 .. bidx-1
// applied to 0 (each thread folds a run of them in order, then one block scan).
// Every thread of the block calls it.
__device__ __forceinline__ int block_carry_in(const CarryArgs& a, long long bidx) {
  const long long per = (bidx + kCarryThreads - 1) / kCarryThreads;
  const long long b0 = threadIdx.x * per;
  unsigned f = kIdentityFn;
  for (long long i = b0; i < b0 + per && i < bidx; ++i) f = compose(a.fblock[i], f);
  unsigned ex, tot;
  block_fn_scan<kCarryThreads>(f, &ex, &tot);
  return apply_fn(tot, 0);
}

// SCAN: the block finds its own carry-in from the blocks' carry functions (no
// separate block-scan launch); otherwise it reads cin_block.
template <bool SCAN = false>
__device__ __forceinline__ void carry_apply_body(CarryArgs a0, const uint3 bid, const uint3 gdim) {
  CarryArgs a = a0;
  if (a0.items) {
    const CarryItem it = a0.items[bid.y];
    a.c = it.c; a.nS = it.nS; a.round_bit = it.round_bit; a.shift_bits = it.shift_bits;
    a.nout = it.nout; a.top_mask = it.top_mask; a.out = it.out; a.r = it.r;
    a.fblock = it.fblock; a.cin_block = it.cin_block;
  }
  pdl_trigger();
  pdl_wait();
  const long long my_blocks = (a.nS + kCarryThreads - 1) / kCarryThreads;
  if (bid.x >= my_blocks) return;     // uniform per block
  int cin_blk = 0;
  if (SCAN) cin_blk = block_carry_in(a, bid.x);
  else cin_blk = int(a.cin_block[bid.x]) - 1;
  const long long L = bid.x * (long long)kCarryThreads + threadIdx.x;
  if (L >= a.nS) return;
  const long long sw = a.shift_bits >> 6;
  const int sb = int(a.shift_bits & 63);
  const long long j = L - sw;                // output limb whose low part comes from L
  if (j < 0 || j >= a.nout) return;
  const unsigned long long lo = a.r[2 * L], w1 = a.r[2 * L + 1];
  const int hi = (int)(signed char)(w1 & 0xFFu);
  const unsigned pfx = unsigned(w1 >> 8) & 0x3Fu;
  const int cin = apply_fn(pfx, cin_blk);
  unsigned long long o = (lo + (unsigned long long)(long long)cin) >> sb;
  if (sb) {
    // carry out of limb L: floor((r_L + cin) / 2^64)
    const int cnext = hi + ((cin > 0 && lo == ~0ull) ? 1 : 0) - ((cin < 0 && lo == 0ull) ? 1 : 0);
    o |= resolved_lo(a, L + 1, cnext) << (64 - sb);
  }
  if (j == a.nout - 1) o &= a.top_mask;
  a.out[j] = o;
}

__global__ void __launch_bounds__(kCarryThreads) k_carry_apply(CarryArgs a0) {
  carry_apply_body(a0, blockIdx, gridDim);
}

__global__ void __launch_bounds__(kCarryThreads) k_carry_apply_scan(CarryArgs a0) {
  carry_apply_body<true>(a0, blockIdx, gridDim);
}

__global__ void k_status_publish(DevStatus* status, DevStatus* host) {
  pdl_trigger();
  pdl_wait();
  if (threadIdx.x == 0) {
    const DevStatus v = *status;
    *host = v;
    status->margin_fx = 0ull;
    status->flags = 0u;
  }
}

void launch_status_publish(DevStatus* status, DevStatus* host, cudaStream_t s) {
  launch_pdl(k_status_publish, dim3(1), dim3(32), 0, s, status, host);
}

// Single products with at most this many carry blocks (131072 limbs) skip the
// block-scan launch: each apply block scans the carry functions of the blocks before
// it itself. Measured on GB300: 1.5-2.5 us less per product at n = 2^16 and 2^20,
// no change at 2^22-2^24, 4 us more at 2^26 and 30 us at 2^28, where every apply
// block walks thousands of functions.
constexpr long long kCarryScanBlocks = 256;

void launch_carry(const CarryArgs& a, int batch, cudaStream_t s) {
  const long long nblocks =
      a.items ? a.nblocks_max : (a.nS + kCarryThreads - 1) / kCarryThreads;
  const dim3 grid(static_cast<unsigned>(nblocks), static_cast<unsigned>(batch));
  launch_pdl(k_carry_local, grid, dim3(kCarryThreads), 0, s, a);
  if (!a.items && nblocks <= kCarryScanBlocks) {
    launch_pdl(k_carry_apply_scan, grid, dim3(kCarryThreads), 0, s, a);
    return;
  }
  launch_pdl(k_carry_blocks, dim3(1, unsigned(batch)), dim3(1024), 0, s, a);
  launch_pdl(k_carry_apply, grid, dim3(kCarryThreads), 0, s, a);
}


// ------------------------------------------------ single-launch products

// Grid-wide barrier of a cooperative launch (every CTA resident). Thread 0 of
// each CTA counts itself in and waits for the generation word to move. The wait
// is bounded by the global nanosecond timer (kBarrierTimeoutNs, one second): on
// timeout it sets kFlagTimeout in the status word, and every CTA returns at its
// next barrier instead of waiting on a CTA that has left. Returns false once any
// CTA timed out. leave = true: this CTA leaves without counting itself in (the
// host-side fault injection of the single-launch paths).
constexpr unsigned long long kBarrierTimeoutNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_barrier(unsigned* sync, DevStatus* status, bool leave = false) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vs = sync;
    if (leave) {
      if (gridDim.x == 1) atomicOr(&status->flags, kFlagTimeout);   // nobody else to wait
    } else {
      const unsigned gen = vs[1];
      __threadfence();
      const unsigned arrived = atomicAdd(sync, 1u) + 1u;
      if (arrived == gridDim.x) {
        atomicExch(sync, 0u);                 // ready for the next barrier
        __threadfence();
        atomicAdd(sync + 1, 1u);              // release the others
      } else {
        const unsigned long long t0 = global_ns();
        while (vs[1] == gen) {
          if (global_ns() - t0 > kBarrierTimeoutNs) {
            atomicOr(&status->flags, kFlagTimeout);
            break;
          }
          __nanosleep(32);
        }
      }
      __threadfence();
    }
    s_ok = !leave && (((volatile unsigned*)&status->flags)[0] & kFlagTimeout) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Every phase of one product in one cooperative launch: forward maps, forward FFT
// passes, twist, inverse passes, back map and rounding, carry scan, separated by
// grid barriers. Each phase runs the same block bodies as the per-phase kernels,
// over its virtual blocks (block v of a phase on CTA v mod grid), so the
// arithmetic is identical to the multi-kernel path.
template <int KIND>
__global__ void __launch_bounds__(kFusedThreads, 2) k_fused_product(FusedArgs A) {
  __shared__ FwdShared fsh;
  const unsigned G = gridDim.x;
  {                                                   // 1. split + convert
    const unsigned bx = unsigned((A.fa.N + kFwdTile - 1) / kFwdTile);
    for (unsigned v = blockIdx.x; v < bx; v += G) {
      if (KIND == TM_HI)
        fwd_hi_body<0>(A.fa, make_uint3(v, 0, 0), make_uint3(bx, 1, 1), fsh.hi);
      else
        fwd_lo_full_body<0>(A.fa, KIND, make_uint3(v, 0, 0), make_uint3(bx, 1, 1), fsh.lo);
      __syncthreads();
    }
  }
  if (!grid_barrier(A.sync, A.status, A.leave_barrier && blockIdx.x == gridDim.x - 1)) return;
  const unsigned nb = A.square ? 1u : 2u;
  for (int i = 0; i < A.npass; ++i) {                 // 2. forward FFTs
    const PassArgs& p = A.fwd[i];
    const unsigned bx = unsigned((p.Q + p.C - 1) / p.C);
    for (unsigned v = blockIdx.x; v < bx * nb; v += G) {
      fft_pass_body<-1>(A.fwd_in[i], A.fwd_out[i], p, make_uint3(v % bx, v / bx, 0),
                        make_uint3(bx, nb, 1));
      __syncthreads();
    }
    if (!grid_barrier(A.sync, A.status)) return;
  }
  {                                                   // 3. twist + pointwise product
    const unsigned bx = unsigned((A.M / 2 + kFusedThreads) / kFusedThreads);
    for (unsigned v = blockIdx.x; v < bx; v += G) {
      if (A.square)
        twist_body<true>(A.Zu, A.Zv, A.Q, A.M, A.tc, A.two_over_N, 0, 0, make_uint3(v, 0, 0),
                         make_uint3(bx, 1, 1));
      else
        twist_body<false>(A.Zu, A.Zv, A.Q, A.M, A.tc, A.two_over_N, 0, 0, make_uint3(v, 0, 0),
                          make_uint3(bx, 1, 1));
    }
  }
  if (!grid_barrier(A.sync, A.status)) return;
  for (int i = 0; i < A.npass; ++i) {                 // 4. inverse FFT
    const PassArgs& p = A.inv[i];
    const unsigned bx = unsigned((p.Q + p.C - 1) / p.C);
    for (unsigned v = blockIdx.x; v < bx; v += G) {
      fft_pass_body<1>(A.inv_in[i], A.inv_out[i], p, make_uint3(v, 0, 0), make_uint3(bx, 1, 1));
      __syncthreads();
    }
    if (!grid_barrier(A.sync, A.status)) return;
  }
  {                                                   // 5. convert back + round
    if (KIND == TM_FULL) {
      long long nvb = (A.ba.count + kFusedThreads - 1) / kFusedThreads;
      if (nvb > 152 * 8) nvb = 152 * 8;
      for (unsigned v = blockIdx.x; v < unsigned(nvb); v += G) {
        back_full_body(A.ba, make_uint3(v, 0, 0), make_uint3(unsigned(nvb), 1, 1));
        __syncthreads();
      }
    } else if (A.back_small) {
      if (blockIdx.x == 0 && threadIdx.x < 32)
        back_small_body_k(A.ba, KIND, make_uint3(0, 0, 0), make_uint3(1, 1, 1));
    } else {
      const unsigned bx = unsigned((A.ba.N + kBackTile - 1) / kBackTile);
      for (unsigned v = blockIdx.x; v < bx; v += G) {
        if (KIND == TM_LO)
          back_lo_body<0>(A.ba, make_uint3(v, 0, 0), make_uint3(bx, 1, 1));
        else
          back_hi_body<0>(A.ba, make_uint3(v, 0, 0), make_uint3(bx, 1, 1));
        __syncthreads();
      }
    }
  }
  if (!grid_barrier(A.sync, A.status)) return;
  const unsigned cb = unsigned((A.ca.nS + kCarryThreads - 1) / kCarryThreads);
  for (unsigned v = blockIdx.x; v < cb; v += G) {     // 6. overlap-add + carries
    carry_local_body(A.ca, make_uint3(v, 0, 0), make_uint3(cb, 1, 1));
    __syncthreads();
  }
  if (!grid_barrier(A.sync, A.status)) return;
  if (blockIdx.x == 0) carry_blocks_body<kFusedThreads>(A.ca, make_uint3(0, 0, 0));
  if (!grid_barrier(A.sync, A.status)) return;
  for (unsigned v = blockIdx.x; v < cb; v += G) {
    carry_apply_body(A.ca, make_uint3(v, 0, 0), make_uint3(cb, 1, 1));
    __syncthreads();
  }
}

// the opt-in limit covers static and dynamic shared memory together
template <int KIND>
void set_fused_attribute(int bytes) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k_fused_product<KIND>) == cudaSuccess)
    cudaFuncSetAttribute(k_fused_product<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes - int(fa.sharedSizeBytes));
  (void)cudaGetLastError();
}

void set_fused_smem_attribute(int bytes) {
  set_fused_attribute<TM_FULL>(bytes);
  set_fused_attribute<TM_LO>(bytes);
  set_fused_attribute<TM_HI>(bytes);
}

int fused_max_blocks(int kind, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (kind == TM_HI)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused_product<TM_HI>,
                                                      kFusedThreads, smem);
  else if (kind == TM_LO)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused_product<TM_LO>,
                                                      kFusedThreads, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused_product<TM_FULL>,
                                                      kFusedThreads, smem);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return per * sms;
}

cudaError_t launch_fused(int kind, const FusedArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kFusedThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (kind == TM_HI) return cudaLaunchKernelEx(&cfg, k_fused_product<TM_HI>, a);
  if (kind == TM_LO) return cudaLaunchKernelEx(&cfg, k_fused_product<TM_LO>, a);
  return cudaLaunchKernelEx(&cfg, k_fused_product<TM_FULL>, a);
}

// ------------------------------------------------ persistent batch

// The segment of [a, b) holding running block index x (largest k with seg_start[k] <= x).
__device__ __forceinline__ int batch_segment_of(const long long* seg_start, int a, int b,
                                                long long x) {
  int lo = a, hi = b - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg_start[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One virtual block of phase ph of group B (batch_units gives the counts).
__device__ void batch_unit(int ph, const BatchGroup& B, long long local, FwdShared& fsh) {
  const unsigned cnt = unsigned(B.cnt);
  if (ph == kPhFwdMap) {
    const unsigned bx = unsigned((B.fa.N + kFwdTile - 1) / kFwdTile);
    const uint3 bid = make_uint3(unsigned(local % bx), unsigned(local / bx), 0);
    const uint3 gd = make_uint3(bx, cnt, 1);
    // unrolled bodies for the row counts the planner produces (register arrays)
#define TM_FWD_ROWS(R)                                              \
  case R:                                                           \
    if (B.kind == TM_HI) fwd_hi_body<R>(B.fa, bid, gd, fsh.hi);     \
    else fwd_lo_full_body<R>(B.fa, B.kind, bid, gd, fsh.lo);        \
    break;
    switch (B.fa.lam - 1) {
      TM_FWD_ROWS(3) TM_FWD_ROWS(4) TM_FWD_ROWS(5) TM_FWD_ROWS(6) TM_FWD_ROWS(7)
      default:
        if (B.kind == TM_HI) fwd_hi_body<0>(B.fa, bid, gd, fsh.hi);
        else fwd_lo_full_body<0>(B.fa, B.kind, bid, gd, fsh.lo);
    }
#undef TM_FWD_ROWS
  } else if (ph >= kPhFwdPass && ph < kPhFwdPass + kMaxPasses) {
    const int i = ph - kPhFwdPass;
    const PassArgs& p = B.fwd[i];
    const unsigned bx = unsigned((p.Q + p.C - 1) / p.C);
    fft_pass_body<-1>(B.fwd_in[i], B.fwd_out[i], p,
                      make_uint3(unsigned(local % bx), unsigned(local / bx), 0),
                      make_uint3(bx, 2 * cnt, 1));
  } else if (ph == kPhTwist) {
    const unsigned bx = unsigned((B.M / 2 + kFusedThreads) / kFusedThreads);
    twist_body<false>(B.Zu, B.Zu + B.M, B.Q, B.M, B.tc, B.two_over_N, 2 * B.M, 2 * B.M,
                      make_uint3(unsigned(local % bx), unsigned(local / bx), 0),
                      make_uint3(bx, cnt, 1));
  } else if (ph >= kPhInvPass && ph < kPhInvPass + kMaxPasses) {
    const int i = ph - kPhInvPass;
    const PassArgs& p = B.inv[i];
    const unsigned bx = unsigned((p.Q + p.C - 1) / p.C);
    fft_pass_body<1>(B.inv_in[i], B.inv_out[i], p,
                     make_uint3(unsigned(local % bx), unsigned(local / bx), 0),
                     make_uint3(bx, cnt, 1));
  } else if (ph == kPhBack) {
    if (B.kind == TM_FULL) {
      const unsigned bx = unsigned(B.back_nvb);
      back_full_body(B.ba, make_uint3(unsigned(local % bx), unsigned(local / bx), 0),
                     make_uint3(bx, cnt, 1));
    } else if (B.back_small) {
      if (threadIdx.x < 32)
        back_small_body_k(B.ba, B.kind, make_uint3(0, unsigned(local), 0), make_uint3(1, cnt, 1));
    } else {
      const unsigned bx = unsigned((B.ba.N + kBackTile - 1) / kBackTile);
      const uint3 bid = make_uint3(unsigned(local % bx), unsigned(local / bx), 0);
      const uint3 gd = make_uint3(bx, cnt, 1);
#define TM_BACK_ROWS(R)                                             \
  case R:                                                           \
    if (B.kind == TM_LO) back_lo_body<R>(B.ba, bid, gd);            \
    else back_hi_body<R>(B.ba, bid, gd);                            \
    break;
      switch (B.kind == TM_LO ? B.ba.lam - 1 : B.ba.lam) {
        TM_BACK_ROWS(3) TM_BACK_ROWS(4) TM_BACK_ROWS(5) TM_BACK_ROWS(6) TM_BACK_ROWS(7)
        default:
          if (B.kind == TM_LO) back_lo_body<0>(B.ba, bid, gd);
          else back_hi_body<0>(B.ba, bid, gd);
      }
#undef TM_BACK_ROWS
    }
  } else if (ph == kPhCarryLocal || ph == kPhCarryApply) {
    const unsigned bx = unsigned(B.ca.nblocks_max);
    const uint3 bid = make_uint3(unsigned(local % bx), unsigned(local / bx), 0);
    if (ph == kPhCarryLocal) carry_local_body(B.ca, bid, make_uint3(bx, cnt, 1));
    else carry_apply_body(B.ca, bid, make_uint3(bx, cnt, 1));
  } else if (ph == kPhCarryBlocks) {
    carry_blocks_body<kFusedThreads>(B.ca, make_uint3(0, unsigned(local), 0));
  }
}

// Every product of a batch in one cooperative launch. The units (the virtual blocks of
// each group's maps, FFT passes, twist, back map and carry steps) are taken in list
// order by ticket; each waits, bounded by the global timer, until its group's
// earlier phases have finished, so groups advance independently and no grid-wide
// barrier is needed. The block bodies are the per-phase kernels'.
__global__ void __launch_bounds__(kFusedThreads, 2) k_batch_persistent(BatchArgs A) {
  __shared__ FwdShared fsh;
  // the unit's group descriptor, staged in shared memory: the block bodies copy
  // their argument structs per thread, and shared-memory reads of one address
  // are broadcast to the warp
  __shared__ __align__(16) unsigned long long gsh[(sizeof(BatchGroup) + 7) / 8];
  __shared__ int s_group, s_ok;
  __shared__ long long s_v;
  if (threadIdx.x == 0) s_group = -1;
  for (;;) {
    if (threadIdx.x == 0) s_v = (long long)atomicAdd(A.ticket, 1u);
    __syncthreads();
    const long long v = s_v;
    if (v >= A.total) break;                          // uniform
    const int k = batch_segment_of(A.seg_start, 0, A.nseg, v);
    const int g = A.seg_group[k];
    if (threadIdx.x == 0) {
      // the group's earlier phases: their units were taken before this one by CTAs
      // that are resident, so the wait ends; it is bounded all the same
      const long long need = A.seg_wait[k];
      const volatile unsigned* d = A.done + g;
      int ok = 1;
      if ((long long)*d < need) {
        const unsigned long long t0 = global_ns();
        while ((long long)*d < need) {
          if (global_ns() - t0 > kBarrierTimeoutNs) {
            atomicOr(&A.status->flags, kFlagTimeout);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;                                // uniform
    if (g != s_group) {                               // uniform: every thread reads s_group
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(A.groups + g);
      for (int t = threadIdx.x; t < int((sizeof(BatchGroup) + 7) / 8); t += blockDim.x)
        gsh[t] = src[t];
      __syncthreads();
      if (threadIdx.x == 0) s_group = g;
    }
    batch_unit(A.seg_phase[k], *reinterpret_cast<const BatchGroup*>(gsh), v - A.seg_start[k],
               fsh);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();                                // the unit's writes, then its count
      if (!(A.withhold && v == 0)) atomicAdd(A.done + g, 1u);
    }
  }
}

int batch_max_blocks(size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncAttributes fa{};
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (cudaFuncGetAttributes(&fa, k_batch_persistent) == cudaSuccess)
    cudaFuncSetAttribute(k_batch_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         optin - int(fa.sharedSizeBytes));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_persistent, kFusedThreads,
                                                    smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return per * sms;
}

cudaError_t launch_batch_persistent(const BatchArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(kFusedThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_batch_persistent, a);
}

// ------------------------------------------------ CTA-resident products

// In-shared-memory FFT of C sequences of length M (single pass, natural order).
template <int S>
__device__ void smem_fft(double2* Z, int M, int C, const SmallPlan& P, const double2* tws,
                         const Tan4* tw4s) {
  int Ns = 1;
  double2 xs[8];
  int base[4], kk[4];
  for (int st = 0; st < P.nstages; ++st) {
    const int R = P.radix[st];
    switch (R) {
      case 2: stockham_stage<2, S>(Z, M, C, Ns, tws, xs, base, kk); break;
      case 3: stockham_stage<3, S>(Z, M, C, Ns, tws, xs, base, kk); break;
      case 4:
        if (Ns > 1) stockham_stage4t<S>(Z, M, C, Ns, tw4s + P.tw4_off[st], xs, base, kk);
        else stockham_stage<4, S>(Z, M, C, Ns, tws, xs, base, kk);
        break;
      case 5: stockham_stage<5, S>(Z, M, C, Ns, tws, xs, base, kk); break;
      default: stockham_stage<7, S>(Z, M, C, Ns, tws, xs, base, kk); break;
    }
    __syncthreads();
    Ns *= R;
  }
}

// r_L = (A_L mod 2^64) + floor(A_(L-1) / 2^64), see the carry scan kernels
__device__ __forceinline__ __int128 limb_r(const CarryArgs& a, long long L) {
  if (L >= a.nS) return 0;
  const __int128 AL = limb_sum(a, L), Ap = limb_sum(a, L - 1);
  return (__int128)(unsigned long long)AL + (Ap >> 64);
}

size_t small_smem_bytes(long long N, long long M, int tw4_len, bool need_wL) {
  const size_t z = size_t((2 * M + 1) & ~1LL) + 2 * size_t(tw4_len) + (need_wL ? size_t(M) : 0);
  return z * sizeof(double2) + size_t(N + 2) * 8;
}

__global__ void __launch_bounds__(kSmallThreads, 1) k_small_products(SmallArgs A) {
  extern __shared__ double2 sm[];
  __shared__ int s_item;
  __shared__ unsigned long long s_bmax;
  __shared__ unsigned s_flags;
  __shared__ unsigned fs[kSmallThreads];
  __shared__ double s_theta[2], s_top[2];
  __shared__ double Pw[kMaxLam];
  __shared__ double Hh[kMaxLam + 64 + 1];
  // the current product's descriptor and plan, staged in shared memory (from the
  // arrays of a batch, or from the arguments for one product)
  __shared__ SmallItem s_it;
  __shared__ SmallPlan s_plan;
  const int tid = threadIdx.x;
  for (int round = 0;; ++round) {
    if (tid == 0) {
      s_item = A.items ? atomicAdd(A.counter, 1) : (round == 0 ? 0 : A.count);
      s_bmax = 0;
      s_flags = 0;
      if (s_item < A.count) {
        s_it = A.items ? A.items[s_item] : A.item0;
        s_plan = A.items ? A.plans[s_it.plan] : A.plan0;
      }
    }
    __syncthreads();
    const int idx = s_item;
    if (idx >= A.count) return;                       // uniform
    const SmallItem& it = s_it;
    const SmallPlan& P = s_plan;
    const int kind = P.kind, b = P.b;
    const int N = int(P.N), M = int(P.M);
    double2* Z = sm;
    const int off4 = (2 * M + 1) & ~1;
    Tan4* tw4s = reinterpret_cast<Tan4*>(sm + off4);
    double2* tws = sm + off4 + 2 * P.tw4_len;
    char* scratch = reinterpret_cast<char*>(tws + (P.need_wL ? M : 0));
    int* du = reinterpret_cast<int*>(scratch);
    int* dv = du + N;
    long long* cc = reinterpret_cast<long long*>(scratch);
    // 1. digits (split step) and the tables of this plan
    for (int p = tid; p < N; p += kSmallThreads) {
      int xu = 0, xv = 0;
      if (kind == TM_HI) {
        xu = balanced_digit(it.u, it.nlimbs, it.n, it.s0, b, p, N, true);
        xv = balanced_digit(it.v, it.nlimbs, it.n, it.s0, b, p, N, true);
      } else if (p < it.nd) {
        xu = balanced_digit(it.u, it.nlimbs, it.n, 0, b, p, it.nd - 1, false);
        xv = balanced_digit(it.v, it.nlimbs, it.n, 0, b, p, it.nd - 1, false);
      }
      du[p] = xu;
      dv[p] = xv;
    }
    if (kind == TM_HI && tid < 2) {
      const unsigned long long* src = tid == 0 ? it.u : it.v;
      s_top[tid] = i2d_exact(balanced_digit(src, it.nlimbs, it.n, it.s0, b, N, N, true));
    }
    for (int t = tid; t < P.tw4_len; t += kSmallThreads) tw4s[t] = P.tw4[t];
    if (P.need_wL)
      for (int t = tid; t < M; t += kSmallThreads) tws[t] = __ldg(P.tw_sub + t);
    __syncthreads();
    // 2. forward map (convert step): U~ at Z as doubles [0, N), V~ at [N, 2N)
    double* X = reinterpret_cast<double*>(Z);
    const int lam = kind == TM_FULL ? 0 : P.lam_fwd;
    const int Q = fx_q(b);
    const int headj = kind == TM_HI ? P.nkappa + lam - 1 : 0;
    for (int j = tid; j < N; j += kSmallThreads) {
      if (kind == TM_FULL) {
        X[j] = i2d_exact(du[j]);
        X[N + j] = i2d_exact(dv[j]);
      } else if (j < headj) {                        // high product, kappa-corrected F'
        double su = 0.0, sv = 0.0;
        for (int r = 0; r < lam; ++r) {
          int k = j - r;
          if (k < 0) k += N;
          double fu = i2d_exact(du[k]), fv = i2d_exact(dv[k]);
          if (k < P.nkappa) {
            const double kp = __ldg(P.kappa + k);
            fu = fma(kp, s_top[0], fu);
            fv = fma(kp, s_top[1], fv);
          }
          if (r == 0) {
            su = fu;
            sv = fv;
          } else {
            const double g = fx_coef(P.fwd_tab, N, r, k, Q, b);
            su = fma(g, fu, su);
            sv = fma(g, fv, sv);
          }
        }
        X[j] = su;
        X[N + j] = sv;
      } else {
        long long su = (long long)du[j] << Q, sv = (long long)dv[j] << Q;
        for (int r = 1; r < lam; ++r) {
          int k = j - r;
          if (k < 0) k += N;
          const long long Ac = __ldg(P.fwd_tab + (long long)(r - 1) * N + k);
          su += (Ac * du[k]) >> (r * b);
          sv += (Ac * dv[k]) >> (r * b);
        }
        X[j] = scale2(__ll2double_rn(su), -Q);
        X[N + j] = scale2(__ll2double_rn(sv), -Q);
      }
    }
    if (kind == TM_HI && (tid == 0 || tid == 32)) {   // theta = sum_j rho^-j F_(N-j)
      const int* d = tid == 0 ? du : dv;
      const double top = s_top[tid == 0 ? 0 : 1];
      double th = 0.0;
      for (int j = P.ntheta - 1; j >= 0; --j) {
        const int p = N - j;
        if (p < 0) continue;
        const double f = p == N ? top : i2d_exact(d[p]);
        th = fma(__ldg(P.rho_pow + j), f, th);
      }
      s_theta[tid == 0 ? 0 : 1] = th;
    }
    __syncthreads();
    // 3.-5. forward FFTs, twist + pointwise product, inverse FFT (convolution)
    smem_fft<-1>(Z, M, 2, P, tws, tw4s);
    for (int k = tid; k <= M / 2; k += kSmallThreads)
      twist_pair<false>(Z, Z + M, Z, M, k, P.twc, 2.0 / double(N));
    __syncthreads();
    smem_fft<1>(Z, M, 1, P, tws, tw4s);
    // 6. back map and rounding (convert back)
    BackArgs ba{};
    ba.w = X;
    ba.N = N;
    ba.b = b;
    ba.lam = kind == TM_FULL ? 0 : P.lam_bwd;
    ba.tab = P.bwd_tab;
    ba.tab2 = kind == TM_HI ? P.bwd_tab2 : P.bwd_tab;
    ba.kappa = P.kappa;
    ba.nkappa = P.nkappa;
    ba.theta = s_theta;
    ba.rho = P.rho;
    ba.c = cc;
    ba.count = kind == TM_HI ? N + 1 : N;
    ba.emax_fx = it.emax_fx;
    ba.status = A.status;
    if (kind == TM_FULL) {
      back_full_loop(ba, tid, kSmallThreads, &s_bmax);
    } else if (N <= 64 || N < 2 * ba.lam + ba.nkappa + 2) {
      if (tid == 0) back_small_body(ba, kind);
    } else if (kind == TM_LO) {
      back_lo_loop(ba, tid, kSmallThreads, &s_bmax, &s_flags);
    } else {
      back_hi_interior(ba, tid, kSmallThreads, &s_bmax);
      if (tid < 32) back_hi_head(ba, tid, Pw, Hh, &s_bmax, &s_flags);
    }
    __syncthreads();
    // 7. overlap-add and carries (one chunk of limbs per thread)
    CarryArgs ca{};
    ca.c = cc;
    ca.K = kind == TM_HI ? N + 1 : N;
    ca.b = b;
    ca.kind = kind;
    ca.nS = it.nS;
    ca.round_bit = it.round_bit;
    const long long chunk = (it.nS + kSmallThreads - 1) / kSmallThreads;
    const long long L0 = tid * chunk, L1 = L0 + chunk < it.nS ? L0 + chunk : it.nS;
    unsigned f = kIdentityFn;
    for (long long L = L0; L < L1; ++L) f = compose(carry_fn(limb_r(ca, L)), f);
    fs[tid] = f;
    __syncthreads();
    block_compose_scan(fs, kSmallThreads);
    int cin = apply_fn(tid ? fs[tid - 1] : kIdentityFn, 0);
    const long long sw = it.shift_bits >> 6;
    const int sb = int(it.shift_bits & 63);
    for (long long L = L0; L < L1; ++L) {
      const __int128 r = limb_r(ca, L);
      const unsigned long long limb = (unsigned long long)(r + cin);
      const int cnext = apply_fn(carry_fn(r), cin);
      const long long j = L - sw;
      if (j >= 0 && j < it.nout) {
        unsigned long long o = limb >> sb;
        if (sb) o |= (unsigned long long)(limb_r(ca, L + 1) + cnext) << (64 - sb);
        if (j == it.nout - 1) o &= it.top_mask;
        it.out[j] = o;
      }
      cin = cnext;
    }
    __syncthreads();
    if (tid == 0) {
      unsigned fl = s_flags;
      if (s_bmax) atomicMax(&A.status->margin_fx, s_bmax);
      if (s_bmax > it.emax_fx) fl |= kFlagPrecision;
      if (fl) atomicOr(&A.status->flags, fl);
    }
    __syncthreads();
  }
}

void set_small_smem_attribute(int bytes) {
  // the opt-in limit covers static and dynamic shared memory together
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k_small_products) == cudaSuccess)
    cudaFuncSetAttribute(k_small_products, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         bytes - int(fa.sharedSizeBytes));
  (void)cudaGetLastError();
}

void launch_small(const SmallArgs& a, int grid, size_t smem, cudaStream_t s) {
  if (a.count <= 0 || grid <= 0) return;
  k_small_products<<<grid, kSmallThreads, smem, s>>>(a);
}

// ------------------------------------------------------------ tables

// one thread per run of kTwRun entries, small blocks spread over the SMs
unsigned tw_blocks(long long count) {
  const long long per = (long long)kTwThreads * kTwRun;
  return unsigned((count + per - 1) / per);
}

void launch_init_twist_coef(double2* tab, long long N, long long count, cudaStream_t s) {
  if (count <= 0) return;
  k_init_twist_coef<<<tw_blocks(count), kTwThreads, 0, s>>>(tab, N, count);
}

void launch_init_twiddles(double2* tab, long long len, long long count, cudaStream_t s) {
  if (count <= 0) return;
  k_init_twiddles<<<tw_blocks(count), kTwThreads, 0, s>>>(tab, len, count);
}

void launch_init_outer(double2* tab, long long Mp, long long Qc, cudaStream_t s) {
  if (Mp <= 0 || Qc <= 0) return;
  k_init_outer<<<tw_blocks(Mp), kTwThreads, 0, s>>>(tab, Mp, Qc);
}

void launch_init_tw4(Tan4* tab, int Ns, cudaStream_t s) {
  if (Ns <= 0) return;
  k_init_tw4<<<tw_blocks(Ns), kTwThreads, 0, s>>>(tab, Ns);
}

void launch_init_maptab_fx(long long* tab, int which, long long N, int b, int rows, int Q,
                           cudaStream_t s) {
  if (rows <= 0) return;
  k_init_maptab_fx<<<unsigned((N + 255) / 256), 256, 0, s>>>(tab, which, N, b, rows, Q);
}

// FP64 FMA issue-rate probe: every thread runs 8 independent chains of `iters`
// dependent FMAs (2 flops each), then thread 0 of each block stores the block's
// first thread's sum, so the chains cannot be dropped.
__device__ double g_probe_sink[4096];
__global__ void __launch_bounds__(256) k_probe_dfma(int iters, double a, double c) {
  double x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 1e-3 * threadIdx.x + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (threadIdx.x == 0) g_probe_sink[blockIdx.x & 4095] = s;
}

double launch_probe_dfma(int iters, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;              // 8 CTAs of 256 threads: every warp slot
  k_probe_dfma<<<blocks, 256, 0, s>>>(iters, 0.9999999, 1e-7);
  return 2.0 * 8.0 * double(iters) * 256.0 * double(blocks);
}

// Holds the stream for about `ns` nanoseconds (one thread reads the global timer;
// at most 2^24 polls, so the kernel ends even if the timer stands still). The
// autotuners launch it before a timed run so that the host has enqueued the run
// before the device reaches it.
__global__ void k_delay(unsigned long long ns) {
  const unsigned long long t0 = global_ns();
  for (int i = 0; i < (1 << 24); ++i)
    if (global_ns() - t0 >= ns) break;
}

void launch_delay(unsigned long long ns, cudaStream_t s) {
  k_delay<<<1, 1, 0, s>>>(ns);
}

void launch_init_rho_powers(double* tab, int nkappa, int ntheta, int b, double lr,
                            cudaStream_t s) {
  if (nkappa + ntheta <= 0) return;
  k_init_rho_powers<<<unsigned((nkappa + ntheta + 127) / 128), 128, 0, s>>>(tab, nkappa, ntheta,
                                                                           b, lr);
}

void launch_init_maptab(double* tab, int which, long long N, int b, int rows, cudaStream_t s) {
  if (rows <= 0) return;
  k_init_maptab<<<unsigned((N + 255) / 256), 256, 0, s>>>(tab, which, N, b, rows);
}

}  // namespace tmul
