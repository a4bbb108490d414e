// Host-side plan of one product: digit size b, transform length, map lengths,
// FP64 error bound, FFT pass decomposition and kernel launch shapes.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

namespace tmul {

constexpr int kMaxStages = 16;     // radix stages inside one sub-FFT
constexpr int kMaxPasses = 3;      // HBM passes of one complex FFT
constexpr int kMaxSubLen = 4096;   // longest sub-FFT held in shared memory
constexpr int kMaxCL = 4096;       // sequences x length per CTA (2 buffers of 16 B each)

// One HBM pass of a complex FFT: Q independent sub-FFTs of length L. Sequence q
// has qc = q % Qc, qa = q / Qc; its element j is read at qa*IA + qc*IC + j*IS and
// its output k is written at qa*OA + qc*OC + k*OS, multiplied by
// omega_Mp^(qc*k) when Mp != 0 (the four-step twiddle).
struct FftPass {
  int L = 0;
  int nstages = 0;
  int radix[kMaxStages] = {};
  int64_t Q = 0, Qc = 0;
  int64_t IA = 0, IC = 0, IS = 0;
  int64_t OA = 0, OC = 0, OS = 0;
  int64_t Mp = 0;
  int C = 1;         // sequences per CTA
  int threads = 32;  // CTA size
  size_t tw_sub = 0;     // offset (in double2) of omega_L^k, k < L, in the twiddle table
  size_t tw_outer = 0;   // offset of omega_Mp^(qc k) at k Qc + qc (Mp = Qc L entries)
  // radix-4 stages with twiddles use tangent-form tables (t1, c1, t2, c2s) per
  // twiddle index: tw4 is their offset (double2 units, even), tw4_len the number
  // of double4 entries, tw4_off[s] the first entry of stage s (-1: none)
  size_t tw4 = 0;
  int tw4_len = 0;
  int tw4_off[kMaxStages] = {};
  bool need_wL = false;  // some stage still multiplies by omega_L^k
};

struct FftPlan {
  int64_t M = 0;         // complex length
  int npass = 0;
  FftPass pass[kMaxPasses];
};

struct PlanParams {
  int kind = 0;          // TM_FULL / TM_LO / TM_HI
  uint64_t n = 0;        // operand bits
  int b = 0;             // digit bits
  int64_t N = 0;         // real transform length
  int64_t n_digits = 0;  // digits per operand
  int lam_fwd = 0, lam_bwd = 0;
  double e_max = 0.0;    // bound on the rounding distance
  double rho = 0.0;      // auxiliary real root (high product only)
  double limit = 0.0;    // largest distance the device accepts (0: e_max)
};

// Chooses (b, N, lambda) for kind and n; returns 0 or a TM_E* code. Allocates no
// heap memory.
int choose_params(int kind, uint64_t n, PlanParams* out);

// The plan for a caller's digit size b and transform length N (the cyclic length
// of Algorithm 1 for the full product): lambda from the same tail budgets as the
// planner, e_max the worst-case bound for (b, N), which may exceed 1/2. TM_EINVAL
// when b is outside [4, 24], N is not a supported length, or (b, N) violates the
// hypotheses of Theorems 2.1-2.3 for n.
int explicit_params(int kind, uint64_t n, int b, int64_t N, PlanParams* out);

// Every certified plan (worst-case bound within the target) of (kind, n) whose
// transform length is at most `span` times the planner's, the planner's own plan
// first, the others by increasing N; at most max_count.
int certified_candidates(int kind, uint64_t n, double span, int max_count,
                         std::vector<PlanParams>* out);

// Layout choices of the FFT passes that the autotuner varies: points a CTA aims to
// hold (sequences per CTA = points / L), how the odd primes of M are distributed
// over the passes (0: each prime to the currently shortest pass, largest primes
// first; 1: all odd primes to the first pass; 2: all to the last pass), and the
// number of passes (0: 1 up to M = 64, 2 up to M = 2^22, else 3).
struct FftShape {
  int points = 1024;
  int split = 0;
  int passes = 0;
};

// Splits the complex length M into at most kMaxPasses sub-FFT passes and picks
// their radices and launch shapes. Twiddle offsets are left for the caller.
// single = true: one sub-FFT of length M (M <= kMaxSubLen), for CTA-resident products.
// Returns TM_ERANGE / TM_EINVAL when `shape` cannot lay out M. Allocates no heap
// memory.
int make_fft_plan(int64_t M, FftPlan* out, bool single = false, const FftShape* shape = nullptr);

// Data-dependent digit size. Measured norms of the balanced digits of u and v for
// one (b, N): nu, nv = ||U||_2, ||V||_2 (high product: of F_0 .. F_(N-1)), tu, tv
// = the high product's top digits F_N.
struct DigitNorms {
  double nu = 0, nv = 0, tu = 0, tv = 0;
};
// The length a plan with digit size b would take (the shortest admissible smooth
// length for (kind, n, b)); -1 when b is outside the planner's range.
int64_t measured_length(int kind, uint64_t n, int b);
// The plan (b, N) with its error bound evaluated on the measured norms (e_max):
// TM_OK when the bound is <= the target, TM_ERANGE when it is above (out still
// filled) or (b, N) is not admissible.
int measured_params(int kind, uint64_t n, int b, int64_t N, const DigitNorms& dn,
                    PlanParams* out);
// The worst-case norms for (kind, n, b, N) (every digit at its largest magnitude),
// and the target every plan's bound must meet.
DigitNorms worst_norms(int kind, uint64_t n, int b, int64_t N);
double bound_target();
// eta with |computed_k - (x*y)_k| <= eta ||x||_2 ||y||_2 for the FP64 cyclic
// convolution of real length L as the FFT kernels compute it (any pass layout).
double conv_error_bound(int64_t L);

// Exposed for tests of the planner.
bool is_valid_length(int64_t L);
int64_t smooth_at_least(int64_t x);

}  // namespace tmul
