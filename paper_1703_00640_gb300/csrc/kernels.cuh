// Kernel parameter blocks and launcher declarations shared by kernels.cu and api.cu.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "plan.h"

namespace tmul {

// Programmatic dependent launch (sm_90+): every kernel of the product pipeline lets
// the next launch proceed as soon as all of its own CTAs have started
// (griddepcontrol.launch_dependents), and waits for the previous kernel to complete
// and its writes to be visible (griddepcontrol.wait) before it touches data that
// kernel produced; only static tables are read before the wait. Kernels launched
// without the attribute see both as no-ops.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// <<<grid, block, smem, s>>> with the programmatic-serialization attribute.
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Device-side outcome of asynchronous calls on one workspace.
struct DevStatus {
  unsigned long long margin_fx;  // largest rounding distance, units of 2^-63
  unsigned int flags;            // kFlagPrecision | kFlagC0 | kFlagTimeout
  unsigned int pad;
};
constexpr unsigned kFlagPrecision = 1u;  // a distance above the plan's bound
constexpr unsigned kFlagC0 = 2u;         // 2^b does not divide c_0
constexpr unsigned kFlagTimeout = 4u;    // a bounded grid-wide wait gave up

// Tangent-form twiddle pair of one radix-4 butterfly (see launch_init_tw4).
struct __align__(32) Tan4 {
  double t1, c1, t2, c2s;
};

// Pass descriptor as seen by the FFT kernel (plan.h's FftPass plus pointers).
struct PassArgs {
  int L, nstages, C;
  int radix[kMaxStages];
  long long Q, Qc, IA, IC, IS, OA, OC, OS, Mp;
  long long batch_stride;        // complex elements between batch entries
  const double2* tw_sub;         // omega_L^k
  const double2* tw_outer;       // omega_Mp^(qc k) at k Qc + qc (or nullptr)
  const Tan4* tw4;            // tangent-form radix-4 stage tables
  int tw4_len;
  int tw4_off[kMaxStages];
  int need_wL;
  // Full product's split computed as the first pass loads: element m is the pair of
  // balanced digits (2m, 2m + 1) of the operand in map_limbs (0 from map_limit on),
  // as the forward map kernel forms them. map_limbs == nullptr: read `in`. Batch
  // entry 1 (blockIdx.y = 1) reads the second operand, map_limbs2.
  const unsigned long long* map_limbs;
  const unsigned long long* map_limbs2;
  unsigned long long map_n;
  long long map_nlimbs, map_limit;
  int map_b;
};

// Per-product fields of the forward map, back map and carry kernels. A batch of
// products with the same plan passes an array of items indexed by blockIdx.y;
// a single product passes items = nullptr and the fields of the args block.
struct FwdItem {
  const unsigned long long* u;
  const unsigned long long* v;
  unsigned long long n;
  long long nlimbs, nd, s0;
  double* X;
  double* theta;
};

// Digit unpack + forward map parameters.
struct FwdArgs {
  const FwdItem* items;
  const unsigned long long* u;
  const unsigned long long* v;
  unsigned long long n;          // operand bits
  long long nlimbs;
  int b;
  long long N;                   // transform length (real)
  long long nd;                  // digits per operand
  int lam;                       // map terms (0 for the full product)
  const long long* tab;          // (lam-1) x N fixed-point rows, r = 1..lam-1:
                                 // round(coef_{k,r} 2^(Q + r b)), Q = fx_q(b)
  const double* kappa;           // high: kappa_i = 2^b / rho^(i+1), i < nkappa
  int nkappa;
  const double* rho_pow;         // high: rho^-j, j < ntheta
  int ntheta;
  long long s0;                  // high: (N+1) b - n
  double* X;                     // out: u at X[0..N), v at X[N..2N)
  double* theta;                 // high: theta_U, theta_V
  int one_operand;               // 1: map u only (a square, a kept v, or v on another stream)
  const double* theta_v;         // one_operand: theta_V to copy into theta[1]
  int square_theta;              // one_operand: theta[1] = theta_U (a square)
  int tile;                      // positions per block, <= kFwdTile (0: kFwdTile)
};

struct BackItem {
  const double* w;
  long long* c;
  const double* theta;
  unsigned long long emax_fx;
};

struct BackArgs {
  const BackItem* items;
  const double* w;               // N real values (inverse FFT output)
  long long N;
  int b;
  int lam;
  const double* tab;             // low: beta rows r=1..lam-1; high: delta' rows r=1..lam
  const double* tab2;            // high: plain delta rows r=1..lam-1 (head positions)
  const double* kappa;
  int nkappa;
  const double* theta;           // high: theta_U, theta_V
  double rho;
  long long* c;                  // out: rounded coefficients
  long long count;               // number of c values (N, N+1 or L)
  unsigned long long emax_fx;    // bound, units of 2^-63
  DevStatus* status;
  int tile;                      // coefficients per block, <= kBackTile (0: kBackTile)
};

struct CarryItem {
  const long long* c;
  long long nS, round_bit, shift_bits, nout;
  unsigned long long top_mask;
  unsigned long long* out;
  unsigned long long* r;
  unsigned char* fblock;
  unsigned char* cin_block;
};

struct CarryArgs {
  const CarryItem* items;
  long long nblocks_max;         // grid width of the batched carry kernels
  const long long* c;
  long long K;                   // number of coefficients
  int b;
  int kind;
  long long nS;                  // limbs of S that are resolved
  long long round_bit;           // high: bit s-1 receives +1 (round half up); else -1
  long long shift_bits;          // output starts at this bit of S
  long long nout;                // output limbs
  unsigned long long top_mask;   // mask of the last output limb
  unsigned long long* out;
  unsigned long long* r;         // scratch: 2 x nS words (r_L as 128-bit)
  unsigned char* fblock;         // scratch: per-block carry functions
  unsigned char* cin_block;      // scratch: per-block carry-in (+1 encoded)
};

// One product in one cooperative launch (all phases, grid barriers between them).
constexpr int kFusedThreads = 512;
struct FusedArgs {
  int square;                    // u == v: one forward map and transform, squared twist
  int npass;
  FwdArgs fa;
  PassArgs fwd[kMaxPasses], inv[kMaxPasses];
  const double2* fwd_in[kMaxPasses];
  double2* fwd_out[kMaxPasses];
  const double2* inv_in[kMaxPasses];
  double2* inv_out[kMaxPasses];
  const double2* Zu;             // twist inputs and output
  const double2* Zv;
  double2* Q;
  long long M;
  const double2* tc;
  double two_over_N;
  BackArgs ba;
  int back_small;                // the back map of small N (one thread)
  CarryArgs ca;
  unsigned* sync;                // grid barrier: arrivals, generation (zeroed before launch)
  DevStatus* status;
  int leave_barrier;             // fault injection: the last CTA leaves at the first barrier
};
void set_fused_smem_attribute(int bytes);
// CTAs of kFusedThreads a cooperative launch of `kind` can keep resident with `smem`
// bytes of dynamic shared memory (0 when it cannot be determined).
int fused_max_blocks(int kind, size_t smem);
cudaError_t launch_fused(int kind, const FusedArgs& a, int grid, size_t smem, cudaStream_t s);

// Positions per block of the forward and back map kernels.
constexpr int kFwdTile = 1024;
constexpr int kBackTile = 1024;

// A batch in one cooperative launch: per plan group, the arguments of every phase
// in the items form of the per-phase kernels (product index in the block's y).
constexpr int kPhFwdMap = 0, kPhFwdPass = 1, kPhTwist = kPhFwdPass + kMaxPasses,
              kPhInvPass = kPhTwist + 1, kPhBack = kPhInvPass + kMaxPasses,
              kPhCarryLocal = kPhBack + 1, kPhCarryBlocks = kPhCarryLocal + 1,
              kPhCarryApply = kPhCarryBlocks + 1, kBatchPhases = kPhCarryApply + 1;
struct BatchGroup {
  int kind, npass, cnt, back_small;
  long long back_nvb;            // full product: back-map blocks per product
  FwdArgs fa;
  PassArgs fwd[kMaxPasses], inv[kMaxPasses];
  const double2* fwd_in[kMaxPasses];
  double2* fwd_out[kMaxPasses];
  const double2* inv_in[kMaxPasses];
  double2* inv_out[kMaxPasses];
  const double2* Zu;             // twist: product i's spectra at Zu + 2 M i (u), + M (v)
  double2* Q;
  long long M;
  const double2* tc;
  double two_over_N;
  BackArgs ba;
  CarryArgs ca;
};
// The launch runs nsteps steps separated by grid barriers. Step s is a list of
// segments [step_seg[s], step_seg[s+1]); segment k is phase seg_phase[k] of group
// seg_group[k], its virtual blocks numbered from seg_start[k] (a running sum over all
// segments). Staggering the groups' phases mixes FFT passes with maps and carries.
// The batch as one launch: the virtual blocks ("units") of every (group, phase)
// segment in one list, phases in order and the largest groups first within a phase.
// CTAs take units by ticket; a unit of phase p of group g starts once every unit of
// g's earlier phases has finished (seg_wait of them), so groups move through their
// phases independently.
struct BatchArgs {
  const BatchGroup* groups;
  int ngroups;
  int nseg;
  long long total;               // units of all segments
  const long long* seg_start;    // first unit of each segment (nseg + 1 entries)
  const int* seg_group;
  const int* seg_phase;
  const long long* seg_wait;     // units of the segment's group in earlier phases
  unsigned* ticket;              // next unit; zeroed before each launch
  unsigned* done;                // finished units per group; zeroed before each launch
  DevStatus* status;
  int withhold;                  // fault injection: unit 0 is never reported as finished
};
int batch_max_blocks(size_t smem);
cudaError_t launch_batch_persistent(const BatchArgs& a, int grid, size_t smem, cudaStream_t s);

// Fraction bits of the fixed-point forward maps: coefficient products
// (coef 2^(Q + r b)) x digit stay below 2^61.
__host__ __device__ inline int fx_q(int b) { return 61 - b; }

// CTA-resident products: one CTA computes a whole product of complex length
// M <= kSmallMaxM in shared memory (single-pass FFT tables).
constexpr long long kSmallMaxM = 2048;
constexpr int kSmallThreads = 1024;

struct SmallPlan {
  int kind, b, lam_fwd, lam_bwd, nkappa, ntheta;
  long long N, M;
  double rho;
  int nstages;
  int radix[kMaxStages];
  int tw4_off[kMaxStages];
  int tw4_len, need_wL;
  const double2* tw_sub;         // omega_M^k, k < M
  const Tan4* tw4;
  const double2* twc;            // twist coefficients (1 + omega_N^(2k)) / (2N), k <= M/2
  const long long* fwd_tab;
  const double* bwd_tab;
  const double* bwd_tab2;
  const double* kappa;
  const double* rho_pow;
};

struct SmallItem {
  const unsigned long long* u;
  const unsigned long long* v;
  unsigned long long* out;
  unsigned long long n;
  long long nlimbs, nd, s0;
  long long nS, round_bit, shift_bits, nout;
  unsigned long long top_mask, emax_fx;
  int plan;
};

struct SmallArgs {
  const SmallItem* items;        // nullptr: the one product item0 of plan plan0
  int count;
  const SmallPlan* plans;
  int* counter;                  // next item to take (zeroed before the launch; unused for one)
  DevStatus* status;
  SmallItem item0;
  SmallPlan plan0;
};

// shared memory a CTA-resident product of this plan needs
size_t small_smem_bytes(long long N, long long M, int tw4_len, bool need_wL);
void launch_small(const SmallArgs& a, int grid, size_t smem, cudaStream_t s);

// table initialisation
// tab[m] = omega_len^m = exp(-2 pi i m / len), m < count
void launch_init_twiddles(double2* tab, long long len, long long count, cudaStream_t s);
// tab[k Qc + qc] = omega_Mp^(qc k mod Mp), qc < Qc, k < Mp / Qc (Qc divides Mp): the
// four-step twiddles in a pass's output order
void launch_init_outer(double2* tab, long long Mp, long long Qc, cudaStream_t s);
// tab[k] = (1 + omega_N^(2k)) / (2N), k < count (coefficients of the fused twist)
void launch_init_twist_coef(double2* tab, long long N, long long count, cudaStream_t s);
// Tangent-form twiddles of one radix-4 Stockham stage with Ns > 1: entry k < Ns
// holds (t1, c1, t2, c2s) with omega_(4Ns)^k = c1 (1 - i t1) and
// omega_(4Ns)^(2k) = c2 (1 - i t2) when its angle is below pi/2, else
// -i c (1 - i t2) stored with c2s = -c.
void launch_init_tw4(Tan4* tab, int Ns, cudaStream_t s);
void launch_init_maptab(double* tab, int which, long long N, int b, int rows, cudaStream_t s);
// The same coefficients in fixed point: tab[(r-1) N + k] = round(coef_{k,r} 2^(Q + r b)).
void launch_init_maptab_fx(long long* tab, int which, long long N, int b, int rows, int Q,
                           cudaStream_t s);

// FP64 FMA issue-rate probe on every SM; returns the flops it enqueued.
double launch_probe_dfma(int iters, cudaStream_t s);

// High product: tab[i] = 2^b / rho^(i+1), i < nkappa, then tab[nkappa + j] = rho^-j,
// j < ntheta (lr = ln rho).
void launch_init_rho_powers(double* tab, int nkappa, int ntheta, int b, double lr,
                            cudaStream_t s);

// Sums of squares of the balanced digits of u and v (and the top digits of the high
// product) into sums[0..3] (zeroed by the caller).
void launch_digit_norms(const unsigned long long* u, const unsigned long long* v,
                        long long nlimbs, unsigned long long n, long long shift, int b,
                        long long count, long long top, bool top_unbalanced,
                        unsigned long long* sums, cudaStream_t s);

// pipeline stages
void launch_fwd(int kind, const FwdArgs& a, int batch, cudaStream_t s);
void set_fft_smem_attribute();
void launch_fft_pass(int dir, const double2* in, double2* out, const PassArgs& p, int batch,
                     int threads, cudaStream_t s);
// Spectra Zu + y zstride (u) and Zv + y zstride (v) -> Q + y qstride for product
// y < batch (real transform length N, complex length M = N/2, coefficients tc from
// launch_init_twist_coef). Zv == Zu squares u's spectrum.
void launch_twist(const double2* Zu, const double2* Zv, double2* Q, long long M,
                  const double2* tc, long long N, int batch, long long zstride,
                  long long qstride, cudaStream_t s);
void launch_back(int kind, const BackArgs& a, int batch, cudaStream_t s);
void launch_carry(const CarryArgs& a, int batch, cudaStream_t s);
// Copies the status word to page-locked host memory mapped into the device's
// address space and resets it, in stream order after the work before it.
void launch_status_publish(DevStatus* status, DevStatus* host, cudaStream_t s);

// map table selectors for launch_init_maptab
constexpr int kTabAlpha = 0, kTabBeta = 1, kTabGamma = 2, kTabDelta = 3, kTabDeltaPrime = 4;

}  // namespace tmul
