// Internal runtime of the library shared by api.cu and batch.cu: resident plan
// tables, workspaces, the per-product launch sequence.
#pragma once
#include <atomic>
#include <cstdint>
#include <memory>

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "plan.h"

namespace tmul {

// Resident device tables of one (device, kind, n).
struct PlanEntry {
  PlanParams p;
  FftPlan fft;
  int64_t M = 0;
  double2* tw = nullptr;       // all twiddle tables
  size_t twc_off = 0;          // (1 + omega_N^(2k)) / (2N), k <= M/2 (fused twist)
  long long* fwd_tab = nullptr;   // alpha or gamma rows r = 1..lam_fwd-1, fixed point
  double* bwd_tab = nullptr;   // beta rows (low) or delta' rows (high)
  double* bwd_tab2 = nullptr;  // high: delta rows r = 1..lam_bwd-1
  double* small = nullptr;     // high: kappa[nkappa] then rho^-j[ntheta]
  int nkappa = 0, ntheta = 0;
  size_t table_bytes = 0;
};

struct Workspace {
  char* base = nullptr;
  size_t size = 0;
  DevStatus* status = nullptr;
  char* io = nullptr;          // staging for tm_mul_host
  size_t io_size = 0;
  // second stream for the operand v's split and forward FFT, forked from and
  // joined into the workspace's stream (nullptr: one stream)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  unsigned long long* norms = nullptr;   // 4 words for the measured digit norms
  DevStatus* status_host = nullptr;      // page-locked copy of the status (tm_mul_host)
  bool sync_ready = false;               // the single-launch barrier words are zeroed
  // set around enqueue when the operands are mapped host memory: the forward map then
  // runs as its own kernel, which reads each limb once
  bool operands_mapped = false;
};

size_t align_up(size_t x);
// The margin bound the device checks, e_max in units of 2^-63. Fault injection on
// the host: the environment variable TRUNCMUL_FAULT_EMAX_SCALE (a number in (0, 1],
// read once per process) scales every bound down, so that the device-side margin
// check fails and the TM_EPRECISION path can be exercised without a GPU fault.
unsigned long long emax_fixed(double e_max);
int64_t limbs_of(uint64_t n);
int64_t out_limbs(int kind, uint64_t n);
void carry_shape(const PlanParams& p, int64_t* nS, int64_t* shift, int64_t* round_bit);
size_t workspace_bytes(const PlanParams& p);
// (kind, n) -> parameters, cached (host only)
int get_params(int kind, uint64_t n, PlanParams* out);
// resident tables for the plan's (kind, b, N) on the current device; single_pass
// lays the FFT out as one sub-FFT of length N/2 (for CTA-resident products)
int get_tables(const PlanParams& p, bool single_pass, cudaStream_t s,
               std::shared_ptr<PlanEntry>* out);
// FFT passes of a batch of `batch` sequences of length M (stride `stride`),
// ping-ponging bufs[cur] <-> bufs[cur ^ 1]; returns the buffer index holding the result
// With map_limbs, the first pass of a forward transform computes its input, the full
// product's split (Algorithm 1) of the operand map_limbs under the call's plan *map_p
// (its n and digit count, which tables shared across n do not carry), as it loads
// it, instead of reading bufs[cur]; with batch 2, sequence 1 is the split of
// map_limbs2.
int launch_fft(const PlanEntry& pe, double2* const* bufs, int cur, int dir, int batch,
               long long stride, cudaStream_t s, const uint64_t* map_limbs = nullptr,
               const PlanParams* map_p = nullptr, const uint64_t* map_limbs2 = nullptr);
// True when every pass of the plan's FFT fills the GPU with one sequence (at least
// 1024 threads per SM): only then do two sequences gain from running on two streams.
bool fft_fills_gpu(const FftPlan& fft);
// a one-thread kernel (csrc/kernels.cu) that holds the stream for about ns
// nanoseconds (bounded): the autotuners' timed runs start behind it
void launch_delay(unsigned long long ns, cudaStream_t s);
void ensure_kernel_attributes();
// Forward transform of one operand kept on the device: the spectrum of V~ (complex
// length M, the order the forward FFT leaves it in) and theta_V (high product).
struct KeptOperand {
  const double2* spec;
  const double* theta;
};
// One whole product on stream s with workspace ws (see api.cu). u == v squares
// (one forward map and one forward FFT); kept != nullptr takes v's transform from
// it (v is then ignored).
// Fault injection for tests of the single-launch paths: with TRUNCMUL_FAULT_BARRIER=1
// (read once) the last CTA of each cooperative launch leaves at the first grid
// barrier, so the others' bounded waits run out and the call reports TM_ETIMEOUT.
bool fault_leave_barrier();
// How products run (tm_set_fused): 0 automatic, 1 per-phase launches only, 2 one
// cooperative launch wherever the layout allows.
extern std::atomic<int> g_fused_mode;
// The pass arguments of pass i of a plan's FFT (stride: elements between batch
// entries), and the dynamic shared memory of that pass with C sequences per CTA.
PassArgs pass_args(const PlanEntry& pe, int i, long long stride);
size_t pass_smem(const FftPass& fp, int C);
void ensure_kernel_attributes();

int enqueue(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n,
            cudaStream_t s, const PlanParams& p, const PlanEntry& pe, Workspace& ws,
            int64_t* coeff_out, void* const* events, const KeptOperand* kept = nullptr);
// Split, forward map and forward FFT of v alone into spec (M complex) and theta (2
// doubles), through workspace ws.
int enqueue_transform(int kind, const uint64_t* v, uint64_t n, cudaStream_t s,
                      const PlanParams& p, const PlanEntry& pe, Workspace& ws, double2* spec,
                      double* theta);
// Single-pass plan tables of a CTA-resident product, and its per-product item.
SmallPlan small_plan_of(const PlanParams& p, const PlanEntry& pe);
// The CTA-resident kernel's descriptor of one product (plan index `plan`).
SmallItem small_item_for(const void* out, const void* u, const void* v, uint64_t n,
                         const PlanParams& q, int plan);
// Waits for s, reads the status word into *rep and resets it. may_allocate = false
// keeps to calls that allocate nothing (no page-locked status buffer).
int read_status(cudaStream_t s, DevStatus* status, tm_report* rep, bool may_allocate = true);
// Waits for s and copies the status word of its workspace out (save) or back in.
int stream_status_word(cudaStream_t s, DevStatus* word, bool save);
void fill_plan_report(const PlanParams& p, const FftPlan& f, tm_report* rep);

}  // namespace tmul
