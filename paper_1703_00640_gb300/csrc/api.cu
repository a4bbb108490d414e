// C ABI of the library (declared in include/truncmul.h): plan cache, per-stream
// workspaces and the launch sequence of one product.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/truncmul.h"
#include "kernels.cuh"
#include "plan.h"
#include "runtime.h"

namespace tmul {

namespace {
std::mutex g_mu;
std::map<std::tuple<int, int, int, int64_t, int>, std::shared_ptr<PlanEntry>> g_plans;
std::map<std::pair<int, uint64_t>, PlanParams> g_params;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;
// FFT layouts chosen by tm_autotune, per (device, complex length M), and plan
// entries replaced after tuning (still referenced by batches; freed by tm_release)
std::map<std::pair<int, int64_t>, FftShape> g_tuned;
std::vector<std::shared_ptr<PlanEntry>> g_retired;

// Makes `shape` (nullptr: the default) the layout of every later plan of
// transform length N on device `dev`. Plans of that length built before keep
// their layout for their holders (batches); the cache rebuilds them.
void apply_layout(int dev, int64_t N, const FftShape* shape) {
  std::lock_guard<std::mutex> lk(g_mu);
  const auto key = std::make_pair(dev, N / 2);
  if (!shape) g_tuned.erase(key);
  else g_tuned[key] = *shape;
  for (auto it = g_plans.begin(); it != g_plans.end();) {
    if (std::get<0>(it->first) == dev && std::get<3>(it->first) == N &&
        std::get<4>(it->first) == 0) {
      g_retired.push_back(it->second);
      it = g_plans.erase(it);
    } else {
      ++it;
    }
  }
}

// tm_mul_host's whole sequence (copies in, product, copies out, status) recorded once
// per (device, stream, kind, n, square) as a CUDA graph; later calls only point the
// three host copies at the new buffers and launch it. Valid while the io buffer,
// workspace and plan tables it was recorded with are the current ones.
struct HostGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t in_u = nullptr, in_v = nullptr, out = nullptr;
  char* io = nullptr;
  char* ws_base = nullptr;
  const PlanEntry* pe = nullptr;
};
std::map<std::tuple<int, cudaStream_t, int, uint64_t, bool>, HostGraph> g_host_graphs;

void drop_host_graph(HostGraph& h) {
  if (h.exec) cudaGraphExecDestroy(h.exec);
  if (h.graph) cudaGraphDestroy(h.graph);
  h = HostGraph{};
}

int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return TM_ENOMEM;
  return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

#define TM_CHECK(x)                                   \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) {                          \
      (void)cudaGetLastError();                       \
      return cuda_fail(e_);                           \
    }                                                 \
  } while (0)

}  // namespace

size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

bool fault_leave_barrier() {
  static const bool on = [] {
    const char* v = std::getenv("TRUNCMUL_FAULT_BARRIER");
    return v && v[0] == '1' && v[1] == 0;
  }();
  return on;
}

unsigned long long emax_fixed(double e_max) {
  static const double scale = [] {
    const char* v = std::getenv("TRUNCMUL_FAULT_EMAX_SCALE");
    if (!v) return 1.0;
    char* end = nullptr;
    const double x = std::strtod(v, &end);
    return (end != v && x > 0.0 && x <= 1.0) ? x : 1.0;
  }();
  return (unsigned long long)std::ldexp(e_max * scale, 63);
}

int64_t limbs_of(uint64_t n) { return int64_t((n + 63) / 64); }
int64_t out_limbs(int kind, uint64_t n) {
  if (kind == TM_FULL) return 2 * limbs_of(n);
  if (kind == TM_LO) return limbs_of(n);
  return int64_t(n / 64) + 1;
}

// Limbs of S the carry scan resolves, and where the output window starts.
void carry_shape(const PlanParams& p, int64_t* nS, int64_t* shift, int64_t* round_bit) {
  const int64_t nout = out_limbs(p.kind, p.n);
  if (p.kind == TM_HI) {
    const int64_t s = (p.N + 3) * int64_t(p.b) - int64_t(p.n);   // Algorithm 3, overlap-add
    *shift = s;
    *round_bit = s - 1;
    *nS = (s + 64 * nout + 63) / 64 + 1;
  } else {
    *shift = 0;
    *round_bit = -1;
    *nS = nout;
  }
}

size_t workspace_bytes(const PlanParams& p) {
  const int64_t M = p.N / 2;
  const size_t region = align_up(size_t(2) * M * sizeof(double2));
  int64_t nS, sh, rb;
  carry_shape(p, &nS, &sh, &rb);
  const size_t carry = align_up(size_t(2) * nS * 8) + 2 * align_up(size_t(nS / 512 + 2));
  const size_t coeff = align_up(size_t(p.N + 2) * 8);
  return std::max(region, coeff) + std::max(region, carry) + 256;
}

// Offsets of every twiddle table of a plan inside one double2 allocation:
// per pass omega_L (when a stage needs it), omega_Mp^(qc k) in output order (Mp
// entries), the radix-4 tangent
// tables; then the twist coefficients (1 + omega_N^(2k)) / (2N), k <= M/2.
// Returns the count.
size_t layout_twiddles(PlanEntry* e) {
  size_t cnt = 0;
  for (int i = 0; i < e->fft.npass; ++i) {
    FftPass& fp = e->fft.pass[i];
    int Ns = 1, len4 = 0;
    fp.need_wL = false;
    for (int st = 0; st < fp.nstages; ++st) {
      const int R = fp.radix[st];
      if (R == 4 && Ns > 1) {
        fp.tw4_off[st] = len4;
        len4 += Ns;
      } else {
        fp.tw4_off[st] = -1;
        if (Ns > 1) fp.need_wL = true;
      }
      Ns *= R;
    }
    fp.tw_sub = cnt;
    cnt += size_t(fp.L);
    if (fp.Mp) { fp.tw_outer = cnt; cnt += size_t(fp.Mp); }
    cnt = (cnt + 1) & ~size_t(1);
    fp.tw4 = cnt;
    fp.tw4_len = len4;
    cnt += 2 * size_t(len4);
  }
  e->twc_off = cnt;
  cnt += size_t(e->M / 2 + 1);
  return cnt;
}

void init_twiddles(const PlanEntry& e, cudaStream_t s) {
  for (int i = 0; i < e.fft.npass; ++i) {
    const FftPass& fp = e.fft.pass[i];
    launch_init_twiddles(e.tw + fp.tw_sub, fp.L, fp.L, s);
    if (fp.Mp) launch_init_outer(e.tw + fp.tw_outer, fp.Mp, fp.Qc, s);
    int Ns = 1;
    for (int st = 0; st < fp.nstages; ++st) {
      if (fp.tw4_off[st] >= 0)
        launch_init_tw4(reinterpret_cast<Tan4*>(e.tw + fp.tw4) + fp.tw4_off[st], Ns, s);
      Ns *= fp.radix[st];
    }
  }
  launch_init_twist_coef(e.tw + e.twc_off, e.p.N, e.M / 2 + 1, s);
}

namespace {

int build_tables(const PlanParams& p, bool single, cudaStream_t s, std::shared_ptr<PlanEntry>* out) {
  auto e = std::make_shared<PlanEntry>();
  e->p = p;
  const int kind = p.kind;
  e->M = e->p.N / 2;
  const FftShape* shape = nullptr;
  if (!single) {
    int dev = 0;
    TM_CHECK(cudaGetDevice(&dev));
    auto t = g_tuned.find(std::make_pair(dev, e->M));
    if (t != g_tuned.end()) shape = &t->second;
  }
  int rc = make_fft_plan(e->M, &e->fft, single, shape);
  if (rc) return rc;
  const size_t cnt = layout_twiddles(e.get());
  TM_CHECK(cudaMalloc(&e->tw, cnt * sizeof(double2)));
  e->table_bytes += cnt * sizeof(double2);
  init_twiddles(*e, s);
  const int64_t N = e->p.N;
  const int b = e->p.b;
  if (kind == TM_LO || kind == TM_HI) {
    const int rf = e->p.lam_fwd - 1;
    const int rb = kind == TM_LO ? e->p.lam_bwd - 1 : e->p.lam_bwd;
    if (rf > 0) {
      TM_CHECK(cudaMalloc(&e->fwd_tab, size_t(rf) * N * 8));
      launch_init_maptab_fx(e->fwd_tab, kind == TM_LO ? kTabAlpha : kTabGamma, N, b, rf,
                            fx_q(b), s);
      e->table_bytes += size_t(rf) * N * 8;
    }
    if (rb > 0) {
      TM_CHECK(cudaMalloc(&e->bwd_tab, size_t(rb) * N * 8));
      launch_init_maptab(e->bwd_tab, kind == TM_LO ? kTabBeta : kTabDeltaPrime, N, b,
                         kind == TM_LO ? rb : e->p.lam_bwd, s);
      e->table_bytes += size_t(rb) * N * 8;
    }
    if (kind == TM_HI && e->p.lam_bwd > 1) {
      const int r2 = e->p.lam_bwd - 1;
      TM_CHECK(cudaMalloc(&e->bwd_tab2, size_t(r2) * N * 8));
      launch_init_maptab(e->bwd_tab2, kTabDelta, N, b, r2, s);
      e->table_bytes += size_t(r2) * N * 8;
    }
  }
  if (kind == TM_HI) {
    // kappa_i = 2^b / rho^(i+1) (eq. 4.4) while it can still reach the rounded
    // coefficients: i <= 3 + (lg N + 64) / b; theta needs rho^-j, j <= 60/b + 3.
    int lgN = 0;
    while ((int64_t(1) << lgN) < N) ++lgN;
    e->nkappa = int(std::min<int64_t>(N, 3 + (lgN + 64 + b - 1) / b));
    e->ntheta = int(std::min<int64_t>(N + 1, (60 + b - 1) / b + 3));
    std::vector<double> host(size_t(e->nkappa + e->ntheta));
    const double rho = e->p.rho;
    const double lr = std::log(rho);
    for (int i = 0; i < e->nkappa; ++i) host[i] = std::exp(b * std::log(2.0) - (i + 1) * lr);
    for (int j = 0; j < e->ntheta; ++j) host[e->nkappa + j] = std::exp(-j * lr);
    TM_CHECK(cudaMalloc(&e->small, host.size() * 8));
    TM_CHECK(cudaMemcpyAsync(e->small, host.data(), host.size() * 8, cudaMemcpyHostToDevice, s));
    e->table_bytes += host.size() * 8;
  }
  TM_CHECK(cudaGetLastError());
  TM_CHECK(cudaStreamSynchronize(s));
  *out = e;
  return TM_OK;
}

}  // namespace

int get_params(int kind, uint64_t n, PlanParams* out) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_params.find(std::make_pair(kind, n));
    if (it != g_params.end()) { *out = it->second; return TM_OK; }
  }
  PlanParams p;
  const int rc = choose_params(kind, n, &p);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  g_params[std::make_pair(kind, n)] = p;
  *out = p;
  return TM_OK;
}

int get_tables(const PlanParams& p, bool single, cudaStream_t s, std::shared_ptr<PlanEntry>* out) {
  int dev = 0;
  TM_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_tuple(dev, p.kind, p.b, p.N, single ? 1 : 0);
  auto it = g_plans.find(key);
  if (it != g_plans.end()) { *out = it->second; return TM_OK; }
  std::shared_ptr<PlanEntry> e;
  const int rc = build_tables(p, single, s, &e);
  if (rc) return rc;
  g_plans[key] = e;
  *out = e;
  return TM_OK;
}

namespace {

int get_workspace(cudaStream_t s, size_t bytes, Workspace** out) {
  int dev = 0;
  TM_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace& w = g_ws[std::make_pair(dev, s)];
  if (!w.status) {
    TM_CHECK(cudaMalloc(&w.status, sizeof(DevStatus)));
    TM_CHECK(cudaMemsetAsync(w.status, 0, sizeof(DevStatus), s));
    TM_CHECK(cudaMalloc(&w.norms, 4 * sizeof(unsigned long long)));
    TM_CHECK(cudaMallocHost(&w.status_host, sizeof(DevStatus)));
    TM_CHECK(cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking));
    TM_CHECK(cudaEventCreateWithFlags(&w.fork, cudaEventDisableTiming));
    TM_CHECK(cudaEventCreateWithFlags(&w.join, cudaEventDisableTiming));
  }
  if (bytes && w.size < bytes) {
    if (w.base) {
      TM_CHECK(cudaStreamSynchronize(s));
      TM_CHECK(cudaFree(w.base));
      w.base = nullptr;
      w.size = 0;
    }
    TM_CHECK(cudaMalloc(&w.base, bytes));
    w.size = bytes;
  }
  *out = &w;
  return TM_OK;
}

int get_io(cudaStream_t s, size_t bytes, char** out) {
  Workspace* w = nullptr;
  int rc = get_workspace(s, 0, &w);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  if (w->io_size < bytes) {
    if (w->io) {
      TM_CHECK(cudaStreamSynchronize(s));
      TM_CHECK(cudaFree(w->io));
      w->io = nullptr;
      w->io_size = 0;
    }
    TM_CHECK(cudaMalloc(&w->io, bytes));
    w->io_size = bytes;
  }
  *out = w->io;
  return TM_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + nb && y < x + na;
}

// The device address of page-locked host memory mapped into the device's address
// space, or nullptr (pageable memory, device memory, an unknown pointer).
const uint64_t* mapped_host(const void* h) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? static_cast<const uint64_t*>(a.devicePointer) : nullptr;
}

}  // namespace

void ensure_kernel_attributes() {
  static std::once_flag once;
  std::call_once(once, [] { set_fft_smem_attribute(); });
}

int launch_fft(const PlanEntry& pe, double2* const* bufs, int cur, int dir, int batch,
               long long stride, cudaStream_t s, const uint64_t* map_limbs,
               const PlanParams* map_p, const uint64_t* map_limbs2) {
  for (int i = 0; i < pe.fft.npass; ++i) {
    const FftPass& fp = pe.fft.pass[i];
    PassArgs a{};
    if (i == 0 && map_limbs && map_p) {
      const PlanParams& p = *map_p;
      a.map_limbs = reinterpret_cast<const unsigned long long*>(map_limbs);
      a.map_limbs2 = reinterpret_cast<const unsigned long long*>(map_limbs2);
      a.map_n = p.n;
      a.map_nlimbs = limbs_of(p.n);
      a.map_limit = std::min<int64_t>(p.N, p.n_digits);
      a.map_b = p.b;
    }
    a.L = fp.L; a.nstages = fp.nstages; a.C = fp.C;
    std::copy(fp.radix, fp.radix + kMaxStages, a.radix);
    a.Q = fp.Q; a.Qc = fp.Qc; a.IA = fp.IA; a.IC = fp.IC; a.IS = fp.IS;
    a.OA = fp.OA; a.OC = fp.OC; a.OS = fp.OS; a.Mp = fp.Mp;
    a.batch_stride = stride;
    a.tw_sub = pe.tw + fp.tw_sub;
    a.tw_outer = fp.Mp ? pe.tw + fp.tw_outer : nullptr;
    a.tw4 = reinterpret_cast<const Tan4*>(pe.tw + fp.tw4);
    a.tw4_len = fp.tw4_len;
    std::copy(fp.tw4_off, fp.tw4_off + kMaxStages, a.tw4_off);
    a.need_wL = fp.need_wL ? 1 : 0;
    launch_fft_pass(dir, bufs[cur], bufs[cur ^ 1], a, batch, fp.threads, s);
    cur ^= 1;
  }
  return cur;
}

bool fft_fills_gpu(const FftPlan& fft) {
  static const long long sm_threads = [] {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      (void)cudaGetLastError();
      sms = 152;
    }
    return 1024LL * sms;
  }();
  for (int i = 0; i < fft.npass; ++i) {
    const FftPass& fp = fft.pass[i];
    if ((fp.Q + fp.C - 1) / fp.C * fp.threads < sm_threads) return false;
  }
  return true;
}

namespace {
// One page-locked status word per host thread (mapped: the device writes it).
DevStatus* thread_status_host() {
  thread_local struct Holder {
    DevStatus* p = nullptr;
    ~Holder() { if (p) cudaFreeHost(p); }
  } h;
  if (!h.p && cudaHostAlloc(&h.p, sizeof(DevStatus),
                            cudaHostAllocPortable | cudaHostAllocMapped) != cudaSuccess) {
    (void)cudaGetLastError();
    h.p = nullptr;
  }
  return h.p;
}
}  // namespace

int stream_status_word(cudaStream_t s, DevStatus* word, bool save) {
  int dev = 0;
  TM_CHECK(cudaGetDevice(&dev));
  DevStatus* st = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ws.find(std::make_pair(dev, s));
    if (it != g_ws.end()) st = it->second.status;
  }
  if (!st) {                     // no workspace yet: nothing pending, nothing to restore
    if (save) *word = DevStatus{};
    return TM_OK;
  }
  TM_CHECK(cudaStreamSynchronize(s));
  if (save)
    TM_CHECK(cudaMemcpy(word, st, sizeof(DevStatus), cudaMemcpyDeviceToHost));
  else
    TM_CHECK(cudaMemcpy(st, word, sizeof(DevStatus), cudaMemcpyHostToDevice));
  return TM_OK;
}

int read_status(cudaStream_t s, DevStatus* status, tm_report* rep, bool may_allocate) {
  DevStatus st{};
  DevStatus* h = may_allocate ? thread_status_host() : nullptr;
  DevStatus* hd = nullptr;
  if (h && cudaHostGetDevicePointer(reinterpret_cast<void**>(&hd), h, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    hd = nullptr;
  }
  if (hd) {                      // one kernel and one wait
    launch_status_publish(status, hd, s);
    TM_CHECK(cudaGetLastError());
    TM_CHECK(cudaStreamSynchronize(s));
    const volatile DevStatus* vh = h;
    st.margin_fx = vh->margin_fx;
    st.flags = vh->flags;
  } else {
    TM_CHECK(cudaStreamSynchronize(s));
    TM_CHECK(cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
    TM_CHECK(cudaMemsetAsync(status, 0, sizeof(DevStatus), s));
    TM_CHECK(cudaStreamSynchronize(s));
  }
  const int code = (st.flags & kFlagTimeout) ? TM_ETIMEOUT : st.flags ? TM_EPRECISION : TM_OK;
  if (rep) {
    rep->margin = std::ldexp(double(st.margin_fx), -63);
    rep->status = code;
  }
  return code;
}

void fill_plan_report(const PlanParams& p, const FftPlan& f, tm_report* rep) {
  rep->kind = p.kind;
  rep->status = TM_OK;
  rep->b = uint32_t(p.b);
  rep->N = uint32_t(p.N);
  rep->n_digits = uint32_t(p.n_digits);
  rep->lam_fwd = uint32_t(p.lam_fwd);
  rep->lam_bwd = uint32_t(p.lam_bwd);
  rep->fft_passes = uint32_t(f.npass);
  rep->fwd_streams = fft_fills_gpu(f) ? 2u : 1u;
  rep->margin = 0.0;
  rep->e_max = p.e_max;
  rep->workspace_bytes = workspace_bytes(p);
  rep->table_bytes = 0;
}

// Enqueues one whole product with parameters p and tables pe; `coeff_out`
// receives the rounded coefficients and stops the pipeline before the carry
// scan when non-null.
namespace {

// Digits and forward map (split and convert steps of Algorithms 1-3) of u and v,
// or of u alone (one_operand), into X.
void fwd_args(int kind, const uint64_t* u, const uint64_t* v, uint64_t n, const PlanParams& p,
              const PlanEntry& pe, double* X, double* theta, bool one_operand,
              const double* theta_v, bool square_theta, FwdArgs* out) {
  FwdArgs fa{};
  fa.u = reinterpret_cast<const unsigned long long*>(u);
  fa.v = reinterpret_cast<const unsigned long long*>(v);
  fa.n = n;
  fa.nlimbs = limbs_of(n);
  fa.b = p.b;
  fa.N = p.N;
  fa.nd = p.n_digits;
  fa.lam = kind == TM_FULL ? 0 : p.lam_fwd;
  fa.tab = pe.fwd_tab;
  fa.kappa = pe.small;
  fa.nkappa = pe.nkappa;
  fa.rho_pow = pe.small ? pe.small + pe.nkappa : nullptr;
  fa.ntheta = pe.ntheta;
  fa.s0 = int64_t(p.N + 1) * p.b - int64_t(n);
  fa.X = X;
  fa.theta = theta;
  fa.one_operand = one_operand ? 1 : 0;
  fa.theta_v = theta_v;
  fa.square_theta = square_theta ? 1 : 0;
  *out = fa;
}

size_t region_bytes(const PlanParams& p, int64_t M) {
  return std::max(align_up(size_t(2) * M * sizeof(double2)), align_up(size_t(p.N + 2) * 8));
}

}  // namespace

int enqueue_transform(int kind, const uint64_t* v, uint64_t n, cudaStream_t s,
                      const PlanParams& p, const PlanEntry& pe, Workspace& ws, double2* spec,
                      double* theta) {
  ensure_kernel_attributes();
  const int64_t M = pe.M;
  double2* R0 = reinterpret_cast<double2*>(ws.base);
  double2* R1 = reinterpret_cast<double2*>(ws.base + region_bytes(p, M));
  // the passes alternate buffers: start where the last pass lands in spec
  double2* bufs[2] = {R0, R1};
  bufs[pe.fft.npass & 1] = spec;
  FwdArgs fa;
  fwd_args(kind, v, v, n, p, pe, reinterpret_cast<double*>(bufs[0]), theta, true, nullptr, true,
           &fa);
  launch_fwd(kind, fa, 1, s);
  const int cur = launch_fft(pe, bufs, 0, -1, 1, M, s);
  if (bufs[cur] != spec) return TM_ECUDA;   // (cannot happen: npass passes alternate)
  TM_CHECK(cudaGetLastError());
  return TM_OK;
}

namespace {
// NVTX ranges (header-only NVTX 3: inert unless a profiler injects its library):
// one per product, named by kind, with one nested range per phase, so that a
// timeline tool groups each product's kernel launches by the paper's steps.
const char* const kPhaseNames[TM_NPHASES] = {"split+convert", "forward FFT",
                                             "twist+pointwise", "inverse FFT",
                                             "convert back+round", "overlap-add+carry"};
const char* const kKindNames[3] = {"tm_mul full", "tm_mul lo", "tm_mul hi"};
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

// ------------------------------------------------ single-launch products

// tm_set_fused: 0 = automatic, 1 = never, 2 = whenever the layout allows it. A grid
// barrier of the single-launch kernel (global atomics, about 3-4 us on GB300) costs
// as much as a launch gap under programmatic dependent launch, and the persistent
// batch kernel (one CTA pair per SM running every phase's block bodies) reaches 45%
// of the FP64 pipe against the per-phase graph's overlapping branches, so automatic
// mode uses per-phase launches and the per-phase batch graph.
std::atomic<int> g_fused_mode{0};

PassArgs pass_args(const PlanEntry& pe, int i, long long stride) {
  const FftPass& fp = pe.fft.pass[i];
  PassArgs a{};
  a.L = fp.L; a.nstages = fp.nstages; a.C = fp.C;
  std::copy(fp.radix, fp.radix + kMaxStages, a.radix);
  a.Q = fp.Q; a.Qc = fp.Qc; a.IA = fp.IA; a.IC = fp.IC; a.IS = fp.IS;
  a.OA = fp.OA; a.OC = fp.OC; a.OS = fp.OS; a.Mp = fp.Mp;
  a.batch_stride = stride;
  a.tw_sub = pe.tw + fp.tw_sub;
  a.tw_outer = fp.Mp ? pe.tw + fp.tw_outer : nullptr;
  a.tw4 = reinterpret_cast<const Tan4*>(pe.tw + fp.tw4);
  a.tw4_len = fp.tw4_len;
  std::copy(fp.tw4_off, fp.tw4_off + kMaxStages, a.tw4_off);
  a.need_wL = fp.need_wL ? 1 : 0;
  return a;
}

size_t pass_smem(const FftPass& fp, int C) {
  return (size_t((C * fp.L + 1) & ~1) + 2 * size_t(fp.tw4_len) +
          (fp.need_wL ? size_t(fp.L) : 0)) * sizeof(double2);
}

// Sequences per CTA in a single-launch product: spread the pass over the resident
// CTAs, at most as many points as kFusedThreads threads hold one radix-4 butterfly
// each.
int fused_C(const FftPass& fp, int resident) {
  const int64_t cap = std::max(1, 4 * kFusedThreads / fp.L);
  const int64_t spread = (fp.Q + resident - 1) / std::max(1, resident);
  return int(std::max<int64_t>(1, std::min(cap, spread)));
}

// Resident CTAs of the single-launch kernel per (device, kind, shared memory),
// queried once.
int fused_resident(int kind, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, int, size_t>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const auto key = std::make_tuple(dev, kind, (smem + 1023) / 1024 * 1024);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const int r = fused_max_blocks(kind, std::get<2>(key));
  cache[key] = r;
  return r;
}

// Whether a product of this plan runs as one cooperative launch.
bool use_fused(const PlanEntry& pe) {
  if (g_fused_mode.load() != 2) return false;
  for (int i = 0; i < pe.fft.npass; ++i)
    if (pe.fft.pass[i].L > 4 * kFusedThreads) return false;
  return true;
}

// Every phase of the product in one cooperative launch (k_fused_product), on the
// same buffers and with the same block arguments as the per-phase launches.
int enqueue_fused(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n,
                  cudaStream_t s, const PlanParams& p, const PlanEntry& pe, Workspace& ws) {
  const int64_t N = p.N, M = pe.M;
  const size_t region = region_bytes(p, M);
  double2* R0 = reinterpret_cast<double2*>(ws.base);
  double2* R1 = reinterpret_cast<double2*>(ws.base + region);
  double* theta = reinterpret_cast<double*>(ws.base + ws.size - 256);
  unsigned* sync = reinterpret_cast<unsigned*>(ws.base + ws.size - 64);
  const bool square = u == v;
  FusedArgs A{};
  A.square = square ? 1 : 0;
  A.npass = pe.fft.npass;
  fwd_args(kind, u, v, n, p, pe, reinterpret_cast<double*>(R0), theta, square, nullptr, square,
           &A.fa);
  double2* bufs[2] = {R0, R1};
  int cur = 0;
  size_t smem = 0, smem_cap = 0;
  for (int i = 0; i < pe.fft.npass; ++i) {
    const FftPass& fp = pe.fft.pass[i];
    smem_cap = std::max(smem_cap, pass_smem(fp, std::max(1, 4 * kFusedThreads / fp.L)));
  }
  const int resident = fused_resident(kind, smem_cap);
  if (resident <= 0) return TM_ECUDA;
  for (int i = 0; i < pe.fft.npass; ++i) {
    A.fwd[i] = pass_args(pe, i, M);
    A.fwd[i].C = fused_C(pe.fft.pass[i], resident);
    A.fwd_in[i] = bufs[cur];
    A.fwd_out[i] = bufs[cur ^ 1];
    cur ^= 1;
    smem = std::max(smem, pass_smem(pe.fft.pass[i], A.fwd[i].C));
  }
  A.Zu = bufs[cur];
  A.Zv = square ? bufs[cur] : bufs[cur] + M;
  A.Q = bufs[cur ^ 1];
  A.M = M;
  A.tc = pe.tw + pe.twc_off;
  A.two_over_N = 2.0 / double(N);
  cur ^= 1;
  for (int i = 0; i < pe.fft.npass; ++i) {
    A.inv[i] = pass_args(pe, i, 0);
    A.inv[i].C = A.fwd[i].C;
    A.inv_in[i] = bufs[cur];
    A.inv_out[i] = bufs[cur ^ 1];
    cur ^= 1;
  }
  double2* wbuf = bufs[cur];
  long long* cbuf = reinterpret_cast<long long*>(bufs[cur ^ 1]);
  BackArgs& ba = A.ba;
  ba.w = reinterpret_cast<const double*>(wbuf);
  ba.N = N;
  ba.b = p.b;
  ba.lam = kind == TM_FULL ? 0 : p.lam_bwd;
  ba.tab = pe.bwd_tab;
  ba.tab2 = kind == TM_HI ? pe.bwd_tab2 : pe.bwd_tab;
  ba.kappa = pe.small;
  ba.nkappa = pe.nkappa;
  ba.theta = theta;
  ba.rho = p.rho;
  ba.c = cbuf;
  ba.count = kind == TM_HI ? N + 1 : N;
  ba.emax_fx = emax_fixed(p.limit > 0.0 ? p.limit : p.e_max);
  ba.status = ws.status;
  A.back_small = kind != TM_FULL && (N <= 64 || N < 2 * ba.lam + ba.nkappa + 2) ? 1 : 0;
  int64_t nS, shift, rbit;
  carry_shape(p, &nS, &shift, &rbit);
  char* scratch = reinterpret_cast<char*>(wbuf);
  CarryArgs& ca = A.ca;
  ca.c = cbuf;
  ca.K = kind == TM_HI ? N + 1 : N;
  ca.b = p.b;
  ca.kind = kind;
  ca.nS = nS;
  ca.round_bit = rbit;
  ca.shift_bits = shift;
  ca.nout = out_limbs(kind, n);
  ca.top_mask = (kind == TM_LO && n % 64) ? ((1ull << (n % 64)) - 1ull) : ~0ull;
  ca.out = reinterpret_cast<unsigned long long*>(out);
  ca.r = reinterpret_cast<unsigned long long*>(scratch);
  ca.fblock = reinterpret_cast<unsigned char*>(scratch + align_up(size_t(2) * nS * 8));
  ca.cin_block = ca.fblock + align_up(size_t(nS / 512 + 2));
  A.sync = sync;
  A.status = ws.status;
  A.leave_barrier = fault_leave_barrier() ? 1 : 0;
  // grid: the widest phase, at most what stays resident
  int64_t want = (N + 1023) / 1024;
  for (int i = 0; i < pe.fft.npass; ++i) {
    const int64_t C = A.fwd[i].C;
    want = std::max<int64_t>(want, ((pe.fft.pass[i].Q + C - 1) / C) * (square ? 1 : 2));
  }
  want = std::max<int64_t>(want, (M / 2 + kFusedThreads) / kFusedThreads);
  want = std::max<int64_t>(want, (nS + 511) / 512);
  const int grid = int(std::min<int64_t>(want, resident));
  if (!ws.sync_ready) {               // the barrier words restore themselves after use
    TM_CHECK(cudaMemsetAsync(sync, 0, 8, s));
    ws.sync_ready = true;
  }
  TM_CHECK(launch_fused(kind, A, grid, smem, s));
  return TM_OK;
}

int enqueue(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n,
            cudaStream_t s, const PlanParams& p, const PlanEntry& pe, Workspace& ws,
            int64_t* coeff_out, void* const* events, const KeptOperand* kept) {
  NvtxRange product(kKindNames[kind]);
  if (!events && !coeff_out && !kept && use_fused(pe)) {
    ensure_kernel_attributes();
    return enqueue_fused(kind, out, u, v, n, s, p, pe, ws);
  }
  bool phase_open = false;
  auto mark = [&](int i) {
    if (events) cudaEventRecord(static_cast<cudaEvent_t>(events[i]), s);
    if (phase_open) nvtxRangePop();
    phase_open = i < TM_NPHASES;
    if (phase_open) nvtxRangePushA(kPhaseNames[i]);
  };
  struct ClosePhase {                   // an early return leaves no phase range open
    bool* open;
    ~ClosePhase() { if (*open) nvtxRangePop(); }
  } close_phase{&phase_open};
  ensure_kernel_attributes();
  mark(0);
  const int64_t N = p.N, M = pe.M;
  const size_t region = region_bytes(p, M);
  double2* R0 = reinterpret_cast<double2*>(ws.base);
  double2* R1 = reinterpret_cast<double2*>(ws.base + region);
  double* theta = reinterpret_cast<double*>(ws.base + ws.size - 256);
  const bool square = !kept && u == v;
  const bool one = square || kept;
  double2* bufs[2] = {R0, R1};
  int cur;
  // full product: the first forward pass computes the split of its operand as it
  // loads it, so steps 1 and 2 are one launch per pass. (The low product's map on
  // load measured slower: the first pass reads columns, so each thread walks a
  // serial chain of digit and table loads per element; its own kernel reads tiles.)
  const bool map_on_load = kind == TM_FULL && !ws.operands_mapped;
  // u's and v's forward FFTs on two streams when one transform's passes fill the GPU
  // (each fills the SMs the other's last partial wave leaves idle); otherwise both
  // in one launch per pass on s, which keeps the chain of programmatic dependent
  // launches unbroken (on GB300: 87 against 118 us for the low product at n = 2^20,
  // 477 against 488 us the other way at 2^24)
  const bool two_streams = !one && ws.side && fft_fills_gpu(pe.fft);
  double2* bufs_v[2] = {R0 + M, R1 + M};
  PlanParams mp = p;                 // this call's operand size and digit count
  mp.n = n;
  if (map_on_load) {
    mark(1);
    if (two_streams) {             // u's transform on s, v's on the side stream
      TM_CHECK(cudaEventRecord(ws.fork, s));
      TM_CHECK(cudaStreamWaitEvent(ws.side, ws.fork, 0));
      cur = launch_fft(pe, bufs, 0, -1, 1, M, s, u, &mp);
      launch_fft(pe, bufs_v, 0, -1, 1, M, ws.side, v, &mp);
      TM_CHECK(cudaEventRecord(ws.join, ws.side));
      TM_CHECK(cudaStreamWaitEvent(s, ws.join, 0));
    } else {
      cur = launch_fft(pe, bufs, 0, -1, one ? 1 : 2, M, s, u, &mp, v);
    }
  } else if (two_streams) {
    // 1. digits + forward maps of both operands in one launch (one pass over the map
    // table); 2. u's forward FFT on s, v's on the side stream, so that each
    // operand's passes fill the SMs the other's leave idle
    FwdArgs fa;
    fwd_args(kind, u, v, n, p, pe, reinterpret_cast<double*>(R0), theta, false, nullptr, false,
             &fa);
    launch_fwd(kind, fa, 1, s);
    mark(1);
    TM_CHECK(cudaEventRecord(ws.fork, s));
    TM_CHECK(cudaStreamWaitEvent(ws.side, ws.fork, 0));
    cur = launch_fft(pe, bufs, 0, -1, 1, M, s);
    launch_fft(pe, bufs_v, 0, -1, 1, M, ws.side);
    TM_CHECK(cudaEventRecord(ws.join, ws.side));
    TM_CHECK(cudaStreamWaitEvent(s, ws.join, 0));
  } else {
    // 1. digits + forward map (split and convert steps of Algorithms 1-3)
    FwdArgs fa;
    fwd_args(kind, u, v, n, p, pe, reinterpret_cast<double*>(R0), theta, one,
             kept ? kept->theta : nullptr, square, &fa);
    launch_fwd(kind, fa, 1, s);
    mark(1);
    // 2. forward FFTs of both operands (complex length M, batch 2), or of u alone
    cur = launch_fft(pe, bufs, 0, -1, one ? 1 : 2, M, s);
  }
  mark(2);
  // 3. real-FFT twist, pointwise product, inverse pre-twist
  const double2* Zu = bufs[cur];
  const double2* Zv = kept ? kept->spec : (square ? Zu : Zu + M);
  launch_twist(Zu, Zv, bufs[cur ^ 1], M, pe.tw + pe.twc_off, N, 1, 0, 0, s);
  cur ^= 1;
  mark(3);
  // 4. inverse FFT (batch 1)
  cur = launch_fft(pe, bufs, cur, 1, 1, M, s);
  mark(4);
  // 5. back map + round (convert-back and rounding of Algorithms 1-3)
  double2* wbuf = bufs[cur];
  long long* cbuf = reinterpret_cast<long long*>(bufs[cur ^ 1]);
  BackArgs ba{};
  ba.w = reinterpret_cast<const double*>(wbuf);
  ba.N = N;
  ba.b = p.b;
  ba.lam = kind == TM_FULL ? 0 : p.lam_bwd;
  ba.tab = pe.bwd_tab;
  ba.tab2 = kind == TM_HI ? pe.bwd_tab2 : pe.bwd_tab;
  ba.kappa = pe.small;
  ba.nkappa = pe.nkappa;
  ba.theta = theta;
  ba.rho = p.rho;
  ba.c = cbuf;
  ba.count = kind == TM_HI ? N + 1 : N;
  ba.emax_fx = emax_fixed(p.limit > 0.0 ? p.limit : p.e_max);
  ba.status = ws.status;
  launch_back(kind, ba, 1, s);
  mark(5);
  if (coeff_out) {
    TM_CHECK(cudaMemcpyAsync(coeff_out, cbuf, size_t(ba.count) * 8, cudaMemcpyDeviceToDevice, s));
    TM_CHECK(cudaGetLastError());
    return TM_OK;
  }
  // 6. overlap-add and carries into the output limbs
  int64_t nS, shift, rbit;
  carry_shape(p, &nS, &shift, &rbit);
  char* scratch = reinterpret_cast<char*>(wbuf);   // the inverse output is consumed
  CarryArgs ca{};
  ca.c = cbuf;
  ca.K = kind == TM_HI ? N + 1 : N;
  ca.b = p.b;
  ca.kind = kind;
  ca.nS = nS;
  ca.round_bit = rbit;
  ca.shift_bits = shift;
  ca.nout = out_limbs(kind, n);
  ca.top_mask = (kind == TM_LO && n % 64) ? ((1ull << (n % 64)) - 1ull) : ~0ull;
  ca.out = reinterpret_cast<unsigned long long*>(out);
  ca.r = reinterpret_cast<unsigned long long*>(scratch);
  ca.fblock = reinterpret_cast<unsigned char*>(scratch + align_up(size_t(2) * nS * 8));
  ca.cin_block = ca.fblock + align_up(size_t(nS / 512 + 2));
  launch_carry(ca, 1, s);
  mark(6);
  TM_CHECK(cudaGetLastError());
  return TM_OK;
}

namespace {

constexpr long long kSmallSingleMaxM = 640;   // one product in one CTA up to this M

int run(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n, void* stream,
        tm_report* rep, int64_t* coeff_out, void* const* events = nullptr,
        const tm_params* explicit_prm = nullptr) {
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n == 0 || !u || !v || (!out && !coeff_out)) return TM_EINVAL;
  if (n > TM_MAX_BITS) return TM_ERANGE;
  const size_t in_bytes = size_t(limbs_of(n)) * 8;
  if (out) {
    const size_t ob = size_t(out_limbs(kind, n)) * 8;
    if (overlaps(out, ob, u, in_bytes) || overlaps(out, ob, v, in_bytes)) return TM_EALIAS;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PlanParams p;
  int rc;
  if (explicit_prm) {
    const double lim = explicit_prm->limit;
    if (!(lim >= 0.0 && lim <= 0.5)) return TM_EINVAL;
    rc = explicit_params(kind, n, int(explicit_prm->b), int64_t(explicit_prm->N), &p);
    if (rc) return rc;
    p.limit = lim > 0.0 ? lim : (p.e_max < 0.5 ? p.e_max : 0.375);
  } else {
    rc = get_params(kind, n, &p);
  }
  if (rc) return rc;
  const bool certified = p.e_max < 0.5;
  // a small product runs whole in the CTA-resident kernel, one launch in place of
  // the per-phase sequence. Measured on GB300: faster up to M = 560 (28 against 36 us
  // at n = 100, 42 against 56 us at 4096, 49 against 55 us at 10000), slower from
  // M = 960 on (69 against 66 us at 20000), where one SM's FP64 work outweighs the
  // launch chain; kSmallSingleMaxM sits between.
  if (out && !coeff_out && !events && p.N / 2 <= kSmallSingleMaxM &&
      g_fused_mode.load() == 0) {
    std::shared_ptr<PlanEntry> spe;
    rc = get_tables(p, true, s, &spe);
    if (rc) return rc;
    Workspace* ws = nullptr;
    rc = get_workspace(s, 0, &ws);
    if (rc) return rc;
    ensure_kernel_attributes();
    SmallArgs a{};
    a.count = 1;
    a.status = ws->status;
    a.item0 = small_item_for(out, u, v, n, p, 0);
    a.plan0 = small_plan_of(p, *spe);
    const FftPass& fp = spe->fft.pass[0];
    launch_small(a, 1, small_smem_bytes(p.N, spe->M, fp.tw4_len, fp.need_wL), s);
    if (cudaGetLastError() != cudaSuccess) return TM_ECUDA;
    if (!rep) return certified ? TM_OK : TM_UNCERTIFIED;
    fill_plan_report(p, spe->fft, rep);
    rep->table_bytes = spe->table_bytes;
    rc = read_status(s, ws->status, rep);
    if (rc == TM_OK && !certified) {
      rc = TM_UNCERTIFIED;
      rep->status = rc;
    }
    return rc;
  }
  std::shared_ptr<PlanEntry> pe;
  rc = get_tables(p, false, s, &pe);
  if (rc) return rc;
  Workspace* ws = nullptr;
  rc = get_workspace(s, workspace_bytes(p), &ws);
  if (rc) return rc;
  rc = enqueue(kind, out, u, v, n, s, p, *pe, *ws, coeff_out, events);
  if (rc) return rc;
  // a caller's (b, N) outside the worst-case bound never reports plain success
  if (!rep) return certified ? TM_OK : TM_UNCERTIFIED;
  fill_plan_report(p, pe->fft, rep);
  rep->table_bytes = pe->table_bytes;
  rc = read_status(s, ws->status, rep);
  if (rc == TM_ETIMEOUT) ws->sync_ready = false;   // barrier words left mid-count
  if (rc == TM_OK && !certified) {
    rc = TM_UNCERTIFIED;
    rep->status = rc;
  }
  return rc;
}

// ------------------------------------------- products without allocation

// The scratch of tm_mul_static: one device array per GPU, kept for the life of
// the process. Host code cannot use its name as a device address; the address is
// looked up once per device with cudaGetSymbolAddress.
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kMaxDevices] = {};
// the plan whose tables the array holds, per device
struct StaticTables {
  bool valid;
  int kind, b;
  int64_t N;
};
StaticTables g_static_last[kMaxDevices] = {};

}  // namespace
}  // namespace tmul

static __device__ __align__(256) unsigned char g_static_scratch[TM_STATIC_SCRATCH_BYTES];

namespace tmul {
namespace {

// Device address of g_static_scratch on the current device (set-up on first use).
int static_scratch(char** out) {
  int dev = 0;
  TM_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return TM_EINVAL;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return TM_ECUDA;
    }
    g_static_addr[dev] = p;
  }
  *out = static_cast<char*>(g_static_addr[dev]);
  return TM_OK;
}

// Lays out the plan tables, the status word and the workspace inside `base`
// (TM_STATIC_SCRATCH_BYTES) and enqueues the table initialisation. Returns
// TM_ERANGE when they do not fit.
int static_plan(int kind, char* base, cudaStream_t s, PlanEntry* e, Workspace* ws) {
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off += align_up(bytes); return at; };
  const size_t status_off = take(sizeof(DevStatus));
  const size_t cnt = layout_twiddles(e);
  const size_t tw_off = take(cnt * sizeof(double2));
  const int64_t N = e->p.N;
  const int b = e->p.b;
  const int rf = kind == TM_FULL ? 0 : e->p.lam_fwd - 1;
  const int rb = kind == TM_FULL ? 0 : (kind == TM_LO ? e->p.lam_bwd - 1 : e->p.lam_bwd);
  const int r2 = kind == TM_HI ? e->p.lam_bwd - 1 : 0;
  const size_t fwd_off = take(size_t(std::max(rf, 0)) * N * 8);
  const size_t bwd_off = take(size_t(std::max(rb, 0)) * N * 8);
  const size_t bwd2_off = take(size_t(std::max(r2, 0)) * N * 8);
  int lgN = 0;
  while ((int64_t(1) << lgN) < N) ++lgN;
  const int nkappa = kind == TM_HI ? int(std::min<int64_t>(N, 3 + (lgN + 64 + b - 1) / b)) : 0;
  const int ntheta = kind == TM_HI ? int(std::min<int64_t>(N + 1, (60 + b - 1) / b + 3)) : 0;
  if (nkappa + ntheta > 96) return TM_ERANGE;
  const size_t small_off = take(size_t(nkappa + ntheta) * 8);
  const size_t ws_bytes = workspace_bytes(e->p);
  const size_t ws_off = take(ws_bytes);
  if (off > TM_STATIC_SCRATCH_BYTES) return TM_ERANGE;
  e->tw = reinterpret_cast<double2*>(base + tw_off);
  e->fwd_tab = rf > 0 ? reinterpret_cast<long long*>(base + fwd_off) : nullptr;
  e->bwd_tab = rb > 0 ? reinterpret_cast<double*>(base + bwd_off) : nullptr;
  e->bwd_tab2 = r2 > 0 ? reinterpret_cast<double*>(base + bwd2_off) : nullptr;
  e->small = kind == TM_HI ? reinterpret_cast<double*>(base + small_off) : nullptr;
  e->nkappa = nkappa;
  e->ntheta = ntheta;
  ws->base = base + ws_off;
  ws->size = ws_bytes;
  ws->status = reinterpret_cast<DevStatus*>(base + status_off);
  // the previous call's contents stay in the array: clear the status word, and
  // rebuild the tables unless the previous call on this device built the same plan
  // (the tables and their offsets depend only on kind, b and N)
  TM_CHECK(cudaMemsetAsync(ws->status, 0, sizeof(DevStatus), s));
  int dev = 0;
  TM_CHECK(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticTables& last = g_static_last[dev];
    if (last.valid && last.kind == kind && last.b == b && last.N == N) return TM_OK;
    last.valid = false;
  }
  init_twiddles(*e, s);
  if (rf > 0)
    launch_init_maptab_fx(e->fwd_tab, kind == TM_LO ? kTabAlpha : kTabGamma, N, b, rf, fx_q(b), s);
  if (rb > 0)
    launch_init_maptab(e->bwd_tab, kind == TM_LO ? kTabBeta : kTabDeltaPrime, N, b,
                       kind == TM_LO ? rb : e->p.lam_bwd, s);
  if (r2 > 0) launch_init_maptab(e->bwd_tab2, kTabDelta, N, b, r2, s);
  // kappa and rho^-j computed on the device: no host-to-device copy, so a call
  // without a report enqueues only kernels and one memset
  if (kind == TM_HI) launch_init_rho_powers(e->small, nkappa, ntheta, b, std::log(e->p.rho), s);
  TM_CHECK(cudaGetLastError());
  std::lock_guard<std::mutex> lk(g_static_mu);
  g_static_last[dev] = StaticTables{true, kind, b, N};
  return TM_OK;
}

int run_static(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n,
               void* stream, tm_report* rep) {
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n == 0 || !u || !v || !out) return TM_EINVAL;
  if (n > TM_STATIC_MAX_BITS) return TM_ERANGE;
  const size_t in_bytes = size_t(limbs_of(n)) * 8;
  const size_t ob = size_t(out_limbs(kind, n)) * 8;
  if (overlaps(out, ob, u, in_bytes) || overlaps(out, ob, v, in_bytes)) return TM_EALIAS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PlanEntry pe;
  int rc = TM_OK;
  {
    // the planner's choice for the last (kind, n), kept in a fixed record (no
    // allocation): planning a high product costs milliseconds of host time
    static std::mutex mu;
    static struct { bool valid; int kind; uint64_t n; PlanParams p; } last = {};
    std::lock_guard<std::mutex> lk(mu);
    if (last.valid && last.kind == kind && last.n == n) {
      pe.p = last.p;
    } else {
      rc = choose_params(kind, n, &pe.p);
      if (rc == TM_OK) last = {true, kind, n, pe.p};
    }
  }
  if (rc) return rc;
  pe.M = pe.p.N / 2;
  rc = make_fft_plan(pe.M, &pe.fft);
  if (rc) return rc;
  char* base = nullptr;
  rc = static_scratch(&base);
  if (rc) return rc;
  Workspace ws;
  rc = static_plan(kind, base, s, &pe, &ws);
  if (rc) return rc;
  rc = enqueue(kind, out, u, v, n, s, pe.p, pe, ws, nullptr, nullptr);
  if (rc) return rc;
  if (!rep) return TM_OK;
  fill_plan_report(pe.p, pe.fft, rep);
  rep->table_bytes = 0;
  return read_status(s, ws.status, rep, false);
}

}  // namespace
}  // namespace tmul

// A kept forward transform (tm_operand_create): one device allocation holding the
// spectrum of V~ and theta_V.
struct tm_operand {
  int kind;
  uint64_t n;
  int device;
  tmul::PlanParams p;
  double2* spec;
  double* theta;
  size_t bytes;
};

extern "C" {

int tm_mul_static(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v,
                  uint64_t n_bits, void* stream, tm_report* rep) {
  return tmul::run_static(kind, out, u, v, n_bits, stream, rep);
}


int tm_mul(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
           void* stream, tm_report* rep) {
  return tmul::run(kind, out, u, v, n_bits, stream, rep, nullptr);
}

int tm_mul_params(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v,
                  uint64_t n_bits, const tm_params* prm, void* stream, tm_report* rep) {
  if (!prm) return TM_EINVAL;
  return tmul::run(kind, out, u, v, n_bits, stream, rep, nullptr, nullptr, prm);
}

int tm_mul_events(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v,
                  uint64_t n_bits, void* stream, void* const* events, tm_report* rep) {
  if (!events) return TM_EINVAL;
  for (int i = 0; i <= TM_NPHASES; ++i)
    if (!events[i]) return TM_EINVAL;
  return tmul::run(kind, out, u, v, n_bits, stream, rep, nullptr, events);
}

int tm_mul_full(uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
                void* stream, tm_report* rep) {
  return tmul::run(TM_FULL, out, u, v, n_bits, stream, rep, nullptr);
}

int tm_mul_lo(uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
              void* stream, tm_report* rep) {
  return tmul::run(TM_LO, out, u, v, n_bits, stream, rep, nullptr);
}

int tm_mul_hi(uint64_t* out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
              void* stream, tm_report* rep) {
  return tmul::run(TM_HI, out, u, v, n_bits, stream, rep, nullptr);
}

int tm_coeffs(int kind, int64_t* c_out, const uint64_t* u, const uint64_t* v, uint64_t n_bits,
              void* stream, tm_report* rep) {
  if (!rep || !c_out) return TM_EINVAL;
  return tmul::run(kind, nullptr, u, v, n_bits, stream, rep, c_out);
}

int tm_mul_host(int kind, uint64_t* out_host, const uint64_t* u_host, const uint64_t* v_host,
                uint64_t n_bits, void* stream, tm_report* rep) {
  if (!out_host || !u_host || !v_host || n_bits == 0) return TM_EINVAL;
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n_bits > TM_MAX_BITS) return TM_ERANGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t in_bytes = size_t(tmul::limbs_of(n_bits)) * 8;
  const size_t out_bytes = size_t(tmul::out_limbs(kind, n_bits)) * 8;
  char* io = nullptr;
  int rc = tmul::get_io(s, tmul::align_up(in_bytes) * 2 + tmul::align_up(out_bytes), &io);
  if (rc) return rc;
  uint64_t* du = reinterpret_cast<uint64_t*>(io);
  uint64_t* dv = reinterpret_cast<uint64_t*>(io + tmul::align_up(in_bytes));
  uint64_t* dout = reinterpret_cast<uint64_t*>(io + 2 * tmul::align_up(in_bytes));
  if (u_host == v_host) dv = du;              // a square: one copy, the squaring path
  tmul::PlanParams p;
  rc = tmul::get_params(kind, n_bits, &p);
  if (rc) return rc;
  std::shared_ptr<tmul::PlanEntry> pe;
  rc = tmul::get_tables(p, false, s, &pe);
  if (rc) return rc;
  tmul::Workspace* ws = nullptr;
  rc = tmul::get_workspace(s, tmul::workspace_bytes(p), &ws);
  if (rc) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
  const bool square = dv == du;
  // Page-locked host buffers that the device addresses directly (mapped pinned
  // memory; a GB300's Grace memory is reached over NVLink-C2C): the forward map
  // reads the operands and the carry kernel writes the product where they are,
  // with no staging copies. The operands are read before the product is written,
  // but overlapping buffers still take the staged path.
  const uint64_t* mu = tmul::mapped_host(u_host);
  const uint64_t* mv = square ? mu : tmul::mapped_host(v_host);
  uint64_t* mo = const_cast<uint64_t*>(tmul::mapped_host(out_host));
  const bool direct = mu && mv && mo && !tmul::overlaps(out_host, out_bytes, u_host, in_bytes) &&
                      !tmul::overlaps(out_host, out_bytes, v_host, in_bytes);
  bool done = false;
  if (direct) {
    ws->operands_mapped = true;
    rc = tmul::enqueue(kind, mo, mu, mv, n_bits, s, p, *pe, *ws, nullptr, nullptr);
    ws->operands_mapped = false;
    if (rc) return rc;
    tmul::DevStatus* sh = nullptr;        // the status word, published by one kernel
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&sh), ws->status_host, 0) ==
        cudaSuccess) {
      tmul::launch_status_publish(ws->status, sh, s);
      if (cudaGetLastError() != cudaSuccess) return TM_ECUDA;
    } else if (cudaMemcpyAsync(ws->status_host, ws->status, sizeof(tmul::DevStatus),
                               cudaMemcpyDeviceToHost, s) != cudaSuccess ||
               cudaMemsetAsync(ws->status, 0, sizeof(tmul::DevStatus), s) != cudaSuccess) {
      return TM_ECUDA;
    }
    done = true;
  }
  // the recorded sequence, if this stream has one for (kind, n) that is still valid
  if (!done && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread) {
    std::lock_guard<std::mutex> lk(tmul::g_mu);
    tmul::HostGraph& h = tmul::g_host_graphs[std::make_tuple(dev, s, kind, n_bits, square)];
    if (h.exec && (h.io != io || h.ws_base != ws->base || h.pe != pe.get()))
      tmul::drop_host_graph(h);
    if (!h.exec) {
      tmul::ensure_kernel_attributes();
      bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const bool rec =
            cudaMemcpyAsync(du, u_host, in_bytes, cudaMemcpyHostToDevice, s) == cudaSuccess &&
            (square ||
             cudaMemcpyAsync(dv, v_host, in_bytes, cudaMemcpyHostToDevice, s) == cudaSuccess) &&
            tmul::enqueue(kind, dout, du, dv, n_bits, s, p, *pe, *ws, nullptr, nullptr) ==
                TM_OK &&
            cudaMemcpyAsync(out_host, dout, out_bytes, cudaMemcpyDeviceToHost, s) ==
                cudaSuccess &&
            cudaMemcpyAsync(ws->status_host, ws->status, sizeof(tmul::DevStatus),
                            cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaMemsetAsync(ws->status, 0, sizeof(tmul::DevStatus), s) == cudaSuccess;
        cudaGraph_t g = nullptr;
        ok = cudaStreamEndCapture(s, &g) == cudaSuccess && rec && g;
        size_t count = 0;
        if (ok) ok = cudaGraphGetNodes(g, nullptr, &count) == cudaSuccess;
        std::vector<cudaGraphNode_t> nodes(count);
        if (ok && count) ok = cudaGraphGetNodes(g, nodes.data(), &count) == cudaSuccess;
        for (size_t i = 0; ok && i < count; ++i) {
          cudaGraphNodeType t;
          if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeMemcpy)
            continue;
          cudaMemcpy3DParms m{};
          if (cudaGraphMemcpyNodeGetParams(nodes[i], &m) != cudaSuccess) { ok = false; break; }
          if (m.dstPtr.ptr == du) h.in_u = nodes[i];
          else if (m.dstPtr.ptr == dv) h.in_v = nodes[i];
          else if (m.srcPtr.ptr == dout) h.out = nodes[i];
        }
        ok = ok && h.in_u && h.out && (square || h.in_v);
        if (ok) ok = cudaGraphInstantiate(&h.exec, g, 0) == cudaSuccess;
        if (ok) {
          h.graph = g;
          h.io = io;
          h.ws_base = ws->base;
          h.pe = pe.get();
          // the recording did not run: run it now
          done = cudaGraphLaunch(h.exec, s) == cudaSuccess;
        } else {                       // e.g. pageable host buffers: no recording
          if (g) cudaGraphDestroy(g);
          h = tmul::HostGraph{};
        }
      }
      (void)cudaGetLastError();
    } else if (h.exec) {
      done = cudaGraphExecMemcpyNodeSetParams1D(h.exec, h.in_u, du, u_host, in_bytes,
                                                cudaMemcpyHostToDevice) == cudaSuccess &&
             (square || cudaGraphExecMemcpyNodeSetParams1D(h.exec, h.in_v, dv, v_host, in_bytes,
                                                           cudaMemcpyHostToDevice) ==
                            cudaSuccess) &&
             cudaGraphExecMemcpyNodeSetParams1D(h.exec, h.out, out_host, dout, out_bytes,
                                                cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaGraphLaunch(h.exec, s) == cudaSuccess;
      if (!done) {
        (void)cudaGetLastError();
        tmul::drop_host_graph(h);
      }
    }
  }
  if (!done) {
    if (cudaMemcpyAsync(du, u_host, in_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (!square &&
         cudaMemcpyAsync(dv, v_host, in_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess))
      return TM_ECUDA;
    rc = tmul::enqueue(kind, dout, du, dv, n_bits, s, p, *pe, *ws, nullptr, nullptr);
    if (rc) return rc;
    // result, status word and its reset in stream order: one wait for all of it
    if (cudaMemcpyAsync(out_host, dout, out_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(ws->status_host, ws->status, sizeof(tmul::DevStatus),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(ws->status, 0, sizeof(tmul::DevStatus), s) != cudaSuccess)
      return TM_ECUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return TM_ECUDA;
  rc = ws->status_host->flags ? TM_EPRECISION : TM_OK;
  if (rep) {
    tmul::fill_plan_report(p, pe->fft, rep);
    rep->table_bytes = pe->table_bytes;
    rep->margin = std::ldexp(double(ws->status_host->margin_fx), -63);
    rep->status = rc;
  }
  return rc;
}

int tm_mul_adaptive(int kind, uint64_t* out, const uint64_t* u, const uint64_t* v,
                    uint64_t n_bits, void* stream, tm_report* rep) {
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n_bits == 0 || !u || !v || !out) return TM_EINVAL;
  if (n_bits > TM_MAX_BITS) return TM_ERANGE;
  const size_t in_bytes = size_t(tmul::limbs_of(n_bits)) * 8;
  const size_t ob = size_t(tmul::out_limbs(kind, n_bits)) * 8;
  if (tmul::overlaps(out, ob, u, in_bytes) || tmul::overlaps(out, ob, v, in_bytes))
    return TM_EALIAS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tmul::PlanParams use;
  int rc = tmul::get_params(kind, n_bits, &use);
  if (rc) return rc;
  tmul::Workspace* ws = nullptr;
  rc = tmul::get_workspace(s, 0, &ws);
  if (rc) return rc;
  // candidate: one more bit per digit at its shortest admissible length, measured
  // only when its worst-case bound is within kMeasure of the target (random digits
  // bring the norm product down by about 3)
  constexpr double kMeasure = 3.5;
  const int b1 = use.b + 1;
  const int64_t N1 = tmul::measured_length(kind, n_bits, b1);
  tmul::PlanParams pw;
  const bool worth =
      N1 > 0 && N1 < use.N &&
      tmul::measured_params(kind, n_bits, b1, N1, tmul::worst_norms(kind, n_bits, b1, N1),
                            &pw) != TM_EINVAL &&
      pw.N == N1 && pw.e_max <= kMeasure * tmul::bound_target();
  if (worth) {
    const int64_t count = kind == TM_FULL ? (int64_t(n_bits) + 1 + b1 - 1) / b1 : N1;
    const int64_t shift = kind == TM_HI ? (N1 + 1) * b1 - int64_t(n_bits) : 0;
    const int64_t top = kind == TM_HI ? N1 : count - 1;
    unsigned long long sums[4] = {0, 0, 0, 0};
    if (cudaMemsetAsync(ws->norms, 0, sizeof(sums), s) != cudaSuccess) return TM_ECUDA;
    tmul::launch_digit_norms(reinterpret_cast<const unsigned long long*>(u),
                             reinterpret_cast<const unsigned long long*>(v),
                             tmul::limbs_of(n_bits), n_bits, shift, b1,
                             count, top, kind == TM_HI, ws->norms, s);
    if (cudaMemcpyAsync(sums, ws->norms, sizeof(sums), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return TM_ECUDA;
    // upper bounds on the norms (the sums are exact integers; a few ulps of slack)
    const double up = 1.0 + std::ldexp(1.0, -48);
    tmul::DigitNorms dn;
    dn.nu = std::sqrt(double(sums[0])) * up;
    dn.nv = std::sqrt(double(sums[1])) * up;
    dn.tu = double(sums[2]);
    dn.tv = double(sums[3]);
    tmul::PlanParams p1;
    if (tmul::measured_params(kind, n_bits, b1, N1, dn, &p1) == TM_OK) use = p1;
  }
  std::shared_ptr<tmul::PlanEntry> pe;
  rc = tmul::get_tables(use, false, s, &pe);
  if (rc) return rc;
  rc = tmul::get_workspace(s, tmul::workspace_bytes(use), &ws);
  if (rc) return rc;
  rc = tmul::enqueue(kind, out, u, v, n_bits, s, use, *pe, *ws, nullptr, nullptr);
  if (rc) return rc;
  if (!rep) return TM_OK;
  tmul::fill_plan_report(use, pe->fft, rep);
  rep->table_bytes = pe->table_bytes;
  return tmul::read_status(s, ws->status, rep);
}

int tm_operand_create(int kind, uint64_t n_bits, const uint64_t* v, void* stream,
                      tm_operand** out) {
  if (!out || !v) return TM_EINVAL;
  *out = nullptr;
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n_bits == 0) return TM_EINVAL;
  if (n_bits > TM_MAX_BITS) return TM_ERANGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
  tmul::PlanParams p;
  int rc = tmul::get_params(kind, n_bits, &p);
  if (rc) return rc;
  std::shared_ptr<tmul::PlanEntry> pe;
  rc = tmul::get_tables(p, false, s, &pe);
  if (rc) return rc;
  tmul::Workspace* ws = nullptr;
  rc = tmul::get_workspace(s, tmul::workspace_bytes(p), &ws);
  if (rc) return rc;
  const size_t spec_bytes = tmul::align_up(size_t(pe->M) * sizeof(double2));
  char* base = nullptr;
  cudaError_t e = cudaMalloc(&base, spec_bytes + 256);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TM_ENOMEM : TM_ECUDA;
  }
  tm_operand* op = new tm_operand;
  op->kind = kind;
  op->n = n_bits;
  op->device = dev;
  op->p = p;
  op->spec = reinterpret_cast<double2*>(base);
  op->theta = reinterpret_cast<double*>(base + spec_bytes);
  op->bytes = spec_bytes + 256;
  rc = tmul::enqueue_transform(kind, v, n_bits, s, p, *pe, *ws, op->spec, op->theta);
  if (rc) {
    cudaFree(base);
    delete op;
    return rc;
  }
  *out = op;
  return TM_OK;
}

int tm_mul_operand(uint64_t* out, const uint64_t* u, const tm_operand* v, void* stream,
                   tm_report* rep) {
  if (!out || !u || !v) return TM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
  if (dev != v->device) return TM_EINVAL;
  const int kind = v->kind;
  const uint64_t n = v->n;
  const size_t in_bytes = size_t(tmul::limbs_of(n)) * 8;
  const size_t ob = size_t(tmul::out_limbs(kind, n)) * 8;
  if (tmul::overlaps(out, ob, u, in_bytes) || tmul::overlaps(out, ob, v->spec, v->bytes))
    return TM_EALIAS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::shared_ptr<tmul::PlanEntry> pe;
  int rc = tmul::get_tables(v->p, false, s, &pe);
  if (rc) return rc;
  tmul::Workspace* ws = nullptr;
  rc = tmul::get_workspace(s, tmul::workspace_bytes(v->p), &ws);
  if (rc) return rc;
  const tmul::KeptOperand kept{v->spec, v->theta};
  rc = tmul::enqueue(kind, out, u, u, n, s, v->p, *pe, *ws, nullptr, nullptr, &kept);
  if (rc) return rc;
  if (!rep) return TM_OK;
  tmul::fill_plan_report(v->p, pe->fft, rep);
  rep->table_bytes = pe->table_bytes;
  return tmul::read_status(s, ws->status, rep);
}

int tm_operand_destroy(tm_operand* op) {
  if (!op) return TM_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
  if (dev != op->device && cudaSetDevice(op->device) != cudaSuccess) return TM_ECUDA;
  const cudaError_t e = cudaFree(op->spec);
  if (dev != op->device) cudaSetDevice(dev);
  delete op;
  return e == cudaSuccess ? TM_OK : TM_ECUDA;
}

// An autotuner replaces the default only for a candidate at least 1% faster.
constexpr double kTuneGain = 0.99;
// the delay before each timed run of the autotuners: longer than the host's planning
// and launch work for one product (about 30 us)
constexpr unsigned long long kTuneDelayNs = 200000ull;

int tm_autotune(int kind, uint64_t n_bits, void* stream, tm_tune* out) {
  if (!out) return TM_EINVAL;
  std::memset(out, 0, sizeof(*out));
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n_bits == 0) return TM_EINVAL;
  if (n_bits > TM_MAX_BITS) return TM_ERANGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tmul::PlanParams p;
  int rc = tmul::get_params(kind, n_bits, &p);
  if (rc) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
  tmul::ensure_kernel_attributes();
  const int64_t M = p.N / 2;
  // candidate layouts: default first, then every distinct valid variation
  std::vector<tmul::FftShape> shapes;
  std::vector<tmul::FftPlan> plans;
  for (int passes : {0, 2, 3})
    for (int split : {0, 1, 2})
      for (int points : {1024, 512, 2048}) {
        const tmul::FftShape sh{points, split, passes};
        tmul::FftPlan f;
        if (tmul::make_fft_plan(M, &f, false, &sh) != TM_OK) continue;
        bool dup = false;
        for (const auto& g : plans) {
          bool same = g.npass == f.npass;
          for (int i = 0; same && i < f.npass; ++i)
            same = g.pass[i].L == f.pass[i].L && g.pass[i].C == f.pass[i].C &&
                   g.pass[i].threads == f.pass[i].threads;
          dup = dup || same;
        }
        if (!dup) { shapes.push_back(sh); plans.push_back(f); }
      }
  if (plans.empty()) return TM_ERANGE;
  double2* buf = nullptr;
  const size_t region = size_t(2) * M * sizeof(double2);
  if (cudaMalloc(&buf, 2 * region) != cudaSuccess) { (void)cudaGetLastError(); return TM_ENOMEM; }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<double> ms(plans.size(), 0.0);
  rc = TM_OK;
  for (size_t c = 0; c < plans.size() && rc == TM_OK; ++c) {
    tmul::PlanEntry e;
    e.p = p;
    e.M = M;
    e.fft = plans[c];
    const size_t cnt = tmul::layout_twiddles(&e);
    if (cudaMalloc(&e.tw, cnt * sizeof(double2)) != cudaSuccess) {
      (void)cudaGetLastError();
      rc = TM_ENOMEM;
      break;
    }
    tmul::init_twiddles(e, s);
    double2* bufs[2] = {buf, reinterpret_cast<double2*>(reinterpret_cast<char*>(buf) + region)};
    // one warm-up, then the median of five isolated timings: a delay kernel holds the
    // stream while the host enqueues the transforms, so the time is the device's
    // latency for one forward pair and one inverse, as a single product sees it
    std::vector<float> t;
    for (int rep = 0; rep < 6; ++rep) {
      cudaMemsetAsync(buf, 0x3f, 2 * region, s);  // bounded values in every repetition
      tmul::launch_delay(kTuneDelayNs, s);
      cudaEventRecord(e0, s);
      const int cur = tmul::launch_fft(e, bufs, 0, -1, 2, M, s);
      tmul::launch_fft(e, bufs, cur, 1, 1, M, s);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = TM_ECUDA; break; }
      float x = 0;
      cudaEventElapsedTime(&x, e0, e1);
      if (rep) t.push_back(x);
    }
    cudaFree(e.tw);
    if (rc) break;
    std::sort(t.begin(), t.end());
    ms[c] = t[t.size() / 2];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc == TM_OK && cudaGetLastError() != cudaSuccess) rc = TM_ECUDA;
  if (rc) return rc;
  size_t best = 0;
  for (size_t c = 1; c < ms.size(); ++c)
    if (ms[c] < ms[best]) best = c;
  if (ms[best] > kTuneGain * ms[0]) best = 0;     // within the noise: keep the default
  out->candidates = int32_t(plans.size());
  out->points = shapes[best].points;
  out->split = shapes[best].split;
  out->passes = shapes[best].passes;
  out->npass = plans[best].npass;
  out->ms_default = ms[0];
  out->ms_best = ms[best];
  tmul::apply_layout(dev, p.N, best == 0 ? nullptr : &shapes[best]);
  return TM_OK;
}

int tm_plan_set(int kind, uint64_t n_bits, uint32_t b, uint32_t N) {
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n_bits == 0) return TM_EINVAL;
  if (n_bits > TM_MAX_BITS) return TM_ERANGE;
  const auto key = std::make_pair(kind, n_bits);
  if (b == 0 && N == 0) {
    std::lock_guard<std::mutex> lk(tmul::g_mu);
    tmul::g_params.erase(key);             // the planner's choice again
    return TM_OK;
  }
  tmul::PlanParams p;
  const int rc = tmul::explicit_params(kind, n_bits, int(b), int64_t(N), &p);
  if (rc) return rc;
  if (p.e_max > tmul::bound_target()) return TM_ERANGE;   // not certified
  std::lock_guard<std::mutex> lk(tmul::g_mu);
  tmul::g_params[key] = p;
  return TM_OK;
}

int tm_autotune_plan(int kind, uint64_t n_bits, void* stream, tm_plan_tune* out) {
  if (!out) return TM_EINVAL;
  std::memset(out, 0, sizeof(*out));
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n_bits == 0) return TM_EINVAL;
  if (n_bits > TM_MAX_BITS) return TM_ERANGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<tmul::PlanParams> cands;
  int rc = tmul::certified_candidates(kind, n_bits, 1.15, 8, &cands);
  if (rc) return rc;
  // operands: any bits do (the work does not depend on the values)
  const size_t in_bytes = size_t(tmul::limbs_of(n_bits)) * 8;
  const size_t out_bytes = size_t(tmul::out_limbs(kind, n_bits)) * 8;
  char* buf = nullptr;
  if (cudaMalloc(&buf, 2 * tmul::align_up(in_bytes) + out_bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    return TM_ENOMEM;
  }
  uint64_t* du = reinterpret_cast<uint64_t*>(buf);
  uint64_t* dv = reinterpret_cast<uint64_t*>(buf + tmul::align_up(in_bytes));
  uint64_t* dout = reinterpret_cast<uint64_t*>(buf + 2 * tmul::align_up(in_bytes));
  cudaMemsetAsync(du, 0x5a, in_bytes, s);
  cudaMemsetAsync(dv, 0xa7, in_bytes, s);
  tmul::DevStatus saved{};
  if (tmul::stream_status_word(s, &saved, true) != TM_OK) {
    cudaFree(buf);
    return TM_ECUDA;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const auto key = std::make_pair(kind, n_bits);
  std::vector<double> ms(cands.size(), 0.0);
  for (size_t c = 0; c < cands.size() && rc == TM_OK; ++c) {
    {
      std::lock_guard<std::mutex> lk(tmul::g_mu);
      tmul::g_params[key] = cands[c];
    }
    // each candidate runs with the layout already set for its length (the default
    // unless tm_autotune or tm_set_layout chose one): tm_autotune's choice comes from
    // timing the transforms alone, and at n = 2^20 a layout it ranked 3% faster there
    // made whole products 35% slower, so the plan tuner does not re-tune layouts
    // one warm-up product (it builds the tables), then the median of five isolated
    // products: a delay kernel holds the stream while the host plans and enqueues the
    // product, so the time is the device's latency for one product, without the
    // host's work and without overlap with a neighbouring product
    rc = tmul::run(kind, dout, du, dv, n_bits, s, nullptr, nullptr);
    if (rc == TM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = TM_ECUDA;
    std::vector<float> t;
    for (int rep = 0; rep < 5 && rc == TM_OK; ++rep) {
      tmul::launch_delay(kTuneDelayNs, s);
      cudaEventRecord(e0, s);
      rc = tmul::run(kind, dout, du, dv, n_bits, s, nullptr, nullptr);
      cudaEventRecord(e1, s);
      if (rc == TM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = TM_ECUDA;
      float x = 0;
      cudaEventElapsedTime(&x, e0, e1);
      t.push_back(x);
    }
    if (rc) break;
    std::sort(t.begin(), t.end());
    ms[c] = t[t.size() / 2];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  // the stream's status word as the caller left it: the trial products' margins must
  // not reach the next reported call
  if (rc == TM_OK && tmul::stream_status_word(s, &saved, false) != TM_OK) rc = TM_ECUDA;
  tmul::PlanParams chosen = cands[0];
  size_t best = 0;
  if (rc == TM_OK) {
    for (size_t c = 1; c < ms.size(); ++c)
      if (ms[c] < ms[best]) best = c;
    if (ms[best] > kTuneGain * ms[0]) best = 0;   // within the noise: keep the planner's
    chosen = cands[best];
  }
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(tmul::g_mu);
    if (best == 0) tmul::g_params.erase(key);
    else tmul::g_params[key] = chosen;
    // tables of the candidates that lost and that nothing else holds
    for (size_t c = 1; c < cands.size(); ++c) {
      if (c == best) continue;
      auto it = tmul::g_plans.find(std::make_tuple(dev, kind, cands[c].b, cands[c].N, 0));
      if (it == tmul::g_plans.end()) continue;
      if (it->second.use_count() == 1) {
        tmul::PlanEntry& e = *it->second;
        cudaFree(e.tw); cudaFree(e.fwd_tab); cudaFree(e.bwd_tab); cudaFree(e.bwd_tab2);
        cudaFree(e.small);
      } else {
        tmul::g_retired.push_back(it->second);
      }
      tmul::g_plans.erase(it);
    }
  }
  if (rc) return rc;
  if (cudaGetLastError() != cudaSuccess) return TM_ECUDA;
  out->b = uint32_t(chosen.b);
  out->N = uint32_t(chosen.N);
  out->candidates = uint32_t(cands.size());
  out->ms_default = ms[0];
  out->ms_best = ms[best];
  return TM_OK;
}

int tm_set_layout(int kind, uint64_t n_bits, const tm_tune* layout) {
  if (!layout) return TM_EINVAL;
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n_bits == 0) return TM_EINVAL;
  if (n_bits > TM_MAX_BITS) return TM_ERANGE;
  const tmul::FftShape sh{layout->points, layout->split, layout->passes};
  if (sh.points < 32 || sh.points > 4096 || sh.split < 0 || sh.split > 2 ||
      (sh.passes != 0 && sh.passes != 2 && sh.passes != 3))
    return TM_EINVAL;
  tmul::PlanParams p;
  int rc = tmul::get_params(kind, n_bits, &p);
  if (rc) return rc;
  tmul::FftPlan f;
  rc = tmul::make_fft_plan(p.N / 2, &f, false, &sh);
  if (rc) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return TM_ECUDA;
  }
  const tmul::FftShape def{};
  const bool is_default = sh.points == def.points && sh.split == def.split &&
                          sh.passes == def.passes;
  tmul::apply_layout(dev, p.N, is_default ? nullptr : &sh);
  return TM_OK;
}

int tm_plan_query(int kind, uint64_t n_bits, tm_report* rep) {
  if (!rep) return TM_EINVAL;
  tmul::PlanParams p;
  int rc = tmul::get_params(kind, n_bits, &p);
  if (rc) return rc;
  // the layout a product would use: the tuned one for this device, if any
  tmul::FftShape shape;
  bool tuned = false;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) {
    std::lock_guard<std::mutex> lk(tmul::g_mu);
    auto t = tmul::g_tuned.find(std::make_pair(dev, p.N / 2));
    if (t != tmul::g_tuned.end()) { shape = t->second; tuned = true; }
  } else {
    (void)cudaGetLastError();
  }
  tmul::FftPlan f;
  rc = tmul::make_fft_plan(p.N / 2, &f, false, tuned ? &shape : nullptr);
  if (rc) return rc;
  tmul::fill_plan_report(p, f, rep);
  return TM_OK;
}

int tm_stream_status(void* stream, tm_report* rep) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
  tmul::Workspace* ws = nullptr;
  {
    std::lock_guard<std::mutex> lk(tmul::g_mu);
    auto it = tmul::g_ws.find(std::make_pair(dev, static_cast<cudaStream_t>(stream)));
    if (it == tmul::g_ws.end()) {
      if (rep) { rep->margin = 0; rep->status = TM_OK; }
      return TM_OK;
    }
    ws = &it->second;
  }
  return tmul::read_status(static_cast<cudaStream_t>(stream), ws->status, rep);
}

int tm_release(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TM_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return TM_ECUDA;
  std::lock_guard<std::mutex> lk(tmul::g_mu);
  for (auto it = tmul::g_plans.begin(); it != tmul::g_plans.end();) {
    if (std::get<0>(it->first) == dev) {
      tmul::PlanEntry& e = *it->second;
      cudaFree(e.tw); cudaFree(e.fwd_tab); cudaFree(e.bwd_tab); cudaFree(e.bwd_tab2);
      cudaFree(e.small);
      it = tmul::g_plans.erase(it);
    } else {
      ++it;
    }
  }
  for (auto& kv : tmul::g_host_graphs) tmul::drop_host_graph(kv.second);
  tmul::g_host_graphs.clear();
  for (auto& r : tmul::g_retired) {
    cudaFree(r->tw); cudaFree(r->fwd_tab); cudaFree(r->bwd_tab); cudaFree(r->bwd_tab2);
    cudaFree(r->small);
    r->tw = nullptr; r->fwd_tab = nullptr; r->bwd_tab = nullptr; r->bwd_tab2 = nullptr;
    r->small = nullptr;
  }
  tmul::g_retired.clear();
  for (auto it = tmul::g_ws.begin(); it != tmul::g_ws.end();) {
    if (it->first.first == dev) {
      cudaFree(it->second.base);
      cudaFree(it->second.status);
      cudaFree(it->second.io);
      if (it->second.norms) cudaFree(it->second.norms);
      if (it->second.status_host) cudaFreeHost(it->second.status_host);
      if (it->second.side) cudaStreamDestroy(it->second.side);
      if (it->second.fork) cudaEventDestroy(it->second.fork);
      if (it->second.join) cudaEventDestroy(it->second.join);
      it = tmul::g_ws.erase(it);
    } else {
      ++it;
    }
  }
  return TM_OK;
}

int tm_set_fused(int mode) {
  if (mode < 0 || mode > 2) return TM_EINVAL;
  tmul::g_fused_mode.store(mode);
  return TM_OK;
}

int tm_convolution(double* out, const double* x, const double* y, int64_t N, void* stream,
                   double* eta) {
  using namespace tmul;
  if (!out || !x || !y || N < 4 || N > (int64_t(1) << 31) || !is_valid_length(N))
    return TM_EINVAL;
  if (eta) *eta = conv_error_bound(N);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PlanParams p;
  p.kind = TM_FULL;               // twiddle and twist tables only (no map rows)
  p.b = 0;                        // a cache key of its own
  p.n = 64;
  p.N = N;
  std::shared_ptr<PlanEntry> pe;
  int rc = get_tables(p, false, s, &pe);
  if (rc) return rc;
  Workspace* ws = nullptr;
  rc = get_workspace(s, workspace_bytes(p), &ws);
  if (rc) return rc;
  ensure_kernel_attributes();
  const int64_t M = N / 2;
  double2* R0 = reinterpret_cast<double2*>(ws->base);
  double2* R1 = reinterpret_cast<double2*>(ws->base + region_bytes(p, M));
  double2* bufs[2] = {R0, R1};
  // the real sequences are their packed complex sequences (x_2j + i x_2j+1)
  TM_CHECK(cudaMemcpyAsync(R0, x, size_t(N) * 8, cudaMemcpyDeviceToDevice, s));
  TM_CHECK(cudaMemcpyAsync(R0 + M, y, size_t(N) * 8, cudaMemcpyDeviceToDevice, s));
  int cur = launch_fft(*pe, bufs, 0, -1, 2, M, s);
  launch_twist(bufs[cur], bufs[cur] + M, bufs[cur ^ 1], M, pe->tw + pe->twc_off, N, 1, 0, 0, s);
  cur = launch_fft(*pe, bufs, cur ^ 1, 1, 1, M, s);
  TM_CHECK(cudaMemcpyAsync(out, bufs[cur], size_t(N) * 8, cudaMemcpyDeviceToDevice, s));
  return cudaGetLastError() == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_table_values(int which, int64_t len, int64_t count, double* out, void* stream) {
  if (!out || len < 1 || count < 0 || len > (int64_t(1) << 40)) return TM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (which) {
    case 0: tmul::launch_init_twiddles(reinterpret_cast<double2*>(out), len, count, s); break;
    case 1:
      if (count != len || len > (int64_t(1) << 30)) return TM_EINVAL;
      tmul::launch_init_tw4(reinterpret_cast<tmul::Tan4*>(out), int(len), s);
      break;
    case 2: tmul::launch_init_twist_coef(reinterpret_cast<double2*>(out), len, count, s); break;
    case 3:
      if (count < 1 || len % count) return TM_EINVAL;
      tmul::launch_init_outer(reinterpret_cast<double2*>(out), len, count, s);
      break;
    default: return TM_EINVAL;
  }
  return cudaGetLastError() == cudaSuccess ? TM_OK : TM_ECUDA;
}

int tm_probe_dfma(int iters, void* stream, double* flops) {
  if (iters <= 0 || !flops) return TM_EINVAL;
  *flops = tmul::launch_probe_dfma(iters, static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? TM_OK : TM_ECUDA;
}

const char* tm_strerror(int code) {
  switch (code) {
    case TM_OK: return "ok";
    case TM_UNCERTIFIED: return "ok within the caller's limit, not certified by the error bound";
    case TM_EINVAL: return "invalid argument";
    case TM_ENOMEM: return "out of memory";
    case TM_EPRECISION: return "rounding margin above the error bound: result not trusted";
    case TM_ETIMEOUT: return "a bounded device-side wait timed out";
    case TM_ECUDA: return "CUDA runtime error";
    case TM_ERANGE: return "operand size outside the supported range";
    case TM_EALIAS: return "output overlaps an input";
    default: return "unknown status";
  }
}

}  // extern "C"
