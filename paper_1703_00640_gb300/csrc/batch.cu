// Batched products: plan groups, one workspace per group, one CUDA graph.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/truncmul.h"
#include "kernels.cuh"
#include "runtime.h"

namespace tmul {
namespace {

constexpr int kBranches = 12;  // concurrent graph branches

#define TB_CHECK(x)                                    \
  do {                                                 \
    cudaError_t e_ = (x);                              \
    if (e_ != cudaSuccess) {                           \
      (void)cudaGetLastError();                        \
      return e_ == cudaErrorMemoryAllocation ? TM_ENOMEM : TM_ECUDA; \
    }                                                  \
  } while (0)

struct Group {
  PlanParams p;                        // kind, b, N, lambdas of the group
  std::shared_ptr<PlanEntry> pe;
  std::vector<uint32_t> members;       // indices into the descriptor array
  size_t carry_bytes = 0;              // per-product carry scratch
  size_t off = 0;                      // offset of the group's memory
  size_t bytes = 0;
  long long nblocks_max = 0;
  unsigned long long emax_fx_min = ~0ull;
};

size_t carry_scratch(const PlanParams& p) {
  int64_t nS, sh, rb;
  carry_shape(p, &nS, &sh, &rb);
  return align_up(size_t(2) * nS * 8) + 2 * align_up(size_t(nS / 512 + 2));
}

}  // namespace
}  // namespace tmul

struct tm_batch {
  int dev = 0;
  std::vector<tm_desc> descs;
  std::vector<tmul::PlanParams> params;
  std::vector<tmul::Group> groups;
  // CTA-resident products
  std::vector<uint32_t> small;
  std::vector<tmul::SmallPlan> small_plans;
  std::vector<std::shared_ptr<tmul::PlanEntry>> small_tables;
  size_t small_off = 0, small_smem = 0;
  char* mem = nullptr;
  tmul::DevStatus* status = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double e_max_min = 1.0;
  // one persistent launch (k_batch_persistent) in place of the per-phase graph
  bool persistent = false;
  tmul::BatchArgs pargs{};
  int pgrid = 0;
  size_t psmem = 0;
  size_t pcounter_bytes = 0;     // ticket and per-group counters, zeroed before each launch
};

namespace tmul {
namespace {

// Enqueues every phase of one group as batched launches.
int enqueue_group(tm_batch* B, const Group& g, cudaStream_t s) {
  const PlanParams& p = g.p;
  const PlanEntry& pe = *g.pe;
  const int kind = p.kind;
  const int64_t N = p.N, M = pe.M;
  const int cnt = int(g.members.size());
  char* base = B->mem + g.off;
  const size_t slab = size_t(cnt) * 2 * M * sizeof(double2);
  double2* R0 = reinterpret_cast<double2*>(base);
  double2* R1 = reinterpret_cast<double2*>(base + align_up(slab));
  char* items = base + 2 * align_up(slab);
  FwdItem* fi = reinterpret_cast<FwdItem*>(items);
  BackItem* bi = reinterpret_cast<BackItem*>(items + align_up(cnt * sizeof(FwdItem)));
  CarryItem* ci = reinterpret_cast<CarryItem*>(reinterpret_cast<char*>(bi) +
                                               align_up(cnt * sizeof(BackItem)));
  FwdArgs fa{};
  fa.items = fi;
  fa.b = p.b;
  fa.N = N;
  fa.lam = kind == TM_FULL ? 0 : p.lam_fwd;
  fa.tab = pe.fwd_tab;
  fa.kappa = pe.small;
  fa.nkappa = pe.nkappa;
  fa.rho_pow = pe.small ? pe.small + pe.nkappa : nullptr;
  fa.ntheta = pe.ntheta;
  launch_fwd(kind, fa, cnt, s);
  double2* bufs[2] = {R0, R1};
  int cur = launch_fft(pe, bufs, 0, -1, 2 * cnt, M, s);
  launch_twist(bufs[cur], bufs[cur] + M, bufs[cur ^ 1], M, pe.tw + pe.twc_off, N, cnt, 2 * M,
               2 * M, s);
  cur ^= 1;
  cur = launch_fft(pe, bufs, cur, 1, cnt, 2 * M, s);
  if (cur != 1) return TM_EINVAL;       // the item layout assumes the output in R1
  BackArgs ba{};
  ba.items = bi;
  ba.N = N;
  ba.b = p.b;
  ba.lam = kind == TM_FULL ? 0 : p.lam_bwd;
  ba.tab = pe.bwd_tab;
  ba.tab2 = kind == TM_HI ? pe.bwd_tab2 : pe.bwd_tab;
  ba.kappa = pe.small;
  ba.nkappa = pe.nkappa;
  ba.rho = p.rho;
  ba.count = kind == TM_HI ? N + 1 : N;
  ba.status = B->status;
  launch_back(kind, ba, cnt, s);
  CarryArgs ca{};
  ca.items = ci;
  ca.nblocks_max = g.nblocks_max;
  ca.K = kind == TM_HI ? N + 1 : N;
  ca.b = p.b;
  ca.kind = kind;
  launch_carry(ca, cnt, s);
  TB_CHECK(cudaGetLastError());
  return TM_OK;
}

// Host images of the per-product items of one group.
void build_items(tm_batch* B, const Group& g, std::vector<char>* host) {
  const PlanParams& p = g.p;
  const int64_t N = p.N, M = g.pe->M;
  const int cnt = int(g.members.size());
  char* base = B->mem + g.off;
  const size_t slab = size_t(cnt) * 2 * M * sizeof(double2);
  char* R0 = base;
  char* R1 = base + align_up(slab);
  const size_t items_off = 2 * align_up(slab);
  const size_t fbytes = align_up(cnt * sizeof(FwdItem));
  const size_t bbytes = align_up(cnt * sizeof(BackItem));
  const size_t cbytes = align_up(cnt * sizeof(CarryItem));
  double* theta = reinterpret_cast<double*>(base + items_off + fbytes + bbytes + cbytes);
  char* carry = reinterpret_cast<char*>(theta) + align_up(size_t(cnt) * 2 * 8);
  host->assign(fbytes + bbytes + cbytes, 0);
  FwdItem* fi = reinterpret_cast<FwdItem*>(host->data());
  BackItem* bi = reinterpret_cast<BackItem*>(host->data() + fbytes);
  CarryItem* ci = reinterpret_cast<CarryItem*>(host->data() + fbytes + bbytes);
  for (int i = 0; i < cnt; ++i) {
    const tm_desc& d = B->descs[g.members[i]];
    const PlanParams& q = B->params[g.members[i]];
    const uint64_t n = d.n_bits;
    double* X = reinterpret_cast<double*>(R0 + size_t(i) * 2 * M * sizeof(double2));
    fi[i].u = reinterpret_cast<const unsigned long long*>(d.u);
    fi[i].v = reinterpret_cast<const unsigned long long*>(d.v);
    fi[i].n = n;
    fi[i].nlimbs = limbs_of(n);
    fi[i].nd = q.n_digits;
    fi[i].s0 = int64_t(N + 1) * p.b - int64_t(n);
    fi[i].X = X;
    fi[i].theta = theta + 2 * i;
    bi[i].w = reinterpret_cast<const double*>(R1 + size_t(i) * 2 * M * sizeof(double2));
    bi[i].c = reinterpret_cast<long long*>(X);
    bi[i].theta = theta + 2 * i;
    bi[i].emax_fx = emax_fixed(q.e_max);
    int64_t nS, shift, rbit;
    carry_shape(q, &nS, &shift, &rbit);
    char* scratch = carry + size_t(i) * g.carry_bytes;
    ci[i].c = reinterpret_cast<const long long*>(X);
    ci[i].nS = nS;
    ci[i].round_bit = rbit;
    ci[i].shift_bits = shift;
    ci[i].nout = out_limbs(p.kind, n);
    ci[i].top_mask = (p.kind == TM_LO && n % 64) ? ((1ull << (n % 64)) - 1ull) : ~0ull;
    ci[i].out = reinterpret_cast<unsigned long long*>(d.out);
    ci[i].r = reinterpret_cast<unsigned long long*>(scratch);
    ci[i].fblock = reinterpret_cast<unsigned char*>(scratch + align_up(size_t(2) * nS * 8));
    ci[i].cin_block = ci[i].fblock + align_up(size_t(nS / 512 + 2));
  }
}

size_t group_bytes(const Group& g) {
  const int cnt = int(g.members.size());
  const size_t slab = size_t(cnt) * 2 * g.pe->M * sizeof(double2);
  return 2 * align_up(slab) + align_up(cnt * sizeof(FwdItem)) + align_up(cnt * sizeof(BackItem)) +
         align_up(cnt * sizeof(CarryItem)) + align_up(size_t(cnt) * 2 * 8) +
         size_t(cnt) * g.carry_bytes + 256;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + nb && y < x + na;
}

void destroy(tm_batch* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  cudaFree(B->mem);
  delete B;
}

// ------------------------------------------------ the batch as one persistent launch

// Virtual blocks of every phase of group g (the counts k_batch_persistent walks).
void phase_units(const BatchGroup& G, long long* units) {
  const long long cnt = G.cnt;
  for (int ph = 0; ph < kBatchPhases; ++ph) units[ph] = 0;
  units[kPhFwdMap] = (G.fa.N + kFwdTile - 1) / kFwdTile * cnt;
  for (int i = 0; i < G.npass; ++i) {
    const long long bx = (G.fwd[i].Q + G.fwd[i].C - 1) / G.fwd[i].C;
    units[kPhFwdPass + i] = bx * 2 * cnt;
    units[kPhInvPass + i] = bx * cnt;
  }
  units[kPhTwist] = (G.M / 2 + kFusedThreads) / kFusedThreads * cnt;
  if (G.kind == TM_FULL) units[kPhBack] = G.back_nvb * cnt;
  else if (G.back_small) units[kPhBack] = cnt;
  else units[kPhBack] = (G.ba.N + kBackTile - 1) / kBackTile * cnt;
  units[kPhCarryLocal] = G.ca.nblocks_max * cnt;
  units[kPhCarryBlocks] = cnt;
  units[kPhCarryApply] = G.ca.nblocks_max * cnt;
}

// The arguments of every phase of one group, on the group's buffers and items (the
// same layout as enqueue_group).
BatchGroup batch_group(tm_batch* B, const Group& g, size_t* smem) {
  const PlanParams& p = g.p;
  const PlanEntry& pe = *g.pe;
  const int kind = p.kind;
  const int64_t N = p.N, M = pe.M;
  const int cnt = int(g.members.size());
  char* base = B->mem + g.off;
  const size_t slab = size_t(cnt) * 2 * M * sizeof(double2);
  double2* R0 = reinterpret_cast<double2*>(base);
  double2* R1 = reinterpret_cast<double2*>(base + align_up(slab));
  char* items = base + 2 * align_up(slab);
  FwdItem* fi = reinterpret_cast<FwdItem*>(items);
  BackItem* bi = reinterpret_cast<BackItem*>(items + align_up(cnt * sizeof(FwdItem)));
  CarryItem* ci = reinterpret_cast<CarryItem*>(reinterpret_cast<char*>(bi) +
                                               align_up(cnt * sizeof(BackItem)));
  BatchGroup G{};
  G.kind = kind;
  G.npass = pe.fft.npass;
  G.cnt = cnt;
  FwdArgs& fa = G.fa;
  fa.items = fi;
  fa.b = p.b;
  fa.N = N;
  fa.lam = kind == TM_FULL ? 0 : p.lam_fwd;
  fa.tab = pe.fwd_tab;
  fa.kappa = pe.small;
  fa.nkappa = pe.nkappa;
  fa.rho_pow = pe.small ? pe.small + pe.nkappa : nullptr;
  fa.ntheta = pe.ntheta;
  double2* bufs[2] = {R0, R1};
  int cur = 0;
  for (int i = 0; i < G.npass; ++i) {
    const FftPass& fp = pe.fft.pass[i];
    // sequences per CTA: as many points as the CTA's threads hold radix-4 butterflies
    const int C = int(std::max<int64_t>(1, std::min<int64_t>(4 * kFusedThreads / fp.L, fp.Q)));
    G.fwd[i] = pass_args(pe, i, M);
    G.fwd[i].C = C;
    G.fwd_in[i] = bufs[cur];
    G.fwd_out[i] = bufs[cur ^ 1];
    cur ^= 1;
    *smem = std::max(*smem, pass_smem(fp, C));
  }
  G.Zu = bufs[cur];
  G.Q = bufs[cur ^ 1];
  G.M = M;
  G.tc = pe.tw + pe.twc_off;
  G.two_over_N = 2.0 / double(N);
  cur ^= 1;
  for (int i = 0; i < G.npass; ++i) {
    G.inv[i] = pass_args(pe, i, 2 * M);
    G.inv[i].C = G.fwd[i].C;
    G.inv_in[i] = bufs[cur];
    G.inv_out[i] = bufs[cur ^ 1];
    cur ^= 1;
  }
  BackArgs& ba = G.ba;
  ba.items = bi;
  ba.N = N;
  ba.b = p.b;
  ba.lam = kind == TM_FULL ? 0 : p.lam_bwd;
  ba.tab = pe.bwd_tab;
  ba.tab2 = kind == TM_HI ? pe.bwd_tab2 : pe.bwd_tab;
  ba.kappa = pe.small;
  ba.nkappa = pe.nkappa;
  ba.rho = p.rho;
  ba.count = kind == TM_HI ? N + 1 : N;
  ba.status = B->status;
  G.back_small = kind != TM_FULL && (N <= 64 || N < 2 * ba.lam + ba.nkappa + 2) ? 1 : 0;
  G.back_nvb = std::min<long long>((ba.count + kFusedThreads - 1) / kFusedThreads, 152 * 8);
  CarryArgs& ca = G.ca;
  ca.items = ci;
  ca.nblocks_max = g.nblocks_max;
  ca.K = kind == TM_HI ? N + 1 : N;
  ca.b = p.b;
  ca.kind = kind;
  return G;
}

}  // namespace

SmallItem small_item_for(const void* out, const void* u, const void* v, uint64_t n,
                         const PlanParams& q, int plan) {
  SmallItem it{};
  it.u = static_cast<const unsigned long long*>(u);
  it.v = static_cast<const unsigned long long*>(v);
  it.out = static_cast<unsigned long long*>(const_cast<void*>(out));
  it.n = n;
  it.nlimbs = limbs_of(n);
  it.nd = q.n_digits;
  it.s0 = int64_t(q.N + 1) * q.b - int64_t(n);
  int64_t nS, shift, rbit;
  carry_shape(q, &nS, &shift, &rbit);
  it.nS = nS;
  it.round_bit = rbit;
  it.shift_bits = shift;
  it.nout = out_limbs(q.kind, n);
  it.top_mask = (q.kind == TM_LO && n % 64) ? ((1ull << (n % 64)) - 1ull) : ~0ull;
  it.emax_fx = emax_fixed(q.limit > 0.0 ? q.limit : q.e_max);
  it.plan = plan;
  return it;
}

SmallPlan small_plan_of(const PlanParams& p, const PlanEntry& pe) {
  SmallPlan sp{};
  const FftPass& fp = pe.fft.pass[0];
  sp.kind = p.kind;
  sp.b = p.b;
  sp.lam_fwd = p.lam_fwd;
  sp.lam_bwd = p.lam_bwd;
  sp.nkappa = pe.nkappa;
  sp.ntheta = pe.ntheta;
  sp.N = p.N;
  sp.M = pe.M;
  sp.rho = p.rho;
  sp.nstages = fp.nstages;
  std::copy(fp.radix, fp.radix + kMaxStages, sp.radix);
  std::copy(fp.tw4_off, fp.tw4_off + kMaxStages, sp.tw4_off);
  sp.tw4_len = fp.tw4_len;
  sp.need_wL = fp.need_wL ? 1 : 0;
  sp.tw_sub = pe.tw + fp.tw_sub;
  sp.tw4 = reinterpret_cast<const Tan4*>(pe.tw + fp.tw4);
  sp.twc = pe.tw + pe.twc_off;
  sp.fwd_tab = pe.fwd_tab;
  sp.bwd_tab = pe.bwd_tab;
  sp.bwd_tab2 = p.kind == TM_HI ? pe.bwd_tab2 : pe.bwd_tab;
  sp.kappa = pe.small;
  sp.rho_pow = pe.small ? pe.small + pe.nkappa : nullptr;
  return sp;
}

namespace {

// The persistent form: every group's phase arguments and the unit tables in device
// memory, then one graph of two nodes, the counters' reset and one cooperative launch
// (a reset and a direct launch per tm_batch_launch when the runtime cannot record it).
int create_persistent(tm_batch* B, size_t groups_off, size_t start_off, size_t sync_off,
                      cudaStream_t s) {
  const int ng = int(B->groups.size());
  std::vector<BatchGroup> gs(ng);
  std::vector<std::array<long long, kBatchPhases>> units(ng);
  size_t smem = 0;
  std::vector<std::pair<double, int>> order(ng);
  for (int g = 0; g < ng; ++g) {
    gs[g] = batch_group(B, B->groups[g], &smem);
    phase_units(gs[g], units[g].data());
    const double N = double(B->groups[g].p.N);
    order[g] = {double(B->groups[g].members.size()) * N * (std::log2(N) + 8.0), g};
  }
  std::sort(order.rbegin(), order.rend());             // largest estimated work first
  // the unit list: phase by phase, each group's segment with the count of its units
  // in earlier phases, which the segment's units wait for
  std::vector<int> seg_group, seg_phase;
  std::vector<long long> seg_start(1, 0), seg_wait, before(ng, 0);
  for (int ph = 0; ph < kBatchPhases; ++ph)
    for (const auto& o : order) {
      const int g = o.second;
      if (units[g][ph] == 0) continue;
      seg_group.push_back(g);
      seg_phase.push_back(ph);
      seg_wait.push_back(before[g]);
      seg_start.push_back(seg_start.back() + units[g][ph]);
      before[g] += units[g][ph];
    }
  const size_t nseg = seg_group.size();
  // device copies: groups, then the segment tables, then the counters
  BatchGroup* dg = reinterpret_cast<BatchGroup*>(B->mem + groups_off);
  char* tab = B->mem + start_off;
  long long* d_start = reinterpret_cast<long long*>(tab);
  long long* d_wait = reinterpret_cast<long long*>(tab + align_up((nseg + 1) * sizeof(long long)));
  int* d_group = reinterpret_cast<int*>(reinterpret_cast<char*>(d_wait) +
                                        align_up(nseg * sizeof(long long) + 8));
  int* d_phase = reinterpret_cast<int*>(reinterpret_cast<char*>(d_group) +
                                        align_up(nseg * sizeof(int) + 4));
  unsigned* counters = reinterpret_cast<unsigned*>(B->mem + sync_off);   // ticket, done[ng]
  if (ng) TB_CHECK(cudaMemcpyAsync(dg, gs.data(), ng * sizeof(BatchGroup), cudaMemcpyHostToDevice, s));
  TB_CHECK(cudaMemcpyAsync(d_start, seg_start.data(), seg_start.size() * sizeof(long long),
                           cudaMemcpyHostToDevice, s));
  if (nseg) {
    TB_CHECK(cudaMemcpyAsync(d_wait, seg_wait.data(), nseg * sizeof(long long),
                             cudaMemcpyHostToDevice, s));
    TB_CHECK(cudaMemcpyAsync(d_group, seg_group.data(), nseg * sizeof(int),
                             cudaMemcpyHostToDevice, s));
    TB_CHECK(cudaMemcpyAsync(d_phase, seg_phase.data(), nseg * sizeof(int),
                             cudaMemcpyHostToDevice, s));
  }
  TB_CHECK(cudaStreamSynchronize(s));
  const int resident = batch_max_blocks(smem);
  if (resident <= 0) return TM_ECUDA;
  B->pargs.groups = dg;
  B->pargs.ngroups = ng;
  B->pargs.nseg = int(nseg);
  B->pargs.total = seg_start.back();
  B->pargs.seg_start = d_start;
  B->pargs.seg_group = d_group;
  B->pargs.seg_phase = d_phase;
  B->pargs.seg_wait = d_wait;
  B->pargs.ticket = counters;
  B->pargs.done = counters + 1;
  B->pargs.status = B->status;
  B->pargs.withhold = fault_leave_barrier() ? 1 : 0;
  B->pcounter_bytes = size_t(ng + 1) * sizeof(unsigned);
  B->pgrid = int(std::min<long long>(seg_start.back(), resident));
  B->psmem = smem;
  if (ng == 0) return TM_OK;
  // one graph: zero the counters, then the launch
  cudaStream_t cs;
  TB_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    cudaError_t le = cudaMemsetAsync(counters, 0, B->pcounter_bytes, cs);
    if (le == cudaSuccess) le = launch_batch_persistent(B->pargs, B->pgrid, B->psmem, cs);
    ce = cudaStreamEndCapture(cs, &B->graph);
    if (le == cudaSuccess && ce == cudaSuccess) ce = cudaGraphInstantiate(&B->exec, B->graph, 0);
    else if (ce == cudaSuccess) ce = le;
  }
  cudaStreamDestroy(cs);
  if (ce != cudaSuccess) {            // launch directly instead
    (void)cudaGetLastError();
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
  }
  return TM_OK;
}

int create(tm_batch** out, const tm_desc* descs, uint32_t count, cudaStream_t s) {
  if (!out || (!descs && count)) return TM_EINVAL;
  std::unique_ptr<tm_batch, void (*)(tm_batch*)> B(new tm_batch(), destroy);
  TB_CHECK(cudaGetDevice(&B->dev));
  B->descs.assign(descs, descs + count);
  B->params.resize(count);
  B->persistent = g_fused_mode.load() == 2;
  std::map<std::tuple<int, int, int64_t>, size_t> index;
  for (uint32_t i = 0; i < count; ++i) {
    const tm_desc& d = B->descs[i];
    if (d.kind != TM_FULL && d.kind != TM_LO && d.kind != TM_HI) return TM_EINVAL;
    if (d.n_bits == 0 || !d.u || !d.v || !d.out) return TM_EINVAL;
    if (d.n_bits > TM_MAX_BITS) return TM_ERANGE;
    const size_t ib = size_t(limbs_of(d.n_bits)) * 8, ob = size_t(out_limbs(d.kind, d.n_bits)) * 8;
    if (overlap(d.out, ob, d.u, ib) || overlap(d.out, ob, d.v, ib)) return TM_EALIAS;
    int rc = get_params(d.kind, d.n_bits, &B->params[i]);
    if (rc) return rc;
    const PlanParams& q = B->params[i];
    B->e_max_min = std::min(B->e_max_min, q.e_max);
    if (!B->persistent && q.N / 2 <= kSmallMaxM) {   // CTA-resident
      B->small.push_back(i);
      continue;
    }
    auto key = std::make_tuple(q.kind, q.b, q.N);
    auto it = index.find(key);
    if (it == index.end()) {
      Group g;
      g.p = q;
      rc = get_tables(q, false, s, &g.pe);
      if (rc) return rc;
      index[key] = B->groups.size();
      B->groups.push_back(std::move(g));
      it = index.find(key);
    }
    Group& g = B->groups[it->second];
    g.members.push_back(i);
    g.carry_bytes = std::max(g.carry_bytes, carry_scratch(q));
    int64_t nS, sh, rb;
    carry_shape(q, &nS, &sh, &rb);
    g.nblocks_max = std::max<long long>(g.nblocks_max, (nS + 511) / 512);
  }
  // plans of the CTA-resident products (single-pass tables)
  std::map<std::tuple<int, int, int64_t>, int> small_index;
  std::vector<SmallItem> small_items;
  for (uint32_t i : B->small) {
    const PlanParams& q = B->params[i];
    auto key = std::make_tuple(q.kind, q.b, q.N);
    auto it = small_index.find(key);
    if (it == small_index.end()) {
      std::shared_ptr<PlanEntry> pe;
      const int rc = get_tables(q, true, s, &pe);
      if (rc) return rc;
      small_index[key] = int(B->small_plans.size());
      B->small_plans.push_back(small_plan_of(q, *pe));
      B->small_tables.push_back(pe);
      const FftPass& fp = pe->fft.pass[0];
      B->small_smem = std::max(B->small_smem,
                               small_smem_bytes(q.N, pe->M, fp.tw4_len, fp.need_wL));
      it = small_index.find(key);
    }
    small_items.push_back(small_item_for(B->descs[i].out, B->descs[i].u, B->descs[i].v,
                                          B->descs[i].n_bits, q, it->second));
  }
  // device memory: status word, CTA-resident items and plans, one region per group
  size_t total = 256;
  B->small_off = total;
  total += align_up(small_items.size() * sizeof(SmallItem)) +
           align_up(B->small_plans.size() * sizeof(SmallPlan)) + 256;
  for (Group& g : B->groups) {
    g.off = total;
    g.bytes = group_bytes(g);
    total += align_up(g.bytes);
  }
  const size_t ng = B->groups.size();
  const size_t pgroups_off = total;
  const size_t pstart_off = pgroups_off + align_up(ng * sizeof(BatchGroup));
  const size_t nseg_max = size_t(kBatchPhases) * ng;
  const size_t psync_off = pstart_off + align_up((nseg_max + 1) * sizeof(long long)) +
                           align_up(nseg_max * sizeof(long long) + 8) +
                           2 * align_up(nseg_max * sizeof(int) + 4);
  if (B->persistent) total = psync_off + align_up((ng + 1) * sizeof(unsigned)) + 256;
  TB_CHECK(cudaMalloc(&B->mem, total));
  B->status = reinterpret_cast<DevStatus*>(B->mem);
  TB_CHECK(cudaMemsetAsync(B->status, 0, sizeof(DevStatus), s));
  SmallArgs sa{};
  if (!small_items.empty()) {
    char* sbase = B->mem + B->small_off;
    const size_t ib = align_up(small_items.size() * sizeof(SmallItem));
    const size_t pb = align_up(B->small_plans.size() * sizeof(SmallPlan));
    TB_CHECK(cudaMemcpyAsync(sbase, small_items.data(), small_items.size() * sizeof(SmallItem),
                             cudaMemcpyHostToDevice, s));
    TB_CHECK(cudaMemcpyAsync(sbase + ib, B->small_plans.data(),
                             B->small_plans.size() * sizeof(SmallPlan), cudaMemcpyHostToDevice, s));
    TB_CHECK(cudaStreamSynchronize(s));
    sa.items = reinterpret_cast<const SmallItem*>(sbase);
    sa.count = int(small_items.size());
    sa.plans = reinterpret_cast<const SmallPlan*>(sbase + ib);
    sa.counter = reinterpret_cast<int*>(sbase + ib + pb);
    sa.status = B->status;
  }
  std::vector<char> host;
  for (Group& g : B->groups) {
    build_items(B.get(), g, &host);
    const int cnt = int(g.members.size());
    const size_t items_off = 2 * align_up(size_t(cnt) * 2 * g.pe->M * sizeof(double2));
    TB_CHECK(cudaMemcpyAsync(B->mem + g.off + items_off, host.data(), host.size(),
                             cudaMemcpyHostToDevice, s));
    TB_CHECK(cudaStreamSynchronize(s));
  }
  ensure_kernel_attributes();
  for (const Group& g : B->groups)         // one radix-4 butterfly per thread at most
    for (int i = 0; i < g.pe->fft.npass; ++i)
      if (g.pe->fft.pass[i].L > 4 * kFusedThreads) B->persistent = false;
  if (B->persistent) {
    const int rc = create_persistent(B.get(), pgroups_off, pstart_off, psync_off, s);
    if (rc) return rc;
    *out = B.release();
    return TM_OK;
  }
  // record the graph: groups spread over kBranches forked capture streams
  cudaStream_t cs[kBranches];
  cudaEvent_t fork, join[kBranches];
  for (int i = 0; i < kBranches; ++i) {
    TB_CHECK(cudaStreamCreateWithFlags(&cs[i], cudaStreamNonBlocking));
    TB_CHECK(cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming));
  }
  TB_CHECK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  int rc = TM_OK;
  cudaError_t ce = cudaStreamBeginCapture(cs[0], cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    cudaEventRecord(fork, cs[0]);
    for (int i = 1; i < kBranches; ++i) cudaStreamWaitEvent(cs[i], fork, 0);
    if (sa.count > 0) {                     // CTA-resident products on branch 0
      cudaMemsetAsync(sa.counter, 0, sizeof(int), cs[0]);
      launch_small(sa, std::min(sa.count, 152), B->small_smem, cs[0]);
    }
    // largest groups first, each to the branch with the least estimated work so far
    // (longest-processing-time order); work ~ products x N (log2 N + 8)
    auto work = [](double N, double count) { return count * N * (std::log2(N) + 8.0); };
    double load[kBranches] = {};
    if (sa.count > 0)
      for (const SmallItem& it : small_items) load[0] += work(double(B->small_plans[it.plan].N), 1.0);
    std::vector<size_t> order(B->groups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](size_t x, size_t y) {
      return work(double(B->groups[x].p.N), double(B->groups[x].members.size())) >
             work(double(B->groups[y].p.N), double(B->groups[y].members.size()));
    });
    for (size_t i = 0; i < order.size() && rc == TM_OK; ++i) {
      int br = 0;
      for (int j = 1; j < kBranches; ++j)
        if (load[j] < load[br]) br = j;
      const Group& g = B->groups[order[i]];
      load[br] += work(double(g.p.N), double(g.members.size()));
      rc = enqueue_group(B.get(), g, cs[br]);
    }
    for (int i = 1; i < kBranches; ++i) {
      cudaEventRecord(join[i], cs[i]);
      cudaStreamWaitEvent(cs[0], join[i], 0);
    }
    ce = cudaStreamEndCapture(cs[0], &B->graph);
    if (ce == cudaSuccess && rc == TM_OK) ce = cudaGraphInstantiate(&B->exec, B->graph, 0);
  }
  for (int i = 0; i < kBranches; ++i) {
    cudaStreamDestroy(cs[i]);
    cudaEventDestroy(join[i]);
  }
  cudaEventDestroy(fork);
  if (rc) return rc;
  TB_CHECK(ce);
  *out = B.release();
  return TM_OK;
}

}  // namespace
}  // namespace tmul

extern "C" {

int tm_batch_create(tm_batch** batch, const tm_desc* descs, uint32_t count, void* stream) {
  return tmul::create(batch, descs, count, static_cast<cudaStream_t>(stream));
}

int tm_batch_launch(tm_batch* batch, void* stream) {
  if (!batch) return TM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (batch->persistent) {
    if (batch->pargs.ngroups == 0) return TM_OK;
    cudaError_t e = cudaSuccess;
    if (batch->exec) {
      e = cudaGraphLaunch(batch->exec, s);
    } else {                           // the recorded graph zeroes the counters itself
      e = cudaMemsetAsync(batch->pargs.ticket, 0, batch->pcounter_bytes, s);
      if (e == cudaSuccess)
        e = tmul::launch_batch_persistent(batch->pargs, batch->pgrid, batch->psmem, s);
    }
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return TM_ECUDA;
    }
    return TM_OK;
  }
  if (!batch->exec) return TM_OK;
  const cudaError_t e = cudaGraphLaunch(batch->exec, s);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return TM_ECUDA;
  }
  return TM_OK;
}

int tm_batch_status(tm_batch* batch, void* stream, tm_report* rep) {
  if (!batch) return TM_EINVAL;
  const int rc = tmul::read_status(static_cast<cudaStream_t>(stream), batch->status, rep);
  if (rep) rep->e_max = batch->e_max_min;
  return rc;
}

int tm_batch_destroy(tm_batch* batch) {
  tmul::destroy(batch);
  return TM_OK;
}

int tm_mul_batch(const tm_desc* descs, uint32_t count, void* stream, tm_report* rep) {
  tm_batch* b = nullptr;
  int rc = tm_batch_create(&b, descs, count, stream);
  if (rc) return rc;
  rc = tm_batch_launch(b, stream);
  if (rc == TM_OK) rc = tm_batch_status(b, stream, rep);
  tm_batch_destroy(b);
  return rc;
}

}  // extern "C"
