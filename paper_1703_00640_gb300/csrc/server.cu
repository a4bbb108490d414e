// Serving layer: continuous batching of queued requests into stream slots under
// a device-memory budget.
#include <algorithm>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/truncmul.h"
#include "kernels.cuh"
#include "runtime.h"

namespace tmul {
namespace {

constexpr int kMicro = 256;            // most small requests per micro-batch launch

struct Request {
  int64_t ticket;
  int kind;
  uint64_t n;
  uint64_t* out;
  const uint64_t* u;
  const uint64_t* v;
  PlanParams p;
  bool small;
};

struct Slot {
  cudaStream_t s = nullptr;
  cudaEvent_t done = nullptr;
  Workspace ws;                        // large products
  SmallItem* d_items = nullptr;        // micro-batches of small products
  SmallPlan* d_plans = nullptr;
  int* d_counter = nullptr;
  SmallItem* h_items = nullptr;        // page-locked staging
  SmallPlan* h_plans = nullptr;
  DevStatus* d_status = nullptr;
  DevStatus* h_status = nullptr;
  std::vector<int64_t> tickets;
  uint64_t held = 0;
  bool busy = false;
};

}  // namespace
}  // namespace tmul

struct tm_server {
  std::mutex mu;
  uint64_t budget = 0, used = 0;
  std::vector<tmul::Slot> slots;
  std::deque<tmul::Request> queue;
  std::deque<tm_completion> done;
  int64_t next_ticket = 0;
  int in_flight = 0;
};

namespace tmul {
namespace {

#define TS_CHECK(x)                                    \
  do {                                                 \
    cudaError_t e_ = (x);                              \
    if (e_ != cudaSuccess) {                           \
      (void)cudaGetLastError();                        \
      return e_ == cudaErrorMemoryAllocation ? TM_ENOMEM : TM_ECUDA; \
    }                                                  \
  } while (0)

void free_slot(Slot& sl) {
  if (sl.s) cudaStreamSynchronize(sl.s);
  cudaFree(sl.ws.base);
  cudaFree(sl.d_items);
  cudaFree(sl.d_plans);
  cudaFree(sl.d_counter);
  cudaFree(sl.d_status);
  cudaFreeHost(sl.h_items);
  cudaFreeHost(sl.h_plans);
  cudaFreeHost(sl.h_status);
  if (sl.done) cudaEventDestroy(sl.done);
  if (sl.s) cudaStreamDestroy(sl.s);
}

int init_slot(Slot& sl) {
  TS_CHECK(cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking));
  TS_CHECK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
  TS_CHECK(cudaMalloc(&sl.d_items, kMicro * sizeof(SmallItem)));
  TS_CHECK(cudaMalloc(&sl.d_plans, kMicro * sizeof(SmallPlan)));
  TS_CHECK(cudaMalloc(&sl.d_counter, sizeof(int)));
  TS_CHECK(cudaMalloc(&sl.d_status, sizeof(DevStatus)));
  TS_CHECK(cudaMallocHost(&sl.h_items, kMicro * sizeof(SmallItem)));
  TS_CHECK(cudaMallocHost(&sl.h_plans, kMicro * sizeof(SmallPlan)));
  TS_CHECK(cudaMallocHost(&sl.h_status, sizeof(DevStatus)));
  sl.ws.status = sl.d_status;
  return TM_OK;
}

// Retires finished slots into S->done.
void retire(tm_server* S) {
  for (Slot& sl : S->slots) {
    if (!sl.busy) continue;
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    int status = TM_OK;
    if (q != cudaSuccess) {
      (void)cudaGetLastError();
      status = TM_ECUDA;
    } else if (sl.h_status->flags) {
      status = TM_EPRECISION;
    }
    for (int64_t t : sl.tickets) S->done.push_back(tm_completion{t, status, 0});
    S->in_flight -= int(sl.tickets.size());
    sl.tickets.clear();
    S->used -= sl.held;
    sl.held = 0;
    sl.busy = false;
  }
}

// Launches up to kMicro consecutive small requests from the queue head on sl.
int admit_small(tm_server* S, Slot& sl) {
  std::map<std::tuple<int, int, int64_t>, int> index;
  int count = 0, nplans = 0;
  size_t smem = 0;
  while (!S->queue.empty() && S->queue.front().small && count < kMicro) {
    Request r = S->queue.front();
    auto key = std::make_tuple(r.p.kind, r.p.b, r.p.N);
    auto it = index.find(key);
    if (it == index.end()) {
      std::shared_ptr<PlanEntry> pe;
      const int rc = get_tables(r.p, true, sl.s, &pe);
      if (rc) return rc;
      sl.h_plans[nplans] = small_plan_of(r.p, *pe);
      const FftPass& fp = pe->fft.pass[0];
      smem = std::max(smem, small_smem_bytes(r.p.N, pe->M, fp.tw4_len, fp.need_wL));
      it = index.emplace(key, nplans++).first;
    }
    sl.h_items[count++] = small_item_for(r.out, r.u, r.v, r.n, r.p, it->second);
    sl.tickets.push_back(r.ticket);
    S->queue.pop_front();
  }
  TS_CHECK(cudaMemcpyAsync(sl.d_items, sl.h_items, count * sizeof(SmallItem),
                           cudaMemcpyHostToDevice, sl.s));
  TS_CHECK(cudaMemcpyAsync(sl.d_plans, sl.h_plans, nplans * sizeof(SmallPlan),
                           cudaMemcpyHostToDevice, sl.s));
  TS_CHECK(cudaMemsetAsync(sl.d_counter, 0, sizeof(int), sl.s));
  TS_CHECK(cudaMemsetAsync(sl.d_status, 0, sizeof(DevStatus), sl.s));
  SmallArgs a{};
  a.items = sl.d_items;
  a.count = count;
  a.plans = sl.d_plans;
  a.counter = sl.d_counter;
  a.status = sl.d_status;
  launch_small(a, std::min(count, 152), smem, sl.s);
  TS_CHECK(cudaGetLastError());
  return count;
}

int admit_large(tm_server* S, Slot& sl, const Request& r) {
  const size_t need = workspace_bytes(r.p);
  if (sl.ws.size < need) {
    if (sl.ws.base) TS_CHECK(cudaFree(sl.ws.base));
    sl.ws.base = nullptr;
    sl.ws.size = 0;
    TS_CHECK(cudaMalloc(&sl.ws.base, need));
    sl.ws.size = need;
  }
  std::shared_ptr<PlanEntry> pe;
  int rc = get_tables(r.p, false, sl.s, &pe);
  if (rc) return rc;
  TS_CHECK(cudaMemsetAsync(sl.d_status, 0, sizeof(DevStatus), sl.s));
  rc = enqueue(r.kind, r.out, r.u, r.v, r.n, sl.s, r.p, *pe, sl.ws, nullptr, nullptr);
  if (rc) return rc;
  sl.tickets.push_back(r.ticket);
  sl.held = need;
  S->used += need;
  return 1;
}

// Admits queued requests into free slots.
int admit(tm_server* S) {
  for (Slot& sl : S->slots) {
    if (S->queue.empty()) break;
    if (sl.busy) continue;
    const Request& head = S->queue.front();
    int got;
    if (head.small) {
      got = admit_small(S, sl);
    } else {
      const size_t need = workspace_bytes(head.p);
      if (S->in_flight > 0 && S->used + need > S->budget) break;   // wait for memory
      Request r = head;
      S->queue.pop_front();
      got = admit_large(S, sl, r);
      if (got < 0) {
        S->done.push_back(tm_completion{r.ticket, got, 0});
        continue;
      }
    }
    if (got < 0) return got;
    TS_CHECK(cudaMemcpyAsync(sl.h_status, sl.d_status, sizeof(DevStatus),
                             cudaMemcpyDeviceToHost, sl.s));
    TS_CHECK(cudaEventRecord(sl.done, sl.s));
    sl.busy = true;
    S->in_flight += got;
  }
  return TM_OK;
}

}  // namespace
}  // namespace tmul

extern "C" {

int tm_server_create(tm_server** server, uint64_t budget_bytes, int slots) {
  if (!server || slots <= 0 || slots > 64) return TM_EINVAL;
  std::unique_ptr<tm_server> S(new tm_server());
  S->budget = budget_bytes;
  S->slots.resize(size_t(slots));
  tmul::ensure_kernel_attributes();
  for (tmul::Slot& sl : S->slots) {
    const int rc = tmul::init_slot(sl);
    if (rc) {
      for (tmul::Slot& x : S->slots) tmul::free_slot(x);
      return rc;
    }
  }
  *server = S.release();
  return TM_OK;
}

int64_t tm_server_submit(tm_server* S, int kind, uint64_t* out, const uint64_t* u,
                         const uint64_t* v, uint64_t n_bits) {
  if (!S || !out || !u || !v || n_bits == 0) return TM_EINVAL;
  if (kind != TM_FULL && kind != TM_LO && kind != TM_HI) return TM_EINVAL;
  if (n_bits > TM_MAX_BITS) return TM_ERANGE;
  tmul::Request r{};
  const int rc = tmul::get_params(kind, n_bits, &r.p);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(S->mu);
  r.ticket = S->next_ticket++;
  r.kind = kind;
  r.n = n_bits;
  r.out = out;
  r.u = u;
  r.v = v;
  r.small = r.p.N / 2 <= tmul::kSmallMaxM;
  S->queue.push_back(r);
  return r.ticket;
}

int tm_server_progress(tm_server* S, tm_completion* done, int max_done) {
  if (!S || (max_done > 0 && !done)) return TM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  tmul::retire(S);
  const int rc = tmul::admit(S);
  int k = 0;
  while (k < max_done && !S->done.empty()) {
    done[k++] = S->done.front();
    S->done.pop_front();
  }
  return rc < 0 ? rc : k;
}

int tm_server_pending(tm_server* S) {
  if (!S) return TM_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  return int(S->queue.size()) + S->in_flight + int(S->done.size());
}

int tm_server_destroy(tm_server* S) {
  if (!S) return TM_EINVAL;
  for (tmul::Slot& sl : S->slots) tmul::free_slot(sl);
  delete S;
  return TM_OK;
}

}  // extern "C"
