// Serving: continuous batching of C_D / torque queries over resident meshes.
//
// tpmc_submit queues a query; one scheduler thread per context repeatedly
//   1. admits queued queries into free slots while device memory allows
//      (panel buffers are charged to the context's budget); a query whose
//      panel buffer does not fit yet waits without holding back the queries
//      behind it,
//   2. builds a step: the admitted query with the least work left, less the
//      time it has waited (aging), runs whole (once started a query is not
//      split, so nothing overtakes it midway), and queries behind it join the
//      step while together they stay tiny,
//   3. enqueues the step -- set-up of newly admitted queries, one persistent
//      trace launch per (mesh, kernel variant) group over work items from all of
//      the group's queries, the FP64 reduction of the queries that finish,
//      the read-back -- while the previous step may still run.  Each of the
//      two step buffers has its own streams, so a step's trace launches start
//      on the SMs that the previous step's launch tails free up; the
//      reduction waits for the traces of both steps, since a finishing query
//      may have had work in the previous one, and
//   4. waits for the older step on the host (a CUDA event; no device-side
//      wait), publishes its finished results and frees their slots.
// A query's particles keep their ids 0..N-1 whatever steps they land in, and
// its sums are exact integers, so its force and C_D do not depend on what else
// is in flight.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <thread>
#include <vector>

#include "runtime.h"

namespace tpmc {

namespace {
using Clock = std::chrono::steady_clock;
constexpr uint32_t kSlots = 1024;
constexpr size_t kMaxQueue = 1u << 16;
static_assert(kMaxQueue <= kMaxLaunchQueries, "a step's query slots must fit the queue word");
constexpr uint64_t kTinyBatch = 1ull << 22;  // queries behind the head share its step up to this many particles
constexpr double kNominalParticlesPerMs = 4e6;  // work-to-time scale of the queue order (about the GPU's rate)
// Weight of the time waited against the work left.  Measured with 1,000
// Poisson queries at 100 to 800 per second against one query per launch: 0.5,
// 1 and 2 give p50 and p99 within 1-2 ms of one another (0.5 the lowest); no
// aging starves large queries under overload (p99 1.4 s against 0.8 s at 400/s).
constexpr double kAging = 0.5;
// Arrival order for queues of up to 3 or 5 waiting queries measured worse at
// 100/s (p99 29.5-30 ms against 25.3): small queries then wait behind large
// ones, and those waits make the tail.
constexpr int kInFlight = 2;                     // steps enqueued ahead of the host
constexpr int kMaxGroups = 64;                   // trace launches per step
constexpr int kGroupStreams = 4;                 // streams the groups of a step run on
}  // namespace

struct Request {
  tpmc_query_id id = 0;
  tpmc_mesh_id mesh = 0;
  uint32_t variant = 0;     // trace-kernel variant (precision and surface model)
  uint32_t n_tri = 0;
  bool want_panels = false;
  QueryDev q;                  // inputs (set-up runs on the device at admission)
  uint64_t N = 0, next_pid = 0;
  int slot = -1;
  bool set_up = false;         // set-up enqueued
  bool done = false;
  tpmc_result result;
  void* d_panel = nullptr;
  Clock::time_point t_submit;
};

// Buffers of one step in flight.
struct StepBuf {
  ItemDev* h_items = nullptr;
  uint32_t* h_fresh = nullptr;
  uint32_t* h_fin = nullptr;
  tpmc_result* h_res = nullptr;
  int* h_err = nullptr;
  ItemDev* d_items = nullptr;
  uint32_t* d_fresh = nullptr;
  uint32_t* d_fin = nullptr;
  tpmc_result* d_res = nullptr;
  unsigned long long* d_counters = nullptr;
  int* d_err = nullptr;
  cudaEvent_t ev = nullptr;
  cudaStream_t st = nullptr;                     // set-up, reduction, read-back
  cudaStream_t group_stream[kGroupStreams] = {};  // trace launches
  cudaEvent_t group_done[kGroupStreams] = {};
  cudaEvent_t ready = nullptr;                   // set-up done
  cudaEvent_t traces_done = nullptr;             // every trace launch of the step done
  std::vector<Request*> members, finishing;
};

struct ServeState {
  Ctx* ctx = nullptr;
  std::thread th;
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  bool mem_wait = false;       // queued queries wait for device memory to be released
  std::deque<Request*> queue;
  std::map<tpmc_query_id, Request*> all;
  std::vector<Request*> slots;
  QueryDev* d_q = nullptr;
  AccStripe* d_acc = nullptr;  // stripe-major, kSlots query slots per stripe
  StepBuf buf[kInFlight];
  std::deque<int> inflight;    // buffer indices, oldest first
  void* d_block = nullptr;
  void* h_block = nullptr;
  uint64_t steps = 0;
};

namespace {

// Admits queued requests into free slots (caller holds s->m), in arrival
// order.  A request whose panel buffer does not fit now stays queued while
// memory may still be released (queries in flight, or panel loads not yet
// read by tpmc_panels), and the requests behind it are admitted meanwhile; it
// fails with ENOMEM only when nothing can free memory.
void admit(ServeState* s) {
  Ctx* c = s->ctx;
  s->mem_wait = false;
  for (auto qit = s->queue.begin(); qit != s->queue.end();) {
    Request* r = *qit;
    int slot = -1;
    for (uint32_t i = 0; i < kSlots; ++i) if (!s->slots[i]) { slot = (int)i; break; }
    if (slot < 0) return;
    if (r->want_panels && r->n_tri > 0) {
      std::lock_guard<std::recursive_mutex> ck(c->mu);
      if (c->alloc(&r->d_panel, (size_t)r->n_tri * 3 * sizeof(long long), "serving panel loads") != TPMC_OK) {
        bool may_free = !s->inflight.empty() || !c->panels.empty();
        for (Request* a : s->slots) may_free = may_free || a;
        if (may_free) {  // wait for memory; later queries may still fit
          s->mem_wait = true;
          ++qit;
          continue;
        }
        r->done = true;  // cannot ever fit
        std::memset(&r->result, 0, sizeof(r->result));
        r->result.status = TPMC_ENOMEM;
        r->result.query_id = r->id;
        auto mit = c->meshes.find(r->mesh);
        if (mit != c->meshes.end()) --mit->second.in_use;
        qit = s->queue.erase(qit);
        s->cv_done.notify_all();
        continue;
      }
    }
    qit = s->queue.erase(qit);
    r->slot = slot;
    s->slots[slot] = r;
  }
}

// Builds and enqueues one step in buffer b (caller does not hold s->m).
// Returns false when there was nothing to run.
bool enqueue_step(ServeState* s, int b, int prev, const std::vector<Request*>& cand, cudaError_t& e) {
  Ctx* c = s->ctx;
  StepBuf& B = s->buf[b];
  B.members.clear();
  B.finishing.clear();
  // Shortest remaining work first, aged: a query's key is its remaining work
  // in GPU time (at a nominal rate) minus kAging times the time it has
  // waited, so small queries overtake young large ones, and a large query that
  // has waited long enough goes before any newcomer (no starvation under
  // overload).  The head query runs whole (once started a query is not split,
  // so nothing overtakes it midway), and the queries behind it join its step
  // while all of them together stay tiny.
  const Clock::time_point now = Clock::now();
  auto key = [&](const Request* r) {
    const double waited_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
    return (double)(r->N - r->next_pid) / kNominalParticlesPerMs - kAging * waited_ms;
  };
  std::vector<Request*> order(cand);
  std::sort(order.begin(), order.end(), [&](const Request* x, const Request* y) {
    const double kx = key(x), ky = key(y);
    return kx != ky ? kx < ky : x->id < y->id;
  });
  std::map<Request*, uint64_t> take;
  uint64_t cum = 0;
  for (Request* r : order) {
    const uint64_t rem = r->N - r->next_pid;
    if (!take.empty() && cum + rem > kTinyBatch) break;
    take[r] = rem;
    cum += rem;
  }
  // groups by (mesh, kernel variant) in the order of `order`
  std::vector<std::pair<std::pair<tpmc_mesh_id, uint32_t>, std::vector<Request*>>> groups;
  for (Request* r : order) {
    if (take[r] == 0) continue;
    const auto key = std::make_pair(r->mesh, r->variant);
    auto it = std::find_if(groups.begin(), groups.end(), [&](const auto& g) { return g.first == key; });
    if (it == groups.end()) {
      if ((int)groups.size() == kMaxGroups) continue;  // later groups wait for the next step
      groups.push_back({key, {}});
      it = groups.end() - 1;
    }
    it->second.push_back(r);
  }
  if (groups.empty()) return false;
  cudaStream_t st = B.st;
  // set-up of newly admitted queries, straight into their slots
  uint32_t n_fresh = 0;
  for (auto& g : groups)
    for (Request* r : g.second) {
      if (r->set_up) continue;
      r->q.panel = (long long*)r->d_panel;
      B.h_fresh[n_fresh++] = (uint32_t)r->slot;
      if (e == cudaSuccess) e = cudaMemcpyAsync(s->d_q + r->slot, &r->q, sizeof(QueryDev), cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess && r->d_panel)
        e = cudaMemsetAsync(r->d_panel, 0, (size_t)r->n_tri * 3 * sizeof(long long), st);
      r->set_up = true;
    }
  if (n_fresh > 0 && e == cudaSuccess) {
    e = cudaMemcpyAsync(B.d_fresh, B.h_fresh, n_fresh * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    // the set-up also clears the fresh slots' accumulators
    if (e == cudaSuccess)
      e = launch_setup(s->d_q, n_fresh, nullptr, nullptr, nullptr, nullptr, B.d_fresh, s->d_acc, kSlots, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(B.d_counters, 0, kMaxGroups * sizeof(unsigned long long), st);
  // the groups run on their own streams once the set-up is done, so that one
  // launch's tail overlaps the next launch's start
  if (e == cudaSuccess) e = cudaEventRecord(B.ready, st);
  bool used[kGroupStreams] = {};
  uint32_t n_items = 0;
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const uint32_t first_item = n_items;
    uint64_t g = 0;
    for (Request* r : groups[gi].second) {
      ItemDev& it = B.h_items[n_items++];
      it.g_begin = g;
      it.pid_begin = r->next_pid;
      it.count = take[r];
      it.query = (uint32_t)r->slot;
      it.pad = 0;
      g += take[r];
      r->next_pid += take[r];
      B.members.push_back(r);
      if (r->next_pid == r->N) B.finishing.push_back(r);
    }
    MeshDev md;
    LaunchCfg cfg;
    {
      std::lock_guard<std::recursive_mutex> ck(c->mu);
      const MeshRec& mr = c->meshes.at(groups[gi].first.first);
      md = mr.dev;
      cfg = c->schedule(mr, groups[gi].first.second, g);
    }
    const int gs = (int)(gi % kGroupStreams);
    cudaStream_t gst = B.group_stream[gs];
    if (!used[gs] && e == cudaSuccess) e = cudaStreamWaitEvent(gst, B.ready, 0);
    used[gs] = true;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(B.d_items + first_item, B.h_items + first_item, (n_items - first_item) * sizeof(ItemDev),
                          cudaMemcpyHostToDevice, gst);
    TraceArgs a{};
    a.mesh = md;
    a.queries = s->d_q;
    a.acc = s->d_acc;
    a.acc_stride = kSlots;
    a.items = B.d_items + first_item;
    a.n_items = n_items - first_item;
    a.total = g;
    a.counter = B.d_counters + gi;
    a.error = B.d_err;
    a.count_work = c->counters ? 1u : 0u;
    a.vn_table = c->vn_table;
    a.chunk = cfg.chunk;
    a.smem_nodes = cfg.smem_nodes;
    a.refill_at = cfg.refill_at;
    if (e == cudaSuccess) e = launch_trace(a, groups[gi].first.second, cfg, c->num_sms, gst);
  }
  for (int gs = 0; gs < kGroupStreams && e == cudaSuccess; ++gs) {
    if (!used[gs]) continue;
    e = cudaEventRecord(B.group_done[gs], B.group_stream[gs]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, B.group_done[gs], 0);
  }
  if (e == cudaSuccess) e = cudaEventRecord(B.traces_done, st);
  // the reduction also waits for the previous step's traces (still in flight)
  if (prev >= 0 && e == cudaSuccess) e = cudaStreamWaitEvent(st, s->buf[prev].traces_done, 0);
  for (size_t i = 0; i < B.finishing.size(); ++i) B.h_fin[i] = (uint32_t)B.finishing[i]->slot;
  if (!B.finishing.empty() && e == cudaSuccess) {
    e = cudaMemcpyAsync(B.d_fin, B.h_fin, B.finishing.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = launch_finalize(s->d_q, s->d_acc, kSlots, (uint32_t)B.finishing.size(), B.d_fin, B.d_res, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(B.h_res, B.d_res, B.finishing.size() * sizeof(tpmc_result), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(B.h_err, B.d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(B.ev, st);
  return true;
}

// Waits for the oldest step and publishes its results (caller does not hold s->m).
void retire_step(ServeState* s, cudaError_t e_enqueue) {
  Ctx* c = s->ctx;
  const int b = s->inflight.front();
  StepBuf& B = s->buf[b];
  cudaError_t e = e_enqueue;
  // Poll rather than sleep on the event: a blocking wait wakes through an
  // interrupt, tens of microseconds after the step ends, and that delay lands
  // on every query's latency.  The loop thread has a core to itself.
  if (e == cudaSuccess) {
    while ((e = cudaEventQuery(B.ev)) == cudaErrorNotReady) std::this_thread::yield();
  }
  ++s->steps;
  const Clock::time_point now = Clock::now();
  std::unique_lock<std::mutex> lk(s->m);
  s->inflight.pop_front();
  std::vector<Request*> done;
  if (e != cudaSuccess || *B.h_err != 0) {
    // a failed step fails every query that had work in it
    for (Request* r : B.members) {
      if (r->done) continue;
      r->done = true;
      std::memset(&r->result, 0, sizeof(r->result));
      r->result.status = TPMC_ECUDA;
      r->result.query_id = r->id;
      done.push_back(r);
    }
    *B.h_err = 0;
    cudaGetLastError();
  } else {
    for (size_t i = 0; i < B.finishing.size(); ++i) {
      Request* r = B.finishing[i];
      r->result = B.h_res[i];
      r->result.query_id = r->id;
      r->result.ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
      r->done = true;
      done.push_back(r);
    }
  }
  std::lock_guard<std::recursive_mutex> ck(c->mu);
  for (Request* r : done) {
    if (r->slot >= 0 && s->slots[r->slot] == r) s->slots[r->slot] = nullptr;
    auto mit = c->meshes.find(r->mesh);
    if (mit != c->meshes.end()) --mit->second.in_use;
    if (r->d_panel && r->result.status == TPMC_OK) {
      PanelRec pr;
      pr.d_panel = r->d_panel;
      pr.query = r->q;
      pr.query.gamma = r->result.gamma;
      pr.query.c_mp = r->result.c_mp;
      pr.query.quantum = r->result.fixed_quantum;
      pr.mesh = r->mesh;
      pr.n_tri = r->n_tri;
      c->panels[r->id] = pr;
      r->d_panel = nullptr;
    } else if (r->d_panel) {
      c->release(r->d_panel);
      r->d_panel = nullptr;
    }
  }
  s->mem_wait = false;  // slots and maybe memory were freed: admission may proceed
  s->cv_done.notify_all();
}

void loop(ServeState* s) {
  cudaSetDevice(s->ctx->device);
  std::vector<Request*> cand;
  for (;;) {
    int free_buf = -1;
    {
      std::unique_lock<std::mutex> lk(s->m);
      auto has_work = [&] {
        for (Request* r : s->slots)
          if (r && !r->done && r->next_pid < r->N) return true;
        return false;
      };
      s->cv_work.wait(lk, [&] {
        return s->stop || !s->inflight.empty() || (!s->queue.empty() && !s->mem_wait) || has_work();
      });
      if (s->stop) break;
      admit(s);
      cand.clear();
      for (Request* r : s->slots)
        if (r && !r->done && r->next_pid < r->N) cand.push_back(r);
      if ((int)s->inflight.size() < kInFlight && !cand.empty()) {
        for (int b = 0; b < kInFlight; ++b)
          if (std::find(s->inflight.begin(), s->inflight.end(), b) == s->inflight.end()) { free_buf = b; break; }
      }
    }
    cudaError_t e = cudaSuccess;
    if (free_buf >= 0) {
      // inflight is changed only by this thread, so it can be read here unlocked
      const int prev = s->inflight.empty() ? -1 : s->inflight.back();
      const bool pushed = enqueue_step(s, free_buf, prev, cand, e);
      if (pushed) {
        std::lock_guard<std::mutex> lk(s->m);
        s->inflight.push_back(free_buf);
      }
      if (pushed && e == cudaSuccess) continue;  // keep the next step ready while this one runs
    }
    bool any;
    {
      std::lock_guard<std::mutex> lk(s->m);
      any = !s->inflight.empty();
    }
    if (any) retire_step(s, e);
  }
  while (!s->inflight.empty()) retire_step(s, cudaSuccess);
}

// Waits for and destroys the streams and events of the step buffers (null ones are skipped).
void destroy_streams(ServeState* s) {
  for (int b = 0; b < kInFlight; ++b) {
    StepBuf& B = s->buf[b];
    for (int g = 0; g < kGroupStreams; ++g) {
      if (B.group_stream[g]) { cudaStreamSynchronize(B.group_stream[g]); cudaStreamDestroy(B.group_stream[g]); }
      if (B.group_done[g]) cudaEventDestroy(B.group_done[g]);
    }
    if (B.st) { cudaStreamSynchronize(B.st); cudaStreamDestroy(B.st); }
    if (B.ev) cudaEventDestroy(B.ev);
    if (B.ready) cudaEventDestroy(B.ready);
    if (B.traces_done) cudaEventDestroy(B.traces_done);
  }
}

tpmc_status start_serving(Ctx* c) {
  ServeState* s = new ServeState();
  s->ctx = c;
  s->slots.assign(kSlots, nullptr);
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < kInFlight && e == cudaSuccess; ++b) {
    StepBuf& B = s->buf[b];
    e = cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B.ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B.traces_done, cudaEventDisableTiming);
    for (int g = 0; g < kGroupStreams && e == cudaSuccess; ++g) {
      e = cudaStreamCreateWithFlags(&B.group_stream[g], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B.group_done[g], cudaEventDisableTiming);
    }
  }
  if (e != cudaSuccess) {
    destroy_streams(s);
    delete s;
    return cuda_fail(e, "serving stream");
  }
  const size_t per_buf_dev = kSlots * (sizeof(ItemDev) + 2 * sizeof(uint32_t) + sizeof(tpmc_result)) +
                             kMaxGroups * sizeof(unsigned long long) + 256;
  const size_t dev_bytes = kSlots * (sizeof(QueryDev) + kAccStripes * sizeof(AccStripe)) + kInFlight * per_buf_dev + 256;
  tpmc_status st = c->alloc(&s->d_block, dev_bytes, "serving slots");
  if (st != TPMC_OK) {
    destroy_streams(s);
    delete s;
    return st;
  }
  char* p = (char*)s->d_block;
  // the accumulators first: cudaMalloc's alignment keeps each stripe on its own line
  s->d_acc = (AccStripe*)p; p += kSlots * kAccStripes * sizeof(AccStripe);
  s->d_q = (QueryDev*)p; p += kSlots * sizeof(QueryDev);
  const size_t per_buf_host = kSlots * (sizeof(ItemDev) + 2 * sizeof(uint32_t) + sizeof(tpmc_result)) + 64;
  if ((e = cudaMallocHost(&s->h_block, kInFlight * per_buf_host)) != cudaSuccess) {
    c->release(s->d_block);
    destroy_streams(s);
    delete s;
    return cuda_fail(e, "serving host buffers");
  }
  char* h = (char*)s->h_block;
  for (int b = 0; b < kInFlight; ++b) {
    StepBuf& B = s->buf[b];
    B.d_items = (ItemDev*)p; p += kSlots * sizeof(ItemDev);
    B.d_res = (tpmc_result*)p; p += kSlots * sizeof(tpmc_result);
    B.d_counters = (unsigned long long*)p; p += kMaxGroups * sizeof(unsigned long long);
    B.d_fresh = (uint32_t*)p; p += kSlots * sizeof(uint32_t);
    B.d_fin = (uint32_t*)p; p += kSlots * sizeof(uint32_t);
    B.d_err = (int*)p; p += 256;
    B.h_items = (ItemDev*)h; h += kSlots * sizeof(ItemDev);
    B.h_res = (tpmc_result*)h; h += kSlots * sizeof(tpmc_result);
    B.h_fresh = (uint32_t*)h; h += kSlots * sizeof(uint32_t);
    B.h_fin = (uint32_t*)h; h += kSlots * sizeof(uint32_t);
    B.h_err = (int*)h; h += 64;
    *B.h_err = 0;
    cudaMemset(B.d_err, 0, sizeof(int));
  }
  c->serve = s;
  s->th = std::thread(loop, s);
  return TPMC_OK;
}

}  // namespace

void serve_memory_released(Ctx* c) {
  ServeState* s = c->serve;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->mem_wait = false;
  }
  s->cv_work.notify_all();
}

void stop_serving(Ctx* c) {
  ServeState* s = c->serve;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  destroy_streams(s);
  for (auto& kv : s->all) {
    if (kv.second->d_panel) c->release(kv.second->d_panel);
    delete kv.second;
  }
  c->release(s->d_block);
  cudaFreeHost(s->h_block);
  delete s;
  c->serve = nullptr;
}

}  // namespace tpmc

using namespace tpmc;

extern "C" {

tpmc_status tpmc_submit(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* params, uint64_t N,
                        tpmc_query_id* out) {
  if (!ctx || !out) return fail(TPMC_EINVAL, "NULL argument");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  tpmc_status st = validate_params(params);
  if (st != TPMC_OK) return st;
  if (N == 0 || N > (1ull << 34)) return fail(TPMC_EINVAL, "N must be in [1, 2^34]");
  std::unique_ptr<Request> r(new Request());
  {
    std::lock_guard<std::recursive_mutex> ck(c->mu);
    cudaSetDevice(c->device);
    auto it = c->meshes.find(mesh);
    if (it == c->meshes.end()) return fail(TPMC_ENOTFOUND, "unknown mesh id");
    if ((st = fill_query(it->second, params, N, &r->q)) != TPMC_OK) return st;
    r->n_tri = it->second.dev.n_tri;
    r->variant = trace_variant(params, it->second.dev);
    if (!c->serve && (st = start_serving(c)) != TPMC_OK) return st;
    ++it->second.in_use;
    r->id = c->next_query++;
  }
  r->mesh = mesh;
  r->want_panels = params->want_panels != 0;
  r->N = N;
  r->t_submit = Clock::now();
  ServeState* s = c->serve;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->mem_wait = false;  // the new query may fit
    if (s->queue.size() >= kMaxQueue) {
      std::lock_guard<std::recursive_mutex> ck(c->mu);
      --c->meshes.at(mesh).in_use;
      return fail(TPMC_EBUSY, "serving queue is full");
    }
    *out = r->id;
    s->all[r->id] = r.get();
    s->queue.push_back(r.release());
  }
  s->cv_work.notify_all();
  return TPMC_OK;
}

tpmc_status tpmc_poll(tpmc_ctx* ctx, tpmc_query_id query, int timeout_ms, tpmc_result* out) {
  if (!ctx || !out) return fail(TPMC_EINVAL, "NULL argument");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  ServeState* s = c->serve;
  if (!s) return fail(TPMC_ENOTFOUND, "no query was submitted");
  std::unique_lock<std::mutex> lk(s->m);
  auto it = s->all.find(query);
  if (it == s->all.end()) return fail(TPMC_ENOTFOUND, "unknown query id");
  Request* r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) s->cv_done.wait(lk, ready);
  else if (timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  if (!r->done) return fail(TPMC_ETIMEOUT, "query not finished");
  *out = r->result;
  const tpmc_status st = (tpmc_status)r->result.status;
  s->all.erase(it);
  delete r;
  if (st != TPMC_OK) return fail(st, "query failed");
  return TPMC_OK;
}

}  // extern "C"
