// Serving: continuous batching of C_D / torque queries over resident meshes.
//
// tpmc_submit queues a query; one scheduler thread per context repeatedly
//   1. admits queued queries into free slots while device memory allows
//      (panel buffers are charged to the context's budget),
//   2. gives every admitted query a share of the next launch's particle budget
//      (a query of at most that share finishes in one launch),
//   3. enqueues, per (mesh, precision) group, one persistent trace launch
//      over work items from all of the group's queries, then the FP64
//      reduction of the queries that finish, and
//   4. waits for the launch on the host (a CUDA event; no device-side wait),
//      publishes finished results and frees their slots.
// A query's particles keep their ids 0..N-1 whatever launches they land in,
// and its sums are exact integers, so its force and C_D do not depend on what
// else is in flight.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <vector>

#include "runtime.h"

namespace tpmc {

namespace {
using Clock = std::chrono::steady_clock;
constexpr uint32_t kSlots = 1024;
constexpr size_t kMaxQueue = 1u << 16;
constexpr uint64_t kLaunchParticles = 1ull << 23;  // particle budget of one scheduler step
constexpr uint64_t kMinShare = 1ull << 16;
}  // namespace

struct Request {
  tpmc_query_id id = 0;
  tpmc_mesh_id mesh = 0;
  uint32_t precision = 0;
  uint32_t n_tri = 0;
  bool want_panels = false;
  QueryDev q;                  // inputs (set-up runs on the device at admission)
  uint64_t N = 0, next_pid = 0;
  int slot = -1;
  bool done = false;
  tpmc_result result;
  void* d_panel = nullptr;
  Clock::time_point t_submit;
};

struct ServeState {
  Ctx* ctx = nullptr;
  std::thread th;
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::deque<Request*> queue;
  std::map<tpmc_query_id, Request*> all;
  std::vector<Request*> slots;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  // device
  QueryDev* d_q = nullptr;
  AccDev* d_acc = nullptr;
  ItemDev* d_items = nullptr;
  uint32_t* d_slots = nullptr;
  tpmc_result* d_res = nullptr;
  unsigned long long* d_counters = nullptr;
  int* d_err = nullptr;
  // pinned host
  ItemDev* h_items = nullptr;
  uint32_t* h_slots = nullptr;
  tpmc_result* h_res = nullptr;
  int* h_err = nullptr;
  void* d_block = nullptr;
  void* h_block = nullptr;
  uint64_t launches = 0;
};

namespace {

void loop(ServeState* s) {
  Ctx* c = s->ctx;
  cudaSetDevice(c->device);
  std::vector<Request*> fresh, active, finishing;
  for (;;) {
    fresh.clear();
    active.clear();
    finishing.clear();
    {
      std::unique_lock<std::mutex> lk(s->m);
      s->cv_work.wait(lk, [&] {
        if (s->stop) return true;
        if (!s->queue.empty()) return true;
        for (Request* r : s->slots) if (r) return true;
        return false;
      });
      if (s->stop) return;
      // 1. admission: a free slot and the panel memory
      while (!s->queue.empty()) {
        Request* r = s->queue.front();
        int slot = -1;
        for (uint32_t i = 0; i < kSlots; ++i) if (!s->slots[i]) { slot = (int)i; break; }
        if (slot < 0) break;
        if (r->want_panels && r->n_tri > 0) {
          std::lock_guard<std::recursive_mutex> ck(c->mu);
          if (c->alloc(&r->d_panel, (size_t)r->n_tri * 3 * sizeof(long long), "serving panel loads") != TPMC_OK) {
            bool any = false;
            for (Request* a : s->slots) any = any || a;
            if (any) break;  // wait for memory to free up
            r->done = true;  // cannot ever fit
            std::memset(&r->result, 0, sizeof(r->result));
            r->result.status = TPMC_ENOMEM;
            r->result.query_id = r->id;
            auto mit = c->meshes.find(r->mesh);
            if (mit != c->meshes.end()) --mit->second.in_use;
            s->queue.pop_front();
            s->cv_done.notify_all();
            continue;
          }
        }
        s->queue.pop_front();
        r->slot = slot;
        s->slots[slot] = r;
        fresh.push_back(r);
      }
      for (Request* r : s->slots) if (r) active.push_back(r);
    }
    if (active.empty()) continue;
    cudaError_t e = cudaSuccess;
    // 2. set-up of newly admitted queries, straight into their slots
    for (size_t i = 0; i < fresh.size() && e == cudaSuccess; ++i) {
      Request* r = fresh[i];
      r->q.panel = (long long*)r->d_panel;
      s->h_slots[i] = (uint32_t)r->slot;
      e = cudaMemcpyAsync(s->d_q + r->slot, &r->q, sizeof(QueryDev), cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s->d_acc + r->slot, 0, sizeof(AccDev), s->stream);
      if (e == cudaSuccess && r->d_panel)
        e = cudaMemsetAsync(r->d_panel, 0, (size_t)r->n_tri * 3 * sizeof(long long), s->stream);
    }
    if (!fresh.empty() && e == cudaSuccess) {
      e = cudaMemcpyAsync(s->d_slots, s->h_slots, fresh.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess)
        e = launch_setup(s->d_q, (uint32_t)fresh.size(), nullptr, nullptr, nullptr, nullptr, s->d_slots, s->stream);
    }
    // 3. shares of this step, grouped by (mesh, precision)
    const uint64_t share = std::max<uint64_t>(kMinShare, kLaunchParticles / active.size());
    std::map<std::pair<tpmc_mesh_id, uint32_t>, std::vector<Request*>> groups;
    for (Request* r : active) groups[{r->mesh, r->precision}].push_back(r);
    uint32_t n_items = 0, group_idx = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_counters, 0, 64 * sizeof(unsigned long long), s->stream);
    for (auto& kv : groups) {
      if (group_idx == 64) break;  // one counter per launch; later groups wait for the next step
      const uint32_t first_item = n_items;
      uint64_t g = 0;
      for (Request* r : kv.second) {
        const uint64_t take = std::min<uint64_t>(r->N - r->next_pid, share);
        if (take == 0) continue;
        ItemDev& it = s->h_items[n_items++];
        it.g_begin = g;
        it.pid_begin = r->next_pid;
        it.count = take;
        it.query = (uint32_t)r->slot;
        it.pad = 0;
        g += take;
        r->next_pid += take;
        if (r->next_pid == r->N) finishing.push_back(r);
      }
      if (n_items == first_item || e != cudaSuccess) continue;
      MeshDev md;
      LaunchCfg cfg;
      {
        std::lock_guard<std::recursive_mutex> ck(c->mu);
        const MeshRec& mr = c->meshes.at(kv.first.first);
        md = mr.dev;
        cfg = c->schedule(mr, kv.first.second, g);
      }
      e = cudaMemcpyAsync(s->d_items + first_item, s->h_items + first_item, (n_items - first_item) * sizeof(ItemDev),
                          cudaMemcpyHostToDevice, s->stream);
      TraceArgs a{};
      a.mesh = md;
      a.queries = s->d_q;
      a.acc = s->d_acc;
      a.items = s->d_items + first_item;
      a.n_items = n_items - first_item;
      a.total = g;
      a.counter = s->d_counters + (group_idx++ % 64);
      a.error = s->d_err;
      a.count_work = c->counters ? 1u : 0u;
      a.vn_table = c->vn_table;
      a.chunk = cfg.chunk;
      a.smem_nodes = cfg.smem_nodes;
      if (e == cudaSuccess) e = launch_trace(a, kv.first.second, cfg, c->num_sms, s->stream);
    }
    // 4. reduction of finishing queries, read-back, host-side wait
    for (size_t i = 0; i < finishing.size(); ++i) s->h_slots[kSlots + i] = (uint32_t)finishing[i]->slot;
    if (!finishing.empty() && e == cudaSuccess) {
      e = cudaMemcpyAsync(s->d_slots + kSlots, s->h_slots + kSlots, finishing.size() * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess)
        e = launch_finalize(s->d_q, s->d_acc, (uint32_t)finishing.size(), s->d_slots + kSlots, s->d_res, s->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->h_res, s->d_res, finishing.size() * sizeof(tpmc_result), cudaMemcpyDeviceToHost,
                            s->stream);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->ev, s->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(s->ev);
    ++s->launches;
    const Clock::time_point now = Clock::now();
    {
      std::unique_lock<std::mutex> lk(s->m);
      if (e != cudaSuccess || *s->h_err != 0) {
        // a failed step fails every query that was in it
        for (Request* r : active) {
          r->done = true;
          std::memset(&r->result, 0, sizeof(r->result));
          r->result.status = TPMC_ECUDA;
          r->result.query_id = r->id;
          s->slots[r->slot] = nullptr;
        }
        *s->h_err = 0;
        cudaGetLastError();
      } else {
        for (size_t i = 0; i < finishing.size(); ++i) {
          Request* r = finishing[i];
          r->result = s->h_res[i];
          r->result.query_id = r->id;
          r->result.ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
          r->done = true;
          s->slots[r->slot] = nullptr;
        }
      }
      std::lock_guard<std::recursive_mutex> ck(c->mu);
      for (Request* r : active) {
        if (!r->done) continue;
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
      s->cv_done.notify_all();
    }
  }
}

tpmc_status start_serving(Ctx* c) {
  ServeState* s = new ServeState();
  s->ctx = c;
  s->slots.assign(kSlots, nullptr);
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev, cudaEventBlockingSync | cudaEventDisableTiming);
  if (e != cudaSuccess) { delete s; return cuda_fail(e, "serving stream"); }
  const size_t dev_bytes = kSlots * (sizeof(QueryDev) + sizeof(AccDev) + 2 * sizeof(ItemDev) + 2 * sizeof(uint32_t) +
                                     sizeof(tpmc_result)) + 64 * sizeof(unsigned long long) + 256;
  tpmc_status st = c->alloc(&s->d_block, dev_bytes, "serving slots");
  if (st != TPMC_OK) { cudaStreamDestroy(s->stream); cudaEventDestroy(s->ev); delete s; return st; }
  char* p = (char*)s->d_block;
  s->d_q = (QueryDev*)p; p += kSlots * sizeof(QueryDev);
  s->d_acc = (AccDev*)p; p += kSlots * sizeof(AccDev);
  s->d_items = (ItemDev*)p; p += 2 * kSlots * sizeof(ItemDev);
  s->d_res = (tpmc_result*)p; p += kSlots * sizeof(tpmc_result);
  s->d_counters = (unsigned long long*)p; p += 64 * sizeof(unsigned long long);
  s->d_slots = (uint32_t*)p; p += 2 * kSlots * sizeof(uint32_t);
  s->d_err = (int*)p;
  cudaMemset(s->d_err, 0, sizeof(int));
  const size_t host_bytes = 2 * kSlots * sizeof(ItemDev) + 2 * kSlots * sizeof(uint32_t) + kSlots * sizeof(tpmc_result) + 64;
  if ((e = cudaMallocHost(&s->h_block, host_bytes)) != cudaSuccess) {
    c->release(s->d_block);
    cudaStreamDestroy(s->stream);
    cudaEventDestroy(s->ev);
    delete s;
    return cuda_fail(e, "serving host buffers");
  }
  char* h = (char*)s->h_block;
  s->h_items = (ItemDev*)h; h += 2 * kSlots * sizeof(ItemDev);
  s->h_slots = (uint32_t*)h; h += 2 * kSlots * sizeof(uint32_t);
  s->h_res = (tpmc_result*)h; h += kSlots * sizeof(tpmc_result);
  s->h_err = (int*)h;
  *s->h_err = 0;
  c->serve = s;
  s->th = std::thread(loop, s);
  return TPMC_OK;
}

}  // namespace

void stop_serving(Ctx* c) {
  ServeState* s = c->serve;
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->m);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaStreamSynchronize(s->stream);
  for (auto& kv : s->all) {
    if (kv.second->d_panel) c->release(kv.second->d_panel);
    delete kv.second;
  }
  c->release(s->d_block);
  cudaFreeHost(s->h_block);
  cudaEventDestroy(s->ev);
  cudaStreamDestroy(s->stream);
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
    if (!c->serve && (st = start_serving(c)) != TPMC_OK) return st;
    ++it->second.in_use;
    r->id = c->next_query++;
  }
  r->mesh = mesh;
  r->precision = params->precision;
  r->want_panels = params->want_panels != 0;
  r->N = N;
  r->t_submit = Clock::now();
  ServeState* s = c->serve;
  {
    std::lock_guard<std::mutex> lk(s->m);
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
