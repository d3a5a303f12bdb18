// tpmc_sweep_noalloc: the batched sweep for callers that may not allocate
// device memory once they are running.
//
// Who needs it: code on a real-time or flight-software loop where allocation
// after start-up is forbidden (cudaMalloc can block, fragment memory or fail
// at an arbitrary point), code embedded in a framework that owns all device
// memory through its own pool and does not let a library call cudaMalloc, and
// code that must keep the memory footprint fixed after initialisation.  Such a
// caller creates the context and loads its meshes at start-up (those calls do
// allocate) and then calls this entry point in the loop.
//
// The per-call scratch of the sweep (query table, accumulators, work items,
// inputs staged for the device, results, work counter, error word) lives in
// one file-scope device array of fixed size, so the call itself performs no
// allocation.  Every GPU that loads this library holds the array until the
// process exits.  All calls on a device share it: each call clears what must
// start at zero, and two calls that overlap on the GPU (different streams or
// threads of different contexts on one device) race on it.
#include <chrono>
#include <mutex>

#include "runtime.h"

namespace tpmc {
namespace {

constexpr uint32_t kNoAllocMaxQueries = 64;

struct NoAllocArea {
  QueryDev base;
  QueryDev queries[kNoAllocMaxQueries];
  AccStripe acc[kAccStripes * kNoAllocMaxQueries];  // stripe-major, kNoAllocMaxQueries slots per stripe
  ItemDev items[kNoAllocMaxQueries];
  double dirs[3 * kNoAllocMaxQueries];
  double S[kNoAllocMaxQueries];
  tpmc_result results[kNoAllocMaxQueries];
  unsigned long long counter;
  int error;
  int pad;
};

// Fixed scratch of tpmc_sweep_noalloc (about 100 KB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocArea)];

constexpr int kMaxDevices = 64;
std::mutex g_area_mu;
NoAllocArea* g_area[kMaxDevices] = {};

// Device address of the scratch array on `device` (which must be current).
// In host code the array's name is only a host-side stand-in, so its device
// address is looked up once per device and kept.
cudaError_t area_on_device(int device, NoAllocArea** out) {
  std::lock_guard<std::mutex> lk(g_area_mu);
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  if (g_area[device] == nullptr) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_area[device] = static_cast<NoAllocArea*>(ptr);
  }
  *out = g_area[device];
  return cudaSuccess;
}

}  // namespace
}  // namespace tpmc

using namespace tpmc;

extern "C" tpmc_status tpmc_sweep_noalloc(tpmc_ctx* ctx, tpmc_mesh_id mesh, const tpmc_params* base,
                                          const double* h_dirs, const double* h_S, uint32_t K, uint64_t N_each,
                                          tpmc_result* h_out) {
  if (!ctx || !h_out) return fail(TPMC_EINVAL, "NULL argument");
  if (K == 0 || K > kNoAllocMaxQueries)
    return fail(TPMC_EINVAL, "tpmc_sweep_noalloc: K must be in [1, 64], the capacity of its fixed scratch");
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  std::lock_guard<std::recursive_mutex> lk(c->mu);
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  tpmc_status st = validate_params(base);
  if (st != TPMC_OK) return st;
  if (N_each == 0 || N_each > (1ull << 34)) return fail(TPMC_EINVAL, "N_each must be in [1, 2^34]");
  auto it = c->meshes.find(mesh);
  if (it == c->meshes.end()) return fail(TPMC_ENOTFOUND, "unknown mesh id");
  const MeshRec& m = it->second;
  QueryDev q;
  if ((st = fill_query(m, base, N_each, &q)) != TPMC_OK) return st;
  q.panel = nullptr;  // per-panel loads need memory sized by the mesh: not kept here
  NoAllocArea* A = nullptr;
  if ((e = area_on_device(c->device, &A)) != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
  cudaStream_t s = c->stream;
  // inputs (host sources are pageable, so each copy is staged before the call returns)
  e = cudaMemcpyAsync(&A->base, &q, sizeof(QueryDev), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && h_dirs)
    e = cudaMemcpyAsync(A->dirs, h_dirs, (size_t)K * 3 * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && h_S) e = cudaMemcpyAsync(A->S, h_S, (size_t)K * sizeof(double), cudaMemcpyHostToDevice, s);
  // the array keeps the previous call's contents: clear the work counter and the error word (the
  // set-up clears the sums)
  if (e == cudaSuccess) e = cudaMemsetAsync(&A->counter, 0, sizeof(unsigned long long) + 2 * sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "tpmc_sweep_noalloc inputs");
  if ((e = launch_setup(A->queries, K, &A->base, h_dirs ? A->dirs : nullptr, h_S ? A->S : nullptr, A->items, nullptr,
                        A->acc, kNoAllocMaxQueries, s)) != cudaSuccess)
    return cuda_fail(e, "setup kernel");
  TraceArgs a{};
  a.mesh = m.dev;
  a.queries = A->queries;
  a.acc = A->acc;
  a.acc_stride = kNoAllocMaxQueries;
  a.items = A->items;
  a.n_items = K;
  a.total = (uint64_t)K * N_each;
  a.counter = &A->counter;
  a.error = &A->error;
  a.count_work = c->counters ? 1u : 0u;
  a.vn_table = c->vn_table;
  const LaunchCfg cfg = c->schedule(m, trace_variant(base, m.dev), a.total);
  a.chunk = cfg.chunk;
  a.smem_nodes = cfg.smem_nodes;
  a.refill_at = cfg.refill_at;
  if ((e = launch_trace(a, trace_variant(base, m.dev), cfg, c->num_sms, s)) != cudaSuccess) return cuda_fail(e, "trace kernel");
  if ((e = launch_finalize(A->queries, A->acc, kNoAllocMaxQueries, K, nullptr, A->results, s)) != cudaSuccess)
    return cuda_fail(e, "finalize kernel");
  int err_word = 0;
  e = cudaMemcpyAsync(h_out, A->results, (size_t)K * sizeof(tpmc_result), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err_word, &A->error, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "tpmc_sweep_noalloc");
  if (err_word != 0) return fail(TPMC_ECUDA, "trace kernel reported a traversal stack overflow");
  // as tpmc_sweep: an item that its set-up rejected reports that in its own
  // status, and every item carries the call's wall time
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (uint32_t k = 0; k < K; ++k) h_out[k].ms = ms;
  return TPMC_OK;
}
